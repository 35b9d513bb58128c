"""CPU FP64 oracle for the GFM dynamic-pressure equation (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It shares no code with the CUDA path: the
arithmetic lives in ``gfm_oracle.c`` (plain C, FP64, -ffp-contract=off), this
file only compiles it and marshals numpy arrays through ctypes.

Every function follows Sec. 3.1 of the paper (Eqs. 12-20) read as documented
in ``gfm_oracle.c``; the readings are listed there.
"""
from __future__ import annotations

import ctypes as ct
import os
import platform
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gfm_oracle.c")
_LIB = os.path.join(_HERE, f"liboracle_{platform.machine()}.so")
_lib = None

(MUT_NONE, MUT_JUMP_SIGN_EQ15, MUT_LAMBDA_FROM_OWNER, MUT_ARITH_BETA, MUT_DROP_JUMP, MUT_SWAP_ALPHA_DERIV,
 MUT_PCG_NO_PRECOND, MUT_PCG_STALE_RZ, MUT_GHOST_SWAP_BETA, MUT_NONORTH_SIGN, MUT_ISO_DOWNWIND) = range(11)
KIND_DRY, KIND_WET, KIND_IF_OWNER_WET, KIND_IF_OWNER_DRY = range(4)


def build(force: bool = False) -> str:
    """Compile gfm_oracle.c into a shared library next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               "-std=c11", "-Wall", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ct.CDLL(_LIB)
        P = ct.c_void_p
        I, D = ct.c_int, ct.c_double
        lib.gfm_oracle_faces.argtypes = [I, I, P, P, P, P, P, D, D, P, P, P, P, P, P, I]
        lib.gfm_oracle_faces.restype = I
        lib.gfm_oracle_assemble.argtypes = [I, I, P, P, P, P, P, I, D, P, P, P, P, P]
        lib.gfm_oracle_assemble.restype = I
        lib.gfm_oracle_spmv.argtypes = [I, P, P, P, P, P]
        lib.gfm_oracle_spmv.restype = None
        lib.gfm_oracle_pcg.argtypes = [I, P, P, P, P, P, D, I, ct.POINTER(I), ct.POINTER(D)]
        lib.gfm_oracle_pcg.restype = I
        lib.gfm_oracle_pcg_fixed.argtypes = [I, P, P, P, P, P, I, I]
        lib.gfm_oracle_pcg_fixed.restype = D
        lib.gfm_oracle_cholesky_solve.argtypes = [I, P, P, P, P, P]
        lib.gfm_oracle_cholesky_solve.restype = I
        lib.gfm_oracle_corrected_flux.argtypes = [I, P, P, P, P, P, P, P]
        lib.gfm_oracle_corrected_flux.restype = None
        lib.gfm_oracle_ghost_route.argtypes = [I, I, P, P, P, P, P, D, D, P, P, P, P, P, P, P]
        lib.gfm_oracle_ghost_route.restype = None
        lib.gfm_oracle_adjoint_chain.argtypes = [I, I, P, P, P, P, P, P, P, P, D, D, P, P, P, P, P, P, I]
        lib.gfm_oracle_adjoint_chain.restype = None
        lib.gfm_oracle_gradient.argtypes = [I, I, P, P, P, P, P, P, P, D, D, P, P, P, I]
        lib.gfm_oracle_gradient.restype = None
        lib.gfm_oracle_reconstruct.argtypes = [I, I, P, P, P, P, P, P, P]
        lib.gfm_oracle_reconstruct.restype = None
        lib.gfm_oracle_nonorth.argtypes = [I, I, P, P, P, P, P, P, P, D, D, P, P, P, P, I]
        lib.gfm_oracle_nonorth.restype = None
        lib.gfm_oracle_iso_flux.argtypes = [I, I, P, P, P, P, D, P, P, I, P, P, P, P, P, P, P, I]
        lib.gfm_oracle_iso_flux.restype = None
        lib.gfm_oracle_iso_advect.argtypes = [I, I, P, P, P, P, P, P]
        lib.gfm_oracle_iso_advect.restype = None
        lib.gfm_oracle_set_threads.argtypes = [I]
        lib.gfm_oracle_set_threads.restype = None
        lib.gfm_oracle_max_threads.restype = I
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ct.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def set_threads(nt: int) -> None:
    _load().gfm_oracle_set_threads(int(nt))


def max_threads() -> int:
    return int(_load().gfm_oracle_max_threads())


@dataclass
class Faces:
    lam: np.ndarray
    gamma: np.ndarray
    jump: np.ndarray
    kind: np.ndarray


@dataclass
class System:
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    diag: np.ndarray
    b: np.ndarray

    @property
    def n(self) -> int:
        return self.diag.size

    def dense(self) -> np.ndarray:
        A = np.zeros((self.n, self.n))
        for i in range(self.n):
            s, e = self.rowptr[i], self.rowptr[i + 1]
            A[i, self.col[s:e]] = self.val[s:e]
        return A

    def matvec(self, x: np.ndarray) -> np.ndarray:
        return spmv(self, x)


def faces(case, alpha=None, mutate: int = MUT_NONE, C=None, rau=None) -> Faces:
    """lambda, gamma, J and the face kind of every internal face (Eqs. 7, 12-18);
    gamma carries the face Rhie-Chow coefficient rau when given."""
    lib = _load()
    n, F = case.n, case.F
    alpha = _f64(case.alpha if alpha is None else alpha)
    C = _f64(case.C if C is None else C)
    lam, gam, jmp = np.empty(F), np.empty(F), np.empty(F)
    kind = np.empty(F, dtype=np.int8)
    g = _f64(case.g)
    rc = lib.gfm_oracle_faces(n, F, _p(_i32(case.owner)), _p(_i32(case.neighbour)), _p(_f64(case.Sf)), _p(C),
                              _p(alpha), case.rho_w, case.rho_a, _p(g),
                              None if rau is None else _p(_f64(rau)), _p(lam), _p(gam), _p(jmp), _p(kind),
                              int(mutate))
    if rc != 0:
        raise ValueError(f"oracle faces: bad mesh ({rc})")
    return Faces(lam, gam, jmp, kind)


def assemble(case, fc: Faces, phi=None, ref_cell=None, ref_value=None) -> System:
    """CSR matrix, diagonal and source of the pinned GFM pressure equation."""
    lib = _load()
    n, F = case.n, case.F
    phi = _f64(case.phi if phi is None else phi)
    rc_ = case.ref_cell if ref_cell is None else ref_cell
    rv = case.ref_value if ref_value is None else ref_value
    rowptr = np.empty(n + 1, dtype=np.int64)
    col = np.empty(n + 2 * F, dtype=np.int32)
    val = np.empty(n + 2 * F)
    diag, b = np.empty(n), np.empty(n)
    rc = lib.gfm_oracle_assemble(n, F, _p(_i32(case.owner)), _p(_i32(case.neighbour)), _p(_f64(fc.gamma)),
                                 _p(_f64(fc.jump)), _p(phi), int(rc_), float(rv), _p(rowptr), _p(col), _p(val),
                                 _p(diag), _p(b))
    if rc != 0:
        raise ValueError(f"oracle assemble failed ({rc})")
    return System(rowptr, col, val, diag, b)


def spmv(sys_: System, x: np.ndarray) -> np.ndarray:
    y = np.empty(sys_.n)
    _load().gfm_oracle_spmv(sys_.n, _p(sys_.rowptr), _p(sys_.col), _p(sys_.val), _p(_f64(x)), _p(y))
    return y


def pcg(sys_: System, b=None, x0=None, rtol: float = 1e-13, maxit: int = 200000):
    """Jacobi-PCG on the pinned system; returns (x, iters, true rel. residual, status)."""
    lib = _load()
    b = _f64(sys_.b if b is None else b)
    x = np.zeros(sys_.n) if x0 is None else _f64(x0).copy()
    it, rel = ct.c_int(0), ct.c_double(0.0)
    st = lib.gfm_oracle_pcg(sys_.n, _p(sys_.rowptr), _p(sys_.col), _p(sys_.val), _p(b), _p(x), float(rtol),
                            int(maxit), ct.byref(it), ct.byref(rel))
    return x, it.value, rel.value, st


def pcg_fixed(sys_: System, iters: int, b=None, x0=None, mutate: int = MUT_NONE):
    """Exactly ``iters`` Jacobi-PCG iterations, no convergence test (timing
    samples).  Returns (x_k, ||r_k||_2 of the recurrence residual)."""
    b = _f64(sys_.b if b is None else b)
    x = np.zeros(sys_.n) if x0 is None else _f64(x0).copy()
    rr = float(_load().gfm_oracle_pcg_fixed(sys_.n, _p(sys_.rowptr), _p(sys_.col), _p(sys_.val), _p(b), _p(x),
                                            int(iters), int(mutate)))
    return x, rr


def cholesky_solve(sys_: System, b=None) -> np.ndarray:
    """Dense textbook Cholesky solve (small n only)."""
    b = _f64(sys_.b if b is None else b)
    x = np.empty(sys_.n)
    rc = _load().gfm_oracle_cholesky_solve(sys_.n, _p(sys_.rowptr), _p(sys_.col), _p(sys_.val), _p(b), _p(x))
    if rc != 0:
        raise np.linalg.LinAlgError(f"oracle Cholesky failed ({rc})")
    return x


def corrected_flux(case, fc: Faces, p: np.ndarray, phi=None) -> np.ndarray:
    out = np.empty(case.F)
    phi = _f64(case.phi if phi is None else phi)
    _load().gfm_oracle_corrected_flux(case.F, _p(_i32(case.owner)), _p(_i32(case.neighbour)), _p(_f64(fc.gamma)),
                                      _p(_f64(fc.jump)), _p(phi), _p(_f64(p)), _p(out))
    return out


def ghost_route(case, p: np.ndarray, alpha=None):
    """Literal Eqs. 12-20 fluxes: returns (q_plus, q_minus, q_ghost, p_plus, p_minus)."""
    F = case.F
    outs = [np.empty(F) for _ in range(5)]
    alpha = _f64(case.alpha if alpha is None else alpha)
    _load().gfm_oracle_ghost_route(case.n, F, _p(_i32(case.owner)), _p(_i32(case.neighbour)), _p(_f64(case.Sf)),
                                   _p(_f64(case.C)), _p(alpha), case.rho_w, case.rho_a, _p(_f64(case.g)),
                                   _p(_f64(p)), *[_p(o) for o in outs])
    return tuple(outs)


def adjoint_chain(case, fc: Faces, p: np.ndarray, mu: np.ndarray, alpha=None, mutate: int = MUT_NONE):
    """dL/dphi*, dL/dalpha, dL/dlambda from the adjoint solution mu (see gfm_oracle.c)."""
    n, F = case.n, case.F
    alpha = _f64(case.alpha if alpha is None else alpha)
    dphi, dalpha, dlam = np.empty(F), np.empty(n), np.empty(F)
    _load().gfm_oracle_adjoint_chain(n, F, _p(_i32(case.owner)), _p(_i32(case.neighbour)), _p(_f64(case.C)),
                                     _p(alpha), _p(_f64(fc.lam)), _p(_f64(fc.gamma)), _p(_f64(fc.jump)),
                                     _p(np.ascontiguousarray(fc.kind, dtype=np.int8)), case.rho_w, case.rho_a,
                                     _p(_f64(case.g)), _p(_f64(p)), _p(_f64(mu)), _p(dphi), _p(dalpha), _p(dlam),
                                     int(mutate))
    return dphi, dalpha, dlam


def gradient(case, p: np.ndarray, alpha=None, xf=None, use_xf: bool = True, mutate: int = MUT_NONE) -> np.ndarray:
    """(1/rho) grad p_d per cell [3, n]: Gauss theorem with the Eq. 20 ghost
    values at interface faces (see gfm_oracle.c).  Face centres: ``xf``, else
    the case's own (case.xf) when use_xf, else midpoints of the centres."""
    n, F = case.n, case.F
    alpha = _f64(case.alpha if alpha is None else alpha)
    if xf is None and use_xf:
        xf = case.xf
    xfp = _p(_f64(xf)) if xf is not None else None
    out = np.empty((3, n))
    _load().gfm_oracle_gradient(n, F, _p(_i32(case.owner)), _p(_i32(case.neighbour)), _p(_f64(case.Sf)),
                                _p(_f64(case.C)), _p(_f64(case.V)), xfp, _p(alpha), case.rho_w, case.rho_a,
                                _p(_f64(case.g)), _p(_f64(p)), _p(out), int(mutate))
    return out


def reconstruct(case, phi: np.ndarray, xf=None, use_xf: bool = True) -> np.ndarray:
    """Cell velocity [3, n] from face fluxes: U_P = sum_f phi_Pf (x_f - x_P) / V_P."""
    n, F = case.n, case.F
    if xf is None and use_xf:
        xf = case.xf
    xfp = _p(_f64(xf)) if xf is not None else None
    out = np.empty((3, n))
    _load().gfm_oracle_reconstruct(n, F, _p(_i32(case.owner)), _p(_i32(case.neighbour)), _p(_f64(case.C)),
                                   _p(_f64(case.V)), xfp, _p(_f64(phi)), _p(out))
    return out


def nonorth_correction(case, p: np.ndarray, rau=None, alpha=None, xf=None, use_xf: bool = True,
                       mutate: int = MUT_NONE) -> np.ndarray:
    """Explicit non-orthogonal correction flux corr_f = rau_f k_f . G_f [F]
    from the gradient of p (see gfm_oracle.c)."""
    n, F = case.n, case.F
    alpha = _f64(case.alpha if alpha is None else alpha)
    if xf is None and use_xf:
        xf = case.xf
    out = np.empty(F)
    _load().gfm_oracle_nonorth(n, F, _p(_i32(case.owner)), _p(_i32(case.neighbour)), _p(_f64(case.Sf)),
                               _p(_f64(case.C)), _p(_f64(case.V)), None if xf is None else _p(_f64(xf)),
                               _p(alpha), case.rho_w, case.rho_a, _p(_f64(case.g)),
                               None if rau is None else _p(_f64(rau)), _p(_f64(p)), _p(out), int(mutate))
    return out


def solve_nonorth(case, correctors: int, rau=None, rtol: float = 1e-13, direct: bool | None = None, phi=None,
                  mutate: int = MUT_NONE):
    """Deferred correction: solve with the implicit part, then `correctors`
    times recompute the explicit non-orthogonal correction from the last
    p_d and solve again.  Returns (p, corr, Faces, System)."""
    fc = faces(case, rau=rau)
    phi = _f64(case.phi if phi is None else phi)
    if direct is None:
        direct = case.n <= 1024
    corr = np.zeros(case.F)
    p = None
    for k in range(correctors + 1):
        sy = assemble(case, fc, phi=phi - corr)
        p = cholesky_solve(sy) if direct else pcg(sy, rtol=rtol, x0=p)[0]
        if k < correctors:
            corr = nonorth_correction(case, p, rau=rau, mutate=mutate)
    return p, corr, fc, sy


def iso_flux(case, phi, dt: float, fv_ptr, fv_xyz, has_iso, xS, nS, UnS, alpha=None, xf=None,
             mutate: int = MUT_NONE):
    """isoAdvector face fluxes (Sec. 3.2): returns (I_f = int alpha_f+ dtau, dV_f = phi_f I_f)."""
    n, F = case.n, case.F
    alpha = _f64(case.alpha if alpha is None else alpha)
    fv_xyz = _f64(fv_xyz).reshape(3, -1)
    I, dV = np.empty(F), np.empty(F)
    _load().gfm_oracle_iso_flux(n, F, _p(_i32(case.owner)), _p(_i32(case.neighbour)), _p(alpha), _p(_f64(phi)),
                                float(dt), _p(_i32(fv_ptr)), _p(np.ascontiguousarray(fv_xyz)), int(fv_xyz.shape[1]),
                                _p(_f64(case.xf if xf is None else xf)),
                                _p(np.ascontiguousarray(has_iso, dtype=np.int8)), _p(_f64(xS)), _p(_f64(nS)),
                                _p(_f64(UnS)), _p(I), _p(dV), int(mutate))
    return I, dV


def iso_advect(case, dV, alpha=None) -> np.ndarray:
    """alpha after the step: alpha - (1/V) sum_f s_f dV_f."""
    out = np.empty(case.n)
    alpha = _f64(case.alpha if alpha is None else alpha)
    _load().gfm_oracle_iso_advect(case.n, case.F, _p(_i32(case.owner)), _p(_i32(case.neighbour)),
                                  _p(_f64(case.V)), _p(alpha), _p(_f64(dV)), _p(out))
    return out


def solve(case, rtol: float | None = None, direct: bool | None = None, alpha=None, phi=None, mutate: int = MUT_NONE,
          C=None):
    """Assemble and solve the pinned system.  Returns (p, Faces, System, info)."""
    fc = faces(case, alpha=alpha, mutate=mutate, C=C)
    sy = assemble(case, fc, phi=phi)
    if direct is None:
        direct = case.n <= 1024
    if direct:
        p = cholesky_solve(sy)
        info = dict(iters=0, relres=float(np.linalg.norm(sy.b - spmv(sy, p)) / max(np.linalg.norm(sy.b), 1e-300)),
                    status=0)
    else:
        p, it, rel, st = pcg(sy, rtol=case.rtol if rtol is None else rtol)
        info = dict(iters=it, relres=rel, status=st)
    return p, fc, sy, info


def adjoint(case, dL_dp: np.ndarray, p=None, rtol: float = 1e-13, direct: bool | None = None, mutate=MUT_NONE):
    """Gradient of L(p) w.r.t. phi* and alpha: returns (dL/dphi, dL/dalpha, mu, p)."""
    fc = faces(case)
    sy = assemble(case, fc)
    if direct is None:
        direct = case.n <= 1024
    if p is None:
        p = cholesky_solve(sy) if direct else pcg(sy, rtol=rtol)[0]
    mu = cholesky_solve(sy, b=dL_dp) if direct else pcg(sy, b=dL_dp, rtol=rtol)[0]
    dphi, dalpha, _ = adjoint_chain(case, fc, p, mu, mutate=mutate)
    return dphi, dalpha, mu, p
