"""GB300-native Ghost Fluid Method pressure solver (arXiv 1804.01130, Sec. 3.1).

A thin ctypes binding over libgfm (C ABI in include/gfm.h).  Every step of the
path -- assembly, solve, corrected flux, adjoint -- runs in libgfm's CUDA
kernels; this module only marshals arguments.  PyTorch supplies device
memory and streams.  There is no CPU fallback: without a built libgfm and a
CUDA device every call raises.
"""
from __future__ import annotations

import ctypes as ct
import os
from dataclasses import dataclass

import torch

from . import build as _build

__all__ = [
    "GFMError", "SolveInfo", "Profile", "GFM", "GFMBatch", "GFMSolve", "load_library", "library_path",
    "solve_csr_noalloc", "NOALLOC_MAX_CELLS",
    "GFM_OK", "GFM_ERR_ARG", "GFM_ERR_CUDA", "GFM_ERR_NOMEM", "GFM_ERR_NOT_CONVERGED", "GFM_ERR_BREAKDOWN",
    "GFM_ERR_TIMEOUT", "GFM_ERR_INCOMPATIBLE", "GFM_ERR_STATE", "EXPORTED_SYMBOLS",
]

(GFM_OK, GFM_ERR_ARG, GFM_ERR_CUDA, GFM_ERR_NOMEM, GFM_ERR_NOT_CONVERGED, GFM_ERR_BREAKDOWN, GFM_ERR_TIMEOUT,
 GFM_ERR_INCOMPATIBLE, GFM_ERR_STATE) = range(9)
GFM_FP64, GFM_MIXED = 0, 1
MODES = {"fp64": GFM_FP64, "mixed": GFM_MIXED}

EXPORTED_SYMBOLS = (
    "gfm_default_opts", "gfm_create", "gfm_destroy", "gfm_assemble", "gfm_export_system", "gfm_solve",
    "gfm_solve_adjoint", "gfm_solve_host", "gfm_set_tuning", "gfm_get_tuning", "gfm_set_profiling",
    "gfm_get_profile", "gfm_get_sizes", "gfm_get_permutation", "gfm_status_string", "gfm_last_error",
    "gfm_set_coarse", "gfm_get_coarse", "gfm_create_batched", "gfm_solve_csr_noalloc", "gfm_autotune",
    "gfm_partition_tanks", "gfm_gradient", "gfm_set_rau", "gfm_nonorth_correct", "gfm_set_table",
    "gfm_get_table", "gfm_piso_step", "gfm_iso_advect",
)

# largest n accepted by gfm_solve_csr_noalloc (its fixed device scratch)
NOALLOC_MAX_CELLS = 262144


class GFMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


class _Mesh(ct.Structure):
    _fields_ = [("n_cells", ct.c_int32), ("n_faces", ct.c_int32), ("owner", ct.c_void_p),
                ("neighbour", ct.c_void_p), ("Sf", ct.c_void_p), ("C", ct.c_void_p), ("V", ct.c_void_p)]


class _Phys(ct.Structure):
    _fields_ = [("rho_w", ct.c_double), ("rho_a", ct.c_double), ("g", ct.c_double * 3), ("ref_cell", ct.c_int32),
                ("ref_value", ct.c_double)]


class _Opts(ct.Structure):
    _fields_ = [("mode", ct.c_int32), ("rtol", ct.c_double), ("inner_rtol", ct.c_double),
                ("max_iters", ct.c_int32), ("max_refine", ct.c_int32), ("use_x0", ct.c_int32),
                ("info_on_device", ct.c_int32), ("timeout_ms", ct.c_double)]


class _Info(ct.Structure):
    _fields_ = [("iters", ct.c_int32), ("refinements", ct.c_int32), ("status", ct.c_int32),
                ("reserved", ct.c_int32), ("rel_res_l2", ct.c_double), ("rel_res_l1", ct.c_double)]


class _Tuning(ct.Structure):
    _fields_ = [("threads", ct.c_int32), ("ctas_per_sm", ct.c_int32), ("form", ct.c_int32)]


class _Profile(ct.Structure):
    _fields_ = [("ms_assemble", ct.c_float), ("ms_solve", ct.c_float), ("ms_total", ct.c_float),
                ("launches", ct.c_int32), ("grid", ct.c_int32), ("threads", ct.c_int32),
                ("launches_total", ct.c_int32)]


@dataclass
class SolveInfo:
    iters: int
    refinements: int
    status: int
    rel_res_l2: float
    rel_res_l1: float


@dataclass
class Profile:
    ms_assemble: float
    ms_solve: float
    ms_total: float
    launches: int
    grid: int
    threads: int
    launches_total: int


_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load libgfm (building it first if needed).  Raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise GFMError(GFM_ERR_CUDA, f"libgfm not built: {path}")
    lib = ct.CDLL(path)
    P, I, S = ct.c_void_p, ct.c_int32, ct.c_int
    sig = {
        "gfm_default_opts": ([ct.POINTER(_Opts)], S),
        "gfm_create": ([ct.POINTER(_Mesh), I, P, ct.POINTER(P)], S),
        "gfm_create_batched": ([P, I, I, P, ct.POINTER(P)], S),
        "gfm_destroy": ([P], S),
        "gfm_assemble": ([P, P, P, ct.POINTER(_Phys), P], S),
        "gfm_export_system": ([P, P, P, P, P, P, P], S),
        "gfm_solve": ([P, ct.POINTER(_Opts), P, P, P, P], S),
        "gfm_solve_adjoint": ([P, ct.POINTER(_Opts), P, P, P, P, P, P, P], S),
        "gfm_solve_host": ([P, P, P, ct.POINTER(_Phys), ct.POINTER(_Opts), P, P, P], S),
        "gfm_set_tuning": ([P, ct.POINTER(_Tuning)], S),
        "gfm_get_tuning": ([P, ct.POINTER(_Tuning)], S),
        "gfm_set_profiling": ([P, I], S),
        "gfm_get_profile": ([P, ct.POINTER(_Profile)], S),
        "gfm_get_sizes": ([P, ct.POINTER(I), ct.POINTER(I), ct.POINTER(I)], S),
        "gfm_get_permutation": ([P, P], S),
        "gfm_set_coarse": ([P, I, I], S),
        "gfm_get_coarse": ([P, ct.POINTER(I), ct.POINTER(I), P, P], S),
        "gfm_solve_csr_noalloc": ([I, I, P, P, P, P, P, ct.c_double, I, I, ct.c_double, P, P], S),
        "gfm_autotune": ([P, ct.POINTER(_Opts), I, ct.POINTER(_Tuning), ct.POINTER(ct.c_float), P], S),
        "gfm_partition_tanks": ([P, I, I, P, P], S),
        "gfm_gradient": ([P, P, P, P, P, P, P, P], S),
        "gfm_set_rau": ([P, P, P], S),
        "gfm_set_table": ([P, I, I], S),
        "gfm_iso_advect": ([P, P, P, ct.c_double, P, P, I, P, P, P, P, P, P, P, P, P, P], S),
        "gfm_piso_step": ([P, ct.POINTER(_Opts), I, I, P, P, ct.POINTER(_Phys), P, P, P, P, P, P, P, P], S),
        "gfm_get_table": ([P, ct.POINTER(I), ct.POINTER(I), ct.POINTER(I)], S),
        "gfm_nonorth_correct": ([P, P, P, P, P, P], S),
        "gfm_status_string": ([S], ct.c_char_p),
        "gfm_last_error": ([P], ct.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda:
        raise GFMError(GFM_ERR_ARG, "libgfm takes CUDA tensors (device memory)")
    if not t.is_contiguous():
        raise GFMError(GFM_ERR_ARG, "libgfm takes contiguous tensors")
    return ct.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ct.c_void_p(s.cuda_stream)


def _f64(x, device) -> torch.Tensor:
    t = torch.as_tensor(x)
    return t.to(device=device, dtype=torch.float64).contiguous()


def _i32(x, device) -> torch.Tensor:
    return torch.as_tensor(x).to(device=device, dtype=torch.int32).contiguous()


class GFM:
    """One mesh's GFM pressure system on the current CUDA device.

    Parameters mirror gfm_create: owner/neighbour [F] int32, Sf [3, F], C [3, n]
    (any array-likes; copied to the device), renumber 0/1/2 (none/RCM/Morton).
    """

    def __init__(self, owner, neighbour, Sf, C, V=None, renumber: int = 1, device=None, stream=None):
        self.lib = load_library()
        if not torch.cuda.is_available():
            raise GFMError(GFM_ERR_CUDA, "no CUDA device: libgfm has no CPU path")
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        d = self.device
        self.owner = _i32(owner, d)
        self.neighbour = _i32(neighbour, d)
        self.Sf = _f64(Sf, d).reshape(3, -1).contiguous()
        self.C = _f64(C, d).reshape(3, -1).contiguous()
        self.n = int(self.C.shape[1])
        self.F = int(self.owner.numel())
        mesh = _Mesh(self.n, self.F, self.owner.data_ptr(), self.neighbour.data_ptr(), self.Sf.data_ptr(),
                     self.C.data_ptr(), None)
        h = ct.c_void_p()
        with torch.cuda.device(d):
            st = self.lib.gfm_create(ct.byref(mesh), int(renumber), _stream(stream), ct.byref(h))
        if st != GFM_OK:
            raise GFMError(st, f"gfm_create: {self.lib.gfm_status_string(st).decode()}")
        self.h = h
        self.phys = None
        self._info_dev = torch.zeros(4, dtype=torch.float64, device=d)  # 32 bytes = gfm_solve_info

    @classmethod
    def from_case(cls, case, renumber: int = 1, **kw) -> "GFM":
        return cls(case.owner, case.neighbour, case.Sf, case.C, renumber=renumber, **kw)

    # -- helpers ----------------------------------------------------------
    def _check(self, st: int, what: str):
        if st != GFM_OK:
            msg = self.lib.gfm_last_error(self.h).decode()
            raise GFMError(st, f"{what}: {self.lib.gfm_status_string(st).decode()}: {msg}")

    def close(self):
        if getattr(self, "h", None):
            self.lib.gfm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def make_phys(rho_w=1000.0, rho_a=1.0, g=(0.0, -9.81, 0.0), ref_cell=0, ref_value=0.0) -> _Phys:
        return _Phys(float(rho_w), float(rho_a), (ct.c_double * 3)(*[float(v) for v in g]), int(ref_cell),
                     float(ref_value))

    def make_opts(self, mode="mixed", rtol=1e-10, inner_rtol=1e-4, max_iters=1_000_000, max_refine=30,
                  use_x0=False, info_on_device=False, timeout_ms=2000.0) -> _Opts:
        o = _Opts()
        self.lib.gfm_default_opts(ct.byref(o))
        o.mode = MODES[mode] if isinstance(mode, str) else int(mode)
        o.rtol = float(rtol)
        o.inner_rtol = float(inner_rtol)
        o.max_iters = int(max_iters)
        o.max_refine = int(max_refine)
        o.use_x0 = int(bool(use_x0))
        o.info_on_device = int(bool(info_on_device))
        o.timeout_ms = float(timeout_ms)
        return o

    # -- ABI calls ----------------------------------------------------------
    def assemble(self, alpha: torch.Tensor, phi: torch.Tensor, rho_w=1000.0, rho_a=1.0, g=(0.0, -9.81, 0.0),
                 ref_cell=0, ref_value=0.0, stream=None):
        alpha = _f64(alpha, self.device)
        phi = _f64(phi, self.device)
        self.phys = self.make_phys(rho_w, rho_a, g, ref_cell, ref_value)
        self._check(self.lib.gfm_assemble(self.h, _ptr(alpha), _ptr(phi), ct.byref(self.phys), _stream(stream)),
                    "gfm_assemble")

    def export_system(self, stream=None) -> dict:
        d = self.device
        out = {k: torch.empty(self.F, dtype=torch.float64, device=d) for k in ("lambda", "gamma", "jump")}
        out.update({k: torch.empty(self.n, dtype=torch.float64, device=d) for k in ("diag", "b")})
        self._check(self.lib.gfm_export_system(self.h, _ptr(out["lambda"]), _ptr(out["gamma"]), _ptr(out["jump"]),
                                               _ptr(out["diag"]), _ptr(out["b"]), _stream(stream)),
                    "gfm_export_system")
        return out

    def solve(self, mode="mixed", rtol=1e-10, inner_rtol=1e-4, p0=None, phi_corr=False, max_iters=1_000_000,
              max_refine=30, info_on_device=False, timeout_ms=2000.0, out=None, raise_on_error=True, stream=None):
        """Solve the assembled system; returns (p, phi_corr or None, SolveInfo or device tensor)."""
        p = out if out is not None else torch.empty(self.n, dtype=torch.float64, device=self.device)
        if p0 is not None:
            p.copy_(_f64(p0, self.device))
        fc = torch.empty(self.F, dtype=torch.float64, device=self.device) if phi_corr else None
        o = self.make_opts(mode, rtol, inner_rtol, max_iters, max_refine, p0 is not None, info_on_device, timeout_ms)
        if info_on_device:
            st = self.lib.gfm_solve(self.h, ct.byref(o), _ptr(p), _ptr(fc), _ptr(self._info_dev), _stream(stream))
            self._check(st, "gfm_solve")
            return p, fc, self._info_dev
        info = _Info()
        st = self.lib.gfm_solve(self.h, ct.byref(o), _ptr(p), _ptr(fc), ct.byref(info), _stream(stream))
        si = SolveInfo(info.iters, info.refinements, info.status, info.rel_res_l2, info.rel_res_l1)
        if st != GFM_OK and (raise_on_error or st not in (GFM_ERR_NOT_CONVERGED, GFM_ERR_BREAKDOWN,
                                                          GFM_ERR_TIMEOUT)):
            self._check(st, "gfm_solve")
        return p, fc, si

    def adjoint(self, p: torch.Tensor, dL_dp: torch.Tensor, mode="fp64", rtol=1e-12, inner_rtol=1e-4,
                max_iters=1_000_000, max_refine=30, timeout_ms=2000.0, raise_on_error=True, stream=None):
        """Returns (dL/dphi [F], dL/dalpha [n], mu [n], SolveInfo)."""
        d = self.device
        p = _f64(p, d)
        g = _f64(dL_dp, d)
        dphi = torch.empty(self.F, dtype=torch.float64, device=d)
        dalpha = torch.empty(self.n, dtype=torch.float64, device=d)
        mu = torch.empty(self.n, dtype=torch.float64, device=d)
        o = self.make_opts(mode, rtol, inner_rtol, max_iters, max_refine, False, False, timeout_ms)
        info = _Info()
        st = self.lib.gfm_solve_adjoint(self.h, ct.byref(o), _ptr(p), _ptr(g), _ptr(dphi), _ptr(dalpha), _ptr(mu),
                                        ct.byref(info), _stream(stream))
        if st != GFM_OK and (raise_on_error or st not in (GFM_ERR_NOT_CONVERGED, GFM_ERR_BREAKDOWN,
                                                          GFM_ERR_TIMEOUT)):
            self._check(st, "gfm_solve_adjoint")
        return dphi, dalpha, mu, SolveInfo(info.iters, info.refinements, info.status, info.rel_res_l2,
                                           info.rel_res_l1)

    def solve_host(self, alpha_host: torch.Tensor, phi_host: torch.Tensor, p_host: torch.Tensor, mode="mixed",
                   rtol=1e-10, inner_rtol=1e-4, rho_w=1000.0, rho_a=1.0, g=(0.0, -9.81, 0.0), ref_cell=0,
                   ref_value=0.0, stream=None) -> SolveInfo:
        """End-to-end call on host (ideally pinned) float64 tensors; p_host is filled."""
        for t in (alpha_host, phi_host, p_host):
            if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
                raise GFMError(GFM_ERR_ARG, "solve_host takes contiguous float64 host tensors")
        self.phys = self.make_phys(rho_w, rho_a, g, ref_cell, ref_value)
        o = self.make_opts(mode, rtol, inner_rtol)
        info = _Info()
        st = self.lib.gfm_solve_host(self.h, ct.c_void_p(alpha_host.data_ptr()), ct.c_void_p(phi_host.data_ptr()),
                                     ct.byref(self.phys), ct.byref(o), ct.c_void_p(p_host.data_ptr()),
                                     ct.byref(info), _stream(stream))
        self._check(st, "gfm_solve_host")
        return SolveInfo(info.iters, info.refinements, info.status, info.rel_res_l2, info.rel_res_l1)

    def gradient(self, p: torch.Tensor, V, xf=None, phi: torch.Tensor | None = None, want_grad: bool = True,
                 stream=None):
        """(1/rho) grad p_d [3, n] with the GFM ghost values (None unless
        want_grad) and, when phi [F] is given, the cell velocity [3, n]
        reconstructed from it (gfm_gradient)."""
        d = self.device
        p = _f64(p, d)
        V = _f64(V, d)
        xf = None if xf is None else _f64(xf, d).reshape(3, -1).contiguous()
        phi = None if phi is None else _f64(phi, d)
        grad = torch.empty((3, self.n), dtype=torch.float64, device=d) if want_grad else None
        U = torch.empty((3, self.n), dtype=torch.float64, device=d) if phi is not None else None
        self._check(self.lib.gfm_gradient(self.h, _ptr(p), _ptr(V), _ptr(xf), _ptr(grad), _ptr(phi), _ptr(U),
                                          _stream(stream)), "gfm_gradient")
        return grad, U

    def piso_step(self, alpha, phi_star: torch.Tensor, p: torch.Tensor, info: torch.Tensor, V=None, xf=None,
                  n_nonorth: int = 0, phi_corr: torch.Tensor | None = None, grad: torch.Tensor | None = None,
                  U: torch.Tensor | None = None, mode="mixed", rtol=1e-10, inner_rtol=1e-4, use_x0=False,
                  rho_w=1000.0, rho_a=1.0, g=(0.0, -9.81, 0.0), ref_cell=0, ref_value=0.0, timeout_ms=2000.0,
                  stream=None):
        """Enqueue the pressure part of one time step (gfm_piso_step):
        phi_star [n_solves, F] predicted fluxes, p [n] solution (x0 when
        use_x0), info a float64 device tensor of 4 * n_solves entries (the
        records), optional outputs phi_corr [F], grad and U [3, n].  Nothing
        is synchronised, so the call can be captured in a CUDA graph; every
        tensor must already be on the device."""
        for t in (alpha, phi_star, p, info):
            if not (isinstance(t, torch.Tensor) and t.is_cuda):
                raise GFMError(GFM_ERR_ARG, "piso_step takes device tensors")
        n_solves = int(phi_star.shape[0]) if phi_star.dim() == 2 else int(phi_star.numel() // self.F)
        if phi_star.numel() != n_solves * self.F or n_solves < 1:
            raise GFMError(GFM_ERR_ARG, f"phi_star must hold n_solves x {self.F} values")
        if info.numel() * info.element_size() < 32 * n_solves:
            raise GFMError(GFM_ERR_ARG, f"info needs {32 * n_solves} bytes")
        self.phys = self.make_phys(rho_w, rho_a, g, ref_cell, ref_value)
        o = self.make_opts(mode, rtol, inner_rtol, 1_000_000, 30, use_x0, True, timeout_ms)
        self._check(self.lib.gfm_piso_step(self.h, ct.byref(o), n_solves, int(n_nonorth), _ptr(alpha),
                                           _ptr(phi_star), ct.byref(self.phys), _ptr(p), _ptr(phi_corr), _ptr(V),
                                           _ptr(xf), _ptr(grad), _ptr(U), _ptr(info), _stream(stream)),
                    "gfm_piso_step")

    def iso_advect(self, alpha, phi, dt: float, fv_ptr, fv_xyz, xf, has_iso, xS, nS, UnS, V=None,
                   stream=None):
        """isoAdvector step (gfm_iso_advect): returns (dV [F], integral [F],
        alpha_new [n] or None without V).  Inputs are array-likes, copied to
        the device."""
        d = self.device
        alpha, phi = _f64(alpha, d), _f64(phi, d)
        fv_ptr = _i32(fv_ptr, d)
        fv_xyz = _f64(fv_xyz, d).reshape(3, -1).contiguous()
        xf = _f64(xf, d).reshape(3, -1).contiguous()
        has = torch.as_tensor(has_iso).to(device=d, dtype=torch.int8).contiguous()
        xS = _f64(xS, d).reshape(3, -1).contiguous()
        nS = _f64(nS, d).reshape(3, -1).contiguous()
        UnS = _f64(UnS, d)
        V = None if V is None else _f64(V, d)
        dV = torch.empty(self.F, dtype=torch.float64, device=d)
        integral = torch.empty(self.F, dtype=torch.float64, device=d)
        a_new = torch.empty(self.n, dtype=torch.float64, device=d) if V is not None else None
        self._check(self.lib.gfm_iso_advect(self.h, _ptr(alpha), _ptr(phi), float(dt), _ptr(fv_ptr), _ptr(fv_xyz),
                                            int(fv_xyz.shape[1]), _ptr(xf), _ptr(has), _ptr(xS), _ptr(nS),
                                            _ptr(UnS), _ptr(V), _ptr(integral), _ptr(dV), _ptr(a_new),
                                            _stream(stream)), "gfm_iso_advect")
        return dV, integral, a_new

    def infos_of_step(self, info: torch.Tensor, n_solves: int):
        """The n_solves records a piso_step wrote."""
        raw = info.detach().cpu().numpy().tobytes()[:32 * n_solves]
        rec = (_Info * n_solves).from_buffer_copy(raw)
        return [SolveInfo(i.iters, i.refinements, i.status, i.rel_res_l2, i.rel_res_l1) for i in rec]

    def set_table(self, compact: bool = False, force_stream: bool = False):
        """Operator-table format of the streamed mixed pass (gfm_set_table)."""
        self._check(self.lib.gfm_set_table(self.h, int(bool(compact)), int(bool(force_stream))), "gfm_set_table")

    def table_info(self) -> dict:
        """{'compact_usable', 'classes', 'compact_valid'} (gfm_get_table)."""
        u, k, v = ct.c_int32(), ct.c_int32(), ct.c_int32()
        self._check(self.lib.gfm_get_table(self.h, ct.byref(u), ct.byref(k), ct.byref(v)), "gfm_get_table")
        return {"compact_usable": bool(u.value), "classes": k.value, "compact_valid": bool(v.value)}

    def set_rau(self, rau=None, stream=None):
        """Face Rhie-Chow coefficient 1/a_P [F] for the next assemblies (None = 1)."""
        self._rau = None if rau is None else _f64(rau, self.device)
        self._check(self.lib.gfm_set_rau(self.h, _ptr(self._rau), _stream(stream)), "gfm_set_rau")

    def nonorth_correct(self, p: torch.Tensor, V, xf=None, return_corr: bool = False, stream=None):
        """Explicit non-orthogonal correction from p_d into the assembled
        source (gfm_nonorth_correct); the next solve uses it.  Returns the
        correction flux [F] when asked."""
        d = self.device
        p = _f64(p, d)
        V = _f64(V, d)
        xf = None if xf is None else _f64(xf, d).reshape(3, -1).contiguous()
        corr = torch.empty(self.F, dtype=torch.float64, device=d) if return_corr else None
        self._check(self.lib.gfm_nonorth_correct(self.h, _ptr(p), _ptr(V), _ptr(xf), _ptr(corr), _stream(stream)),
                    "gfm_nonorth_correct")
        return corr

    def set_tuning(self, threads=0, ctas_per_sm=0, form=0):
        """Launch shape and mixed iteration form (1: two passes, 2: fused); 0 keeps a value."""
        self._check(self.lib.gfm_set_tuning(self.h, ct.byref(_Tuning(int(threads), int(ctas_per_sm), int(form)))),
                    "gfm_set_tuning")

    def get_tuning(self):
        t = _Tuning()
        self._check(self.lib.gfm_get_tuning(self.h, ct.byref(t)), "gfm_get_tuning")
        return t.threads, t.ctas_per_sm

    def iteration_form(self) -> int:
        """The mixed iteration form in use: 1 (two passes per iteration) or 2 (fused, one all-reduce)."""
        t = _Tuning()
        self._check(self.lib.gfm_get_tuning(self.h, ct.byref(t)), "gfm_get_tuning")
        return t.form

    def autotune(self, mode="mixed", rtol=1e-10, inner_rtol=1e-4, trials=3, timeout_ms=2000.0, stream=None):
        """Time the launch shapes (and, batched, the iteration-weighted tank table) on the assembled
        system and keep the fastest; returns (threads, ctas_per_sm, median ms)."""
        o = self.make_opts(mode, rtol, inner_rtol, 1_000_000, 30, False, False, timeout_ms)
        t = _Tuning()
        ms = ct.c_float(0.0)
        self._check(self.lib.gfm_autotune(self.h, ct.byref(o), int(trials), ct.byref(t), ct.byref(ms),
                                          _stream(stream)), "gfm_autotune")
        return t.threads, t.ctas_per_sm, float(ms.value)

    def set_coarse(self, max_vectors: int = 8, min_size: int = 64):
        """Coarse space of the two-level preconditioner (0 vectors = Jacobi only); next assembly on."""
        self._check(self.lib.gfm_set_coarse(self.h, int(max_vectors), int(min_size)), "gfm_set_coarse")

    def coarse_info(self, stream=None):
        """(vectors in use, regions of at least min_size cells, sizes of the kept regions)."""
        import numpy as np
        k, nr = ct.c_int32(), ct.c_int32()
        sizes = np.zeros(8, dtype=np.int32)
        self._check(self.lib.gfm_get_coarse(self.h, ct.byref(k), ct.byref(nr), ct.c_void_p(sizes.ctypes.data),
                                            _stream(stream)), "gfm_get_coarse")
        return k.value, nr.value, sizes[:k.value].tolist()

    def set_profiling(self, on: bool = True):
        self._check(self.lib.gfm_set_profiling(self.h, int(bool(on))), "gfm_set_profiling")

    def profile(self) -> Profile:
        pr = _Profile()
        self._check(self.lib.gfm_get_profile(self.h, ct.byref(pr)), "gfm_get_profile")
        return Profile(pr.ms_assemble, pr.ms_solve, pr.ms_total, pr.launches, pr.grid, pr.threads,
                       pr.launches_total)

    def permutation(self):
        import numpy as np
        perm = np.empty(self.n, dtype=np.int32)
        self._check(self.lib.gfm_get_permutation(self.h, ct.c_void_p(perm.ctypes.data)), "gfm_get_permutation")
        return perm

    @staticmethod
    def info_from_device(t: torch.Tensor) -> SolveInfo:
        raw = t.detach().cpu().numpy().tobytes()
        info = _Info.from_buffer_copy(raw)
        return SolveInfo(info.iters, info.refinements, info.status, info.rel_res_l2, info.rel_res_l1)


class GFMSolve(torch.autograd.Function):
    """p = GFMSolve.apply(alpha, phi, gfm, phys_kwargs, solve_kwargs): differentiable GFM pressure solve.

    Forward assembles and solves; backward solves the adjoint system (A is
    symmetric) in libgfm and returns dL/dalpha and dL/dphi.  Only (alpha, phi,
    p) are saved: no Krylov state is stored; the system is re-assembled in
    backward if the handle was re-assembled since.
    """

    @staticmethod
    def forward(ctx, alpha, phi, gfm: GFM, phys_kwargs: dict, solve_kwargs: dict):
        gfm.assemble(alpha.detach(), phi.detach(), **phys_kwargs)
        p, _, info = gfm.solve(**solve_kwargs)
        ctx.gfm = gfm
        ctx.phys_kwargs = phys_kwargs
        ctx.solve_kwargs = solve_kwargs
        ctx.save_for_backward(alpha.detach(), phi.detach(), p)
        ctx.stamp = id(gfm.phys)
        return p

    @staticmethod
    def backward(ctx, grad_p):
        alpha, phi, p = ctx.saved_tensors
        gfm = ctx.gfm
        if id(gfm.phys) != ctx.stamp:
            gfm.assemble(alpha, phi, **ctx.phys_kwargs)
        kw = dict(mode=ctx.solve_kwargs.get("mode", "fp64"), rtol=min(ctx.solve_kwargs.get("rtol", 1e-10), 1e-10))
        dphi, dalpha, _, _ = gfm.adjoint(p, grad_p.contiguous(), **kw)
        return dalpha, dphi, None, None, None


class GFMBatch(GFM):
    """Many independent tanks solved by one persistent launch (gfm_create_batched).

    ``tanks`` is a list of objects with owner, neighbour, Sf, C (e.g. cases.Case).
    Cell and face arrays of every later call are the tanks' arrays concatenated
    in tank order; physics is given per tank.
    """

    def __init__(self, tanks, renumber: int = 1, device=None, stream=None):
        self.lib = load_library()
        if not torch.cuda.is_available():
            raise GFMError(GFM_ERR_CUDA, "no CUDA device: libgfm has no CPU path")
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        d = self.device
        self.T = len(tanks)
        self._keep = []
        meshes = (_Mesh * self.T)()
        self.ncell, self.nface = [], []
        for k, t in enumerate(tanks):
            own, nb = _i32(t.owner, d), _i32(t.neighbour, d)
            Sf = _f64(t.Sf, d).reshape(3, -1).contiguous()
            C = _f64(t.C, d).reshape(3, -1).contiguous()
            self._keep += [own, nb, Sf, C]
            meshes[k] = _Mesh(int(C.shape[1]), int(own.numel()), own.data_ptr(), nb.data_ptr(), Sf.data_ptr(),
                              C.data_ptr(), None)
            self.ncell.append(int(C.shape[1]))
            self.nface.append(int(own.numel()))
        h = ct.c_void_p()
        with torch.cuda.device(d):
            st = self.lib.gfm_create_batched(ct.cast(meshes, ct.c_void_p), self.T, int(renumber), _stream(stream),
                                             ct.byref(h))
        if st != GFM_OK:
            raise GFMError(st, f"gfm_create_batched: {self.lib.gfm_status_string(st).decode()}")
        self._keep = []  # the handle holds its own copy of the meshes
        self.h = h
        self.n = sum(self.ncell)
        self.F = sum(self.nface)
        self.phys = None
        self._info_dev = torch.zeros(4 * self.T, dtype=torch.float64, device=d)

    def assemble(self, alpha, phi, phys: list, stream=None):
        """phys: list of dicts (rho_w, rho_a, g, ref_cell, ref_value), one per tank."""
        alpha = _f64(alpha, self.device)
        phi = _f64(phi, self.device)
        arr = (_Phys * self.T)()
        for k, ph in enumerate(phys):
            arr[k] = self.make_phys(**ph)
        self.phys = arr
        self._check(self.lib.gfm_assemble(self.h, _ptr(alpha), _ptr(phi), ct.cast(arr, ct.POINTER(_Phys)),
                                          _stream(stream)), "gfm_assemble")

    def solve(self, mode="mixed", rtol=1e-8, inner_rtol=1e-4, p0=None, phi_corr=False, max_iters=1_000_000,
              max_refine=30, info_on_device=False, timeout_ms=2000.0, out=None, raise_on_error=True, stream=None):
        """Returns (p, phi_corr or None, list of SolveInfo or the device records)."""
        p = out if out is not None else torch.empty(self.n, dtype=torch.float64, device=self.device)
        if p0 is not None:
            p.copy_(_f64(p0, self.device))
        fc = torch.empty(self.F, dtype=torch.float64, device=self.device) if phi_corr else None
        o = self.make_opts(mode, rtol, inner_rtol, max_iters, max_refine, p0 is not None, info_on_device, timeout_ms)
        if info_on_device:
            st = self.lib.gfm_solve(self.h, ct.byref(o), _ptr(p), _ptr(fc), _ptr(self._info_dev), _stream(stream))
            self._check(st, "gfm_solve")
            return p, fc, self._info_dev
        infos = (_Info * self.T)()
        st = self.lib.gfm_solve(self.h, ct.byref(o), _ptr(p), _ptr(fc), ct.cast(infos, ct.c_void_p),
                                _stream(stream))
        out_infos = [SolveInfo(i.iters, i.refinements, i.status, i.rel_res_l2, i.rel_res_l1) for i in infos]
        if st != GFM_OK and (raise_on_error or st not in (GFM_ERR_NOT_CONVERGED, GFM_ERR_BREAKDOWN,
                                                          GFM_ERR_TIMEOUT)):
            self._check(st, "gfm_solve")
        return p, fc, out_infos

    def infos_from_device(self, t: torch.Tensor):
        raw = t.detach().cpu().numpy().tobytes()
        rec = (_Info * self.T).from_buffer_copy(raw)
        return [SolveInfo(i.iters, i.refinements, i.status, i.rel_res_l2, i.rel_res_l1) for i in rec]


def _check_csr_noalloc(row_ptr, col, val, b, x, info) -> tuple[int, int]:
    """Host-side checks of solve_csr_noalloc's tensors (no device access):
    dtypes, sizes (row_ptr [n+1], col and val [nnz], x [n], info at least
    one record) and one common device.  Returns (n, nnz)."""
    n = int(b.numel())
    nnz = int(col.numel())
    for name, t, dt in (("row_ptr", row_ptr, torch.int32), ("col", col, torch.int32), ("val", val, torch.float64),
                        ("b", b, torch.float64), ("x", x, torch.float64), ("info", info, torch.uint8)):
        if t.dtype != dt:
            raise GFMError(GFM_ERR_ARG, f"gfm_solve_csr_noalloc: {name} must be {dt}, got {t.dtype}")
        if t.device != b.device:
            raise GFMError(GFM_ERR_ARG, f"gfm_solve_csr_noalloc: {name} is on {t.device}, b on {b.device}")
    if not 1 <= n <= NOALLOC_MAX_CELLS:
        raise GFMError(GFM_ERR_ARG, f"gfm_solve_csr_noalloc: n = {n} is outside 1..{NOALLOC_MAX_CELLS}, the "
                                    "capacity of its fixed device scratch")
    if row_ptr.numel() != n + 1:
        raise GFMError(GFM_ERR_ARG, f"gfm_solve_csr_noalloc: row_ptr has {row_ptr.numel()} entries, need n+1 = {n + 1}")
    if val.numel() != nnz:
        raise GFMError(GFM_ERR_ARG, f"gfm_solve_csr_noalloc: col has {nnz} entries but val {val.numel()}")
    if nnz < n or nnz >= 2**31:
        raise GFMError(GFM_ERR_ARG, f"gfm_solve_csr_noalloc: nnz = {nnz} must be in [n, 2^31)")
    if x.numel() != n:
        raise GFMError(GFM_ERR_ARG, f"gfm_solve_csr_noalloc: x has {x.numel()} entries, b {n}")
    if info.numel() < ct.sizeof(_Info):
        raise GFMError(GFM_ERR_ARG, f"gfm_solve_csr_noalloc: info needs {ct.sizeof(_Info)} bytes")
    return n, nnz


def solve_csr_noalloc(row_ptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor, b: torch.Tensor,
                      x: torch.Tensor | None = None, rtol: float = 1e-10, max_iters: int = 1_000_000,
                      use_x0: bool = False, timeout_ms: float = 2000.0, info: torch.Tensor | None = None,
                      stream=None):
    """FP64 Jacobi-PCG of a CSR system through gfm_solve_csr_noalloc, which
    allocates no device memory (for callers that cannot; its temporaries sit
    in a fixed device array of the library, n <= NOALLOC_MAX_CELLS).  All
    tensors are caller-owned CUDA tensors on one device (int32 row_ptr [n+1]
    and col [nnz], FP64 val [nnz], b [n] and x [n]); x and info (a uint8
    device tensor of at least 32 bytes for the result record) are made here
    when not given.  Sizes, dtypes and devices are checked here; the CSR
    structure (row bounds, column range) is checked by the kernel, which
    then reports GFM_ERR_ARG in the record.  Returns (x, info tensor); read
    the record with GFM.info_from_device.  Enqueues only: nothing is
    synchronised."""
    if x is None:
        x = torch.zeros(b.numel(), dtype=torch.float64, device=b.device)
    if info is None:
        info = torch.zeros(ct.sizeof(_Info), dtype=torch.uint8, device=b.device)
    n, nnz = _check_csr_noalloc(row_ptr, col, val, b, x, info)
    lib = load_library()
    st = lib.gfm_solve_csr_noalloc(n, nnz, _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(b), _ptr(x), float(rtol),
                                   int(max_iters), int(bool(use_x0)), float(timeout_ms), _ptr(info),
                                   _stream(stream))
    if st != GFM_OK:
        raise GFMError(st, f"gfm_solve_csr_noalloc: {lib.gfm_status_string(st).decode()}")
    return x, info
