"""The compact operator table of the streamed mixed pass (gfm_set_table /
gfm_get_table): 4 bytes per slot instead of 8, with the same arithmetic, so
solutions must be bit-identical to the full table's and within the mixed
bar (relative L2 1e-6) of the oracle.  Small meshes are made to stream
their tables (force_stream) so that both formats run on them: 2D and 3D
rows (4- and 6-face instantiations), permuted cell orders, a batch of
tanks; and the cases where the compact form must stand aside (a face
Rhie-Chow coefficient; neighbour offsets beyond 16 bits)."""
import numpy as np
import pytest
import torch

import cases
import oracle

pytestmark = pytest.mark.gpu


def _g():
    import paper_1804_01130_gb300 as g
    return g


def _solve_both(s, c, rtol=1e-10):
    out = []
    for compact in (True, False):
        s.set_table(compact=compact, force_stream=True)
        p, _, info = s.solve(mode="mixed", rtol=rtol)
        assert info.status == 0, (compact, info)
        out.append((p.clone(), info))
    return out


@pytest.mark.parametrize("mk", [
    lambda: cases.box_case(40, 24, 1, seed=3, ka=0.12),
    lambda: cases.box_case(24, 16, 12, seed=5, permute=True, alpha_noise=0.05),
    lambda: cases.box_case(20, 12, 10, seed=7, ka=0.08),
])
@pytest.mark.parametrize("renumber", [1, 2])
def test_compact_table_is_bit_identical_to_the_full_one(mk, renumber):
    c = mk()
    g = _g()
    s = g.GFM.from_case(c, renumber=renumber)
    s.assemble(torch.as_tensor(c.alpha), torch.as_tensor(c.phi), c.rho_w, c.rho_a, c.g, c.ref_cell, c.ref_value)
    info = s.table_info()
    # rounding of the centre differences splits c_f into a few classes
    assert info["compact_usable"] and info["compact_valid"] and 1 <= info["classes"] <= 64
    (p_ct, i_ct), (p_full, i_full) = _solve_both(s, c)
    assert torch.equal(p_ct, p_full) and i_ct.iters == i_full.iters
    p_ref = oracle.solve(c, direct=c.n <= 4096, rtol=1e-13)[0]
    assert np.linalg.norm(p_ct.cpu().numpy() - p_ref) <= 1e-6 * np.linalg.norm(p_ref)


def test_compact_table_in_a_batch():
    g = _g()
    tanks = cases.batch_cases(6, seed0=4300, nx_range=(40, 120), ny_range=(16, 48))
    b = g.GFMBatch(tanks, renumber=1)
    alpha = torch.as_tensor(np.concatenate([t.alpha for t in tanks]))
    phi = torch.as_tensor(np.concatenate([t.phi for t in tanks]))
    phys = [dict(rho_w=t.rho_w, rho_a=t.rho_a, g=t.g, ref_cell=t.ref_cell, ref_value=t.ref_value) for t in tanks]
    b.assemble(alpha, phi, phys)
    assert b.table_info()["compact_valid"]
    runs = []
    for compact in (True, False):
        b.set_table(compact=compact, force_stream=True)
        p, _, infos = b.solve(rtol=1e-10)
        assert all(i.status == 0 for i in infos)
        runs.append((p.clone(), [i.iters for i in infos]))
    assert torch.equal(runs[0][0], runs[1][0]) and runs[0][1] == runs[1][1]
    pn, c0 = runs[0][0].cpu().numpy(), 0
    for t in tanks:
        p_ref = oracle.solve(t, rtol=1e-13, direct=False)[0]
        assert np.linalg.norm(pn[c0:c0 + t.n] - p_ref) <= 1e-6 * np.linalg.norm(p_ref)
        c0 += t.n


def test_compact_table_stands_aside_with_a_face_coefficient():
    c = cases.box_case(24, 16, 8, seed=2, permute=True)
    g = _g()
    s = g.GFM.from_case(c, renumber=1)
    rau = np.random.default_rng(4).uniform(0.5, 2.0, c.F)
    s.set_rau(torch.as_tensor(rau))
    s.assemble(torch.as_tensor(c.alpha), torch.as_tensor(c.phi), c.rho_w, c.rho_a, c.g, c.ref_cell, c.ref_value)
    assert s.table_info()["compact_usable"] and not s.table_info()["compact_valid"]
    s.set_table(compact=True, force_stream=True)
    p, _, info = s.solve(mode="mixed", rtol=1e-10)
    assert info.status == 0
    p_ref = oracle.cholesky_solve(oracle.assemble(c, oracle.faces(c, rau=rau)))
    assert np.linalg.norm(p.cpu().numpy() - p_ref) <= 1e-6 * np.linalg.norm(p_ref)


def test_compact_table_unusable_with_far_neighbours():
    """A permuted 3D mesh kept in the caller's (random) order: neighbour
    offsets exceed 16 bits, so only the full table exists."""
    c = cases.box_case(48, 40, 40, seed=8, permute=True)
    g = _g()
    s = g.GFM.from_case(c, renumber=0)
    s.assemble(torch.as_tensor(c.alpha), torch.as_tensor(c.phi), c.rho_w, c.rho_a, c.g, c.ref_cell, c.ref_value)
    assert not s.table_info()["compact_usable"] and not s.table_info()["compact_valid"]
    s.set_table(compact=True, force_stream=True)
    p, _, info = s.solve(mode="mixed", rtol=1e-8)
    assert info.status == 0
    sy = oracle.assemble(c, oracle.faces(c))
    r = sy.b - oracle.spmv(sy, p.cpu().numpy())
    assert np.linalg.norm(r) <= 1.05e-8 * np.linalg.norm(sy.b)
