"""Parity at the full workload sizes.

* E = 32^3, N = 7 (the benchmarked workload, ~11.4M DOFs): the FP64 and FP32 operators
  in the benchmark's launch configuration are checked on sampled nodes, whose values the
  oracle computes from the (at most 8) elements around each node; full solves in both
  precisions must reach the 1e-8 relative residual, measured with the sample-checked
  FP64 operator.
* E = 16^3, N = 7 -> 3 -> 1, optimized 4th kind, one-sided (4,0): the oracle solves the
  whole problem and the iteration counts must agree within one.
* The opt-in FP32-pair outer product at E = 32^3: sampled parity at the FP64 bar and a full
  mixed solve to a true (FP64) 1e-8 residual within one iteration of the FP64 outer product.
"""
import numpy as np
import pytest

import workloads as W
from oracle import krylov as K
from oracle import multigrid as M
from oracle import problems as P
from oracle.sem import SemLevel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2210_03179_gb300 as cm  # noqa: E402
from gpu_util import N, T, empty  # noqa: E402


def touching_elements(nodes, ne, Nn):
    """Elements (ex, ey, ez) -> flat ids that contain the lattice nodes (gx, gy, gz)."""
    out = set()
    for gx, gy, gz in nodes:
        def cand(g):
            c = {min(g // Nn, ne - 1)}
            if g % Nn == 0 and g > 0:
                c.add(g // Nn - 1)
            return c
        for ez in cand(gz):
            for ey in cand(gy):
                for ex in cand(gx):
                    out.add((ez * ne + ey) * ne + ex)
    return sorted(out)


@pytest.fixture(scope="module")
def big():
    ne, Nn = 32, 7
    v = W.sem_box_vertices(ne, ne, ne)
    s = cm.Solver("sem", verts=v, orders=(7, 3, 1), kind="opt4th", order=2, sided="one-sided", prec="mixed")
    yield ne, Nn, v, s
    s.close()


def test_sampled_operator_parity_32cubed(big):
    ne, Nn, v, s = big
    n = s.size(0)
    NX = ne * Nn + 1
    assert n == NX ** 3 == 11390625
    rng = np.random.default_rng(123)
    x = rng.uniform(-1, 1, n)
    gs = np.concatenate([rng.integers(0, n, 150), [0, n - 1, NX * NX * 7 + NX * 14 + 21, (n - 1) // 2]])
    nodes = [(g % NX, (g // NX) % NX, g // (NX * NX)) for g in gs]
    sub = SemLevel(v, Nn, elements=touching_elements(nodes, ne, Nn))
    ref = sub.apply_A(x)[gs]
    scale = np.abs(ref).max()
    y = empty(n)
    cm.chebmg_apply_A(s.ctx, 0, cm.CHEBMG_F64, T(x), y)
    assert np.abs(N(y)[gs] - ref).max() <= 1e-12 * scale
    # the opt-in FP32-pair outer product, in its launch configuration, at the FP64 bar
    cm.chebmg_set_outer_operator(s.ctx, cm.CHEBMG_OUTER_F32X2)
    yx = empty(n)
    cm.chebmg_apply_outer(s.ctx, T(x), yx)
    cm.chebmg_set_outer_operator(s.ctx, cm.CHEBMG_OUTER_FP64)
    assert np.abs(N(yx)[gs] - ref).max() <= 1e-12 * scale
    y32 = empty(n, True)
    x32 = x.astype(np.float32)
    cm.chebmg_apply_A(s.ctx, 0, cm.CHEBMG_F32, T(x32, torch.float32), y32)
    ref32 = sub.apply_A(x32.astype(np.float64))[gs]
    assert np.abs(N(y32)[gs] - ref32).max() <= 2e-5 * scale


def test_full_solves_32cubed(big):
    ne, Nn, v, s = big
    b = W.sem_rhs(ne, ne, ne, Nn)
    bt = T(b)
    u32 = empty(len(b))
    c32, it32, rel32, _ = cm.chebmg_pcg_solve(s.ctx, bt, u32, 1e-8, 300)
    assert c32 == cm.CHEBMG_OK and rel32 <= 1e-8
    s64 = cm.Solver("sem", verts=v, orders=(7, 3, 1), kind="opt4th", order=2, sided="one-sided", prec="fp64",
                    lmax=[s.lambda_max(0), s.lambda_max(1)])
    u64 = empty(len(b))
    c64, it64, rel64, _ = cm.chebmg_pcg_solve(s64.ctx, bt, u64, 1e-8, 300)
    assert c64 == cm.CHEBMG_OK and rel64 <= 1e-8
    assert abs(it32 - it64) <= 1
    cm.chebmg_set_outer_operator(s.ctx, cm.CHEBMG_OUTER_F32X2)
    ux = empty(len(b))
    cx, itx, relx, _ = cm.chebmg_pcg_solve(s.ctx, bt, ux, 1e-8, 300)
    cm.chebmg_set_outer_operator(s.ctx, cm.CHEBMG_OUTER_FP64)
    assert cx == cm.CHEBMG_OK and relx <= 1e-8 and abs(itx - it32) <= 1
    for u in (u32, u64, ux):
        Au = empty(len(b))
        cm.chebmg_apply_A(s64.ctx, 0, cm.CHEBMG_F64, u, Au)
        assert float(torch.linalg.norm(bt - Au) / torch.linalg.norm(bt)) <= 1.01e-8
    s64.close()


def test_iteration_parity_16cubed():
    ne = 16
    v = W.sem_box_vertices(ne, ne, ne)
    H = P.sem_hierarchy(v, (7, 3, 1), kind="opt4th", k=2, sided="one-sided")
    lmax = [L.lmax for L in H.levels[:-1]]
    b = W.sem_rhs(ne, ne, ne, 7)
    x_ref, it_ref, hist_ref = K.fcg(H.levels[0].apply_A, lambda r: M.vcycle(H, r), b, 1e-8)
    s = cm.Solver("sem", verts=v, orders=(7, 3, 1), kind="opt4th", order=2, sided="one-sided", lmax=lmax)
    u = empty(len(b))
    code, it, rel, hist = cm.chebmg_pcg_solve(s.ctx, T(b), u, 1e-8, 200, history=True)
    assert code == cm.CHEBMG_OK and rel <= 1e-8 and abs(it - it_ref) <= 1
    np.testing.assert_allclose(hist[: min(len(hist), len(hist_ref))], hist_ref[: min(len(hist), len(hist_ref))],
                               rtol=1e-5)
    assert np.abs(N(u) - x_ref).max() <= 1e-6 * np.abs(x_ref).max()
    s.close()
    # the mixed form (FP32 smoother, operator and transfers under the FP64 flexible CG) at the same
    # size: the same iteration count within one, the true FP64 residual at 1e-8, and a solution that
    # differs from the oracle's by no more than the 1e-8 residual allows
    sm = cm.Solver("sem", verts=v, orders=(7, 3, 1), kind="opt4th", order=2, sided="one-sided", prec="mixed",
                   lmax=lmax)
    um = empty(len(b))
    code, itm, relm, _ = cm.chebmg_pcg_solve(sm.ctx, T(b), um, 1e-8, 200)
    assert code == cm.CHEBMG_OK and relm <= 1e-8 and abs(itm - it_ref) <= 1, (itm, it_ref)
    A = H.levels[0].apply_A
    assert np.linalg.norm(b - A(N(um))) <= 1.01e-8 * np.linalg.norm(b)
    assert np.abs(N(um) - x_ref).max() <= 1e-6 * np.abs(x_ref).max()
    sm.close()
    s2 = cm.Solver("sem", verts=v, orders=(7, 3, 1), kind="opt4th", order=2, sided="one-sided")
    for j in range(2):
        assert abs(s2.lambda_max(j) / lmax[j] - 1) < 1e-9
    s2.close()
