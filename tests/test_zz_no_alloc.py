"""The allocation-free smoother entry point, chebmg_fd_smooth_noalloc.

It serves callers that cannot allocate device memory where they smooth (an application that
owns all device memory through its own pool, or a loop in which cudaMalloc/cudaFree are
forbidden because they may synchronise the device).  Its work vectors live in a static device
array shared by all calls, so these tests check that each call's result is the oracle's
whatever the previous call left in that array, that it agrees with the context smoother, that
the size limit is enforced, and that calls leave the device's free memory unchanged.  This
file is named so that pytest collects it last; it must pass alone in a fresh process too.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import __graft_entry__  # noqa: E402
import workloads as W  # noqa: E402
from oracle.chebyshev import smooth as oracle_smooth  # noqa: E402
from oracle.fd import FdLevel, laplacian_5pt  # noqa: E402

__graft_entry__.build()
import paper_2210_03179_gb300 as cm  # noqa: E402

LMIN_RATIO = 0.1


def _t(a):
    return torch.tensor(np.asarray(a), device="cuda:0", dtype=torch.float64)


def _fine_level(m, Lx=1.0, Ly=1.0):
    L = FdLevel(laplacian_5pt(m, m, Lx / (m + 1), Ly / (m + 1)), m, m)
    L.invD = L.inv_diagonal()
    return L


def _lmax(m):
    # lambda_max of S A for the five-point operator on the unit square: 2 sin^2(m pi / (2 (m+1)))
    return 2.0 * np.sin(m * np.pi / (2.0 * (m + 1))) ** 2


def _two_calls(m, seed):
    """Call 1 from a zero guess, call 2 continuing from a nonzero guess with another b."""
    rng = np.random.default_rng(seed)
    return [(True, W.fd_rhs(m, seed=seed), np.zeros(m * m)),
            (False, W.fd_rhs(m, seed=seed + 1), rng.uniform(-1, 1, m * m))]


@pytest.mark.parametrize("m,kind,order", [(63, "opt4th", 4), (63, "4th", 3), (63, "1st", 5),
                                          (512, "opt4th", 4), (512, "1st", 3)])
def test_noalloc_matches_oracle_on_two_calls(m, kind, order):
    L = _fine_level(m)
    lmax = _lmax(m)
    for x_zero, b, x0 in _two_calls(m, 7):
        ref = oracle_smooth(L, b, order, kind, lmax, LMIN_RATIO, x0=None if x_zero else x0)
        x = _t(x0)
        cm.chebmg_fd_smooth_noalloc(m, 1.0, 1.0, kind, order, lmax, LMIN_RATIO, _t(b), x, x_zero)
        torch.cuda.synchronize()
        got = x.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("kind,order", [("opt4th", 4), ("4th", 3), ("1st", 5)])
def test_noalloc_matches_context_smoother_on_two_calls(kind, order):
    m, Lx, Ly = 63, 1.0, 1.0
    lmax = 1.9953
    s = cm.Solver("fd2d", m=m, Lx=Lx, Ly=Ly, coarsening=2, coarsest=7, kind=kind, order=2,
                  sided="one-sided", lmax=[lmax, 1.3, 1.4])
    for x_zero, b, x0 in _two_calls(m, 3):
        x_ref = _t(x0)
        cm.chebmg_smooth(s.ctx, 0, cm.CHEBMG_F64, _t(b), x_ref, order, x_zero)
        x_new = _t(x0)
        cm.chebmg_fd_smooth_noalloc(m, Lx, Ly, kind, order, lmax, LMIN_RATIO, _t(b), x_new, x_zero)
        torch.cuda.synchronize()
        ref = x_ref.cpu().numpy()
        got = x_new.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    s.close()


def test_noalloc_rejects_sizes_beyond_the_scratch_limit():
    m = 513                                   # 263169 > 262144 unknowns
    b = torch.zeros(m * m, device="cuda:0", dtype=torch.float64)
    x = torch.zeros_like(b)
    with pytest.raises(cm.ChebmgError) as e:
        cm.chebmg_fd_smooth_noalloc(m, 1.0, 1.0, "opt4th", 2, 2.0, LMIN_RATIO, b, x, True)
    assert e.value.code == cm.CHEBMG_EINVAL
    assert "262144" in str(e.value)
    assert float(x.abs().max()) == 0.0        # nothing ran


def test_noalloc_leaves_free_device_memory_unchanged():
    vecs = {m: (_t(W.fd_rhs(m, seed=5)), torch.zeros(m * m, device="cuda:0", dtype=torch.float64))
            for m in (63, 512)}
    b, x = vecs[63]
    cm.chebmg_fd_smooth_noalloc(63, 1.0, 1.0, "opt4th", 4, _lmax(63), LMIN_RATIO, b, x, True)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for m in (512, 63, 512):                  # includes calls at the size limit
        b, x = vecs[m]
        cm.chebmg_fd_smooth_noalloc(m, 1.0, 1.0, "1st", 3, _lmax(m), LMIN_RATIO, b, x, False)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
