"""The allocation-free smoother entry point against the context-based smoother.

chebmg_fd_smooth_noalloc serves callers that cannot allocate device memory when they
smooth; its work vectors live in a static device array shared by all calls.  This file is
named so that pytest collects it last; it must pass alone in a fresh process too.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import __graft_entry__  # noqa: E402
import workloads as W  # noqa: E402

__graft_entry__.build()
import paper_2210_03179_gb300 as cm  # noqa: E402


def _t(a):
    return torch.tensor(np.asarray(a), device="cuda:0", dtype=torch.float64)


@pytest.mark.parametrize("kind,order", [("opt4th", 4), ("4th", 3), ("1st", 5)])
def test_noalloc_matches_context_smoother_on_two_calls(kind, order):
    m, Lx, Ly = 63, 1.0, 1.0
    lmax = 1.9953
    s = cm.Solver("fd2d", m=m, Lx=Lx, Ly=Ly, coarsening=2, coarsest=7, kind=kind, order=2,
                  sided="one-sided", lmax=[lmax, 1.3, 1.4])
    rng = np.random.default_rng(31)
    n = m * m
    # call 1 from a zero guess, call 2 continuing from a nonzero guess
    for x_zero, b, x0 in [(True, W.fd_rhs(m, seed=3), np.zeros(n)),
                          (False, W.fd_rhs(m, seed=4), rng.uniform(-1, 1, n))]:
        x_ref = _t(x0)
        cm.chebmg_smooth(s.ctx, 0, cm.CHEBMG_F64, _t(b), x_ref, order, x_zero)
        x_new = _t(x0)
        cm.chebmg_fd_smooth_noalloc(m, Lx, Ly, kind, order, lmax, 0.1, _t(b), x_new, x_zero)
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
        cm.chebmg_fd_smooth_noalloc(m, 1.0, 1.0, "opt4th", 2, 2.0, 0.1, b, x, True)
    assert e.value.code == cm.CHEBMG_EINVAL
    assert "262144" in str(e.value)
    m = 512                                   # exactly at the limit works
    b = _t(W.fd_rhs(m))
    x = torch.zeros_like(b)
    cm.chebmg_fd_smooth_noalloc(m, 1.0, 1.0, "opt4th", 2, 2.0, 0.1, b, x, True)
    torch.cuda.synchronize()
    assert torch.isfinite(x).all() and float(x.abs().max()) > 0
