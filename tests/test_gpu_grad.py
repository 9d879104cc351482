"""GPU adjoint V-cycle: the gradient of the error-reduction ratio of three cycles with respect
to the 4th-kind weights (k = 4) and the lambda_max scale, against the oracle's forward-mode
gradient and against central finite differences (h = 1e-6) of the GPU's own objective.

Workloads: 16 initial errors e0 (uniform[-1,1]) on the 2-D FD problem 255 x 255 and on SEM
E = 8^3, N = 7 (the oracle comparison on SEM uses a 3 x 4 x 5 mesh; the E = 8^3 case is held
to finite differences), symmetric (4,4) cycles, FP64.
"""
import numpy as np
import pytest

import workloads as W
from oracle import problems as P
from oracle import sensitivity as SE
from oracle.chebyshev import optimized_betas

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2210_03179_gb300 as cm  # noqa: E402
from gpu_util import T  # noqa: E402


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.abs(a - b).max() / np.abs(b).max())


def gpu_fd(s, E0, betas, scale, h=1e-6):
    p = list(betas) + [scale]
    g = []
    for i in range(len(p)):
        pp, pm = list(p), list(p)
        pp[i] += h
        pm[i] -= h
        fp = cm.chebmg_cycle_error_grad(s.ctx, E0, pp[:-1], pp[-1])[0]
        fm = cm.chebmg_cycle_error_grad(s.ctx, E0, pm[:-1], pm[-1])[0]
        g.append((fp - fm) / (2 * h))
    return np.array(g)


@pytest.mark.parametrize("m,kind,betas,scale", [
    (31, "opt4th", None, 1.0),
    (31, "4th", np.ones(4), 1.07),
    (255, "opt4th", None, 1.0),
])
def test_fd_gradient_matches_oracle(m, kind, betas, scale):
    H = P.fd_hierarchy(m, kind=kind, k=4, sided="symmetric")
    b = optimized_betas(4) if betas is None else betas
    s = cm.Solver("fd2d", m=m, kind=kind, order=4, sided="symmetric", lmax=[L.lmax for L in H.levels[:-1]])
    nrhs = 16 if m == 255 else 4
    E0 = W.random_vectors(m * m, nrhs, seed=11)
    f, gb, gs, fe = cm.chebmg_cycle_error_grad(s.ctx, T(E0), b, scale)
    f_ref, g_ref = SE.error_ratio_and_gradient(H, E0, b, scale)
    assert f == pytest.approx(f_ref, rel=1e-10)
    assert rel(gb + [gs], g_ref) < 1e-8
    assert np.mean(fe) == pytest.approx(f, rel=1e-12)
    s.close()


def test_fd_255_gradient_matches_central_differences():
    m = 255
    s = cm.Solver("fd2d", m=m, kind="opt4th", order=4, sided="symmetric")
    E0 = T(W.random_vectors(m * m, 16, seed=0))
    b = list(optimized_betas(4))
    f, gb, gs, _ = cm.chebmg_cycle_error_grad(s.ctx, E0, b, 1.0)
    g_fd = gpu_fd(s, E0, b, 1.0)
    assert rel(gb + [gs], g_fd) < 1e-5
    s.close()


def test_sem_gradient_matches_oracle():
    v = W.sem_box_vertices(3, 4, 5)
    H = P.sem_hierarchy(v, (7, 3, 1), kind="opt4th", k=4, sided="symmetric", coarse_rtol=1e-13)
    s = cm.Solver("sem", verts=v, orders=(7, 3, 1), kind="opt4th", order=4, sided="symmetric",
                  lmax=[L.lmax for L in H.levels[:-1]], coarse_rtol=1e-13)
    live = ~H.levels[0].dirichlet
    E0 = W.random_vectors(H.levels[0].n, 3, seed=2) * live[None, :]
    b = optimized_betas(4)
    f, gb, gs, _ = cm.chebmg_cycle_error_grad(s.ctx, T(E0), b, 1.02)
    f_ref, g_ref = SE.error_ratio_and_gradient(H, E0, b, 1.02)
    assert f == pytest.approx(f_ref, rel=1e-9)
    assert rel(gb + [gs], g_ref) < 1e-7
    s.close()


def test_sem_8cubed_gradient_matches_central_differences():
    ne = 8
    v = W.sem_box_vertices(ne, ne, ne)
    s = cm.Solver("sem", verts=v, orders=(7, 3, 1), kind="opt4th", order=4, sided="symmetric",
                  coarse_rtol=1e-13)
    n = s.size(0)
    mask = W.sem_boundary_mask(ne, ne, ne, 7)
    E0 = T(W.random_vectors(n, 16, seed=0) * ~mask[None, :])
    b = list(optimized_betas(4))
    f, gb, gs, _ = cm.chebmg_cycle_error_grad(s.ctx, E0, b, 1.0)
    assert 0.0 < f < 1e-3
    g_fd = gpu_fd(s, E0, b, 1.0)
    assert rel(gb + [gs], g_fd) < 1e-5
    s.close()


def test_autograd_function_and_adam_from_plain_4th_kind():
    from paper_2210_03179_gb300 import tuning
    m = 63
    s = cm.Solver("fd2d", m=m, kind="4th", order=4, sided="symmetric")
    E0 = T(W.random_vectors(m * m, 8, seed=3))
    betas = torch.ones(4, dtype=torch.float64, requires_grad=True)
    scale = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    f = tuning.error_ratio(s.ctx, E0, betas, scale)
    f.backward()
    f2, gb, gs, _ = cm.chebmg_cycle_error_grad(s.ctx, E0, [1.0] * 4, 1.0)
    assert float(f.detach()) == f2
    assert np.allclose(betas.grad.numpy(), gb) and float(scale.grad) == gs
    b_opt, s_opt, hist = tuning.tune_weights(s.ctx, E0, [1.0] * 4, 1.0, iters=25, lr=0.02)
    assert hist[-1] < 0.8 * hist[0]
    s.close()


def test_set_smoother_weights_changes_the_cycle():
    from oracle import multigrid as M
    m = 31
    H = P.fd_hierarchy(m, kind="4th", k=4, sided="symmetric")
    s = cm.Solver("fd2d", m=m, kind="4th", order=4, sided="symmetric", lmax=[L.lmax for L in H.levels[:-1]])
    w = np.array([1.0, 1.05, 1.2, 1.4])
    cm.chebmg_set_smoother_weights(s.ctx, w, 1.0)
    H.betas = {4: w}
    r = W.fd_rhs(m, seed=2)
    z = torch.zeros(m * m, dtype=torch.float64, device="cuda")
    cm.chebmg_vcycle(s.ctx, T(r), z)
    ref = M.vcycle(H, r)
    assert rel(z.cpu().numpy(), ref) < 1e-12
    cm.chebmg_set_smoother_weights(s.ctx, (), 1.0)   # back to the context's kind
    cm.chebmg_vcycle(s.ctx, T(r), z)
    H.betas = None
    assert rel(z.cpu().numpy(), M.vcycle(H, r)) < 1e-12
    with pytest.raises(cm.ChebmgError):
        cm.chebmg_cycle_error_grad(s.ctx, T(W.random_vectors(m * m, 2, seed=0)), [1.0] * 3, 1.0)
    s.close()
