"""Jacobi-scaled polynomial smoothers (FP64 oracle).

Test infrastructure only (see ``oracle/__init__``).

* ``chebyshev_1st`` -- Algorithm 1: 1st-kind Chebyshev on [lambda_min, lambda_max]
  of S A, acting on the preconditioned residual r = S (b - A x).
* ``chebyshev_4th`` -- Algorithm 2: 4th-kind Chebyshev (Lottes), acting on the
  unpreconditioned residual; with ``betas`` from the optimized table (Table 5,
  Sec. 8.1) it is the optimized 4th kind.  The beta_i scale only the update of
  x; the residual r keeps tracking the beta = 1 iteration, exactly as printed.
* ``simple`` -- the simple smoothing iteration of Eq. 2.3,
  x <- x + (omega / lambda_max) S (b - A x).

S is the Jacobi smoother diag(A)^{-1} (the "S_j = diag(A_j)^{-1} A_j" of Sec. 2 is
read as S_j = diag(A_j)^{-1} with S_j A_j the smoothed operator), passed as the
vector ``Sdiag``.  ``x0 = None`` means a zero initial guess, in which case the
initial residual costs no operator application.
"""
from __future__ import annotations

import numpy as np

# Optimized 4th-kind coefficients beta_i^{(k)}, k = 1..16 (Table 5, Sec. 8.1).
BETA_TABLE = {
    1: (1.12500000000000,),
    2: (1.02387287570313, 1.26408905371085),
    3: (1.00842544782028, 1.08867839208730, 1.33753125909618),
    4: (1.00391310427285, 1.04035811188593, 1.14863498546254, 1.38268869241000),
    5: (1.00212930146164, 1.02173711549260, 1.07872433192603, 1.19810065292663, 1.41322542791682),
    6: (1.00128517255940, 1.01304293035233, 1.04678215124113, 1.11616489419675, 1.23829020218444, 1.43524297106744),
    7: (1.00083464397912, 1.00843949430122, 1.03008707768713, 1.07408384092003, 1.15036186707366, 1.27116474046139, 1.45186658649364),
    8: (1.00057246631197, 1.00577427662415, 1.02050187922941, 1.05019803444565, 1.10115572984941, 1.18086042806856, 1.29838585382576, 1.46486073151099),
    9: (1.00040960072832, 1.00412439506106, 1.01460212148266, 1.03561113626671, 1.07139972529194, 1.12688273710962, 1.20785219140729, 1.32121930716746, 1.47529642820699),
    10: (1.00030312229652, 1.00304840660796, 1.01077022715387, 1.02619011597640, 1.05231724933755, 1.09255743207549, 1.15083376663972, 1.23172250870894, 1.34060802024460, 1.48386124407011),
    11: (1.00023058595209, 1.00231675024028, 1.00817245396304, 1.01982986566342, 1.03950210235324, 1.06965042700541, 1.11305754295742, 1.17290876275564, 1.25288300576792, 1.35725579919519, 1.49101672564139),
    12: (1.00017947200828, 1.00180189139619, 1.00634861907307, 1.01537864566306, 1.03056942830760, 1.05376019693943, 1.08699862592072, 1.13259183097913, 1.19316273358172, 1.27171293675110, 1.37169337969799, 1.49708418575562),
    13: (1.00014241921559, 1.00142906932629, 1.00503028986298, 1.01216910518495, 1.02414874342792, 1.04238158880820, 1.06842008128700, 1.10399010936759, 1.15102748242645, 1.21171811910125, 1.28854264865128, 1.38432619380991, 1.50229418757368),
    14: (1.00011490538261, 1.00115246376914, 1.00405357333264, 1.00979590573153, 1.01941300472994, 1.03401425035436, 1.05480599606629, 1.08311420301813, 1.12040891660892, 1.16833095655446, 1.22872122288238, 1.30365305707817, 1.39546814053678, 1.50681646209583),
    15: (1.00009404750752, 1.00094291696343, 1.00331449056444, 1.00800294833816, 1.01584236259140, 1.02772083317705, 1.04459535422831, 1.06750761206125, 1.09760092545889, 1.13613855366157, 1.18452361426236, 1.24432087304475, 1.31728069083392, 1.40536543893560, 1.51077872501845),
    16: (1.00007794828179, 1.00078126847253, 1.00274487974401, 1.00662291017015, 1.01309858836971, 1.02289448329337, 1.03678321409983, 1.05559875719896, 1.08024848405560, 1.11172607131497, 1.15112543431072, 1.19965584614973, 1.25865841744946, 1.32962412656664, 1.41421360695576, 1.51427891730346),
}


def optimized_betas(k: int):
    if k not in BETA_TABLE:
        raise ValueError("optimized 4th-kind coefficients are tabulated for k = 1..16 only")
    return np.array(BETA_TABLE[k], dtype=np.float64)


def chebyshev_1st(apply_A, Sdiag, b, k: int, lmax: float, lmin: float, x0=None):
    """Algorithm 1 (1st-kind Chebyshev smoother), order k >= 1."""
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sigma = theta / delta
    rho = 1.0 / sigma
    if x0 is None:
        x = np.zeros_like(b)
        r = Sdiag * b
    else:
        x = x0.copy()
        r = Sdiag * (b - apply_A(x))
    d = r / theta
    for _ in range(1, k):
        x = x + d
        r = r - Sdiag * apply_A(d)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * r
        rho = rho_new
    return x + d


def chebyshev_4th(apply_A, Sdiag, b, k: int, lmax: float, betas=None, x0=None):
    """Algorithm 2 ((optimized) 4th-kind Chebyshev smoother), order k >= 1."""
    betas = np.ones(k) if betas is None else np.asarray(betas, dtype=np.float64)
    if len(betas) != k:
        raise ValueError("need one beta per smoothing step")
    if x0 is None:
        x = np.zeros_like(b)
        r = b.copy()
    else:
        x = x0.copy()
        r = b - apply_A(x)
    d = (4.0 / 3.0) / lmax * (Sdiag * r)
    for i in range(1, k):
        x = x + betas[i - 1] * d
        r = r - apply_A(d)
        d = (2.0 * i - 1.0) / (2.0 * i + 3.0) * d + (8.0 * i + 4.0) / (2.0 * i + 3.0) / lmax * (Sdiag * r)
    return x + betas[k - 1] * d


def simple(apply_A, Sdiag, b, k: int, omega: float, lmax: float, x0=None):
    """k steps of the simple smoothing iteration (Eq. 2.3) with S scaled by 1/lambda_max."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    for _ in range(k):
        x = x + (omega / lmax) * (Sdiag * (b - apply_A(x)))
    return x


def smooth(level, b, order: int, kind: str, lmax: float, lmin_ratio: float = 0.1,
           x0=None, betas=None):
    """Dispatch one smoother application of the given kind and order on ``level``."""
    if order == 0:
        return np.zeros_like(b) if x0 is None else x0.copy()
    S = level.invD
    if kind == "1st":
        return chebyshev_1st(level.apply_A, S, b, order, lmax, lmin_ratio * lmax, x0)
    if kind == "4th":
        return chebyshev_4th(level.apply_A, S, b, order, lmax, betas=betas, x0=x0)
    if kind == "opt4th":
        bt = optimized_betas(order) if betas is None else betas
        return chebyshev_4th(level.apply_A, S, b, order, lmax, betas=bt, x0=x0)
    raise ValueError(f"unknown smoother kind {kind!r}")
