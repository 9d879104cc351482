"""Writes optimal_betas.json: the optimized 4th-kind weights for smoothing orders the paper's
Table 5 (Sec. 8.1) does not list, computed by the oracle's gamma^{-1} maximisation
(oracle.theory.optimal_betas, which reproduces Table 5 for the orders it lists).  Calls only the
oracle.  Run from the repository root:  python tests/golden/make_optimal_betas.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import theory as T  # noqa: E402

out = {"source": "oracle.theory.optimal_betas: weights of Algorithm 2 maximising gamma^{-1} (Eq. 2.14), "
                 "for the smoothing orders of Table 1 (Sec. 3) beyond Table 5", "orders": {}}
for k in (18, 20):
    betas, gi = T.optimal_betas(k)
    out["orders"][str(k)] = {"betas": [float(b) for b in betas], "gamma_inv": float(gi)}
with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "optimal_betas.json"), "w") as f:
    json.dump(out, f, indent=1)
