#!/usr/bin/env python3
"""Benchmark: time-to-1e-8 residual and smoother GDOF/s, SEM E=32^3 N=7, mixed vs FP64.

Workload: the 3-D spectral-element Poisson problem on the perturbed unit box
(E = 32^3 trilinear hexahedra, N = 7, n = 11,390,625 global DOFs), p-multigrid
7 -> 3 -> 1 with the optimized 4th-kind Chebyshev smoother in the one-sided
(6, 0) V-cycle (k = 3), flexible CG to a 1e-8 relative residual, uniform[-1,1]
right-hand side (seed 1).  One "step" is one complete solve.  Other smoothing orders,
cycle shapes, schedules and kinds at the same size are reported under "schedules".

value      = whole-job solve throughput: n * solves / seconds / 1e9 (GDOF/s solved to 1e-8)
             for the mixed form (FP32 smoother/Ax/transfers, FP64 Krylov, Lanczos and coarse CG),
             inputs resident in HBM.  time_to_1e8_s gives seconds per solve for both forms.
e2e        = the same metric through chebmg_pcg_solve_host with pinned host b and u
             (H2D of b and D2H of u inside the timed region).
roofline   = the fine-level Chebyshev smoother step (element Ax + gather-scatter + recurrence),
             algorithmic bytes w (6 L + 7 n) per step, against the measured HBM copy bandwidth.
cpu_baseline / --impl reference = the FP64 oracle (numpy, single thread) solving the same
             recipe at E = 16^3 (a bounded sample), in the same unit.

Replicas only: with N GPUs every rank solves its own copy (weak scaling, no collective on
the data path); the timed region is bracketed by barriers and the max over ranks is used.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# one-sided (2k,0) cycles with k in {1, 2, 3} are the family the E = 16^3 configuration names; at
# E = 32^3 on GB300, k = 3 takes the least time in it (FP32 smoothing is cheap next to the FP64
# outer operator and coarse solve that each extra iteration costs); the sweep is reported too
NE, NORDER, ORDERS, KIND, K_ORDER, SIDED = 32, 7, (7, 3, 1), "opt4th", 3, "one-sided"
RTOL = 1e-8
SAMPLE_NE = 16
METRIC = "time-to-1e-8 residual and smoother GDOF/s, SEM E=32^3 N=7, mixed vs FP64"
UNIT = "GDOF/s (DOFs solved to 1e-8 rel. residual per second)"


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def recorded_traffic(variant):
    """DRAM bytes per fine step of the order-7 operator variant `variant` from
    profiles/roofline_traffic.json, or None if that variant was not captured or the kernels that
    make up the step changed since the counters were taken."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "roofline_traffic.json")))
        h = hashlib.sha256()
        for f in rec["source_files"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        if h.hexdigest() != rec["source_sha256"]:
            return None
        return rec["variants"][str(variant)]["traffic_bytes_per_step"]
    except Exception:
        return None


def config(extra=None):
    c = {"workload": f"SEM Poisson E={NE}^3 N={NORDER}, p-MG {ORDERS}, {KIND} Chebyshev one-sided "
                     f"({2 * K_ORDER},0), FCG to 1e-8",
         "E": NE ** 3, "N": NORDER, "n_dof": (NE * NORDER + 1) ** 3, "orders": list(ORDERS),
         "smoother": KIND, "k": K_ORDER, "sided": SIDED, "rtol": RTOL,
         "l2": "inputs larger than L2 (FP32+FP64 geometric factors 1.2 GB, vectors 91 MB each)"}
    if extra:
        c.update(extra)
    return c


# ---------------------------------------------------------------------------
# CPU oracle sample (reference arm and cpu_baseline): one FP64 solve at E=16^3
# ---------------------------------------------------------------------------
ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, %(root)r)
import workloads as W
from oracle import krylov as K, multigrid as M, problems as P
ne = %(ne)d
v = W.sem_box_vertices(ne, ne, ne)
H = P.sem_hierarchy(v, %(orders)r, kind=%(kind)r, k=%(k)d, sided=%(sided)r)
b = W.sem_rhs(ne, ne, ne, %(N)d)
times = []
for _ in range(%(reps)d):
    t = time.perf_counter()
    x, it, hist = K.fcg(H.levels[0].apply_A, lambda r: M.vcycle(H, r), b, %(rtol)r)
    times.append(time.perf_counter() - t)
if %(save)r:
    import numpy as np
    np.save(%(save)r, x)
print(json.dumps({"n": H.levels[0].n, "iters": it, "times": times}))
"""


def run_oracle(reps: int, save: str = ""):
    """Time `reps` oracle solves of the E=16^3 sample in a one-thread subprocess; with `save`,
    the last solution is written there (numpy .npy) for the error of the GPU results."""
    code = ORACLE_SNIPPET % dict(root=ROOT, ne=SAMPLE_NE, orders=ORDERS, kind=KIND, k=K_ORDER, sided=SIDED,
                                 N=NORDER, rtol=RTOL, reps=reps, save=save)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def run_oracle_all_cores():
    """One oracle solve per host core, all at once (independent processes, one thread each):
    the host's whole-machine oracle throughput.  Returns (total DOFs, wall seconds, cores)."""
    cores = len(os.sched_getaffinity(0))
    code = ORACLE_SNIPPET % dict(root=ROOT, ne=SAMPLE_NE, orders=ORDERS, kind=KIND, k=K_ORDER, sided=SIDED,
                                 N=NORDER, rtol=RTOL, reps=1, save="")
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    t0 = time.perf_counter()
    procs = [subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                              stderr=subprocess.DEVNULL, text=True) for _ in range(cores)]
    outs = [p.communicate()[0] for p in procs]
    wall = time.perf_counter() - t0
    n = sum(json.loads(o.strip().splitlines()[-1])["n"] for o in outs)
    return n, wall, cores


def sample_desc(r):
    return (f"FP64 numpy oracle, one thread, full FCG solve of the same recipe at E={SAMPLE_NE}^3 "
            f"(n={r['n']}, {r['iters']} iterations), setup excluded")


def sample_config(r):
    """The configuration the oracle sample actually solves: the benchmark's recipe and cycle at
    E = 16^3 (the rate is per DOF, so it compares with the E = 32^3 GPU rate)."""
    return {"workload": f"SEM Poisson E={SAMPLE_NE}^3 N={NORDER}, p-MG {ORDERS}, {KIND} Chebyshev one-sided "
                        f"({2 * K_ORDER},0), FCG to 1e-8 (bounded sample of the E={NE}^3 workload)",
            "E": SAMPLE_NE ** 3, "N": NORDER, "n_dof": r["n"], "orders": list(ORDERS), "smoother": KIND,
            "k": K_ORDER, "sided": SIDED, "rtol": RTOL, "iterations": r["iters"],
            "sample_of": {"E": NE ** 3, "n_dof": (NE * NORDER + 1) ** 3}}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    """nvidia-smi samples every 100 ms.  The sampler is started and its first row awaited before
    the timed region opens (mark()), and only rows written after the mark are kept; a timed
    region shorter than one interval keeps the last row before it and says so."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.start_row = 0
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        t0 = time.time()
        while self.p is not None and not self._rows() and time.time() - t0 < 10 and self.p.poll() is None:
            time.sleep(0.02)

    def _rows(self):
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        return rows

    def mark(self):
        """Called just before the timed region: rows so far were taken before it."""
        self.start_row = len(self._rows()) if self.p is not None else 0

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        all_rows = self._rows()
        os.unlink(self.f.name)
        rows = all_rows[self.start_row:]
        before = False
        if not rows and all_rows:
            rows, before = all_rows[-1:], True
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        out = {"sm_mhz": sm[len(sm) // 2] if sm else None,
               "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
               "reasons": reasons, "samples": len(rows), "interval_ms": 100}
        if before:
            out["note"] = "timed region shorter than one interval: the last sample before it"
        return out


# ---------------------------------------------------------------------------
# ---------------------------------------------------------------------------
# Replicas (N > 1): every rank solves its own copy; the slowest rank sets the job time
# ---------------------------------------------------------------------------
def max_over_ranks(x, dist=None, device="cpu"):
    """The largest of the ranks' values of x (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, dofs_per_rank, seconds):
    """Whole-job GDOF/s: every rank solved dofs_per_rank unknowns; seconds is the max over ranks."""
    return world * dofs_per_rank / seconds / 1e9


BATCH_NE, BATCH_NRHS = 8, 64
UNEVEN = [(ne, Nn) for ne in (4, 6, 8, 12) for Nn in (5, 7, 9)]


# Shared-memory bytes per point and right-hand side of the batched FP32 order-7 operator, counted
# from the kernel source (4-byte words): staging the gathered column 4, the forward r and s
# passes 8 + 8, the factor multiply (two derivatives read and written, six factors read) 40, the
# transposed r and s passes 8 + 12, the scatter read 4 = 84 with the factors staged in shared
# memory; 60 with them in registers (the six factor reads go); 72 taking the right-hand sides in
# pairs (each factor read serves two).  Keyed by the variant's form, (variant % 100) // 10.
BATCHED_SHARED_BYTES = {0: 84, 1: 72, 2: 60}
BATCHED_FORMS = {0: "k_sem_ax8b (factors staged in shared memory once per block)",
                 1: "k_sem_ax8b2 (right-hand sides in pairs through each line pass)",
                 2: "k_sem_ax8bg (factors in registers across the block's right-hand sides)"}


def bench_batched(cm, W, torch, timed, reps, sm_mhz=None):
    """64 right-hand sides on E = 8^3, N = 7 in one batched solve, and the uneven group of meshes
    E in {4^3, 6^3, 8^3, 12^3} x N in {5, 7, 9} (one right-hand side each) in one grouped solve,
    each against the same problems solved one after another by the single-right-hand-side
    FP64 and mixed forms.  Times are seconds for the whole set, inputs resident in HBM."""
    import numpy as np
    common = dict(orders=ORDERS, kind=KIND, order=K_ORDER, sided=SIDED)
    v = W.sem_box_vertices(BATCH_NE, BATCH_NE, BATCH_NE)
    s32 = cm.Solver("sem", verts=v, prec="mixed", **common)
    lmax = [s32.lambda_max(j) for j in range(len(ORDERS) - 1)]
    s64 = cm.Solver("sem", verts=v, prec="fp64", lmax=lmax, **common)
    n = s32.size(0)
    B = torch.tensor(np.stack([W.sem_rhs(BATCH_NE, BATCH_NE, BATCH_NE, NORDER, seed=q)
                               for q in range(BATCH_NRHS)]), device="cuda")
    U = torch.zeros_like(B)
    u = torch.zeros(n, dtype=torch.float64, device="cuda")

    def batched(s, graph):
        code, its, rel = cm.chebmg_pcg_solve_batched(s.ctx, B, U, RTOL, 500, graph=graph)
        assert code == cm.CHEBMG_OK and max(rel) <= RTOL, (code, max(rel))
        return its

    def sequential(s):
        its = []
        for q in range(BATCH_NRHS):
            code, it, rel, _ = cm.chebmg_pcg_solve(s.ctx, B[q], u, RTOL, 500)
            assert code == cm.CHEBMG_OK and rel <= RTOL
            its.append(it)
        return its

    out = {"workload": f"{BATCH_NRHS} RHS (seeds 0..{BATCH_NRHS - 1}) on SEM E={BATCH_NE}^3 N={NORDER}, "
                       f"p-MG {ORDERS}, {KIND} one-sided ({2 * K_ORDER},0), FCG to 1e-8",
           "n_dof_per_rhs": n, "time_s": {}}
    for name, fn in [("batched_mixed_graph", lambda: batched(s32, True)),
                     ("batched_mixed_eager", lambda: batched(s32, False)),
                     ("batched_fp64_graph", lambda: batched(s64, True)),
                     ("sequential_mixed", lambda: sequential(s32)),
                     ("sequential_fp64", lambda: sequential(s64))]:
        fn()
        l0 = cm.chebmg_launch_count()
        t, its = timed(fn, reps)
        out["time_s"][name] = t
        if name == "batched_mixed_graph":
            out["iterations"] = {"min": min(its), "max": max(its)}
            out["gpu_launches"] = (cm.chebmg_launch_count() - l0) // reps
    # opt-in: the outer products in FP64-class arithmetic on FP32 pairs
    cm.chebmg_set_outer_operator(s32.ctx, cm.CHEBMG_OUTER_F32X2)
    batched(s32, True)
    out["time_s"]["batched_mixed_graph_f32x2_outer"], _ = timed(lambda: batched(s32, True), reps)
    cm.chebmg_set_outer_operator(s32.ctx, cm.CHEBMG_OUTER_FP64)
    tb = out["time_s"]["batched_mixed_graph"]
    out["gdofs_batched_mixed_graph"] = BATCH_NRHS * n / tb / 1e9
    out["speedup_vs_sequential_fp64"] = out["time_s"]["sequential_fp64"] / tb
    out["speedup_vs_sequential_mixed"] = out["time_s"]["sequential_mixed"] / tb
    out["ax8_batched_variant"] = {"fp32": cm.chebmg_batch_info(s32.ctx, BATCH_NRHS, 0, cm.CHEBMG_F32)[0],
                                  "fp64": cm.chebmg_batch_info(s64.ctx, BATCH_NRHS, 0, cm.CHEBMG_F64)[0]}
    out["coarse_degree"] = cm.chebmg_batch_info(s32.ctx, BATCH_NRHS, 0, cm.CHEBMG_F32)[1]
    # batched FP32 order-7 operator: G read once for all right-hand sides
    X32 = torch.rand((BATCH_NRHS, n), dtype=torch.float32, device="cuda")
    Y32 = torch.zeros_like(X32)
    cm.chebmg_apply_A_batched(s32.ctx, 0, cm.CHEBMG_F32, X32, Y32)
    t_ax, _ = timed(lambda: cm.chebmg_apply_A_batched(s32.ctx, 0, cm.CHEBMG_F32, X32, Y32), 10)
    t_zero, _ = timed(lambda: Y32.zero_(), 10)      # apply_A_batched zeroes Y first: take that out
    t_k = max(t_ax - t_zero, 1e-9)
    Lb = BATCH_NE ** 3 * (NORDER + 1) ** 3
    alg = 4 * (6 * Lb + 2 * BATCH_NRHS * n)
    hbm = peaks().get("hbm_gbs") or 6800.0
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = sm_mhz or peaks().get("sm_max_mhz") or 2070.0
    form = (out["ax8_batched_variant"]["fp32"] % 100) // 10
    shb = BATCHED_SHARED_BYTES[form] * Lb * BATCH_NRHS
    shared_peak = 128 * sms * mhz * 1e6 / 1e9          # 32 banks x 4 bytes per SM per clock
    # executed FP32 instructions per point and right-hand side: six line passes of 48 per
    # 8-point line (8 even-odd sums, 32 chain FMAs, 8 recombinations) = 36, the factors 9, the
    # two transposed-contribution additions 2
    fp32_instr = 47 * Lb * BATCH_NRHS
    fp32_peak = 128 * sms * mhz * 1e6 / 1e9           # G instructions/s: 128 FP32 lanes per SM
    out["roofline_batched_operator"] = {
        "bound": "shared", "kernel": BATCHED_FORMS[form], "variant": out["ax8_batched_variant"]["fp32"],
        "time_us": t_k * 1e6, "time_with_zeroing_us": t_ax * 1e6,
        "shared_bytes": shb, "shared_bytes_per_point": BATCHED_SHARED_BYTES[form],
        "achieved": shb / t_k / 1e9, "peak": shared_peak, "unit": "GB/s", "frac": shb / t_k / 1e9 / shared_peak,
        "peak_source": f"unit count: 128 bytes / SM / clock x {sms} SMs x {mhz:.0f} MHz",
        "hbm": {"alg_bytes": alg, "achieved": alg / t_k / 1e9, "peak": hbm, "frac": alg / t_k / 1e9 / hbm,
                "peak_source": "of measured" if peaks().get("hbm_gbs") else "of fallback"},
        "fp32_pipe": {"instructions": fp32_instr, "achieved": fp32_instr / t_k / 1e9, "peak": fp32_peak,
                      "unit": "G instructions/s", "frac": fp32_instr / t_k / 1e9 / fp32_peak}}
    del X32, Y32
    s32.close()
    s64.close()

    # ---- uneven group of meshes ----
    g32, g64, bs, us = [], [], [], []
    for k, (ne, Nn) in enumerate(UNEVEN):
        vv = W.sem_box_vertices(ne, ne, ne)
        a = cm.Solver("sem", verts=vv, prec="mixed", **dict(common, orders=(Nn, 3, 1)))
        lm = [a.lambda_max(j) for j in range(2)]
        g32.append(a)
        g64.append(cm.Solver("sem", verts=vv, prec="fp64", lmax=lm, **dict(common, orders=(Nn, 3, 1))))
        bs.append(torch.tensor(W.sem_rhs(ne, ne, ne, Nn, seed=k), device="cuda"))
        us.append(torch.zeros_like(bs[-1]))
    ctxs = [a.ctx for a in g32]
    grp = cm.chebmg_group_create(ctxs)

    def group(graph):
        code, its, rel = cm.chebmg_group_pcg_solve(grp, ctxs, bs, us, RTOL, 500, graph=graph)
        assert code == cm.CHEBMG_OK and max(rel) <= RTOL
        return its

    def seq(solvers):
        its = []
        for a, bb, uu in zip(solvers, bs, us):
            code, it, rel, _ = cm.chebmg_pcg_solve(a.ctx, bb, uu, RTOL, 500)
            assert code == cm.CHEBMG_OK and rel <= RTOL
            its.append(it)
        return its

    un = {"workload": "one RHS each on SEM E in {4,6,8,12}^3 x N in {5,7,9}, p-MG (N,3,1), "
                      f"{KIND} one-sided ({2 * K_ORDER},0), FCG to 1e-8",
          "n_dof_total": int(sum(bb.numel() for bb in bs)), "time_s": {}}
    for name, fn in [("group_mixed_graph", lambda: group(True)), ("group_mixed_eager", lambda: group(False)),
                     ("sequential_mixed", lambda: seq(g32)), ("sequential_fp64", lambda: seq(g64))]:
        fn()
        t, _ = timed(fn, reps)
        un["time_s"][name] = t
    un["speedup_vs_sequential_fp64"] = un["time_s"]["sequential_fp64"] / un["time_s"]["group_mixed_graph"]
    un["speedup_vs_sequential_mixed"] = un["time_s"]["sequential_mixed"] / un["time_s"]["group_mixed_graph"]
    cm.chebmg_group_destroy(grp)
    for a in g32 + g64:
        a.close()
    out["uneven"] = un
    return out


# Table 1 (Sec. 3): configuration with the fewest fine mat-vecs per row, GMRES(20) to 1e-6, n = 128
TABLE1 = [  # Lx, coarsening, complexity, kind, m, n, matvecs, iterations (printed)
    (1, 2, 1.568, "4th", 2, 2, 20, 4), (8, 2, 1.568, "4th", 14, 0, 75, 5),
    (64, 2, 1.568, "opt4th", 20, 0, 252, 12), (128, 2, 1.568, "opt4th", 20, 0, 252, 12),
    (1, 8, 1.023, "4th", 7, 7, 60, 4), (8, 8, 1.023, "opt4th", 14, 0, 195, 13),
    (64, 8, 1.023, "opt4th", 18, 0, 323, 17), (128, 8, 1.023, "opt4th", 20, 0, 294, 14)]


def table1_weights():
    """Optimized 4th-kind weights for the smoothing orders 18 and 20 of Table 1, which Table 5
    does not list: the gamma^{-1}-maximising weights stored beside the tests (computed once from
    Eq. 2.14; they reproduce Table 5 for the orders it lists)."""
    rec = json.load(open(os.path.join(ROOT, "tests", "golden", "optimal_betas.json")))
    return {int(k): v["betas"] for k, v in rec["orders"].items()}


def true_relres(cm, torch, s, b, u):
    """||b - A u|| / ||b|| with the FP64 operator of the finest level (held to the oracle at 1e-12)."""
    y = torch.zeros_like(b)
    cm.chebmg_apply_A(s.ctx, 0, cm.CHEBMG_F64, u, y)
    return float(torch.linalg.norm(b - y) / torch.linalg.norm(b))


def errors_against_oracle(cm, W, torch, np, x_ref, it_ref):
    """The mixed and FP64 GPU solutions of the E = 16^3 sample against the oracle's FCG solution of
    the same problem: iterations, max-norm relative error and the true FP64 relative residual."""
    ne = SAMPLE_NE
    v = W.sem_box_vertices(ne, ne, ne)
    b = torch.tensor(W.sem_rhs(ne, ne, ne, NORDER), device="cuda")
    out = {"workload": f"E={ne}^3 N={NORDER}, the benchmark's recipe and cycle", "oracle_iterations": it_ref}
    xr = torch.tensor(x_ref, device="cuda")
    lmax = None
    for prec in ("mixed", "fp64"):
        s = cm.Solver("sem", verts=v, orders=ORDERS, kind=KIND, order=K_ORDER, sided=SIDED, prec=prec, lmax=lmax)
        if lmax is None:
            lmax = [s.lambda_max(j) for j in range(len(ORDERS) - 1)]
        u = torch.zeros_like(b)
        code, it, rel, _ = cm.chebmg_pcg_solve(s.ctx, b, u, RTOL, 500)
        out[prec] = {"status": code, "iterations": it, "recursive_relres": rel,
                     "true_relres": true_relres(cm, torch, s, b, u),
                     "max_rel_error_vs_oracle": float((u - xr).abs().max() / xr.abs().max())}
        s.close()
    return out


def bench_fd_table1(cm, torch, timed, reps):
    """The paper's FD study on the GPU: all eight Table 1 rows, with the GPU's own Lanczos
    lambda_max, u = sin(3 pi x / Lx) sin(4 pi y) + g (g uniform[-1,1], seed 0), b = A u.  Rows
    whose smoothing order is above 16 (beyond Table 5) run the optimized 4th kind with the
    gamma^{-1}-maximising weights of that order, set through chebmg_set_smoother_weights."""
    import numpy as np
    betas = table1_weights()
    out = []
    for Lx, c, cx, kind, m, nn, mv, its in TABLE1:
        row = {"Lx": Lx, "coarsening": c, "kind": kind, "m": m, "n": nn,
               "paper": {"iterations": its, "matvecs": mv, "grid_complexity": cx}}
        k, sided = (m // 2, "one-sided") if nn == 0 else (m, "symmetric")
        order = m + nn
        s = cm.Solver("fd2d", m=127, Lx=float(Lx), Ly=1.0, coarsening=c, coarsest=1,
                      kind=kind if order <= 16 else "4th", order=k, sided=sided)
        if order > 16:
            cm.chebmg_set_smoother_weights(s.ctx, betas[order], 1.0)
            row["weights"] = f"gamma^-1-optimal weights of order {order} (Table 5 stops at 16)"
        sizes = [int(round(s.size(j) ** 0.5)) for j in range(s.num_levels)]
        nnz = [5 * sizes[0] ** 2 - 4 * sizes[0]] + [(3 * q - 2) ** 2 for q in sizes[1:]]
        x = np.arange(1, 128) * (Lx / 128.0)
        y = np.arange(1, 128) / 128.0
        X, Y = np.meshgrid(x, y)
        ue = (np.sin(3 * np.pi * X / Lx) * np.sin(4 * np.pi * Y)).ravel() + \
            np.random.default_rng(0).uniform(-1, 1, 127 * 127)
        b = torch.zeros(127 * 127, dtype=torch.float64, device="cuda")
        cm.chebmg_apply_A(s.ctx, 0, cm.CHEBMG_F64, torch.tensor(ue, device="cuda"), b)
        u = torch.zeros_like(b)

        def solve():
            code, it, rel, _ = cm.chebmg_gmres_solve(s.ctx, b, u, 1e-6, 20, 500)
            assert code == cm.CHEBMG_OK
            return it
        solve()
        t, it = timed(solve, reps)
        row.update({"levels": sizes, "grid_complexity": sum(nnz) / nnz[0], "iterations": it,
                    "matvecs": it * (m + nn + 1), "time_to_1e6_ms": t * 1e3})
        s.close()
        out.append(row)
    return out


def bench_schedules(cm, W, torch, timed, reps, verts, b):
    """Solves at the benchmark size (E = 32^3, N = 7, mixed form, FCG to 1e-8): the smoothing
    order and cycle shape (one-sided (2k,0) and symmetric (k,k)), the p-MG schedule
    7 -> 5 -> 3 -> 1 beside 7 -> 3 -> 1, and the smoother kind (4th, optimized 4th, 1st kind at
    lambda_min = 0.1 lambda_max and at the gamma^{-1}-optimal lambda_min)."""
    u = torch.zeros_like(b)
    out = {}
    cases = []
    # smoothing order and cycle shape (the paper's question), opt-4th, 7-3-1
    for k in (1, 2, 3, 4):
        cases.append((f"opt4th one-sided ({2 * k},0) (7,3,1)", dict(orders=(7, 3, 1), kind="opt4th", order=k)))
    for k in (2, 3, 4):
        cases.append((f"opt4th symmetric ({k},{k}) (7,3,1)",
                      dict(orders=(7, 3, 1), kind="opt4th", order=k, sided="symmetric")))
    cases += [("opt4th one-sided (6,0) (7,5,3,1)", dict(orders=(7, 5, 3, 1), kind="opt4th", order=3)),
              ("opt4th symmetric (3,3) (7,5,3,1)", dict(orders=(7, 5, 3, 1), kind="opt4th", order=3,
                                                         sided="symmetric")),
              ("4th kind one-sided (6,0) (7,3,1)", dict(orders=(7, 3, 1), kind="4th", order=3)),
              ("1st kind lmin=0.1 one-sided (6,0) (7,3,1)", dict(orders=(7, 3, 1), kind="1st", order=3,
                                                                  lmin_ratio=0.1)),
              ("1st kind lmin optimal one-sided (6,0) (7,3,1)", dict(orders=(7, 3, 1), kind="1st", order=3,
                                                                      lmin_ratio=0.0))]
    for name, kw in cases:
        kw = dict(kw)
        kw.setdefault("order", K_ORDER)
        kw.setdefault("sided", SIDED)
        s = cm.Solver("sem", verts=verts, prec="mixed", **kw)

        def solve():
            code, it, rel, _ = cm.chebmg_pcg_solve(s.ctx, b, u, RTOL, 500)
            assert code == cm.CHEBMG_OK and rel <= RTOL
            return it
        solve()
        t, it = timed(solve, reps)
        rec = {"time_to_1e8_s": t, "iterations": it}
        if kw["kind"] == "1st":
            rec["lmin_ratio"] = cm.chebmg_lambda_min_ratio(s.ctx, 2 * kw["order"])
        out[name] = rec
        s.close()
    return out


DIFF_NRHS, DIFF_ADAM_STEPS = 16, 200


def bench_differentiation(cm, W, torch, timed, reps):
    """Gradient of mean ||(I - B A)^3 e0||^2 / ||e0||^2 over 16 e0 with respect to the k = 4
    weights and the lambda_max scale (symmetric (4,4) cycles, FP64 adjoint on the GPU) on
    FD 255 x 255 and SEM E = 8^3, N = 7: time per objective, per gradient and per central-
    difference gradient, and 200 Adam steps from the plain 4th kind beside the paper's
    optimized weights (Table 5)."""
    import numpy as np
    from paper_2210_03179_gb300 import tuning
    table4 = [1.00391310427285, 1.04035811188593, 1.14863498546254, 1.38268869241000]
    cases = []
    fd = cm.Solver("fd2d", m=255, kind="4th", order=4, sided="symmetric")
    cases.append(("FD 255x255, 6 levels to 7x7", fd, torch.tensor(W.random_vectors(255 * 255, DIFF_NRHS, 0),
                                                                    device="cuda")))
    v = W.sem_box_vertices(BATCH_NE, BATCH_NE, BATCH_NE)
    sem = cm.Solver("sem", verts=v, orders=ORDERS, kind="4th", order=4, sided="symmetric")
    mask = W.sem_boundary_mask(BATCH_NE, BATCH_NE, BATCH_NE, NORDER)
    cases.append((f"SEM E={BATCH_NE}^3 N={NORDER}, p-MG {ORDERS}", sem,
                  torch.tensor(W.random_vectors(sem.size(0), DIFF_NRHS, 0) * ~mask[None, :], device="cuda")))
    out = []
    for name, s, E0 in cases:
        ones = [1.0] * 4
        cm.chebmg_cycle_error_grad(s.ctx, E0, ones, 1.0)
        t_obj, _ = timed(lambda: cm.chebmg_cycle_error(s.ctx, E0, ones, 1.0), reps)
        t_grad, _ = timed(lambda: cm.chebmg_cycle_error_grad(s.ctx, E0, ones, 1.0), reps)
        f_plain = cm.chebmg_cycle_error(s.ctx, E0, ones, 1.0)[0]
        f_table = cm.chebmg_cycle_error(s.ctx, E0, table4, 1.0)[0]
        b_t, s_t, hist = tuning.tune_weights(s.ctx, E0, ones, 1.0, iters=DIFF_ADAM_STEPS, lr=0.01)
        f_tuned = cm.chebmg_cycle_error(s.ctx, E0, b_t.tolist(), s_t)[0]
        b_w, s_w, _ = tuning.tune_weights(s.ctx, E0, ones, 1.0, iters=DIFF_ADAM_STEPS, lr=0.01, tune_scale=False)
        f_tuned_w = cm.chebmg_cycle_error(s.ctx, E0, b_w.tolist(), 1.0)[0]
        out.append({"workload": name + f", symmetric (4,4), {DIFF_NRHS} e0, 3 cycles",
                    "n_dof": s.size(0), "objective_ms": t_obj * 1e3, "gradient_ms": t_grad * 1e3,
                    "central_difference_gradient_ms": 2 * 5 * t_obj * 1e3,
                    "f": {"plain_4th_kind": f_plain, "paper_optimized_table5": f_table,
                          "adam_weights_only": f_tuned_w, "adam_weights_and_scale": f_tuned},
                    "weights": {"paper_table5": table4, "adam_weights_only": [float(x) for x in b_w],
                                "adam_weights_and_scale": [float(x) for x in b_t], "adam_scale": s_t},
                    "adam_steps": DIFF_ADAM_STEPS})
    fd.close()
    sem.close()
    return out


def main():
    global NE
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 20; 5 for --impl reference, whose steps are oracle solves)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-all-cores", action="store_true", help="skip the all-cores oracle throughput")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched / grouped measurements")
    ap.add_argument("--profile-batched", action="store_true",
                    help="set up the 64-RHS E=8^3 batch, warm up, run one batched solve (kernels launched "
                         "one by one) inside the NVTX range 'bsolve' and exit")
    ap.add_argument("--no-diff", action="store_true", help="skip the gradient / weight-tuning measurements")
    ap.add_argument("--no-table1", action="store_true", help="skip the FD study of Table 1")
    ap.add_argument("--no-schedules", action="store_true",
                    help="skip the 7-5-3-1 schedule and optimal-lambda_min solves at E=32^3")
    ap.add_argument("--schedules-only", action="store_true",
                    help="only the 7-5-3-1 schedule and optimal-lambda_min solves at E=32^3")
    ap.add_argument("--table1-only", action="store_true", help="only the FD study of Table 1")
    ap.add_argument("--diff-only", action="store_true",
                    help="only the gradient / weight-tuning measurements (printed as one JSON object)")
    ap.add_argument("--batched-only", action="store_true",
                    help="only the batched / grouped measurements (printed as one JSON object)")
    ap.add_argument("--ne", type=int, default=NE,
                    help="elements per direction (profiling runs only; the benchmark uses 32)")
    ap.add_argument("--profile-smoother", choices=["mixed", "fp64"], default=None,
                    help="set up, then run one order-9 fine-level smoother application inside the NVTX "
                         "range 'smooth' and exit")
    ap.add_argument("--tile", type=int, default=None,
                    help="profiling runs only: force this order-7 kernel variant on the fine level")
    ap.add_argument("--fused", action="store_true",
                    help="profiling runs only (--profile-smoother): force the fused smoother kernel on the fine level")
    ap.add_argument("--profile-outer", choices=["fp64", "f32x2"], default=None,
                    help="apply only the outer operator (FP64 or FP32 pairs) twice, the second inside an "
                         "NVTX range 'outer' (for ncu)")
    ap.add_argument("--pin-tiles", default=None,
                    help="profiling runs only (--profile-solve): JSON {\"level,dtype\": variant} of operator "
                         "variants to set after setup (the autotuner's timings are distorted under a profiler); "
                         "the run prints the variants it used")
    ap.add_argument("--profile-solve", choices=["mixed", "fp64"], default=None,
                    help="set up, warm up, run one solve inside the NVTX range 'solve' and exit "
                         "(for ncu --nvtx-include solve/)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 5 if args.impl == "reference" else 20

    if args.profile_solve or args.profile_smoother or args.profile_outer:
        NE = args.ne
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return 0
        r = run_oracle(args.warmup + args.steps)
        ts = r["times"][args.warmup:]
        t = sum(ts) / len(ts)
        v = r["n"] / t / 1e9
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": sample_config(r),
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample_desc(r),
                                 "config": sample_config(r)},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import numpy as np
    import torch

    import paper_2210_03179_gb300 as cm
    import workloads as W
    from paper_2210_03179_gb300 import _build

    _build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def slowest(x):
        return max_over_ranks(x, dist, "cuda")

    if args.profile_batched:
        v = W.sem_box_vertices(BATCH_NE, BATCH_NE, BATCH_NE)
        s = cm.Solver("sem", verts=v, prec="mixed", orders=ORDERS, kind=KIND, order=K_ORDER, sided=SIDED)
        B = torch.tensor(np.stack([W.sem_rhs(BATCH_NE, BATCH_NE, BATCH_NE, NORDER, seed=q)
                                   for q in range(BATCH_NRHS)]), device="cuda")
        U = torch.zeros_like(B)
        cm.chebmg_pcg_solve_batched(s.ctx, B, U, RTOL, 500, graph=False)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("bsolve")
        code, its, rel = cm.chebmg_pcg_solve_batched(s.ctx, B, U, RTOL, 500, graph=False)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile_batched": BATCH_NRHS, "code": code, "iterations": max(its)}))
        s.close()
        return 0

    verts = W.sem_box_vertices(NE, NE, NE)
    b_np = W.sem_rhs(NE, NE, NE, NORDER)
    n = b_np.size
    common = dict(verts=verts, orders=ORDERS, kind=KIND, order=K_ORDER, sided=SIDED)
    s32 = cm.Solver("sem", prec="mixed", **common)
    lmax = [s32.lambda_max(j) for j in range(len(ORDERS) - 1)]
    s64 = cm.Solver("sem", prec="fp64", lmax=lmax, **common)
    stream = torch.cuda.current_stream()
    b = torch.tensor(b_np, device="cuda")
    u = torch.zeros_like(b)

    def solve(s):
        code, it, rel, _ = cm.chebmg_pcg_solve(s.ctx, b, u, RTOL, 500)
        assert code == cm.CHEBMG_OK and rel <= RTOL, (code, it, rel)
        return it

    if args.profile_smoother:
        s = s32 if args.profile_smoother == "mixed" else s64
        f32 = args.profile_smoother == "mixed"
        dt = cm.CHEBMG_F32 if f32 else cm.CHEBMG_F64
        xb = torch.zeros(n, device="cuda", dtype=torch.float32 if f32 else torch.float64)
        bb = xb.clone().uniform_(-1, 1)
        if args.tile is not None:
            cm.chebmg_set_tile_choice(s.ctx, 0, dt, args.tile)
        # the separate kernels unless the fused one is asked for (whatever the autotuner chose)
        cm.chebmg_set_fused_smoother(s.ctx, 0, dt, (1 if f32 else 2) if args.fused else 0)
        cm.chebmg_smooth(s.ctx, 0, dt, bb, xb, 9, True)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("smooth")
        cm.chebmg_smooth(s.ctx, 0, dt, bb, xb, 9, True)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile_smoother": args.profile_smoother,
                          "elements_per_block": cm.chebmg_tile_choice(s.ctx, 0, dt),
                          "fused_variant": cm.chebmg_fused_smoother(s.ctx, 0, dt)}))
        s32.close()
        s64.close()
        return 0

    if args.profile_outer:
        if args.profile_outer == "f32x2":
            cm.chebmg_set_outer_operator(s32.ctx, cm.CHEBMG_OUTER_F32X2)
        xo = torch.empty(n, dtype=torch.float64, device="cuda").uniform_(-1, 1)
        yo = torch.zeros_like(xo)
        cm.chebmg_apply_outer(s32.ctx, xo, yo)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("outer")
        cm.chebmg_apply_outer(s32.ctx, xo, yo)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile_outer": args.profile_outer}))
        s32.close()
        s64.close()
        return 0

    if args.profile_solve:
        s = s32 if args.profile_solve == "mixed" else s64
        solve(s)
        torch.cuda.synchronize()
        if args.pin_tiles:
            for key, var in json.loads(args.pin_tiles).items():
                lev, dt = (int(x) for x in key.split(","))
                cm.chebmg_set_tile_choice(s.ctx, lev, dt, int(var))
            solve(s)
            torch.cuda.synchronize()
        tiles = {f"{j},{dt}": cm.chebmg_tile_choice(s.ctx, j, dt)
                 for j in range(len(ORDERS)) for dt in ((0, 1) if args.profile_solve == "mixed" else (0,))
                 if cm.chebmg_tile_choice(s.ctx, j, dt)}
        torch.cuda.nvtx.range_push("solve")
        it = solve(s)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile_solve": args.profile_solve, "iterations": it, "tiles": tiles}))
        s32.close()
        s64.close()
        return 0

    def timed(fn, reps):
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = None
        for _ in range(reps):
            out = fn()
        e1.record(stream)
        e1.synchronize()
        barrier()
        return slowest(e0.elapsed_time(e1) / 1e3 / reps), out

    if args.schedules_only:
        s32.close()
        s64.close()
        print(json.dumps({"schedules": bench_schedules(cm, W, torch, timed, max(1, args.steps), verts, b)}))
        return 0

    if args.table1_only:
        s32.close()
        s64.close()
        print(json.dumps({"fd_table1": bench_fd_table1(cm, torch, timed, max(1, args.steps))}))
        return 0

    if args.diff_only:
        s32.close()
        s64.close()
        print(json.dumps({"differentiation": bench_differentiation(cm, W, torch, timed, max(1, args.steps))}))
        return 0

    if args.batched_only:
        s32.close()
        s64.close()
        print(json.dumps({"batched": bench_batched(cm, W, torch, timed, max(1, args.steps))}))
        return 0

    for _ in range(args.warmup):
        it32 = solve(s32)
    it64 = solve(s64)

    # ---- headline: mixed-precision solves, inputs resident in HBM ----
    clocks = Clocks(local)
    clocks.mark()
    l0 = cm.chebmg_launch_count()
    t32, it32 = timed(lambda: solve(s32), args.steps)
    launches = (cm.chebmg_launch_count() - l0) // args.steps
    clk = clocks.stop()
    t64, it64 = timed(lambda: solve(s64), max(1, min(args.steps, 3)))

    # ---- the paper's statistic as well: the fastest of 20 individually timed solves ----
    def best_of(fn, trials=20):
        best = float("inf")
        for _ in range(trials):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        return slowest(best)

    best20 = {"mixed": best_of(lambda: solve(s32)), "fp64": best_of(lambda: solve(s64))}

    # ---- each form's result: true FP64 residual, and the mixed solution against the FP64 one ----
    solve(s64)
    u64 = u.clone()
    solve(s32)
    results = {"mixed": {"iterations": it32, "true_relres": true_relres(cm, torch, s64, b, u)},
               "fp64": {"iterations": it64, "true_relres": true_relres(cm, torch, s64, b, u64)},
               "mixed_vs_fp64_max_rel_diff": float((u - u64).abs().max() / u64.abs().max())}
    del u64

    # ---- end to end through the host-buffer entry point (pinned host memory) ----
    bh = torch.tensor(b_np).pin_memory()
    uh = torch.zeros(n, dtype=torch.float64).pin_memory()
    bh_np, uh_np = bh.numpy(), uh.numpy()

    def solve_host():
        code, it, rel = cm.chebmg_pcg_solve_host(s32.ctx, bh_np, uh_np, RTOL, 500)
        assert code == cm.CHEBMG_OK
        return it

    solve_host()
    te2e, _ = timed(solve_host, args.steps)

    # ---- fine-level smoother step (Ax + gather-scatter + recurrence) ----
    def smoother_step_time(s, dt, f32):
        xb = torch.zeros(n, device="cuda", dtype=torch.float32 if f32 else torch.float64)
        bb = xb.clone().uniform_(-1, 1)
        # orders 9 and 2: both end with the fused last step, so the difference is 7 whole steps
        hi, lo = 9, 2
        cm.chebmg_smooth(s.ctx, 0, dt, bb, xb, hi, True)
        t_hi, _ = timed(lambda: cm.chebmg_smooth(s.ctx, 0, dt, bb, xb, hi, True), 10)
        t_lo, _ = timed(lambda: cm.chebmg_smooth(s.ctx, 0, dt, bb, xb, lo, True), 10)
        return (t_hi - t_lo) / (hi - lo)

    step32 = smoother_step_time(s32, cm.CHEBMG_F32, True)
    step64 = smoother_step_time(s64, cm.CHEBMG_F64, False)
    E = NE ** 3
    L = E * (NORDER + 1) ** 3
    alg_bytes32 = 4 * (6 * L + 7 * n)
    pk = peaks()
    hbm = pk.get("hbm_gbs")
    achieved = alg_bytes32 / step32 / 1e9
    fused32 = cm.chebmg_fused_smoother(s32.ctx, 0, cm.CHEBMG_F32)
    tile32 = cm.chebmg_tile_choice(s32.ctx, 0, cm.CHEBMG_F32)
    roofline = {"bound": "hbm",
                "kernel": ("fine FP32 Chebyshev step, fused: k_sem_smooth8 (one launch per smoother application)"
                           if fused32 else
                           "fine FP32 Chebyshev step: k_sem_ax8p (element Ax + gather-scatter) + k_cheb4_step"),
                "achieved": achieved, "peak": hbm if hbm else 6800.0, "unit": "GB/s",
                "frac": achieved / (hbm if hbm else 6800.0),
                "peak_source": "of measured (MEASURED_PEAKS.json hbm_gbs)" if hbm else "of fallback",
                # the recorded DRAM bytes belong to the separate kernels of that variant
                "traffic": recorded_traffic(tile32) if fused32 == 0 else None,
                "alg_bytes_per_step": alg_bytes32, "step_us": step32 * 1e6,
                "elements_per_block_variant": tile32, "fused_variant": fused32}
    # ---- the FP64 outer operator q = A p (k_sem_ax8<double>), bound by the FP64 pipe ----
    # Executed FP64 instructions per element point, counted from the kernel source: six line
    # passes of 44 per 8-point line (8 even-odd sums, 4 x 9 chain FMAs) = 33, the geometric
    # factors 9 (3 x (1 mul + 2 FMA)), two additions of the transposed contributions = 44.
    FP64_INSTR_PER_POINT = 44
    xo64 = torch.empty(n, dtype=torch.float64, device="cuda").uniform_(-1, 1)
    yo64 = torch.zeros_like(xo64)
    cm.chebmg_apply_A(s32.ctx, 0, cm.CHEBMG_F64, xo64, yo64)
    t_apply64, _ = timed(lambda: cm.chebmg_apply_A(s32.ctx, 0, cm.CHEBMG_F64, xo64, yo64), 10)
    t_zero64, _ = timed(lambda: yo64.zero_(), 10)     # apply_A zeroes y first: take that out
    t_op_kernel = max(t_apply64 - t_zero64, 1e-9)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    sm_mhz = clk.get("sm_mhz") or 2070.0
    # GB300 issues 2 FP64 FMA (or add / mul) instructions per SM per clock: the unit-count rate,
    # 2 x 152 x 2.07 GHz = 629 G instructions/s (1.26 TFLOP/s in FMAs, the nominal 1.25)
    peak_i64 = 2 * sms * sm_mhz * 1e6 / 1e9
    ach_i64 = FP64_INSTR_PER_POINT * L / t_op_kernel / 1e9
    fp64_alu = {"bound": "alu", "kernel": "FP64 outer operator q = A p (k_sem_ax8<double>, element Ax + "
                                          "gather-scatter), 40% of the mixed solve",
                "achieved": ach_i64, "peak": peak_i64, "unit": "G FP64 instructions/s", "frac": ach_i64 / peak_i64,
                "peak_source": f"unit count: 2 FP64 instructions / SM / clock x {sms} SMs x {sm_mhz:.0f} MHz "
                               f"(median SM clock sampled in the timed region)",
                "instructions_per_point": FP64_INSTR_PER_POINT, "points_per_launch": L,
                "kernel_us": t_op_kernel * 1e6,
                "algorithmic_tflops": (111 * L + 8 * n) / t_op_kernel / 1e12,
                "fine_fp64_chebyshev_step_us": step64 * 1e6}
    del xo64, yo64

    # ---- coarse solve (N = 1, FP64 CG to the coarse tolerance) on its own ----
    def coarse_time(s):
        nc = s.size(len(ORDERS) - 1)
        rc = torch.empty(nc, dtype=torch.float64, device="cuda").uniform_(-1, 1)
        zc = torch.zeros_like(rc)
        its = cm.chebmg_coarse_solve(s.ctx, rc, zc)
        t_c, _ = timed(lambda: cm.chebmg_coarse_solve(s.ctx, rc, zc), 20)
        deg, _ = cm.chebmg_coarse_info(s.ctx)
        kern, blocks, rows = cm.chebmg_coarse_shape(s.ctx)
        return {"ms": t_c * 1e3, "iterations": its, "degree": deg,
                "kernel": {cm.CHEBMG_COARSE_GRID: "grid", cm.CHEBMG_COARSE_CLUSTER: "cluster"}.get(kern, "host"),
                "blocks": blocks, "rows_per_block": rows, "n": nc}

    coarse = {"mixed": coarse_time(s32), "fp64": coarse_time(s64)}

    # ---- opt-in: the outer product in FP64-class arithmetic on FP32 pairs ----
    xo = torch.empty(n, dtype=torch.float64, device="cuda").uniform_(-1, 1)
    yo = torch.zeros_like(xo)
    t_op64, _ = timed(lambda: cm.chebmg_apply_outer(s32.ctx, xo, yo), 5)
    cm.chebmg_set_outer_operator(s32.ctx, cm.CHEBMG_OUTER_F32X2)
    cm.chebmg_apply_outer(s32.ctx, xo, yo)
    t_opx2, _ = timed(lambda: cm.chebmg_apply_outer(s32.ctx, xo, yo), 5)
    solve(s32)
    t32x2, it32x2 = timed(lambda: solve(s32), args.steps)
    cm.chebmg_set_outer_operator(s32.ctx, cm.CHEBMG_OUTER_FP64)
    outer = {"fp64_us": t_op64 * 1e6, "f32x2_us": t_opx2 * 1e6,
             "note": "opt-in CHEBMG_OUTER_F32X2: the outer product q = A p in FP64-class arithmetic on "
                     "FP32 pairs (about 48 significant bits); the headline uses FP64; each time includes "
                     "the zeroing of q and a host synchronisation"}

    world_n = world
    value = job_throughput(world_n, n, t32)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world_n, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t32 * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": config({"parallelism": f"replicas x{world_n}",
                              "ax8_elements_per_block": {"fp32": cm.chebmg_tile_choice(s32.ctx, 0, 1),
                                                         "fp64": cm.chebmg_tile_choice(s64.ctx, 0, 0)}}),
            "time_to_1e8_s": {"mixed": t32, "fp64": t64, "mixed_f32x2_outer": t32x2},
            "time_to_1e8_s_min_of_20": best20,
            "iterations": {"mixed": it32, "fp64": it64, "mixed_f32x2_outer": it32x2},
            "results": results,
            "outer_operator": outer,
            "speedup_mixed_vs_fp64": t64 / t32,
            "smoother_gdofs": {"fp32": n / step32 / 1e9, "fp64": n / step64 / 1e9},
            "e2e": {"value": job_throughput(world_n, n, te2e), "unit": UNIT, "h2d_bytes_per_step": 8 * n,
                    "d2h_bytes_per_step": 8 * n},
            "gpu_launches": int(launches),
            "roofline": roofline, "roofline_fp64": fp64_alu,
            "coarse_solve": coarse,
            "clocks": clk}
    if not args.no_batched:
        s32.close()
        s64.close()
        line["batched"] = bench_batched(cm, W, torch, timed, max(1, min(args.steps, 3)), clk.get("sm_mhz"))
    if not args.no_schedules:
        s32.close()
        s64.close()
        line["schedules"] = bench_schedules(cm, W, torch, timed, max(1, min(args.steps, 3)), verts, b)
    if not args.no_table1:
        s32.close()
        s64.close()
        line["fd_table1"] = bench_fd_table1(cm, torch, timed, max(1, min(args.steps, 3)))
    if not args.no_diff:
        s32.close()
        s64.close()
        line["differentiation"] = bench_differentiation(cm, W, torch, timed, max(1, min(args.steps, 3)))
    if rank == 0 and not args.no_cpu_baseline and not args.no_all_cores:
        nall, wall, cores = run_oracle_all_cores()
        line["cpu_baseline_all_cores"] = {"value": nall / wall / 1e9, "unit": UNIT, "cores": cores,
                                          "kind": "oracle",
                                          "sample": f"{cores} concurrent one-thread FP64 oracle solves of the "
                                                    f"E={SAMPLE_NE}^3 recipe (one per core), setup included in "
                                                    f"each process, wall time {wall:.1f} s"}
    if rank == 0 and not args.no_cpu_baseline:
        with tempfile.TemporaryDirectory() as td:
            path = os.path.join(td, "x_oracle.npy")
            r = run_oracle(1, save=path)
            x_ref = np.load(path)
        t = r["times"][0]
        line["cpu_baseline"] = {"value": r["n"] / t / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": sample_desc(r), "seconds": t, "config": sample_config(r)}
        line["error_vs_oracle"] = errors_against_oracle(cm, W, torch, np, x_ref, r["iters"])
    s32.close()
    s64.close()
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
