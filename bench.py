#!/usr/bin/env python3
"""Benchmark: rank-1 bidiagonal updates per second at m = n = 4096.

Workload (the recommender stream): A = Q Bd P^T with Q, P products of 8
Householder reflectors, d ~ U(1, 10), e ~ N(0, 1); each step is one rank-1
"set item column" update A + b e_j^T with b a ratings column (2% of the rows,
values 1..5) and j = h mod n.  A step runs the whole hot path: projection,
FP64 rotation generation and bulge chasing, and the application of the
rotations to Q and P.

The headline form is the mixed one (Q, P in FP32; generation and Bd in FP64),
with its default re-orthogonalization (one Newton-Schulz step after every
column at this size, on the apply stream) inside the timed region; the plain
FP64 form is measured on the same workload and reported beside it with both
forms' residuals, and the mixed form's ||Q^T Q - I||_2, ||P^T P - I||_2 after
the timed run are reported against the 1e-5 tolerance.

Timing: CUDA events on the library's stream after W warm-up steps.  The mixed
form runs overlapped (each update's application to Q and P on a second stream
while the next update's rotations are generated); its K steps are timed back
to back as one region that ends when all their work, the last deferred
application included, is done.  No L2 flush is needed there: every step
streams about 1.2 GB (rotation records, Q, P), far more than the 129 MB L2.
The FP64 form is timed per step with an L2 flush (a 512 MiB write) before
each.  `value` is device-resident throughput (B, C already in HBM,
bdu_update_dev); `e2e` goes through bdu_update with pinned host buffers and
reads the updated bidiagonal back every step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

  python bench.py --thin KR [--thin-fp64] [--size M] [--steps K] [--warmup W]
    rank-KR tracking (bdu_thin_*, Sec. 4; mixed form unless --thin-fp64) on the network edge stream at
    m = n = M: each step is one symmetric edge insertion, i.e. two rank-1
    tracking steps; wall clock (every tracking step completes before it
    returns), with the CPU oracle timed on one tracking step beside it.

With N > 1 (launched by torchrun) every rank updates its own factorization:
the path does not shard, so ranks are independent replicas (weak scaling).
The reference arm times the CPU oracle (the library's plain FP64 reference
implementation) on a bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rank-1 updates/s at m=n=4096 (mixed form; FP64 form beside it)"
UNIT = "updates/s"
M = N = 4096


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--e2e-steps", type=int, default=100,
                    help="updates of the end-to-end run (at least --steps); their wall times give the latency")
    ap.add_argument("--serving-seconds", type=float, default=8.0,
                    help="Poisson phase of the serving measurement per form (0 = no serving measurement)")
    ap.add_argument("--serving-sessions", type=int, default=256)
    ap.add_argument("--oracle-rows", type=int, default=256,
                    help="rows of Q and P the CPU oracle applies in its bounded sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-bhu", action="store_true", help="no BHU (Algorithm 1) measurement in the bench line")
    ap.add_argument("--bhu", action="store_true",
                    help="only the BHU measurement, at m = n = --size (profiling runs; --steps timed updates)")
    ap.add_argument("--size", type=int, default=4096,
                    help="m = n of the workload (4096 is the benchmark; smaller sizes are for profiling)")
    ap.add_argument("--quick", action="store_true",
                    help="mixed form only: no FP64 form, e2e or CPU baseline (profiling runs)")
    ap.add_argument("--thin", type=int, default=0,
                    help="rank of the thin (rank-k tracking) benchmark instead of the headline")
    ap.add_argument("--thin-fp64", action="store_true", help="the FP64 form of rank-k tracking (default: mixed)")
    ap.add_argument("--nb", type=int, default=0,
                    help="apply variant of the mixed form (0: the autotuner's choice; 64/96/128: the blocked "
                         "tensor-core apply; for profiling runs)")
    ap.add_argument("--network", action="store_true",
                    help="full factors on the network edge stream (rank-2 symmetric edge insertions), mixed form, "
                         "at m = n = --size (16384 for this mode unless given)")
    a = ap.parse_args()
    global M, N
    M = N = a.size if (not a.network or any(x.startswith("--size") for x in sys.argv[1:])) else 16384
    return a


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        return parse_clock_samples(self.lines)


def parse_clock_samples(lines):
    """The clocks object of a bench line from nvidia-smi samples of the QUERY
    fields (CSV, no header, no units): the median SM clock under load, the
    maximum, and every throttle reason seen active in any sample."""
    sm, smax, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            smax = float(f[2])
        except ValueError:
            continue
        for name, v in zip(names, f[5:9]):
            if v.lower().startswith("active"):
                reasons.add(name)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
            "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# workload
# --------------------------------------------------------------------------
def workload(rank, steps):
    from paper_2509_02840_gb300 import inputs as I
    Q, d, e, P = I.factorization(M, N, config=1, which=rank)
    ups = [I.recommender_update(M, N, h + 1000 * rank, config=1) for h in range(steps)]
    return Q, d, e, P, ups


def slowest_rank_ms(ms, dist, device):
    """The timed region of the whole job: the largest of every rank's (the job
    ends with its slowest replica).  dist is torch.distributed or None."""
    if dist is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, ms):
    """Whole-job units per second: the units every rank processed over the
    slowest rank's time (the replicas are independent: weak scaling)."""
    return world * units_per_rank / (ms / 1e3)


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# FP32 FMA peak from unit counts and the maximum clock: 152 SMs x 128 FP32
# lanes x 2 flops x 2070 MHz.  FP64: 152 SMs x 2 FP64 FMA per clock x 2 flops
# x 2070 MHz (GB300's FP64 rate).
ALU_FP32_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
ALU_FP64_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# Algorithmic work per rotation: 10 multiplications and 10 additions on the band
# (Sec. 3.4), plus the rotation itself (2 multiplications, 1 addition, 1 square
# root, 2 divisions counted as one flop each).
CHASE_FLOPS_PER_ROTATION = 26
# DRAM bytes (read + write) of one mixed-form chase launch at m = n = 4096, from one
# ncu capture (one pass) of this benchmark's launches with the chase kernel as it is:
# the rotation records written (FP32 (c, s) and an int32 pair index per rotation,
# 12 B x 25.2M = 302 MB, part of which is still in L2 when the launch ends).
CHASE_TRAFFIC_4096 = 5.91e6 + 248.74e6


def roofline(st, precision, rotations_per_update, launches_per_update, steps_per_update=None):
    """Roofline object of the dominant kernel group of one update."""
    ms = {"chase": st["ms_chase"], "apply": st["ms_apply_q"] + st["ms_apply_p"], "project": st["ms_project"]}
    nup = max(st["timed_updates"], 1)
    dom = max(ms, key=ms.get)
    if dom == "chase":
        per_launch_ms = ms["chase"] / nup
        flops = CHASE_FLOPS_PER_ROTATION * rotations_per_update
        ach = flops / (per_launch_ms * 1e-3) / 1e12
        out = {"kernel": "k_chase (FP64 rotation generation + bulge chase)", "bound": "alu",
               "achieved": ach, "peak": ALU_FP64_TFLOPS, "unit": "TFLOP/s", "frac": ach / ALU_FP64_TFLOPS,
               "traffic": CHASE_TRAFFIC_4096 if (M == N == 4096 and precision == 1) else None,
               "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 x 2070 MHz",
               "share": ms["chase"] / sum(ms.values())}
        if steps_per_update:
            # the kernel is bound by its chain of dependent steps, not by a throughput
            out["critical_path"] = {"steps_per_launch": steps_per_update,
                                    "us_per_step": per_launch_ms * 1e3 / steps_per_update}
        return out
    # apply: algorithmic bytes = one read + one write of Q and P per rank-1 column
    es = 8 if precision == 0 else 4
    per_launch_ms = ms["apply"] / max(st["apply_launches"], 1)
    bytes_per_launch = (2 * M * M * es + 2 * N * N * es) / 2
    flops_per_launch = 6 * rotations_per_update / 2 * M
    if precision == 1:
        ach = flops_per_launch / (per_launch_ms * 1e-3) / 1e12
        return {"kernel": "k_apply_slab (FP32 column-pair rotations)", "bound": "alu", "achieved": ach,
                "peak": ALU_FP32_TFLOPS, "unit": "TFLOP/s", "frac": ach / ALU_FP32_TFLOPS, "traffic": None,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz",
                "algorithmic_bytes": bytes_per_launch, "share": ms["apply"] / sum(ms.values())}
    ach = flops_per_launch / (per_launch_ms * 1e-3) / 1e12
    return {"kernel": "k_apply_slab (FP64 column-pair rotations)", "bound": "alu", "achieved": ach,
            "peak": ALU_FP64_TFLOPS, "unit": "TFLOP/s", "frac": ach / ALU_FP64_TFLOPS, "traffic": None,
            "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 x 2070 MHz",
            "share": ms["apply"] / sum(ms.values())}


def latency_summary(samples, what):
    """p50 and p99 when there are at least 100 samples; otherwise the median
    and the maximum (a p99 of fewer samples would only be the maximum)."""
    xs = sorted(samples)
    out = {"samples": len(xs), "what": what, "p50": statistics.median(xs), "max": xs[-1]}
    if len(xs) >= 100:
        out["p99"] = xs[min(len(xs) - 1, int(round(0.99 * (len(xs) - 1))))]
    return out


def apply_roofline(st, rotations_per_update):
    """The rotation apply (mixed form) against HBM: algorithmic bytes per
    launch = one read and one write of the factor in FP32 plus one read of its
    side's FP32 coefficient records (8 B per rotation), over the launch's
    average device time (CUDA events around each launch)."""
    launches = max(st["apply_launches"], 1)
    per_launch_ms = (st["ms_apply_q"] + st["ms_apply_p"]) / launches
    alg = 2 * M * M * 4 + 8 * rotations_per_update / 2
    hbm = peaks().get("hbm_gbs")
    ach = alg / (per_launch_ms * 1e-3) / 1e9
    return {"kernel": "rotation apply to Q or P (mixed form, one rank-1 column per launch)", "bound": "hbm",
            "algorithmic_bytes": alg, "ms_per_launch": per_launch_ms, "achieved": ach, "unit": "GB/s",
            "peak": hbm, "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if hbm else None,
            "frac": ach / hbm if hbm else None,
            # the work the rotations define (6 flops per rotation and row), which the
            # blocked apply (orders >= 1024) performs as tensor-core products of
            # accumulated rotation blocks: far from HBM-bound
            "rotation_tflops": 6.0 * (rotations_per_update / 2) * M / (per_launch_ms * 1e-3) / 1e12,
            "note": "timed beside the concurrent chase of the next update (overlapped form)"}


def serving(args):
    """A short run of the serving mix (256 resident factorizations, m, n
    log-uniform in [64, 2048], rank 1..4 requests, a device budget of a third
    of what all sessions need) in both forms: saturated updates/s, then p50/p99
    latency under Poisson arrivals at 80 % of the saturated rate."""
    from paper_2509_02840_gb300 import bdu, serve as S
    out = {}
    for form, prec in (("mixed", bdu.MIXED), ("fp64", bdu.FP64)):
        r = S.serve(args.serving_sessions, args.serving_seconds, prec, sat_per_session=1)
        out[form] = {"saturated_updates_per_s": r["saturated"]["updates_per_s"],
                     "poisson_updates_per_s": r["poisson"]["updates_per_s"],
                     "offered_requests_per_s": r["offered_requests_per_s"],
                     "latency_ms": r["poisson"]["latency_ms"], "requests": r["poisson"]["requests"],
                     "evictions": r["saturated"]["evictions"] + r["poisson"]["evictions"]}
    out["config"] = {"sessions": args.serving_sessions, "budget_fraction": 1 / 3,
                     "poisson_seconds": args.serving_seconds, "load": 0.8,
                     "saturation": "one request per session, all present at the start"}
    return out


def bhu_bench(steps=2, shapes=None):
    """BHU (Sec. 3.3, Algorithm 1) beside the FP64 Givens form on the same
    rank-1 updates, at m = n = 4096 (the recommender stream) and m = 8192 x
    n = 2048 (dense b, c: a tall factorization, the case Sec. 3.3 names for
    BHU).  Device time per update with CUDA events on the handle's stream (B, C
    already on the device); one untimed update first.  The roofline counts the
    paper's multiplications for the reflectors, (m + 3n) n^2 - 4/3 n^3 (Eq.
    housecplx), two flops each, plus the three products a side that update Q
    and P (4 m^2 k + m k^2 with k reflectors), against the FP64 peak."""
    import numpy as np
    import torch
    from paper_2509_02840_gb300 import bdu, inputs as I
    peak = 152 * 2 * 2 * 2.07e9
    out = {}
    shapes = shapes or ((f"recommender_{M}", M, N), ("tall_8192x2048", 8192, 2048))
    for name, m, n in shapes:
        Q, d, e, P = I.factorization(m, n, config=1 if m == n else 2)
        if m == n:
            ups = [I.recommender_update(m, n, h + 500, config=1) for h in range(steps + 1)]
        else:
            ups = [I.dense_update(m, n, h + 500, config=2, r=1) for h in range(steps + 1)]
        dev = [(torch.from_numpy(np.asfortranarray(B)).cuda(), torch.from_numpy(np.asfortranarray(C)).cuda())
               for B, C in ups]
        res = {}
        for method in ("bhu", "givens"):
            stream = torch.cuda.Stream()
            with bdu.Factorization(Q, d, e, P, precision=bdu.FP64, stream=stream.cuda_stream) as F:
                call = F.update_bhu_dev if method == "bhu" else F.update_dev
                call(dev[0][0].data_ptr(), dev[0][1].data_ptr(), 1)
                F.sync()
                with torch.cuda.stream(stream):
                    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    for Bd, Cd in dev[1:]:
                        call(Bd.data_ptr(), Cd.data_ptr(), 1)
                    e1.record(stream)
                F.sync()
                res[method] = e0.elapsed_time(e1) / steps
                if method == "bhu":
                    s_bhu = F.singular_values(16)
                else:
                    s_giv = F.singular_values(16)
        kl, kr = (n if m > n else n - 1), n - 2
        flops = 2 * ((m + 3 * n) * n * n - 4.0 / 3.0 * n ** 3) + 4 * m * m * kl + m * kl * kl + 4 * n * n * kr + n * kr * kr
        achieved = flops / (res["bhu"] * 1e-3) / 1e12
        out[name] = {"m": m, "n": n, "bhu_ms_per_update": res["bhu"], "givens_fp64_ms_per_update": res["givens"],
                     "bhu_updates_per_s": 1e3 / res["bhu"], "steps": steps,
                     "top16_singular_values_max_rel_diff": float(np.abs(s_bhu - s_giv).max() / s_giv[0]),
                     "roofline": {"bound": "alu", "achieved": achieved, "peak": peak / 1e12, "unit": "TFLOP/s",
                                  "frac": achieved * 1e12 / peak, "flops_per_update": flops,
                                  "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 x 2070 MHz"}}
    # the symmetric variant (Sec. 6): A + rho c c^T for A = Q T Q^T, n = M, in place
    n = M
    k, _, ub = bdu.tri_sizes(n, n)
    g = np.random.default_rng(77)
    # an orthogonal Q (its row-major storage read as column-major is its transpose, also orthogonal)
    Qt = torch.linalg.qr(torch.from_numpy(g.standard_normal((n, n))).cuda())[0].contiguous()
    at = torch.from_numpy(g.uniform(1.0, 10.0, n)).cuda()
    bt = torch.from_numpy(g.standard_normal(n - 1)).cuda()
    cs = [torch.from_numpy(g.standard_normal(n)).cuda() for _ in range(steps + 1)]
    wst = torch.zeros((ub + 7) // 8, dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        bdu.tri_update_dev(n, Qt.data_ptr(), at.data_ptr(), bt.data_ptr(), 1.0, cs[0].data_ptr(), wst.data_ptr(),
                           stream.cuda_stream)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for c in cs[1:]:
            bdu.tri_update_dev(n, Qt.data_ptr(), at.data_ptr(), bt.data_ptr(), 1.0, c.data_ptr(), wst.data_ptr(),
                               stream.cuda_stream)
        e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # multiplications of the reflector products (four passes over the trapezoidal Y a step,
    # sum_j 4 (n - j/2) j ~ 4/3 n^3) and the update of Q (4 n^2 k + n k^2), two flops each
    flops = 2 * (4.0 / 3.0) * n ** 3 + 4 * n * n * k + n * k * k
    out[f"tridiagonal_{n}"] = {"n": n, "ms_per_update": ms, "updates_per_s": 1e3 / ms, "steps": steps,
                               "what": "A + rho c c^T for A = Q T Q^T (bdu_tri_update_dev: u = Q^T c, the "
                                       "tridiagonalization of T + rho u u^T, Q updated), device time",
                               "roofline": {"bound": "alu", "achieved": flops / (ms * 1e-3) / 1e12,
                                            "peak": peak / 1e12, "unit": "TFLOP/s",
                                            "frac": flops / (ms * 1e-3) / peak, "flops_per_update": flops,
                                            "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 x 2070 MHz"}}
    return out


def residual(F, A0_parts, ups):
    """||A+ - Q Bd P^T||_F / ||A+||_F with A+ accumulated in FP64."""
    import numpy as np
    Q0, d0, e0, P0 = A0_parts
    A = Q0 @ (np.diag(d0) + np.diag(e0, 1)) @ P0.T
    for B, C in ups:
        A += B @ C.T
    Q, d, e, P = F.read()
    R = Q @ (np.diag(d) + np.diag(e, 1)) @ P.T
    return float(np.linalg.norm(A - R) / np.linalg.norm(A))


# --------------------------------------------------------------------------
# CPU oracle: a bounded sample of the same workload
# --------------------------------------------------------------------------
def oracle_sample(rows_sample, updates=1):
    """Full rotation generation of one update plus the apply for `rows_sample`
    rows of Q and of P (rows are independent), extrapolated to all rows."""
    import numpy as np
    import oracle as O
    Q, d, e, P, ups = workload(0, updates)
    secs = []
    for B, C in ups:
        t0 = time.perf_counter()
        U, V = O.project(Q, P, B, C)
        d2, e2, L, R, _ = O.generate(M, N, d, e, U, V)
        t1 = time.perf_counter()
        rows = np.arange(rows_sample)
        O.apply_rows(Q, rows, L)
        O.apply_rows(P, rows, R)
        t2 = time.perf_counter()
        secs.append((t1 - t0) + (t2 - t1) * (M / rows_sample))
        d, e = d2, e2
    per = statistics.mean(secs)
    return {"value": 1.0 / per, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": (f"{updates} full m=n=4096 recommender update(s): projection and all "
                       f"~25M rotations generated; rotations applied to {rows_sample} of 4096 rows "
                       f"of Q and of P and extrapolated linearly (rows are independent)"),
            "seconds_per_update": per}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    t_all = time.perf_counter()
    for _ in range(args.warmup):
        oracle_sample(args.oracle_rows, 1)
    t_meas = time.perf_counter()
    samples = [oracle_sample(args.oracle_rows, 1) for _ in range(args.steps)]
    t_meas = time.perf_counter() - t_meas
    t = [x["seconds_per_update"] for x in samples]
    import oracle as O
    per = statistics.mean(t)
    line = {"impl": "reference", "metric": METRIC, "value": 1.0 / per, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3,
            "ms_per_step_kind": ("extrapolated: each step generates all rotations of one full update and "
                                 f"applies them to {args.oracle_rows} of {M} rows of Q and of P; the apply "
                                 "time is scaled to all rows (rows are independent)"),
            "measured_wall_s": {"timed_steps": t_meas, "per_step": t_meas / max(args.steps, 1),
                                "whole_run": time.perf_counter() - t_all},
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "recommender stream m=n=4096, rank-1 set-item-column updates",
                                            "m": M, "n": N, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": 1.0 / per, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": f"per step: one full update's generation + apply on {args.oracle_rows} rows of Q and P, extrapolated"},
            "e2e": {"value": 1.0 / per, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def run_gpu(args):
    import numpy as np
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2509_02840_gb300 import bdu
    bdu.load()
    K, W = args.steps, args.warmup
    n_e2e = max(args.e2e_steps, K)
    Q, d, e, P, ups = workload(rank, W + K + n_e2e + 1 + args.fp64_steps)
    stream = torch.cuda.Stream()
    dev_ups = []
    with torch.cuda.stream(stream):
        for B, C in ups:
            dev_ups.append((torch.from_numpy(np.asfortranarray(B).reshape(-1, order="F")).cuda(),
                            torch.from_numpy(np.asfortranarray(C).reshape(-1, order="F")).cuda()))
    stream.synchronize()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def timed_steps(F, seq):
        times = []
        for Bd, Cd in seq:
            with torch.cuda.stream(stream):
                flush.zero_()
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                F.update_dev(Bd.data_ptr(), Cd.data_ptr(), 1)
                ev1.record(stream)
            times.append((ev0, ev1))
        stream.synchronize()
        return [a.elapsed_time(b) for a, b in times]

    def timed_block(F, seq):
        """The steps back to back, as a stream of updates arrives; the region
        ends when every step's work, the deferred application of the last one
        included, is done.  Returns (total ms, per-step intervals between the
        ends of consecutive steps' chases)."""
        with torch.cuda.stream(stream):
            ev0 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            marks = []
            for Bd, Cd in seq:
                F.update_dev(Bd.data_ptr(), Cd.data_ptr(), 1)
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(stream)
                marks.append(ev)
            F.flush()
            ev1 = torch.cuda.Event(enable_timing=True)
            ev1.record(stream)
        stream.synchronize()
        steps = [(ev0 if i == 0 else marks[i - 1]).elapsed_time(marks[i]) for i in range(len(marks))]
        return ev0.elapsed_time(ev1), steps

    # ---- mixed form (headline), overlapped -------------------------------
    Fm = bdu.Factorization(Q, d, e, P, precision=bdu.MIXED, stream=stream.cuda_stream, device=local,
                           overlap=True, nb=args.nb)
    timed_block(Fm, dev_ups[:W])
    st0 = Fm.stats()
    Fm.set_timing(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    t_wall = time.perf_counter()
    total_ms, ms = timed_block(Fm, dev_ups[W:W + K])
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    torch.cuda.synchronize()
    total_ms = slowest_rank_ms(total_ms, dist, "cuda")
    st = Fm.stats()
    rot_per_update = (sum(st["rot_left"]) + sum(st["rot_right"]) - sum(st0["rot_left"]) - sum(st0["rot_right"])) / K
    launches = (st["launches"] - st0["launches"])
    roof = roofline(st, 1, rot_per_update, launches / K, (st["chase_steps"] - st0["chase_steps"]) / K)
    res_mixed = residual(Fm, (Q, d, e, P), ups[:W + K])
    ortho_q, ortho_p = Fm.check_orthogonality()
    ortho = {"q": ortho_q, "p": ortho_p, "tolerance": 1e-5, "reorth_q": st["reorth_q"] - st0["reorth_q"],
             "reorth_p": st["reorth_p"] - st0["reorth_p"],
             "policy": "one Newton-Schulz step (FP32 products, FP64 diagonal) after every rank-1 column"}

    if args.quick:
        Fm.close()
        line = {"metric": METRIC, "value": job_throughput(world, K, total_ms), "unit": UNIT, "n_gpus": world,
                "steps": K, "warmup": W, "ms_per_step": total_ms / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": f"recommender stream m=n={M} (quick profiling run)", "m": M, "n": N},
                "roofline": roof, "clocks": clk, "gpu_launches": launches,
                "kernel_ms_per_update": {k: st["ms_" + k] / max(st["timed_updates"], 1)
                                         for k in ("project", "chase", "apply_q", "apply_p")}}
        if rank == 0:
            print(json.dumps(line), flush=True)
        return

    # ---- e2e through the host-pointer ABI (pinned buffers, result read back):
    # each update's wall time from its bdu_update call to the return of the
    # bdu_read of its d, e is one latency sample; the region ends after
    # bdu_flush and bdu_sync, so the last update's deferred application to Q
    # and P is inside it
    e2e_seq = ups[W + K:W + K + n_e2e]
    pinned = []
    for B, C in e2e_seq:
        pb = torch.from_numpy(np.asfortranarray(B).reshape(-1, order="F")).pin_memory()
        pc = torch.from_numpy(np.asfortranarray(C).reshape(-1, order="F")).pin_memory()
        pinned.append((pb, pc))
    Fm.set_timing(False)
    dbuf = np.zeros(N); ebuf = np.zeros(N)
    import ctypes
    dp = ctypes.POINTER(ctypes.c_double)
    Fm.sync()
    lat = []

    def e2e_run(seq):
        for pb, pc in seq:
            ts = time.perf_counter()
            code = Fm._L.bdu_update(Fm._h, ctypes.cast(pb.data_ptr(), dp), ctypes.cast(pc.data_ptr(), dp), 1)
            bdu._check(Fm._L, Fm._h, code)
            code = Fm._L.bdu_read(Fm._h, None, dbuf.ctypes.data_as(dp), ebuf.ctypes.data_as(dp), None)
            bdu._check(Fm._L, Fm._h, code)
            lat.append(1e3 * (time.perf_counter() - ts))
        Fm.flush()
        Fm.sync()

    # the throughput region: K updates, as many as the device-timed region,
    # so that both carry the same pipeline fill and drain; the rest of the
    # updates only add latency samples
    t0 = time.perf_counter()
    e2e_run(pinned[:K])
    e2e_s = (time.perf_counter() - t0) / K
    e2e_run(pinned[K:])
    Fm.close()

    # ---- plain FP64 form on the same workload ------------------------------
    F64 = bdu.Factorization(Q, d, e, P, precision=bdu.FP64, stream=stream.cuda_stream, device=local)
    timed_steps(F64, dev_ups[:1])
    ms64 = timed_steps(F64, dev_ups[1:1 + args.fp64_steps])
    res64 = residual(F64, (Q, d, e, P), ups[:1 + args.fp64_steps])
    F64.close()

    if dist:
        dist.barrier()
    value = job_throughput(world, K, total_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (Q, P storage and apply) + f64 (projection, rotations, Bd)",
        "data": "synthetic",
        "config": {"workload": f"recommender stream m=n={M}, rank-1 set-item-column updates (2% ratings column, c=e_j)",
                   "m": M, "n": N, "rank": 1, "form": "mixed", "parallelism": f"replicas x{world}",
                   "overlap": "apply of step h concurrent with the chase of step h+1",
                   "l2": "not flushed: each step streams ~1.2 GB (rotation records, Q, P) > 129 MB L2"},
        "latency_ms": latency_summary(lat, "wall time of one update through the C ABI: bdu_update with pinned "
                                           "host B, C until bdu_read of its d, e returns (overlapped form: "
                                           "the application to Q, P runs behind it)"),
        "step_interval_ms": {"median": statistics.median(ms), "max": max(ms), "samples": len(ms),
                             "what": "interval between the chase ends of consecutive timed steps"},
        "fp64_form": {"value": 1e3 / statistics.mean(ms64), "unit": UNIT, "ms_per_step": statistics.mean(ms64),
                      "steps": len(ms64), "relative_residual": res64},
        "mixed_relative_residual": res_mixed,
        "mixed_orthogonality": ortho,
        "mixed_vs_fp64_speedup": (K / (total_ms / 1e3)) / (1e3 / statistics.mean(ms64)),
        "kernel_ms_per_update": {"project": st["ms_project"] / max(st["timed_updates"], 1),
                                 "chase": st["ms_chase"] / max(st["timed_updates"], 1),
                                 "apply_q": st["ms_apply_q"] / max(st["timed_updates"], 1),
                                 "apply_p": st["ms_apply_p"] / max(st["timed_updates"], 1)},
        "rotations_per_update": rot_per_update,
        "roofline": roof,
        "clocks": clk,
        "e2e": {"value": 1.0 / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": 8 * (M + N), "d2h_bytes_per_step": 8 * (2 * N - 1), "steps": K,
                "path": "bdu_update (pinned host B, C) + bdu_read of d, e per step, wall clock over K updates "
                        "(as many as the device-timed region); the region ends after bdu_flush + bdu_sync "
                        "(the last deferred application included)"},
        "gpu_launches": launches,
        "wall_s_timed": t_wall,
    }
    line["apply_roofline"] = apply_roofline(st, rot_per_update)
    if rank == 0 and world == 1 and args.serving_seconds > 0:
        line["serving"] = serving(args)
    if rank == 0 and world == 1 and not args.no_bhu:
        line["bhu"] = bhu_bench()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample(args.oracle_rows, 1)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_thin(args):
    """Rank-k tracking on the network edge stream (Sec. 4 applied to the
    Chung-Lu edge insertions): wall-clock rank-1 tracking steps per second."""
    import numpy as np
    import torch

    from paper_2509_02840_gb300 import bdu, inputs as I

    m = n = M
    k = args.thin
    Q1, d, e, P1 = I.thin_factors(m, n, k)
    K, W = args.steps, max(args.warmup, 1)
    ups = [I.network_update(n, h) for h in range(W + K)]
    prec = bdu.FP64 if args.thin_fp64 else bdu.MIXED
    with bdu.ThinTracker(Q1, d, e, P1, precision=prec) as T:
        for B, C in ups[:W]:
            for j in range(2):
                T.update(B[:, j], C[:, j])
        torch.cuda.synchronize()
        clocks = Clocks(0)
        clocks.start()
        t0 = time.perf_counter()
        err = 0.0
        for B, C in ups[W:]:
            for j in range(2):
                err += T.update(B[:, j], C[:, j])[1]
        dt = time.perf_counter() - t0
        clk = clocks.stop()
        Qg, dg, eg, Pg = T.read()
    ortho = max(float(np.linalg.norm(Qg.T @ Qg - np.eye(k), 2)), float(np.linalg.norm(Pg.T @ Pg - np.eye(k), 2)))
    steps = 2 * K
    form = "FP64" if args.thin_fp64 else "mixed: FP32 factors, FP64 middle band"
    line = {"metric": f"rank-{k} tracking steps/s at m=n={m} (Sec. 4, {form})", "value": steps / dt,
            "unit": "rank-1 tracking steps/s", "n_gpus": 1, "steps": steps, "warmup": 2 * W,
            "ms_per_step": 1e3 * dt / steps, "higher_is_better": True, "dtype": "f64" if args.thin_fp64 else "f32+f64",
            "data": "synthetic",
            "config": {"workload": f"network edge stream (Chung-Lu, exponent 2.1), m=n={m}, rank {k}",
                       "m": m, "n": n, "k": k},
            "truncation_err2_per_step": err / steps, "orthogonality": ortho, "clocks": clk}
    if not args.no_cpu_baseline:
        import oracle as O
        B, C = ups[0]
        t0 = time.perf_counter()
        O.thin_update(Q1, d, e, P1, B[:, 0], C[:, 0])
        sec = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": 1.0 / sec, "unit": "rank-1 tracking steps/s", "cores": os.cpu_count(),
                                "kind": "oracle", "sample": "one tracking step of the same stream"}
    print(json.dumps(line), flush=True)


def run_network(args):
    """Full factors on the network edge stream (Sec. 4.1: rank-2 symmetric
    edge insertions between Chung-Lu nodes), mixed form: rank-2 updates per
    second, device-timed with B, C resident, the last update's work included."""
    import numpy as np
    import torch

    from paper_2509_02840_gb300 import bdu, inputs as I

    n = M
    K, W = args.steps, max(args.warmup, 1)
    Q0, d0, e0, P0 = I.factorization(n, n, config=3)
    ups = [I.network_update(n, h, config=3) for h in range(W + K)]
    stream = torch.cuda.Stream()
    dev = []
    with torch.cuda.stream(stream):
        for B, C in ups:
            dev.append((torch.from_numpy(np.asfortranarray(B).reshape(-1, order="F")).cuda(),
                        torch.from_numpy(np.asfortranarray(C).reshape(-1, order="F")).cuda()))
    stream.synchronize()
    with bdu.Factorization(Q0, d0, e0, P0, precision=bdu.MIXED, stream=stream.cuda_stream) as F:
        del Q0, P0
        for Bd, Cd in dev[:W]:
            F.update_dev(Bd.data_ptr(), Cd.data_ptr(), 2)
        F.sync()
        st0 = F.stats()
        F.set_timing(True)
        torch.cuda.synchronize()
        clocks = Clocks(0)
        clocks.start()
        with torch.cuda.stream(stream):
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            for Bd, Cd in dev[W:]:
                F.update_dev(Bd.data_ptr(), Cd.data_ptr(), 2)
            F.flush()
            ev1.record(stream)
        stream.synchronize()
        clk = clocks.stop()
        ms = ev0.elapsed_time(ev1)
        st = F.stats()
        q, p = F.check_orthogonality()
    tu = max(st["timed_updates"], 1)
    line = {"metric": f"rank-2 network updates/s at m=n={n} (mixed form)", "value": 1e3 * K / ms,
            "unit": "updates/s", "n_gpus": 1, "steps": K, "warmup": W, "ms_per_step": ms / K,
            "higher_is_better": True, "dtype": "f32 (Q, P) + f64 (projection, rotations, Bd)", "data": "synthetic",
            "config": {"workload": f"network edge stream (Chung-Lu, exponent 2.1), m=n={n}, rank-2 symmetric "
                                   "edge insertions, full factors", "m": n, "n": n, "rank": 2, "form": "mixed",
                       "l2": "not flushed: each update streams > 10 GB"},
            "apply_variant": st["apply_variant"], "orthogonality": {"q": q, "p": p, "tolerance": 1e-5},
            "kernel_ms_per_update": {k: st["ms_" + k] / tu for k in ("project", "chase", "apply_q", "apply_p")},
            "chase_steps_per_update": (st["chase_steps"] - st0["chase_steps"]) / K,
            "clocks": clk, "cpu_baseline": None,
            "note": "no CPU baseline: the oracle does not finish an update at this size in minutes"}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.thin:
        run_thin(args)
        return
    if args.network:
        run_network(args)
        return
    if args.bhu:
        r = bhu_bench(steps=args.steps, shapes=((f"m=n={M}", M, N),))[f"m=n={M}"]
        print(json.dumps({"metric": "BHU updates/s (Algorithm 1, FP64)", "value": r["bhu_updates_per_s"],
                          "unit": "updates/s", "n_gpus": 1, "steps": args.steps, "higher_is_better": True,
                          "dtype": "f64", "data": "synthetic", "config": {"workload": f"recommender m=n={M}"},
                          "bhu": r}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
