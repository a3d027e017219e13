"""Rows/s through the FCT + ℓ1-sampling pass (Figure 2, steps 1-7) on GB300.

One step = fct_embed (Π1·X), l1_condition (QR, M = R⁻¹Π2) and l1_sample (λ,
Σλ, p̂, Bernoulli keep, compaction, coreset gather) over the n = 2^26, d = 64
workload (FP32 A, 0.1% of rows scaled by 1e3, Cauchy(0,1) noise; s = 1024,
r1 = 2130, r2 = 32, m_s = 100000), inputs resident in HBM.  It prints one JSON
line: the step's rows/s (one step captured as a CUDA graph and replayed), the
dominant kernel's algorithmic bytes per second against the measured HBM copy
bandwidth and its issue rate, the end-to-end rate from pinned host memory, the
BF16-streamed form of the same data (tensor-core λ) against the plain FP32 path
with the relative difference of their objectives, the other forms (the n = 2^22,
d = 16 workload plain and as OptimizedFastCauchyRegression, sampling with
replacement and multiple regression; the n = 2^24, d = 32 BF16 workload; a batch
of 256 problems) and the FP64 oracle's rate on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Under torchrun each rank runs its own problem (problem_id = rank) on its own
GPU: weak scaling with no collective on the data path.  `--impl reference`
times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "spiky_n64M_d64"
METRIC = "Rows/s through FCT+ℓ1 sampling, % HBM peak; BF16/batched vs plain FP32"
UNIT = "rows/s"
L2_BYTES = 129 * 2 ** 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-graph", action="store_true",
                    help="time eager calls instead of replays of the step captured as a CUDA graph")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the other forms (measured after the main line's timed region)")
    ap.add_argument("--kernel-case", default=None, choices=sorted(KERNEL_CASES),
                    help="run one small case of one kernel, twice, and exit (for profiler captures; no timing)")
    ap.add_argument("--variants", default="bf16,colscale,optimized,replacement,multi,sct,fct2,t2rows_bf16,batched,canonical",
                    help="comma-separated forms to measure after the main line: bf16 (the main data streamed as "
                         "BF16), colscale (n = 2^22, d = 16, FP32), optimized, replacement, multi, sct (the slow "
                         "Cauchy transform), fct2 (FCT2; these on the n = 2^22 data), t2rows_bf16 (n = 2^24, d = 32, BF16), "
                         "batched, canonical (the canonical-row design of §6.3 at n = 2^26, d = 15: 100 "
                         "coresets and solves from one pass)")
    return ap.parse_args()


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def algorithmic_bytes(n: int, d: int, elem: int, coreset_rows: int) -> dict:
    """Bytes the method must move: X read in phase 1 and phase 2, λ written and read
    back, and the coreset gather (index, weight, FP64 row) — D, C, B, Π2 are
    counter-generated and never stored."""
    q = d + 1
    x_bytes = n * (d * elem + 4)
    phase1 = x_bytes
    phase2 = x_bytes + 4 * n
    phase3 = 4 * n + n // 8 + coreset_rows * (16 + 8 * q + d * elem + 4)
    return {"phase1": phase1, "phase2": phase2, "phase3": phase3, "step": phase1 + phase2 + phase3}


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self) -> dict:
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------- CPU oracle baseline
def cpu_oracle_rows_per_s(pr: dict, w, seconds: float) -> dict:
    """The FP64 oracle as it stands, steps 1-7 (no LP), on a bounded prefix of the workload."""
    import numpy as np

    from oracle import pipeline

    rows = 1 << 17
    A = pr["A"][:rows]
    b = pr["b"][:rows]
    done, t_total, reps = 0, 0.0, 0
    while t_total < seconds or reps == 0:
        t0 = time.perf_counter()
        pipeline.fast_cauchy_regression(A, b, w.s, w.r1, w.r2, w.coreset * rows / w.n, w.seed, w.problem_id,
                                        solve_lp=False)
        t_total += time.perf_counter() - t0
        done += rows
        reps += 1
    threads = None
    try:
        from threadpoolctl import threadpool_info

        threads = max((i.get("num_threads", 1) for i in threadpool_info()), default=1)
    except Exception:
        threads = None
    cores = os.cpu_count()
    return {"value": done / t_total, "unit": UNIT, "cores": threads or cores, "kind": "oracle",
            "sample": f"first {rows} rows of {w.name} (n={w.n}), {reps} passes of Figure 2 steps 1-7 "
                      f"in FP64 numpy, {t_total:.1f} s; m_s scaled to the sample",
            "host_cores": cores}


def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from synth import WORKLOADS, make_problem

    w = WORKLOADS[args.workload]
    pr = make_problem(w, n=1 << 17)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        from oracle import pipeline

        pipeline.fast_cauchy_regression(pr["A"], pr["b"], w.s, w.r1, w.r2, w.coreset * (1 << 17) / w.n,
                                        w.seed, w.problem_id, solve_lp=False)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    rows = 1 << 17
    val = rows * len(times) / sum(times)
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "n": w.n, "d": w.d, "s": w.s, "r1": w.r1,
                                             "r2": w.r2, "coreset": w.coreset, "sample_rows": rows},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step: the FP64 oracle (Figure 2 steps 1-7, numpy) on the "
                                       f"first {rows} rows of {w.name}"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- BF16 and batched forms
def _time_step_ms(step_on, stream, args) -> float:
    """Mean device time of one step enqueued by step_on(stream): captured once as a CUDA
    graph on a side stream and replayed (eager calls on `stream` with --no-graph)."""
    import torch

    if args.no_graph:
        return _time_ms(lambda: step_on(stream), stream, args.warmup, args.steps)
    gs = torch.cuda.Stream(stream.device)
    with torch.cuda.stream(gs):
        step_on(gs)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=gs):
        step_on(gs)
    with torch.cuda.stream(gs):
        ms = _time_ms(g.replay, gs, args.warmup, args.steps)
    return ms


def _time_ms(step, stream, warmup: int, steps: int) -> float:
    """Mean device time of one step: CUDA events on `stream` around `steps` back-to-back steps."""
    import torch

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def _phase_ms(L, A, b, prm, cap, q, dev, stream, warmup, steps) -> dict:
    import torch

    R = torch.empty((q, q), dtype=torch.float64, device=dev)
    M = torch.empty((q, prm.r2), dtype=torch.float64, device=dev)
    pix = torch.empty((prm.r1, q), dtype=torch.float32, device=dev)
    idx = torch.empty(cap, dtype=torch.int64, device=dev)
    wts = torch.empty(cap, dtype=torch.float64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    n, d = A.shape
    ws = L.workspace(prm, n, d, L.BF16 if A.dtype == torch.bfloat16 else L.F32, device=dev)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    acc = [0.0, 0.0, 0.0]
    for it in range(warmup + steps):
        evs[0].record(stream)
        L.fct_embed(A, b, prm, pix, ws, stream=stream)
        evs[1].record(stream)
        L.l1_condition(pix, prm, R, M, ws, stream=stream)
        evs[2].record(stream)
        L.l1_sample(A, b, M, prm, cap, idx, wts, None, cnt, None, ws, stream=stream)
        evs[3].record(stream)
        if it >= warmup:
            torch.cuda.synchronize(dev)
            for k in range(3):
                acc[k] += evs[k].elapsed_time(evs[k + 1])
    return dict(zip(["fct_embed", "l1_condition", "l1_sample"], [a / steps for a in acc]))


def bf16_same_data_variant(L, dev, stream, args, A32, b, w, peak: float, ws32, f32_ms: float) -> dict:
    """The main workload streamed as BF16 (A rounded once, nearest even; λ on tcgen05 tensor
    cores) against the plain FP32 path on the original FP32 data: rows/s of each and the
    relative difference of the objectives ‖A·x̂ − b‖₁, both evaluated on the FP32 data."""
    import torch

    n, d = A32.shape
    q = d + 1
    A16 = A32.to(torch.bfloat16)
    prm = L.make_params(w.s, w.r1, w.r2, w.coreset, seed=w.seed, problem_id=w.problem_id)
    cap = int(2 * w.coreset) + 64
    ws16 = L.workspace(prm, n, d, L.BF16, device=dev)
    idx = torch.empty(cap, dtype=torch.int64, device=dev)
    wts = torch.empty(cap, dtype=torch.float64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    ms = _time_step_ms(lambda st: L.l1_coreset(A16, b, prm, cap, idx, wts, None, cnt, ws16, stream=st), stream, args)
    kept = int(cnt.item())
    ab = algorithmic_bytes(n, d, 2, kept)["step"]
    phase = _phase_ms(L, A16, b, prm, cap, q, dev, stream, 2, max(3, args.steps // 4))
    x16, f16_own, rows16, rc16 = L.l1_regress(A16, b, prm, ws16, stream=stream)
    x32, f32, rows32, rc32 = L.l1_regress(A32, b, prm, ws32, stream=stream)
    out = torch.empty(1, dtype=torch.float64, device=dev)
    L.l1_objective(A32, b, x16.to(dev), out, ws32, stream=stream)
    f16_on32 = float(out.item())
    del ws16, A16
    return {"workload": f"{w.name} streamed as BF16", "value": n / (ms / 1e3), "ms_per_step": ms,
            "step_gbs": ab / (ms / 1e3) / 1e9, "step_frac": ab / (ms / 1e3) / 1e9 / peak, "algorithmic_bytes": ab,
            "coreset_rows": kept, "phase_ms": phase, "status": rc16,
            "objective_bf16_on_f32_data": f16_on32, "objective_f32": f32, "objective_bf16_own_data": f16_own,
            "objective_rel_err_vs_f32": abs(f16_on32 - f32) / f32, "f32_status": rc32,
            "speedup_vs_f32": f32_ms / ms}


def colscale_variant(L, dev, stream, args, peak: float) -> tuple:
    """The n = 2^22, d = 16 FP32 workload (columns scaled by 10^U(−2,2)): the plain pass as CUDA-
    graph replays, its phase split and the phase-1 kernel's share of HBM.  Returns the line and
    the device inputs, which the forms measured on this data reuse."""
    import torch

    from synth import WORKLOADS, make_problem

    w = WORKLOADS["colscale_n4M_d16"]
    pr = make_problem(w)
    n, d = pr["A"].shape
    q = d + 1
    A = torch.from_numpy(pr["A"]).to(dev)
    b = torch.from_numpy(pr["b"]).to(dev)
    prm = L.make_params(w.s, w.r1, w.r2, w.coreset, seed=w.seed, problem_id=w.problem_id)
    ws = L.workspace(prm, n, d, device=dev)
    cap = int(2 * w.coreset) + 64
    idx = torch.empty(cap, dtype=torch.int64, device=dev)
    wts = torch.empty(cap, dtype=torch.float64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    ms = _time_step_ms(lambda st: L.l1_coreset(A, b, prm, cap, idx, wts, None, cnt, ws, stream=st), stream, args)
    kept = int(cnt.item())
    ab = algorithmic_bytes(n, d, 4, kept)
    phase = _phase_ms(L, A, b, prm, cap, q, dev, stream, 2, max(3, args.steps // 4))
    del ws
    return ({"workload": w.name, "n": n, "d": d, "s": w.s, "r1": w.r1, "r2": w.r2, "coreset": w.coreset,
             "value": n / (ms / 1e3), "ms_per_step": ms, "step_frac": ab["step"] / (ms / 1e3) / 1e9 / peak,
             "phase_ms": phase, "phase1_frac": ab["phase1"] / (phase["fct_embed"] / 1e3) / 1e9 / peak,
             "coreset_rows": kept}, A, b, w)


def sct_variant(L, dev, stream, args, A, b, w, plain_ms: float, fct1_ms: float) -> dict:
    """The slow Cauchy transform as Π1 (§3; the conditioning of §6.3) on the same data:
    steps 1-7 with Π1·X = (4/r1)·C·X.  Its cost is drawing r1·n Cauchy variates (one Philox
    call per four), so its phase 1 is reported against the SM issue rate, not HBM."""
    import torch

    n, d = A.shape
    q = d + 1
    prm = L.make_params(1, w.r1, w.r2, w.coreset, seed=w.seed, problem_id=w.problem_id, transform=1)
    ws = L.workspace(prm, n, d, device=dev)
    cap = int(2 * w.coreset) + 64
    idx = torch.empty(cap, dtype=torch.int64, device=dev)
    wts = torch.empty(cap, dtype=torch.float64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    ms = _time_step_ms(lambda st: L.l1_coreset(A, b, prm, cap, idx, wts, None, cnt, ws, stream=st), stream, args)
    kept = int(cnt.item())
    phase = _phase_ms(L, A, b, prm, cap, q, dev, stream, 2, max(3, args.steps // 4))
    del ws
    variates = n * w.r1
    return {"workload": w.name, "transform": "slow Cauchy transform (4/r1)*C", "value": n / (ms / 1e3),
            "ms_per_step": ms, "phase_ms": phase, "coreset_rows": kept,
            "variates_per_s": variates / (phase["fct_embed"] / 1e3),
            "fma_per_s": variates * q / (phase["fct_embed"] / 1e3),
            "phase1_vs_fct1": phase["fct_embed"] / fct1_ms, "speedup_vs_f32_plain": plain_ms / ms}


# Quartiles of the Cauchy-conditioned sampling (CT) row of the relative-error table of §6.3,
# the paper's result on its 5.24e9 × 15 instance: context for this scaled instance, not a target.
PAPER_CT_QUARTILES = {"l1": [0.008, 0.0115], "l2": [0.00895, 0.0146], "linf": [0.0113, 0.0211]}


def canonical_variant(L, dev, stream, args) -> dict:
    """The large-scale experiment of §6.3 scaled to one GPU: the imbalanced, corrupted
    canonical-row design at n = 2^26, d = 15, the slow Cauchy transform as Π1 (the paper's CT)
    and, for comparison, FCT1; 100 coresets of about 10^5 rows from one λ and their 100 solves
    side by side.  Reports each phase's device time, rows/s of the whole 100-solution pass, and
    the quartiles over the 100 solutions of the 1-, 2- and ∞-norm distance from the optimal box
    (per-coordinate medians), relative to the optimum, with entry-wise quartiles."""
    import numpy as np
    import torch

    from paper_1207_4684_gb300 import validation
    from synth import canonical_design, r1_for

    n, d, k, m = 1 << 26, 15, 100, 1e5
    cd = canonical_design(n, d, seed=0)
    cols = torch.from_numpy(cd["cols"]).to(dev).long()
    A = torch.zeros((n, d), dtype=torch.float32, device=dev)
    A.scatter_(1, cols[:, None], 1.0)
    b = torch.from_numpy(cd["b"]).to(dev)
    lo, hi = validation.canonical_box(cols, b, d)
    del cd
    out = {"workload": "canonical_n64M_d15", "n": n, "d": d, "k": k, "coreset": m, "r1": r1_for(d), "r2": 16,
           "irls_max_iter": 20,
           "paper_ct_quartiles": PAPER_CT_QUARTILES}
    for name, prm in (("ct", L.make_params(1, r1_for(d), 16, m, seed=0, transform=1)),
                      ("fct1", L.make_params(128, r1_for(d), 16, m, seed=0))):
        # IRLS capped at 20 iterations: the simplex finish certifies each coreset's optimum, and
        # on this design the certified objectives equal those after 100 iterations (the finish
        # from a rougher start costs less than the FP64 iterations it saves here; on dense
        # Gaussian coresets it does not, so the library's default stays at 100).
        validation.many_solutions(A, b, prm, k, max_iter=20, stream=stream)          # warm-up
        torch.cuda.synchronize()
        res = validation.many_solutions(A, b, prm, k, max_iter=20, stream=stream)
        err = validation.box_errors(res["x"], lo, hi)
        xs = res["x"].cpu().numpy()
        ent = np.maximum(0.0, np.maximum(lo.numpy()[None, :] - xs, xs - hi.numpy()[None, :]))
        total = sum(res["phase_ms"].values())
        out[name] = {
            "phase_ms": res["phase_ms"], "ms_per_pass": total, "rows_per_s": n / (total / 1e3),
            "status": res["status"], "solves_flagged": int((res["solve_flags"] != 0).sum().item()),
            "coreset_rows_median": float(res["count"].double().median().item()),
            "quartiles": {key: [float(np.percentile(v, 25)), float(np.percentile(v, 75))] for key, v in err.items()},
            "entrywise_abs_quartiles": [[float(np.percentile(ent[:, j], 25)), float(np.percentile(ent[:, j], 75))]
                                        for j in range(d)],
        }
        del res
        torch.cuda.empty_cache()
    del A, b, cols
    torch.cuda.empty_cache()
    return out


def fct2_variant(L, dev, stream, args, A, b, w, plain_ms: float, fct1_ms: float) -> dict:
    """FCT2 as Π1 (§3.2) on the same data: one SRHT block G (s = ⌈2d ln d⌉ of t = 2^⌈log₂ 2d²⌉
    rows kept) per t rows of X, then the slow Cauchy transform on the ns/t rows of H̃X."""
    import torch

    n, d = A.shape
    q = d + 1
    t = 1 << math.ceil(math.log2(2 * d * d))
    sf = math.ceil(2 * d * math.log(d))
    prm = L.make_params(t, w.r1, w.r2, w.coreset, seed=w.seed, problem_id=w.problem_id, transform=2, fjlt_rows=sf)
    ws = L.workspace(prm, n, d, device=dev)
    cap = int(2 * w.coreset) + 64
    idx = torch.empty(cap, dtype=torch.int64, device=dev)
    wts = torch.empty(cap, dtype=torch.float64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    ms = _time_step_ms(lambda st: L.l1_coreset(A, b, prm, cap, idx, wts, None, cnt, ws, stream=st), stream, args)
    kept = int(cnt.item())
    phase = _phase_ms(L, A, b, prm, cap, q, dev, stream, 2, max(3, args.steps // 4))
    del ws
    return {"workload": w.name, "transform": f"FCT2: SRHT blocks of t = {t} rows keeping s = {sf}, then (8/r1)*sqrt(pi*t/(2s))*C",
            "value": n / (ms / 1e3), "ms_per_step": ms, "phase_ms": phase, "coreset_rows": kept,
            "rows_of_HX": (-(-n // t)) * sf, "phase1_vs_fct1": phase["fct_embed"] / fct1_ms,
            "speedup_vs_f32_plain": plain_ms / ms}


def bf16_variant(L, dev, stream, args, peak: float) -> dict:
    """The mixed-precision form (A streamed as BF16, λ on tcgen05 tensor cores) against the plain
    FP32 path on the same values widened to FP32: rows/s of each, and the relative difference of
    the final objectives ‖A·x̂ − b‖₁ after the coreset solve."""
    import numpy as np
    import torch

    from synth import WORKLOADS, make_problem

    w = WORKLOADS["t2rows_n16M_d32_bf16"]
    pr = make_problem(w)
    n, d = pr["A"].shape
    q = d + 1
    A16 = torch.from_numpy(pr["A"].view(np.int16)).view(torch.bfloat16).to(dev)
    A32 = A16.float()
    b = torch.from_numpy(pr["b"]).to(dev)
    del pr
    prm = L.make_params(w.s, w.r1, w.r2, w.coreset, seed=w.seed, problem_id=w.problem_id)
    cap = int(2 * w.coreset) + 64
    ws = L.workspace(prm, n, d, L.F32, device=dev)
    assert ws.numel() >= L.l1s_workspace_size(prm, n, d, L.BF16)
    idx = torch.empty(cap, dtype=torch.int64, device=dev)
    wts = torch.empty(cap, dtype=torch.float64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    out = {"workload": w.name, "n": n, "d": d, "s": w.s, "r1": w.r1, "r2": w.r2, "coreset": w.coreset}
    for tag, A, elem in (("bf16", A16, 2), ("f32", A32, 4)):
        ms = _time_step_ms(lambda st: L.l1_coreset(A, b, prm, cap, idx, wts, None, cnt, ws, stream=st), stream, args)
        kept = int(cnt.item())
        ab = algorithmic_bytes(n, d, elem, kept)["step"]
        x, f, rows, rc = L.l1_regress(A, b, prm, ws, stream=stream)
        out[tag] = {"value": n / (ms / 1e3), "ms_per_step": ms, "step_gbs": ab / (ms / 1e3) / 1e9,
                    "step_frac": ab / (ms / 1e3) / 1e9 / peak, "algorithmic_bytes": ab, "coreset_rows": kept,
                    "objective": f, "status": rc,
                    "phase_ms": _phase_ms(L, A, b, prm, cap, q, dev, stream, 2, max(3, args.steps // 4))}
    f16, f32 = out["bf16"]["objective"], out["f32"]["objective"]
    out["objective_rel_err_vs_f32"] = abs(f16 - f32) / f32
    out["speedup_vs_f32"] = out["bf16"]["value"] / out["f32"]["value"]
    return out


def batched_variant(L, dev, stream, args, peak: float) -> dict:
    """256 independent regressions of uneven n and d in one l1_regress_batched call, schedules
    picked by l1s_autotune per (d, s), the call captured into one CUDA graph and replayed."""
    import torch

    from synth import make_batched_problems

    t0 = time.perf_counter()
    prs = make_batched_problems(256)
    gen_s = time.perf_counter() - t0
    members = []
    for pr in prs:
        w = pr["w"]
        A = torch.from_numpy(pr["A"]).to(dev)
        b = torch.from_numpy(pr["b"]).to(dev)
        prm = L.make_params(w.s, w.r1, w.r2, w.coreset, seed=w.seed, problem_id=w.problem_id)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        members.append(dict(w=w, A=A, b=b, prm=prm, cnt=cnt))
    del prs
    # Autotune one representative (the largest n) per (d, s).
    tuned = {}
    t0 = time.perf_counter()
    for m in sorted(members, key=lambda m: -m["w"].n):
        key = (m["w"].d, m["w"].s)
        if key in tuned:
            continue
        ws1 = L.workspace(m["prm"], m["w"].n, m["w"].d, device=dev)
        sched, ms = L.l1s_autotune(L.make_problem(m["A"], m["b"], m["prm"]), ws1, trials=3, stream=stream)
        tuned[key] = {"schedule": sched, "ms": ms, "n": m["w"].n}
        del ws1
    tune_s = time.perf_counter() - t0
    probs = [L.make_problem(m["A"], m["b"], m["prm"], count=m["cnt"]) for m in members]
    ws = L.batched_workspace(probs, device=dev)
    flags = torch.zeros(len(probs), dtype=torch.int32, device=dev)
    side = torch.cuda.Stream(dev)   # graphs are not captured on the legacy default stream
    side.wait_stream(stream)

    def eager():
        L.l1_regress_batched(probs, ws, flags, stream=side)

    with torch.cuda.stream(side):
        c0 = L.l1s_kernel_launches()
        eager()
        launches = L.l1s_kernel_launches() - c0
        eager_ms = _time_ms(eager, side, args.warmup, args.steps)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            eager()
        graph_ms = _time_ms(g.replay, side, args.warmup, args.steps)
    torch.cuda.synchronize()
    fl = flags.cpu().numpy()
    # The batched form against the plain FP32 path (outside the timed region): 16 members,
    # spread over every d, solved through the batch (x̂ and ‖Ax̂ − b‖₁ per member) and one by
    # one through l1_regress; the relative difference of their objectives.
    pick = sorted(range(len(members)), key=lambda i: (members[i]["w"].d, members[i]["w"].n))[::16][:16]
    xs = [torch.empty(members[i]["w"].d, dtype=torch.float64, device=dev) for i in pick]
    objs = [torch.empty(1, dtype=torch.float64, device=dev) for _ in pick]
    sub = [L.make_problem(members[i]["A"], members[i]["b"], members[i]["prm"], x=xs[k], objective=objs[k])
           for k, i in enumerate(pick)]
    sub_ws = L.batched_workspace(sub, device=dev)
    sub_flags = torch.zeros(len(sub), dtype=torch.int32, device=dev)
    L.l1_regress_batched(sub, sub_ws, sub_flags, stream=side)
    torch.cuda.synchronize()
    errs = []
    for k, i in enumerate(pick):
        m = members[i]
        ws1 = L.workspace(m["prm"], m["w"].n, m["w"].d, device=dev)
        _, f_plain, _, rc = L.l1_regress(m["A"], m["b"], m["prm"], ws1, stream=stream)
        errs.append(abs(float(objs[k].item()) - f_plain) / f_plain)
        del ws1
    del sub_ws
    rows = sum(m["w"].n for m in members)
    ab = sum(algorithmic_bytes(m["w"].n, m["w"].d, 4, int(m["cnt"].item()))["step"] for m in members)
    ds = sorted({m["w"].d for m in members})
    return {"workload": "batched_256_n2^12..2^20_d4..64", "problems": len(members), "rows": rows,
            "value": rows / (graph_ms / 1e3), "ms_per_step": graph_ms, "graph": True,
            "eager": {"value": rows / (eager_ms / 1e3), "ms_per_step": eager_ms},
            "step_gbs": ab / (graph_ms / 1e3) / 1e9, "step_frac": ab / (graph_ms / 1e3) / 1e9 / peak,
            "algorithmic_bytes": ab, "gpu_launches_per_step": launches,
            "status_nonzero": int((fl != 0).sum()),
            "objective_rel_err_vs_plain": {"members": len(pick), "max": max(errs), "median": float(sorted(errs)[len(errs) // 2]),
                                           "solve_status_nonzero": int((sub_flags != 0).sum().item())},
            "d_values": ds, "s_by_d": {str(m["w"].d): m["w"].s for m in members},
            "autotuned": {f"d{k[0]}_s{k[1]}": v for k, v in sorted(tuned.items())},
            "host_s": {"generate": gen_s, "autotune": tune_s}}


def optimized_variant(L, dev, stream, args, A, b, w, peak: float, plain_ms: float) -> dict:
    """OptimizedFastCauchyRegression (Figure "mainOpt") on the same data: Gaussian Π2 with
    r2 = 8 and p̂ = min(1, s·λ̂) without Σλ.  s is calibrated once, outside the timed region,
    so that the expected coreset size is m_s (from one λ pass with the same Π1 and Π2)."""
    import torch

    n, d = A.shape
    q = d + 1
    r2 = 8
    prm0 = L.make_params(w.s, w.r1, r2, w.coreset, seed=w.seed, problem_id=w.problem_id, variant=1,
                         sample_scale=1.0)
    ws = L.workspace(prm0, n, d, device=dev)
    pix = torch.empty((w.r1, q), dtype=torch.float32, device=dev)
    R = torch.empty((q, q), dtype=torch.float64, device=dev)
    M = torch.empty((q, r2), dtype=torch.float64, device=dev)
    lam = torch.empty(n, dtype=torch.float32, device=dev)
    tot = torch.zeros(1, dtype=torch.float64, device=dev)
    L.fct_embed(A, b, prm0, pix, ws, stream=stream)
    L.l1_condition(pix, prm0, R, M, ws, stream=stream)
    L.l1_lambda(A, b, M, prm0, lam, tot, ws, stream=stream)
    torch.cuda.synchronize()
    scale = w.coreset / float(tot.item())
    prm = L.make_params(w.s, w.r1, r2, w.coreset, seed=w.seed, problem_id=w.problem_id, variant=1,
                        sample_scale=scale)
    cap = int(2 * w.coreset) + 64
    idx = torch.empty(cap, dtype=torch.int64, device=dev)
    wts = torch.empty(cap, dtype=torch.float64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    ms = _time_step_ms(lambda st: L.l1_coreset(A, b, prm, cap, idx, wts, None, cnt, ws, stream=st), stream, args)
    kept = int(cnt.item())
    flags = L.l1s_status_read(ws, stream=stream)
    # λ̂ and the keep decision share one pass: no λ write and read back (8 bytes per row)
    ab = algorithmic_bytes(n, d, 4, kept)["step"] - 8 * n
    return {"workload": w.name, "variant": "OptimizedFastCauchyRegression (Gaussian Pi2, r2 = 8, no Sum(lambda))",
            "r2": r2, "sample_scale": scale, "value": n / (ms / 1e3), "ms_per_step": ms,
            "step_frac": ab / (ms / 1e3) / 1e9 / peak, "coreset_rows": kept, "status": flags,
            "speedup_vs_f32_plain": plain_ms / ms}


def replacement_variant(L, dev, stream, args, A, b, w, peak: float, plain_ms: float) -> dict:
    """Exactly m_s draws with replacement, p̂_i = λ_i/Σλ (the caption of Figure 2), on the
    same data: steps 1-5, the running sum of λ and the m_s draws."""
    import torch

    n, d = A.shape
    m = int(w.coreset)
    prm = L.make_params(w.s, w.r1, w.r2, float(m), seed=w.seed, problem_id=w.problem_id, variant=2)
    ws = L.workspace(prm, n, d, device=dev)
    cap = 2 * m + 64
    idx = torch.empty(cap, dtype=torch.int64, device=dev)
    wts = torch.empty(cap, dtype=torch.float64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    ms = _time_step_ms(lambda st: L.l1_coreset(A, b, prm, cap, idx, wts, None, cnt, ws, stream=st), stream, args)
    flags = L.l1s_status_read(ws, stream=stream)
    # X twice, λ written and read twice (sum, running sum), C written (8 bytes per row), the draws
    ab = 2 * n * (d * 4 + 4) + 4 * n + 8 * n + 8 * n + m * (16 + 8 * (d + 1) + d * 4 + 4)
    return {"workload": w.name, "variant": "FastCauchyRegression, m_s draws with replacement", "draws": m,
            "value": n / (ms / 1e3), "ms_per_step": ms, "step_frac": ab / (ms / 1e3) / 1e9 / peak,
            "status": flags, "speedup_vs_f32_plain": plain_ms / ms}


def multi_variant(L, dev, stream, args, A, b, w, peak: float) -> dict:
    """Multiple regression (§4.2.1) on the same design: X = [A | B] with k = 4 right-hand
    sides (b and three more columns A·w_j + Laplace noise with 5% 100·Cauchy outliers),
    one coreset for all of them (steps 1-7 on q = d + k columns)."""
    import numpy as np
    import torch

    n, d = A.shape
    k = 4
    g = np.random.default_rng(w.seed + 77)
    extra = torch.empty((n, k - 1), dtype=torch.float32)
    Ah = A.cpu().numpy()
    for j in range(k - 1):
        e = g.laplace(size=n)
        out = g.random(n) < 0.05
        e[out] = 100.0 * g.standard_cauchy(int(out.sum()))
        extra[:, j] = torch.from_numpy((Ah.astype(np.float64) @ g.standard_normal(d) + e).astype(np.float32))
    X = torch.cat([A, b[:, None], extra.to(dev)], dim=1).contiguous()
    del Ah, extra
    from synth import r1_for

    prm = L.make_params(w.s, r1_for(d + k), w.r2, w.coreset, seed=w.seed, problem_id=w.problem_id)
    ws = L.multi_workspace(prm, n, d, k, device=dev)
    cap = int(2 * w.coreset) + 64
    idx = torch.empty(cap, dtype=torch.int64, device=dev)
    wts = torch.empty(cap, dtype=torch.float64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    ms = _time_step_ms(lambda st: L.l1_coreset_multi(X, k, prm, cap, idx, wts, None, cnt, ws, stream=st), stream, args)
    kept = int(cnt.item())
    flags = L.l1s_status_read(ws, stream=stream)
    # the passes read d + k − 1 columns of X and B_k gathered once (read + write 4 bytes per row)
    ab = algorithmic_bytes(n, d + k - 1, 4, kept)["step"] + 8 * n
    return {"workload": f"{w.name} with k = {k} right-hand sides", "k": k, "q": d + k, "r1": prm.r1,
            "value": n / (ms / 1e3),
            "ms_per_step": ms, "step_frac": ab / (ms / 1e3) / 1e9 / peak, "coreset_rows": kept,
            "status": flags}


# ----------------------------------------------------------------- GPU arm
def _parse_cpulist(txt: str) -> set:
    cpus = set()
    for part in txt.strip().split(","):
        if not part:
            continue
        lo, _, hi = part.partition("-")
        cpus.update(range(int(lo), int(hi or lo) + 1))
    return cpus


def bind_near_gpu(dev) -> str:
    """Run this process on the CPUs local to the GPU (sysfs local_cpulist of its PCI
    device), so that pinned host buffers are allocated in the memory next to it and the
    host→device copies of the end-to-end number do not cross the CPU-to-CPU link."""
    import torch

    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid).lower().replace("gpu-", "")
        out = subprocess.run(["nvidia-smi", "--query-gpu=uuid,pci.bus_id", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=30).stdout
        bus = None
        for line in out.splitlines():
            u, _, b = (x.strip() for x in line.partition(","))
            if u.lower().replace("gpu-", "") == uuid:
                bus = b.lower()
        if bus is None:
            return "unbound: GPU not found in nvidia-smi"
        dom, rest = bus.split(":", 1)
        path = f"/sys/bus/pci/devices/{dom[-4:]}:{rest}/local_cpulist"
        cpus = _parse_cpulist(open(path).read()) & os.sched_getaffinity(0)
        if not cpus:
            return "unbound: no local CPUs available"
        os.sched_setaffinity(0, cpus)
        return f"{len(cpus)} CPUs local to the GPU"
    except Exception as e:  # noqa: BLE001 - diagnostics only
        return f"unbound: {type(e).__name__}"


def run_gpu(args) -> None:
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    host_binding = bind_near_gpu(dev)

    import __graft_entry__

    __graft_entry__.build()
    import paper_1207_4684_gb300 as L
    from synth import WORKLOADS, make_problem

    w = WORKLOADS[args.workload]
    pr = make_problem(w)
    n, d = pr["A"].shape
    q = d + 1
    bf16 = pr["A"].dtype == np.uint16
    dt = L.BF16 if bf16 else L.F32
    elem = 2 if bf16 else 4
    if bf16:
        A = torch.from_numpy(pr["A"].view(np.int16)).view(torch.bfloat16).to(dev)
    else:
        A = torch.from_numpy(pr["A"]).to(dev)
    b = torch.from_numpy(pr["b"]).to(dev)
    prm = L.make_params(w.s, w.r1, w.r2, w.coreset, seed=w.seed, problem_id=rank)
    ws = L.workspace(prm, n, d, dt, device=dev)
    cap = int(2 * w.coreset) + 64
    idx = torch.empty(cap, dtype=torch.int64, device=dev)
    wts = torch.empty(cap, dtype=torch.float64, device=dev)
    core = torch.empty((cap, q), dtype=torch.float64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        L.l1_coreset(A, b, prm, cap, idx, wts, core, cnt, ws, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    flags = L.l1s_status_read(ws)
    kept = int(cnt.item())

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # One step captured as a CUDA graph on a side stream: the same launches, replayed
    # without the host's per-call planning.  The eager calls are timed too.
    gstream = torch.cuda.Stream(dev)
    graph = None
    per_step_launches = None
    if not args.no_graph:
        with torch.cuda.stream(gstream):
            L.l1_coreset(A, b, prm, cap, idx, wts, core, cnt, ws, stream=gstream)
        torch.cuda.synchronize(dev)
        graph = torch.cuda.CUDAGraph()
        c0 = L.l1s_kernel_launches()
        with torch.cuda.graph(graph, stream=gstream):
            L.l1_coreset(A, b, prm, cap, idx, wts, core, cnt, ws, stream=gstream)
        per_step_launches = L.l1s_kernel_launches() - c0
        for _ in range(args.warmup):
            graph.replay()
        torch.cuda.synchronize(dev)
    eager_ms = _time_ms(step, stream, 0, args.steps)

    # ---- timed region: K steps, CUDA events on the launching stream
    tstream = gstream if graph is not None else stream
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk, torch.cuda.stream(tstream):
        barrier()
        t_host0 = time.perf_counter()
        launches0 = L.l1s_kernel_launches()
        ev0.record(tstream)
        for _ in range(args.steps):
            if graph is not None:
                graph.replay()
            else:
                step()
        ev1.record(tstream)
        launches = L.l1s_kernel_launches() - launches0
        if graph is not None:
            launches = per_step_launches * args.steps      # graph nodes: counted at capture
        barrier()
        t_host = time.perf_counter() - t_host0
    gpu_ms = ev0.elapsed_time(ev1)
    if world > 1:
        t = torch.tensor([gpu_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        gpu_ms = float(t.item())
    ms_per_step = gpu_ms / args.steps
    value = world * n * args.steps / (gpu_ms / 1e3)

    # ---- per-phase times (same work, split into the three entry points with events between)
    R = torch.empty((q, q), dtype=torch.float64, device=dev)
    M = torch.empty((q, w.r2), dtype=torch.float64, device=dev)
    pix = torch.empty((w.r1, q), dtype=torch.float32, device=dev)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    acc = [0.0, 0.0, 0.0]
    for it in range(args.warmup + args.steps):
        evs[0].record(stream)
        L.fct_embed(A, b, prm, pix, ws, stream=stream)
        evs[1].record(stream)
        L.l1_condition(pix, prm, R, M, ws, stream=stream)
        evs[2].record(stream)
        L.l1_sample(A, b, M, prm, cap, idx, wts, core, cnt, None, ws, stream=stream)
        evs[3].record(stream)
        if it >= args.warmup:
            torch.cuda.synchronize(dev)
            for k in range(3):
                acc[k] += evs[k].elapsed_time(evs[k + 1])
    phase_ms = [a / args.steps for a in acc]

    # ---- end to end through the public API with host buffers (copies inside the timed region)
    ws_h = L.workspace(prm, n, d, dt, host_staging=True, device=dev)
    A_h = torch.from_numpy(pr["A"].view(np.int16) if bf16 else pr["A"]).pin_memory()
    b_h = torch.from_numpy(pr["b"]).pin_memory()
    idx_h = torch.empty(cap, dtype=torch.int64).pin_memory()
    w_h = torch.empty(cap, dtype=torch.float64).pin_memory()
    cnt_h = torch.zeros(1, dtype=torch.int64)
    e2e_steps = max(3, min(args.steps, 10))
    # the host link's own rate for the same bytes (a plain pinned copy), for reference
    dst = torch.empty(A_h.numel() * A_h.element_size(), dtype=torch.uint8, device=dev)
    src = A_h.view(-1).view(torch.uint8)
    h2d = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            dst.copy_(src, non_blocking=True)
            e1.record(stream)
        e1.synchronize()
        h2d.append(dst.numel() / (e0.elapsed_time(e1) / 1e3) / 1e9)
    del dst
    h2d_gbs = statistics.median(h2d)
    for _ in range(2):
        L.l1_coreset_host(A_h, b_h, prm, cap, idx_h, w_h, cnt_h, ws_h, stream=stream)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        rc = L.l1_coreset_host(A_h, b_h, prm, cap, idx_h, w_h, cnt_h, ws_h, stream=stream)
    barrier()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if world > 1:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    del ws_h, A_h, b_h

    # ---- roofline of the dominant kernel (phase-level events bracket it)
    peaks = measured_peaks()
    ab = algorithmic_bytes(n, d, elem, kept)
    names = ["fct_embed", "l1_condition", "l1_sample"]
    dom = max(range(3), key=lambda k: phase_ms[k])
    dom_bytes = [ab["phase1"], 0, ab["phase2"] + ab["phase3"]][dom]
    achieved = dom_bytes / (phase_ms[dom] / 1e3) / 1e9
    step_gbs = ab["step"] / (ms_per_step / 1e3) / 1e9
    traffic = instr = None
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(prof):
        with open(prof) as f:
            tr = json.load(f)
        traffic = tr.get(f"{names[dom]}:{w.name}")
        instr = tr.get(f"{names[dom]}:{w.name}:warp_instructions")

    clocks = clk.summary()
    # The phase-1 kernel is bound by instruction issue and shared-memory atomics, not by
    # HBM: its issue rate against 4 warp instructions per cycle per SM at the sampled clock
    # (warp instructions per launch from the ncu capture in profiles/).
    issue = None
    if instr and clocks.get("sm_mhz"):
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        ach = instr / (phase_ms[dom] / 1e3)
        pk = sms * 4 * clocks["sm_mhz"] * 1e6
        issue = {"warp_instructions": instr, "achieved_per_s": ach, "peak_per_s": pk, "frac": ach / pk,
                 "peak_basis": f"{sms} SMs x 4 warp instructions per cycle x sampled SM clock"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16" if bf16 else "f32", "data": "synthetic",
        "config": {"workload": w.name, "n": n, "d": d, "q": q, "s": w.s, "r1": w.r1, "r2": w.r2,
                   "coreset": w.coreset, "parallelism": f"replicas{world}",
                   "l2": f"inputs {n * (d * elem + 4) / 2**20:.0f} MiB exceed the {L2_BYTES // 2**20} MiB L2; no flush"},
        "roofline": {"kernel": names[dom], "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                     "peak_source": peaks["source"], "algorithmic_bytes": dom_bytes,
                     "launch_ms": phase_ms[dom], "issue": issue},
        "step_roofline": {"achieved": step_gbs, "frac": step_gbs / peaks["hbm_gbs"],
                          "algorithmic_bytes": ab["step"]},
        "phase_ms": dict(zip(names, phase_ms)),
        "launch": {"mode": "cuda_graph" if graph is not None else "eager", "eager_ms_per_step": eager_ms,
                   "launches_per_step": per_step_launches if graph is not None else launches // max(args.steps, 1)},
        "e2e": {"value": world * n / e2e_s, "unit": UNIT, "h2d_bytes_per_step": n * (d * elem + 4),
                "d2h_bytes_per_step": 8 + cap * 16, "status": rc, "host": host_binding,
                "h2d_copy_gbs": h2d_gbs},
        "gpu_launches": launches,
        "clocks": clocks,
        "coreset_rows": kept, "status_flags": flags, "host_wall_s": t_host,
    }
    if rank == 0 and not args.no_variants and world == 1:
        want = {v.strip() for v in args.variants.split(",") if v.strip()}
        variants = {}
        if "bf16" in want and w.dtype == "f32":
            variants["bf16"] = bf16_same_data_variant(L, dev, stream, args, A, b, w, peaks["hbm_gbs"], ws, ms_per_step)
        del ws, A, b
        torch.cuda.empty_cache()
        if want & {"colscale", "optimized", "replacement", "multi", "sct", "fct2"}:
            line_c, A1, b1, w1 = colscale_variant(L, dev, stream, args, peaks["hbm_gbs"])
            if "colscale" in want:
                variants["colscale"] = line_c
            if "optimized" in want:
                variants["optimized"] = optimized_variant(L, dev, stream, args, A1, b1, w1, peaks["hbm_gbs"],
                                                          line_c["ms_per_step"])
            torch.cuda.empty_cache()
            if "replacement" in want:
                variants["replacement"] = replacement_variant(L, dev, stream, args, A1, b1, w1, peaks["hbm_gbs"],
                                                              line_c["ms_per_step"])
            torch.cuda.empty_cache()
            if "multi" in want:
                variants["multi"] = multi_variant(L, dev, stream, args, A1, b1, w1, peaks["hbm_gbs"])
            torch.cuda.empty_cache()
            if "sct" in want:
                variants["sct"] = sct_variant(L, dev, stream, args, A1, b1, w1, line_c["ms_per_step"],
                                              line_c["phase_ms"]["fct_embed"])
            torch.cuda.empty_cache()
            if "fct2" in want:
                variants["fct2"] = fct2_variant(L, dev, stream, args, A1, b1, w1, line_c["ms_per_step"],
                                                line_c["phase_ms"]["fct_embed"])
            del A1, b1
            torch.cuda.empty_cache()
        if "t2rows_bf16" in want:
            variants["t2rows_bf16"] = bf16_variant(L, dev, stream, args, peaks["hbm_gbs"])
            torch.cuda.empty_cache()
        if "batched" in want:
            variants["batched"] = batched_variant(L, dev, stream, args, peaks["hbm_gbs"])
            torch.cuda.empty_cache()
        if "canonical" in want:
            variants["canonical"] = canonical_variant(L, dev, stream, args)
        variants["main_f32"] = {"workload": w.name, "value": value, "ms_per_step": ms_per_step,
                                "step_frac": step_gbs / peaks["hbm_gbs"]}
        line["variants"] = variants
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_rows_per_s(pr, w, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# Small cases of the kernels whose profiles are kept under profiles/: each runs the call
# twice on device-generated data (a few GB at most), so that a capture of one launch
# (ncu -s 1 -c 1) sees a warm launch.  Sizes: phase 1 of the d = 64 headline at n = 2^22
# (and 2^24 for its DRAM traffic), the slow transform at n = 2^21, d = 16, and the d = 64
# tensor-core λ at n = 2^22.
KERNEL_CASES = {"phase1_d64_n4M": (1 << 22,), "phase1_d64_n16M": (1 << 24,), "sct_d16_n2M": (1 << 21,),
                "lambda_tc_d64_n4M": (1 << 22,), "batched_256": (0,),
                "condition_d16": (1 << 20,), "condition_d64": (1 << 20,), "lambda_f32_d64_n4M": (1 << 22,)}


def run_kernel_case(args) -> None:
    import torch

    import paper_1207_4684_gb300 as L

    L.load()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    (n,) = KERNEL_CASES[args.kernel_case]
    if args.kernel_case == "batched_256":
        # the batched form's 256 members (default schedules), one l1_regress_batched call twice
        from synth import make_batched_problems

        probs, keep = [], []
        for pr in make_batched_problems(256):
            w = pr["w"]
            A = torch.from_numpy(pr["A"]).to(dev)
            b = torch.from_numpy(pr["b"]).to(dev)
            prm = L.make_params(w.s, w.r1, w.r2, w.coreset, seed=w.seed, problem_id=w.problem_id)
            cnt = torch.zeros(1, dtype=torch.int64, device=dev)
            keep.append((A, b, cnt))
            probs.append(L.make_problem(A, b, prm, count=cnt))
        ws = L.batched_workspace(probs, device=dev)
        flags = torch.zeros(len(probs), dtype=torch.int32, device=dev)
        for _ in range(2):
            L.l1_regress_batched(probs, ws, flags)
        torch.cuda.synchronize()
        bad = int((flags != 0).sum().item())
        print(json.dumps({"kernel_case": args.kernel_case, "members": len(probs), "status_nonzero": bad}))
        if bad:
            sys.exit(1)
        return
    if args.kernel_case.startswith("condition"):
        # the conditioning of the two measured shapes (r1 = 355, q = 17, r2 = 16 and r1 = 2130,
        # q = 65, r2 = 32) on the embedding of 2^20 random rows, with columns scaled as in the
        # colscale workload: two l1_condition calls as the pipeline makes them (no R copy)
        d, r1, r2 = (16, 355, 16) if args.kernel_case.endswith("d16") else (64, 2130, 32)
        A = torch.randn((n, d), generator=g, device=dev)
        A *= 10.0 ** (torch.rand(d, generator=g, device=dev) * 4.0 - 2.0)
        b = torch.randn(n, generator=g, device=dev)
        prm = L.make_params(256 if d == 16 else 1024, r1, r2, 1e4, seed=1)
        ws = L.workspace(prm, n, d, device=dev)
        pix = torch.empty((r1, d + 1), device=dev)
        M = torch.empty((d + 1, r2), device=dev, dtype=torch.float64)
        L.l1s_status_reset(ws)
        L.fct_embed(A, b, prm, pix, ws)
        for _ in range(2):
            L.l1_condition(pix, prm, None, M, ws)
        torch.cuda.synchronize()
        flags = L.l1s_status_read(ws)
        print(json.dumps({"kernel_case": args.kernel_case, "r1": r1, "q": d + 1, "status": flags}))
        if flags:
            sys.exit(1)
        return
    if args.kernel_case.startswith("phase1"):
        d, r1 = 64, 2130
        A = torch.randn((n, d), generator=g, device=dev)
        b = torch.randn(n, generator=g, device=dev)
        prm = L.make_params(1024, r1, 32, 1e5, seed=1)
    elif args.kernel_case.startswith("sct"):
        d, r1 = 16, 355
        A = torch.randn((n, d), generator=g, device=dev)
        b = torch.randn(n, generator=g, device=dev)
        prm = L.make_params(1, r1, 16, 2e4, seed=1, transform=1)
    else:
        d, r1 = 64, 2130
        A = torch.randn((n, d), generator=g, device=dev)
        if "_tc_" in args.kernel_case:
            A = A.to(torch.bfloat16)
        b = torch.randn(n, generator=g, device=dev)
        prm = L.make_params(1024, r1, 32, 1e5, seed=1)
    dt = L.BF16 if A.dtype == torch.bfloat16 else L.F32
    ws = L.workspace(prm, n, d, dt, device=dev)
    L.l1s_status_reset(ws)
    if args.kernel_case.startswith("lambda"):
        M = torch.randn((d + 1, 32), generator=g, device=dev, dtype=torch.float64) * 0.01
        lam = torch.empty(n, device=dev)
        tot = torch.empty(1, device=dev, dtype=torch.float64)
        for _ in range(2):
            L.l1_lambda(A, b, M, prm, lam, tot, ws)
    else:
        pix = torch.empty((r1, d + 1), device=dev)
        for _ in range(2):
            L.fct_embed(A, b, prm, pix, ws)
    torch.cuda.synchronize()
    flags = L.l1s_status_read(ws)
    print(json.dumps({"kernel_case": args.kernel_case, "n": n, "status": flags}))
    if flags:
        sys.exit(1)


def main():
    args = parse()
    if args.kernel_case:
        run_kernel_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
