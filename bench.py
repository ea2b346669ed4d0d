#!/usr/bin/env python
"""Benchmark: dual-pair solves/s of recycling BiCG on a sequence of slowly changing systems.

Workload (default): 2-D convection-diffusion, 512 x 512 interior grid (n = 262144, nnz =
1308672), 20 dual pairs whose convection (10, 10) drifts 1 % per pair, b and bt ~ N(0, 1),
recycle dimension k = 20, cycle length s = 40, relative tolerance 1e-8, FP64 RBiCG.  One step =
the whole sequence solved from an empty recycle space (all hot-path steps: system start,
initial projection, iterations, cycle refreshes, final correction).  The FP32-refined form,
plain BiCG and an end-to-end (host buffers) pass are reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints ONE JSON line on rank 0.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "dual-pair solves/s at rel.res 1e-8, chosen vs plain FP64; HBM GB/s; p99 ms"


def workload_name(a):
    """Name of the timed workload from its sizes (default: convdiff2d-512x512-seq20-k20)."""
    return "convdiff2d-%dx%d-seq%d-k%d" % (a.grid, a.grid, a.pairs, a.k)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--grid", type=int, default=512)
    ap.add_argument("--pairs", type=int, default=20)
    ap.add_argument("--k", type=int, default=20)
    ap.add_argument("--s", type=int, default=40)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--setup-blocks", type=int, default=0,
                    help="blocks of the refresh Gram launches (rbicg_params.setup_blocks; 0: the default)")
    ap.add_argument("--grid-blocks", type=int, default=0,
                    help="blocks per iteration-phase launch (0: the library default)")
    ap.add_argument("--no-extras", action="store_true", help="skip the FP32-refined, BiCG and e2e passes")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-config4", action="store_true",
                    help="skip the 1024^2 mixed-precision sequence (10 pairs, 0.5 %% drift, tol 1e-10)")
    ap.add_argument("--serving-small", action="store_true",
                    help="serve 64 requests from families of grid sides 64..256 instead of 256 from 64..1024")
    return ap.parse_args()


def make_sequence(a):
    from paper_1010_0762_gb300 import inputs as I
    return I.convdiff_sequence(a.grid, [10.0, 10.0], a.pairs, 0.01, 2000, bt_kind="normal")


# ------------------------------------------------------------------ clocks sampling
class Clocks:
    def __init__(self):
        self.samples = []
        self.stop = threading.Event()
        self.t = None

    def start(self):
        def run():
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            try:
                p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits", "-lms", "200"],
                                     stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            except OSError:
                return
            while not self.stop.is_set():
                line = p.stdout.readline()
                if not line:
                    break
                self.samples.append([v.strip() for v in line.split(",")])
            p.terminate()
        self.t = threading.Thread(target=run, daemon=True)
        self.t.start()

    def finish(self):
        self.stop.set()
        if self.t:
            self.t.join(timeout=3)
        dev = os.environ.get("LOCAL_RANK", "0")
        rows = [s for s in self.samples if s and s[0] == dev] or self.samples
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if len(r) > 5 + i and r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ replicas
def max_over_ranks(value, dist, device):
    """The job's timed region ends with its slowest rank: max of `value` over all ranks."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world, units_per_rank, ms):
    """Whole-job throughput of `world` independent replicas that each processed units_per_rank
    units, with the job's time ms (max over ranks)."""
    return world * units_per_rank / (ms * 1e-3)


# ------------------------------------------------------------------ GPU arm
def algorithmic_phase1(n, nnz, k, w=8):
    """Algorithmic flops and bytes of one phase-1 launch (dual SpMV with on-the-fly p update and
    the 2k projection dots) for real FP64, one A read (values + indices, A^H uses the same
    entries), vectors r, p_old, rt, pt_old read and p, pt, z, zt written, C and Ct read."""
    flops = 4 * nnz + 4 * n + 4 * k * n
    bytes_ = nnz * (w + 4) + 4 * (n + 1) + 8 * n * w + 2 * k * n * w
    return flops, bytes_


def measure_dgemm_tflops(torch):
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    for _ in range(2):
        torch.mm(a, b)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = 0.0
    for _ in range(3):   # best of three back-to-back pairs (cuBLAS FP64 GEMM, 4096^3)
        e0.record()
        reps = 2
        for _ in range(reps):
            torch.mm(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, 2.0 * n ** 3 * reps / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    return best


def run_sequence(R, torch, S, ops, bs, bts, xs, xts, results=None, refresh_every=1):
    S.reset()
    for j in range(len(ops)):
        xs[j].zero_()
        xts[j].zero_()
        if refresh_every > 1:   # Section 6.2: a new recycle space only for every refresh_every-th pair
            S.set_refresh(1 if j % refresh_every == 0 else 0)
        r = S.solve_pair(ops[j], bs[j], bts[j], xs[j], xts[j])
        if results is not None:
            results.append(r)


def flush_l2(torch, buf):
    buf.fill_(1.0)


def gpu_arm(a):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_1010_0762_gb300 import rbicg as R

    seq = make_sequence(a)
    n = seq[0]["A"].n
    nnz = seq[0]["A"].nnz
    # inputs resident in HBM: one pattern, per-pair values and right-hand sides
    rp = torch.as_tensor(seq[0]["A"].row_ptr, device="cuda")
    ci = torch.as_tensor(seq[0]["A"].col_idx, device="cuda")
    ops = [R.Operator(rp, ci, torch.as_tensor(p["A"].val, device="cuda")) for p in seq]
    bs = [torch.as_tensor(p["b"], device="cuda") for p in seq]
    bts = [torch.as_tensor(p["bt"], device="cuda") for p in seq]
    xs = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in seq]
    xts = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in seq]
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2

    def timed(S, steps, warmup, profile=False, refresh_every=1):
        for _ in range(warmup):
            run_sequence(R, torch, S, ops, bs, bts, xs, xts, refresh_every=refresh_every)
        results = []
        clocks = Clocks()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        l0 = S.launch_count()
        clocks.start()
        total_ms = 0.0
        for _ in range(steps):
            flush_l2(torch, flush)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run_sequence(R, torch, S, ops, bs, bts, xs, xts, results, refresh_every=refresh_every)
            e1.record(stream)
            torch.cuda.synchronize()
            total_ms += e0.elapsed_time(e1)
        ck = clocks.finish()
        launches = S.launch_count() - l0
        prof = None
        if profile:
            # per-phase CUDA-event timing on the solver's stream, in one extra untimed step so
            # that the events do not perturb the timed region
            import ctypes as C
            ms = (C.c_double * 8)()
            cnt = (C.c_int64 * 8)()
            R.lib.rbicg_profile(S.h, 1, None, None)
            flush_l2(torch, flush)
            run_sequence(R, torch, S, ops, bs, bts, xs, xts)
            torch.cuda.synchronize()
            R.lib.rbicg_profile(S.h, 0, ms, cnt)
            cols = C.c_int64(0)
            R.lib.rbicg_profile_columns(S.h, C.byref(cols))
            gp = C.c_int64(0)
            R.lib.rbicg_profile_gram_pairs(S.h, C.byref(gp))
            prof = (list(ms), list(cnt), cols.value, gp.value)
            # the same step once more with every refresh run alone (rbicg_profile enable = 2):
            # kernel times not shared with the concurrent next cycle's iterations
            R.lib.rbicg_profile(S.h, 2, None, None)
            flush_l2(torch, flush)
            run_sequence(R, torch, S, ops, bs, bts, xs, xts)
            torch.cuda.synchronize()
            R.lib.rbicg_profile(S.h, 0, ms, cnt)
            R.lib.rbicg_profile_columns(S.h, C.byref(cols))
            R.lib.rbicg_profile_gram_pairs(S.h, C.byref(gp))
            prof = prof + ((list(ms), list(cnt), cols.value, gp.value),)
        if world > 1:
            total_ms = max_over_ranks(total_ms, dist, "cuda")
        return total_ms, results, ck, prof, launches

    # --- plain FP64 RBiCG (the configuration's own form): every step in FP64, the per-cycle
    # Grams, basis products and SpMM of the refresh included (setup_fp32 = 0), as the oracle ---
    S = R.Solver(n, k=a.k, s=a.s, tol=a.tol, grid_blocks=a.grid_blocks, setup_blocks=a.setup_blocks, setup_fp32=0)
    ms64, res64, clocks, prof, launches = timed(S, a.steps, a.warmup, profile=True)
    pairs_done = a.pairs * a.steps
    value = replica_value(world, pairs_done, ms64)
    per_step = res64[:a.pairs]
    iters = [r["iters"] for r in per_step]
    ok = all(r["status"] in (R.OK, R.RECYCLE_EMPTY) for r in res64)
    worst_true = max(max(r["true_relres"], r["true_relres_dual"]) for r in res64)
    kcs = [r["recycle_dim"] for r in per_step]
    # 1 where the stagnation guard dropped the recycle space mid-solve (recycle_dim then reads 0)
    fbs = [r["fallback"] for r in per_step]

    # roofline of the dominant kernel (phase 1: dual SpMV + projections) from live CUDA events
    names = ["dual_spmv_project", "q_and_pq", "update_dots", "refresh_gram", "refresh_eig",
             "refresh_basis", "system_start", "init_finish_adjoint"]
    ms_slots, cnt_slots, pcols, gpairs, serial_prof = prof
    dom = int(np.argmax(ms_slots))
    # algorithmic work of every phase-1 launch of the profiled step: the dual SpMV and p update
    # of each launch plus 2 projections per active recycle column (pcols sums those widths)
    f0, b0 = algorithmic_phase1(n, nnz, 0)
    f1, b1 = algorithmic_phase1(n, nnz, 1)
    fl_tot = f0 * cnt_slots[0] + (f1 - f0) * pcols
    by_tot = b0 * cnt_slots[0] + (b1 - b0) * pcols
    t1 = ms_slots[0] * 1e-3
    dgemm = measure_dgemm_tflops(torch)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"hbm_gbs": 6800.0}
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    # FP64 ALU peak from the unit counts and the SM clock sampled during the timed region:
    # 2 DFMA per clock per SM x 2 flops x SMs
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    fp64_units = 2 * 2 * sms * sm_mhz * 1e6 / 1e12
    # the ALU roofline is the FP64 rate measured live (cuBLAS DGEMM); the unit count is context
    fp64_peak = dgemm
    fp64_src = ("cuBLAS FP64 GEMM 4096^3 measured in this run (of measured); FP64 FMA units: 2 DFMA/clock/SM "
                "x %d SMs at the sampled %.0f MHz = %.4f TFLOP/s" % (sms, sm_mhz, fp64_units))
    ach_tf = fl_tot / t1 / 1e12 if t1 > 0 else 0.0
    ach_gbs = by_tot / t1 / 1e9 if t1 > 0 else 0.0
    alu_frac = ach_tf / fp64_peak
    hbm_frac = ach_gbs / hbm_peak
    bound = "alu" if alu_frac >= hbm_frac else "hbm"
    launches_phase1 = cnt_slots[0]
    # DRAM traffic of one recycled k_phase1 launch on this operator, the compact bases four
    # columns wide (k_phase1<double, double, 4>: ncu dram__bytes_read.sum +
    # dram__bytes_write.sum; summary kept with the profiles), against the algorithmic bytes of
    # the same launch
    traffic_k4 = 52.440576e6 + 0.253952e6
    alg_k4 = algorithmic_phase1(n, nnz, 4)[1]
    rl_phase1 = {
        "kernel": "k_phase1 (dual SpMV + p update + Ct^H z, C^H zt)",
        "bound": bound,
        "achieved": round(ach_tf if bound == "alu" else ach_gbs, 4),
        "peak": round(fp64_peak if bound == "alu" else hbm_peak, 4),
        "unit": "TFLOP/s" if bound == "alu" else "GB/s",
        "frac": round(alu_frac if bound == "alu" else hbm_frac, 4),
        "peak_source": fp64_src if bound == "alu" else "MEASURED_PEAKS.json hbm_gbs (of measured)",
        "traffic": traffic_k4 if n == 262144 and nnz == 1308672 else None,
        "traffic_note": "bytes of one recycled launch (bases 4 columns wide) at 512^2 (ncu); "
                        "algorithmic %.1f MB" % (alg_k4 / 1e6),
        "hbm_view": {"achieved_gbs": round(ach_gbs, 1), "peak_gbs": hbm_peak, "frac": round(hbm_frac, 4)},
        "alu_view": {"achieved_tflops": round(ach_tf, 4), "peak_tflops": round(fp64_peak, 4),
                     "frac": round(alu_frac, 4), "fp64_unit_tflops": round(fp64_units, 4)},
        "avg_launch_us": round(ms_slots[0] * 1e3 / max(1, launches_phase1), 2),
        "mean_projection_columns": round(pcols / max(1, launches_phase1), 3),
        "launches": int(launches_phase1),
        "timing": "CUDA events around each phase launch in one profiled step of the same sequence "
                  "(plain launches), run right after the timed steps",
        "step_share": {names[i]: round(ms_slots[i] / max(1e-9, sum(ms_slots)), 4) for i in range(8)},
        "slot_ms": {names[i]: round(ms_slots[i], 2) for i in range(8)},
        "slot_launches": {names[i]: int(cnt_slots[i]) for i in range(8)},
        "dominant_slot": names[dom],
    }

    # the refresh's Gram Psit^H [Psi U_{j-1}] (Section 4.1): mx my n multiply-adds per launch in
    # FP64, ALU-bound (about 30 multiply-adds per loaded double at these widths)
    tg = ms_slots[3] * 1e-3
    g_tf = 2.0 * gpairs * n / tg / 1e12 if tg > 0 else 0.0
    rl_gram = {
        "kernel": "k_gram (refresh Gram Psit^H [Psi U_{j-1}], FP64)",
        "bound": "alu", "achieved": round(g_tf, 4), "peak": round(fp64_peak, 4), "unit": "TFLOP/s",
        "frac": round(g_tf / fp64_peak, 4),
        "peak_source": fp64_src,
        "frac_of_fp64_units": round(g_tf / fp64_units, 4),
        "traffic": None,
        "avg_launch_us": round(ms_slots[3] * 1e3 / max(1, cnt_slots[3] // 2), 2),
        "launches": int(cnt_slots[3] // 2),
        "mean_column_pairs": round(gpairs / max(1, cnt_slots[3] // 2), 1),
        "timing": rl_phase1["timing"],
    }
    # the same kernels timed alone: a second profiled step in which every refresh waits for the
    # iteration stream and the iteration stream for the refresh (no concurrent work)
    sms_, scnt_, spcols_, sgp_ = serial_prof
    tg_s = sms_[3] * 1e-3
    g_tf_s = 2.0 * sgp_ * n / tg_s / 1e12 if tg_s > 0 else 0.0
    rl_gram["alone"] = {"achieved": round(g_tf_s, 4), "frac": round(g_tf_s / fp64_peak, 4),
                        "avg_launch_us": round(sms_[3] * 1e3 / max(1, scnt_[3] // 2), 2),
                        "mean_column_pairs": round(sgp_ / max(1, scnt_[3] // 2), 1),
                        "timing": "profiled step with every refresh run alone (rbicg_profile enable = 2)"}
    fl_s = f0 * scnt_[0] + (f1 - f0) * spcols_
    t1_s = sms_[0] * 1e-3
    ach_s = fl_s / t1_s / 1e12 if t1_s > 0 else 0.0
    rl_phase1["alone"] = {"achieved_tflops": round(ach_s, 4), "frac": round(ach_s / fp64_peak, 4),
                          "avg_launch_us": round(sms_[0] * 1e3 / max(1, scnt_[0]), 2),
                          "timing": rl_gram["alone"]["timing"]}
    step_alone = {names[i]: round(sms_[i] / max(1e-9, sum(sms_)), 4) for i in range(8)}
    # the dominant kernel of the profiled step by its live CUDA-event time
    roofline = dict(rl_gram if ms_slots[3] > ms_slots[0] else rl_phase1)
    roofline["other_kernel"] = {k: v for k, v in (rl_phase1 if ms_slots[3] > ms_slots[0] else rl_gram).items()
                                if k not in ("step_share", "slot_ms", "slot_launches", "dominant_slot")}
    for key in ("step_share", "slot_ms", "slot_launches", "dominant_slot"):
        roofline[key] = rl_phase1[key]
    roofline["step_share_refresh_alone"] = step_alone

    out = {
        "metric": METRIC,
        "value": round(value, 4),
        "unit": "solves/s",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": round(ms64 / a.steps, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded convection-diffusion sequence, paper_1010_0762_gb300.inputs.convdiff_sequence)",
        "config": {"workload": workload_name(a), "grid": a.grid, "n": n, "nnz": nnz, "pairs": a.pairs, "k": a.k,
                   "s": a.s, "tol": a.tol, "drift": 0.01,
                   "form": "plain FP64 RBiCG (iteration and refresh products in FP64, setup_fp32=0)",
                   "guard": 1.5,
                   "l2": "256 MB flush between steps; working set > L2", "parallelism": "replicas"},
        "iters_per_pair": iters,
        "recycle_dim_per_pair": kcs,
        "guard_fallback_per_pair": fbs,
        "all_converged": ok,
        "worst_true_relres": worst_true,
        "roofline": roofline,
        "clocks": clocks,
        "gpu_launches": int(launches),
    }

    if not a.no_extras:
        # extras are timed over at most two steps each, so that the run stays within minutes
        x_steps = min(a.steps, 2)
        # --- chosen form: FP64 iterative refinement around FP32 inner RBiCG ---
        S32 = R.Solver(n, k=a.k, s=a.s, tol=a.tol, precision="fp32_refined", inner_tol=1e-5,
                       grid_blocks=a.grid_blocks)
        ms32, res32, _, _, _ = timed(S32, x_steps, 1)
        # --- FP64 iteration with the refresh's O(n) products multiplied in FP32 (setup_fp32 = 1) ---
        Sf = R.Solver(n, k=a.k, s=a.s, tol=a.tol, grid_blocks=a.grid_blocks, setup_fp32=1)
        msf, resf, _, _, _ = timed(Sf, x_steps, 1)
        out["fp32_setup"] = {"form": "FP64 iteration; refresh Grams, basis products and SpMM multiplied in FP32 "
                                     "with FP64 accumulation (setup_fp32=1)",
                             "value": round(world * a.pairs * x_steps / (msf * 1e-3), 4), "unit": "solves/s",
                             "ms_per_step": round(msf / x_steps, 3), "steps": x_steps,
                             "iters_per_pair": [r["iters"] for r in resf[:a.pairs]],
                             "guard_fallback_per_pair": [r["fallback"] for r in resf[:a.pairs]],
                             "all_converged": all(r["status"] in (R.OK, R.RECYCLE_EMPTY) for r in resf)}
        # --- the same FP64 form with a new recycle space only for every fifth pair (Section 6.2) ---
        Sr = R.Solver(n, k=a.k, s=a.s, tol=a.tol, grid_blocks=a.grid_blocks, setup_fp32=0)
        msr, resr, _, _, _ = timed(Sr, x_steps, 1, refresh_every=5)
        out["refresh_every_5th_pair"] = {
            "form": "plain FP64 RBiCG (setup_fp32=0), recycle space recomputed for pairs 0, 5, 10, 15 only",
            "value": round(world * a.pairs * x_steps / (msr * 1e-3), 4), "unit": "solves/s",
            "ms_per_step": round(msr / x_steps, 3), "steps": x_steps,
            "iters_per_pair": [r["iters"] for r in resr[:a.pairs]],
            "guard_fallback_per_pair": [r["fallback"] for r in resr[:a.pairs]],
            "all_converged": all(r["status"] in (R.OK, R.RECYCLE_EMPTY) for r in resr)}
        out["chosen"] = {"form": "fp32_refined (FP32 inner RBiCG, FP64 residual refinement)",
                         "value": round(world * a.pairs * x_steps / (ms32 * 1e-3), 4), "unit": "solves/s",
                         "ms_per_step": round(ms32 / x_steps, 3), "steps": x_steps,
                         "iters_per_pair": [r["iters"] for r in res32[:a.pairs]],
                         "refine_steps": [r["refine_steps"] for r in res32[:a.pairs]],
                         "all_converged": all(r["status"] in (R.OK, R.RECYCLE_EMPTY) for r in res32),
                         "fp64_fallback_pairs": sum(1 for r in res32[:a.pairs] if r["fallback"] == 2),
                         "worst_true_relres": max(max(r["true_relres"], r["true_relres_dual"]) for r in res32)}
        # --- non-recycling BiCG on the same sequence ---
        Sb = R.Solver(n, k=a.k, s=a.s, tol=a.tol, recycle=0, grid_blocks=a.grid_blocks)
        msb, resb, _, _, _ = timed(Sb, 1, 1)
        out["bicg"] = {"value": round(world * a.pairs / (msb * 1e-3), 4), "unit": "solves/s",
                       "iters_per_pair": [r["iters"] for r in resb[:a.pairs]]}
        # --- end to end through the C ABI with host buffers (H2D inputs, D2H solutions) ---
        hvals = [torch.as_tensor(p["A"].val).pin_memory() for p in seq]
        hb = [torch.as_tensor(p["b"]).pin_memory() for p in seq]
        hbt = [torch.as_tensor(p["bt"]).pin_memory() for p in seq]
        hrp = torch.as_tensor(seq[0]["A"].row_ptr).pin_memory()
        hci = torch.as_tensor(seq[0]["A"].col_idx).pin_memory()
        hx = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in seq]
        hxt = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in seq]
        dvals = [torch.empty_like(o.val) for o in ops]
        drp, dci = torch.empty_like(rp), torch.empty_like(ci)
        Se = R.Solver(n, k=a.k, s=a.s, tol=a.tol, grid_blocks=a.grid_blocks, setup_fp32=0)   # the headline form
        e_steps = max(1, a.steps // 2)
        h2d = d2h = 0
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(e_steps):
            Se.reset()
            drp.copy_(hrp, non_blocking=True)
            dci.copy_(hci, non_blocking=True)
            h2d += hrp.numel() * 4 + hci.numel() * 4
            for j in range(a.pairs):
                dvals[j].copy_(hvals[j], non_blocking=True)
                bs[j].copy_(hb[j], non_blocking=True)
                bts[j].copy_(hbt[j], non_blocking=True)
                xs[j].zero_()
                xts[j].zero_()
                h2d += (hvals[j].numel() + 2 * n) * 8
                op = R.Operator(drp, dci, dvals[j])
                Se.solve_pair(op, bs[j], bts[j], xs[j], xts[j])
                hx[j].copy_(xs[j], non_blocking=True)
                hxt[j].copy_(xts[j], non_blocking=True)
                d2h += 2 * n * 8
        e1.record(stream)
        torch.cuda.synchronize()
        mse = e0.elapsed_time(e1)
        out["e2e"] = {"value": round(world * a.pairs * e_steps / (mse * 1e-3), 4), "unit": "solves/s",
                      "h2d_bytes_per_step": int(h2d // e_steps), "d2h_bytes_per_step": int(d2h // e_steps),
                      "steps": e_steps}

        extras = [("irka", irka_extra), ("serving", serving_extra)]
        if not a.no_config4:
            extras.append(("config4", config4_extra))
        for key, fn in extras:
            t_ex = time.perf_counter()
            try:
                out[key] = fn(R, torch, a)
            except Exception as exc:   # an extra must not take the headline line down
                out[key] = {"error": "%s: %s" % (type(exc).__name__, exc)}
            out[key]["wall_s"] = round(time.perf_counter() - t_ex, 1)

    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(seq, a)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


# ------------------------------------------------------------------ IRKA (Algorithm 3)
def irka_extra(R, torch, a, N=64, nshift=8, steps=10, k=16):
    """IRKA (Algorithm 3) on a 3-D convection-diffusion model (N^3, real A shared by all shifts,
    E = I), 8 initial shifts in conjugate pairs, 10 steps: each step solves the 8 shifted dual
    systems (sigma I - A) v = b, (sigma I - A)^H w = c in complex128 with RBiCG (recycling
    strategy 1 of Section 5.3, one batched launch per iteration phase for all shifts), forms the
    reduced model and moves the shifts to the mirrored reduced poles.  Compared with the same run
    without recycling (BiCG) and with the shifts solved one after another."""
    from paper_1010_0762_gb300 import inputs as I
    A = I.convdiff(N, [10.0, 10.0, 10.0], dim=3)
    n = A.n
    op = R.Operator.from_csr(A)
    rng = np.random.default_rng(3000)
    b = torch.as_tensor(rng.standard_normal(n), device="cuda")
    c = torch.as_tensor(rng.standard_normal(n), device="cuda")
    shifts0 = I.irka_shifts(nshift, 3001)

    def run(strategy, batched, recycle_count=0, refresh_every=1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = R.irka(op, b, c, shifts0, max_steps=steps, shift_tol=1e-6, strategy=strategy, batched=batched,
                     recycle_count=recycle_count, refresh_every=refresh_every, solver_k=k, solver_s=a.s,
                     solver_tol=a.tol, solver_setup_fp32=0)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, out

    run(1, 1)   # warm-up (adjoints, graphs, lazy module loading)
    t1, o1 = run(1, 1)
    t4, o4 = run(4, 1)
    t2s, o2s = run(1, 1, recycle_count=2)
    tp, op_ = run(1, 1, recycle_count=2, refresh_every=5)
    t0, o0 = run(0, 1)
    ts, os_ = run(1, 0)
    its = lambda o: [int(v) for v in np.asarray(o["iters"]).sum(axis=1)]
    rate = lambda t, o: round(o["steps"] * nshift / t, 4)
    return {"workload": "IRKA, convdiff3d-%d^3 (real A, E = I), %d shifts in conjugate pairs, complex128 dual solves, "
                        "k=%d, up to %d steps, shift tolerance 1e-6" % (N, nshift, k, steps),
            "n": n, "nnz": A.nnz, "steps": o1["steps"], "converged": o1["converged"],
            "last_shift_change": o1["last_change"],
            "solves_per_s": rate(t1, o1),
            "solves_per_s_shared_space": rate(t4, o4),
            "solves_per_s_recycle_two_smallest": rate(t2s, o2s),
            "solves_per_s_two_smallest_refresh_every_5th_step": rate(tp, op_),
            "solves_per_s_bicg": rate(t0, o0),
            "solves_per_s_sequential": rate(ts, os_),
            "batched_over_sequential": round(ts / t1, 3),
            "iters_per_step": its(o1), "iters_per_step_shared_space": its(o4), "iters_per_step_bicg": its(o0),
            "total_iters": o1["total_iters"], "total_iters_shared_space": o4["total_iters"],
            "total_iters_recycle_two_smallest": o2s["total_iters"],
            "total_iters_two_smallest_refresh_every_5th_step": op_["total_iters"],
            "total_iters_bicg": o0["total_iters"],
            "failed_solves": o1["failed_solves"] + o4["failed_solves"] + o0["failed_solves"],
            "final_shifts": [[round(float(z.real), 4), round(float(z.imag), 4)] for z in o1["shifts"]],
            "strategies": "solves_per_s: strategy 1 (per shift index, batched); shared_space: strategy 4 (one space "
                          "for all shifts, one refresh chain per step); recycle_two_smallest: strategy 1 for the two "
                          "shifts of smallest modulus only (Section 6.2 recycles for the small shifts), the others "
                          "BiCG; two_smallest_refresh_every_5th_step: the same with the recycle spaces recomputed only at "
                          "every fifth IRKA step (the paper's practice in its model-reduction experiments); bicg: "
                          "no recycling; sequential: strategy 1, shifts solved one after another.  A step counts "
                          "all 8 shifted dual systems as solves (one shift of each conjugate pair is solved and "
                          "the other is its conjugate)"}


# ------------------------------------------------------------------ serving
def config4_extra(R, torch, a, N=1024, pairs=10, tol=1e-10, restarts=8):
    """Mixed precision at 1024^2 (n = 1048576, nnz = 5238784): 10 pairs with 0.5 % drift, relative
    tolerance 1e-10, the FP32-refined form against all-FP64 RBiCG on the same sequence (one timed
    pass each, after an untimed solve of pair 0); both forms run their refresh products in FP64
    (setup_fp32 = 0), so the refined form's FP64 fallback is the FP64 form itself.  Both restart
    as plain BiCG after a breakdown (`restarts`, as the serving run: at this tolerance a pair can
    end in a BiCG breakdown).  The refined solutions are compared with the FP64 ones."""
    from paper_1010_0762_gb300 import inputs as I
    seq = I.convdiff_sequence(N, [10.0, 10.0], pairs, 0.005, 4000, bt_kind="normal")
    n = seq[0]["A"].n
    rp = torch.as_tensor(seq[0]["A"].row_ptr, device="cuda")
    ci = torch.as_tensor(seq[0]["A"].col_idx, device="cuda")
    ops = [R.Operator(rp, ci, torch.as_tensor(p["A"].val, device="cuda")) for p in seq]
    bs = [torch.as_tensor(p["b"], device="cuda") for p in seq]
    bts = [torch.as_tensor(p["bt"], device="cuda") for p in seq]
    out = {"workload": "convdiff2d-%dx%d-seq%d-k%d, drift 0.5 %%, tol %g" % (N, N, pairs, a.k, tol), "n": n,
           "nnz": seq[0]["A"].nnz}
    sols = {}
    for form, kw in (("fp64", dict(setup_fp32=0)), ("fp32_refined", dict(precision="fp32_refined", setup_fp32=0))):
        S = R.Solver(n, k=a.k, s=a.s, tol=tol, restarts=restarts, **kw)
        xs = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in seq]
        xts = [torch.zeros_like(xs[0]) for _ in seq]
        run_sequence(R, torch, S, ops[:1], bs[:1], bts[:1], xs[:1], xts[:1])   # warm-up (untimed)
        res = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run_sequence(R, torch, S, ops, bs, bts, xs, xts, res)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        sols[form] = xs
        out[form] = {"solves_per_s": round(pairs / dt, 4), "s_per_sequence": round(dt, 3),
                     "iters_per_pair": [r["iters"] for r in res], "refine_steps": [r["refine_steps"] for r in res],
                     "fp64_fallback_pairs": sum(1 for r in res if r["fallback"] == 2),
                     "status_per_pair": [int(r["status"]) for r in res],
                     "fallback_per_pair": [int(r["fallback"]) for r in res],
                     "worst_true_relres": max(max(r["true_relres"], r["true_relres_dual"]) for r in res),
                     "all_converged": all(r["status"] in (R.OK, R.RECYCLE_EMPTY) for r in res)}
        S.destroy()
    out["rel_diff_fp32_refined_vs_fp64_per_pair"] = [
        float("%.3g" % float(torch.linalg.norm(x1 - x0) / torch.linalg.norm(x0)))
        for x0, x1 in zip(sols["fp64"], sols["fp32_refined"])]
    out["max_rel_diff_fp32_refined_vs_fp64"] = max(out["rel_diff_fp32_refined_vs_fp64_per_pair"])
    return out


def serving_extra(R, torch, a, families=16, requests=256, seed=5000, restarts=8):
    """Continuous batching over the engine: Poisson arrivals of dual-pair requests from
    `families` convection-diffusion families (grid sides log-uniform in [64, 1024], 256 requests;
    --serving-small: [64, 256] and 64 requests; (c1, c2) ~ U[1, 50]^2, 1 % drift per request, k ~ U{10..20},
    precision fp32_refined with probability 0.5), recycle spaces resident per family, HBM
    budget 80 % of free memory.  A closed-loop run (all requests at t = 0) measures capacity;
    the open-loop runs offer 0.8 x and 1.2 x that rate.  With (c1 + c2) / 2 up to 50 the
    operators are far from normal (the diagonal that symmetrises them spans about
    e^((c1 + c2) / 2)), so BiCG's shadow and primary residuals lose their correlation and many
    requests break down after ~130 iterations; the requests are served with `restarts`
    restarts after a breakdown (plain BiCG from the iterate; not in the paper)."""
    from paper_1010_0762_gb300 import serving as SV
    side_hi = 256 if a.serving_small else 1024
    requests = 64 if a.serving_small else 256
    specs = SV.random_families(families, seed, side_lo=64, side_hi=side_hi)
    free, _ = torch.cuda.mem_get_info()
    budget = int(0.8 * free)

    def serve(rate, count=None):
        be = SV.GpuBackend(s=a.s, tol=a.tol, restarts=restarts)
        srv = SV.Server(specs, be, budget, s=a.s, max_in_flight=32)
        reqs = SV.poisson_arrivals(requests, rate if rate > 0 else 1.0, specs, seed + 1, p_fp32=0.5)
        if count is not None:
            reqs = reqs[:count]
        if rate <= 0:
            for r in reqs:
                r.t_arrival = 0.0
        st = srv.run(reqs)
        for h in list(srv.resident.values()):
            h.destroy()
        be.engine.close()
        return st

    serve(1e9, count=16)   # warm-up: the first 16 requests of the stream
    closed = serve(0)
    cap = closed["requests_per_s"]
    out = {"workload": "%d families, grid sides 64..%d, %d requests, fp32_refined p=0.5, %d restarts after a "
                       "breakdown" % (families, side_hi, requests, restarts),
           "closed_loop": {k: (round(v, 3) if isinstance(v, float) else v) for k, v in closed.items()}}
    for f in (0.8, 1.2):
        st = serve(f * cap)
        out["open_loop_%.1fx" % f] = dict({"rate_per_s": round(f * cap, 3)},
                                          **{k: (round(v, 3) if isinstance(v, float) else v) for k, v in st.items()})
    return out


# ------------------------------------------------------------------ oracle (CPU) timing
class OracleSampler:
    """Bounded samples of the oracle on the benchmark sequence, in the recycled regime.

    Set-up (untimed): pair 0 for 2 s iterations (two cycles) gives a recycle space.  A sample
    (timed): the system start of pair 1 with that space (Section 4.3 last paragraph) and
    `iters` iterations of Algorithm 2 on it, projections and cycle refreshes included.  Solves
    per second = 1 / (seconds per iteration x the oracle's own iterations per pair over the
    whole sequence), the latter from oracle/bench_counts.json when it describes this workload,
    else from a full oracle BiCG solve of pair 0 (stated in the sample text)."""

    def __init__(self, seq, a):
        from oracle import rbicg_oracle as O
        self.O, self.seq, self.a = O, seq, a
        pr = seq[0]
        n = pr["A"].n
        r = O.rbicg_pair(pr["A"], pr["b"], pr["bt"], np.zeros(n), np.zeros(n), None, k=a.k, s=a.s,
                         tol=a.tol, max_itn=2 * a.s)
        self.U, self.Ut = r.U_next, r.Ut_next
        self.per_pair, self.source = self._iters_per_pair()

    def _iters_per_pair(self):
        path = os.path.join(ROOT, "oracle", "bench_counts.json")
        if os.path.exists(path):
            d = json.load(open(path))
            p = d.get("params", {})
            if d.get("workload") == workload_name(self.a) and p.get("s") == self.a.s and p.get("tol") == self.a.tol:
                return float(d["mean_iters"]), "the oracle's mean iterations per pair over the whole sequence " \
                                               "(oracle/bench_counts.json: %s)" % d["iters_per_pair"]
        pr = self.seq[0]
        n = pr["A"].n
        full = self.O.bicg(pr["A"], pr["b"], pr["bt"], np.zeros(n), np.zeros(n), self.a.tol, 20000)
        return float(full.iters), "the oracle BiCG count of pair 0 (no recorded sequence counts for this workload)"

    def sample(self, iters):
        O, a = self.O, self.a
        pr = self.seq[1 % len(self.seq)]
        n = pr["A"].n
        t = time.perf_counter()
        rec = O.biorth_recycle(pr["A"], self.U, self.Ut, 1e-6)
        r = O.rbicg_pair(pr["A"], pr["b"], pr["bt"], np.zeros(n), np.zeros(n), rec, k=a.k, s=a.s, tol=a.tol,
                         max_itn=iters)
        return time.perf_counter() - t, r.iters

    def rate(self, sec, done):
        return 1.0 / (sec / max(1, done) * self.per_pair)

    def describe(self, iters, sec):
        return ("oracle RBiCG (numpy/scipy FP64) on pair 1 with the recycle space of a two-cycle run of "
                "pair 0: system start + %d iterations per sample (%.1f s of samples); solves/s = 1 / "
                "(seconds per iteration x %.1f, %s)" % (iters, sec, self.per_pair, self.source))


def cpu_baseline(seq, a):
    smp = OracleSampler(seq, a)
    its = 2 * a.s
    sec, done = smp.sample(its)
    return {"value": round(smp.rate(sec, done), 6), "unit": "solves/s", "cores": os.cpu_count(),
            "kind": "oracle", "sample": smp.describe(done, sec)}


def reference_arm(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    seq = make_sequence(a)
    smp = OracleSampler(seq, a)
    for _ in range(a.warmup):
        smp.sample(4)
    its = a.s
    tot = 0.0
    done = 0
    for _ in range(a.steps):
        sec, d = smp.sample(its)
        tot += sec
        done += d
    value = smp.rate(tot, done)
    cpu = {"value": round(value, 6), "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
           "sample": "each step: " + smp.describe(its, tot)}
    A0 = seq[0]["A"]
    # n_gpus: the launch's N (the oracle itself runs on rank 0's host cores, see cpu_baseline)
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "solves/s",
           "n_gpus": int(os.environ.get("WORLD_SIZE", str(a.gpus))),
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(1e3 * tot / max(1, a.steps), 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded convection-diffusion sequence, paper_1010_0762_gb300.inputs.convdiff_sequence)",
           "config": {"workload": workload_name(a), "grid": a.grid, "n": A0.n, "nnz": A0.nnz, "pairs": a.pairs,
                      "k": a.k, "s": a.s, "tol": a.tol, "drift": 0.01,
                      "form": "plain FP64 RBiCG (oracle: numpy/scipy FP64, explicit Grams)", "guard": 1.5},
           "cpu_baseline": cpu, "e2e": {"value": round(value, 6), "unit": "solves/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)
