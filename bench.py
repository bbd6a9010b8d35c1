#!/usr/bin/env python
"""Throughput of the element-local semi-Lagrangian Monte-Carlo step on GB300.

Metric: element-sample SL updates per second (ESU/s; one element of one
Monte-Carlo sample advanced by one SL step), at the stated error against the
FP64 oracle.

Workload (one benchmark step): the 1D non-constant drift-diffusion problem on
periodic [0,2] with K=256 elements, M=4096 samples, u = 1 + 0.5 sin(pi x),
D = 0.01 (1 + 0.5 cos(pi x)), seeded 8-mode Fourier phi0, run for 1000 SL
steps at each order N in {4, 8, 12, 16} (4.19e9 ESU), followed by the sample
moments of each -- every part of the path (Wiener increments, advance, face
values, upwinding, constrained least-squares remap, averaging) in the CUDA
library.  Inputs are synthetic and resident in HBM when the timed region
starts; L2 is flushed (256 MiB write) between timed steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
Under torchrun each rank runs the same workload on its own disjoint sample
range (weak scaling, no collective on the data path); rank 0 prints the line.
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

# CUDA multiplexes streams onto this many in-order hardware queues (default 8);
# the serving leg runs hundreds of request streams, and streams that share a
# queue wait for one another.  Read when CUDA initialises, so set before torch.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import sl_inputs as I  # noqa: E402

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# FP32 step kernel at config 2 (one launch of 1000 steps per order), from one
# ncu capture.  A capture describes one version of the kernel, so it carries
# the SHA-256 (first 16 hex digits) of the kernel's two source files; when
# they change, the figure no longer applies and the bench reports null.
TRAFFIC_CAPTURE = {
    "sources": ("paper_2009_07340_gb300/csrc/sl_step1d.cuh", "paper_2009_07340_gb300/csrc/sl_step1d_fp32.cu"),
    "sha256_16": "c199abc8e2aa0936",
    "bytes_per_launch": {4: 68739328, 8: 110707712, 12: 180182272, 16: 250309120},
}


def _captured_traffic():
    import hashlib

    h = hashlib.sha256()
    for f in TRAFFIC_CAPTURE["sources"]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return TRAFFIC_CAPTURE["bytes_per_launch"] if h.hexdigest()[:16] == TRAFFIC_CAPTURE["sha256_16"] else None


METRIC = "element-sample SL updates/sec at stated error vs FP64 oracle; p50/p99 solve latency"
ORDERS = (4, 8, 12, 16)
SL_STEPS = 1000
K_ELEM, M_SAMPLES = 256, 4096
WORKLOAD = ("1D periodic [0,2], K=256, N in {4,8,12,16}, M=4096, 1000 SL steps per order, "
            "u=1+0.5 sin(pi x), D=0.01(1+0.5 cos(pi x)), 8-mode Fourier phi0 (seed 2), dt=3.665e-7 "
            "(half the N=16 particle-gap bound)")

# GB300: 152 SMs at 2070 MHz max; FP32 128 lanes/SM/clk; FP64 2 FMA/SM/clk
# (nominal 1.25 TFLOP/s; a DFMA probe on this machine measured 1.90 FMA/SM/clk).
N_SM, SM_MHZ = 152, 2070.0
PEAK_FP32_TFLOPS = N_SM * 128 * 2 * SM_MHZ * 1e6 / 1e12   # 80.5
PEAK_FP64_TFLOPS = N_SM * 2 * 2 * SM_MHZ * 1e6 / 1e12     # 1.26


def flops_per_esu_1d(N):
    """Algorithmic flops of one 1D element-sample update: the minimal dense
    work of the reduced (Woodbury) form of the constrained least-squares
    remap, 2N^2 (barycentric weights of the advected nodes) + 3N(N+2) (the
    advected basis at the N nodes and 2 faces, 3 flops per entry) + N(N+2)
    divisions, each division counted as one flop: 6N^2 + 8N (128, 448, 960,
    1664 at N = 4, 8, 12, 16).  The kernel itself issues more: it is
    division-free (products and recurrences in place of the N(N+2)
    divisions) and forms every position difference in two parts."""
    return 6 * N * N + 8 * N


def algorithmic_bytes_1d(N, M, K, steps, state_bytes):
    """HBM bytes one 1D launch must move: the state read and written once
    (the sample fields stay on chip for all steps of a launch) and one
    Wiener increment (8 bytes) per sample and step."""
    return 2 * M * K * N * state_bytes + 8 * M * steps


def _clock_sampler():
    try:
        return subprocess.Popen(
            ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
             "--format=csv,noheader,nounits", "-lms", "200"],
            stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return None


def _clock_summary(proc, device_index):
    if proc is None:
        return None
    proc.terminate()
    try:
        out, _ = proc.communicate(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
        out, _ = proc.communicate()
    sm, mx, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.splitlines():
        f = [t.strip() for t in line.split(",")]
        if len(f) < 9 or f[0] != str(device_index):
            continue
        try:
            sm.append(float(f[1]))
            mx = max(mx, float(f[2]))
        except ValueError:
            continue
        for n, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _dist(backend="nccl"):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group(backend)
        return dist, dist.get_rank(), ws
    return None, 0, 1


def shard_sample0(rank, per_rank):
    """Rank r owns the global samples [r * per_rank, (r + 1) * per_rank): the
    Philox counter is keyed on the global sample index, so the ranks together
    draw exactly the increments of one run over all samples."""
    return rank * per_rank


def max_over_ranks(x, dist, device="cpu"):
    """The largest of every rank's x (the job takes as long as its slowest rank)."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Units all ranks processed per second of the slowest rank (weak scaling)."""
    return world * units_per_rank / seconds


def _cpu_baseline(seconds=15.0):
    """The FP64 CPU oracle as it stands, all host cores, on a bounded sample
    of the workload: all K=256 elements, a few samples per core, each order."""
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    ms = 2 * cores
    # calibrate the step count on a short run, then run ~`seconds`
    probe = 2
    t0 = time.perf_counter()
    for N in ORDERS:
        oracle.run(I.config2(N=N, M=ms, steps=probe), ns=ms, nthreads=cores, want_sums=True)
    tp = time.perf_counter() - t0
    steps = max(1, int(probe * seconds / max(tp, 1e-3)))
    t0 = time.perf_counter()
    for N in ORDERS:
        oracle.run(I.config2(N=N, M=ms, steps=steps), ns=ms, nthreads=cores, want_sums=True)
    t = time.perf_counter() - t0
    esu = len(ORDERS) * K_ELEM * ms * steps
    # the same oracle on one thread: 2 samples, a fifth of the time
    s1 = max(1, int(steps * (seconds / 5.0) / max(t * cores / ms * 2.0, 1e-3)))
    t0 = time.perf_counter()
    for N in ORDERS:
        oracle.run(I.config2(N=N, M=2, steps=s1), ns=2, nthreads=1, want_sums=True)
    t1 = time.perf_counter() - t0
    esu1 = len(ORDERS) * K_ELEM * 2 * s1
    return {"value": esu / t, "unit": "ESU/s", "cores": cores, "kind": "oracle",
            "sample": f"K=256, M={ms}, {steps} steps at each N in {{4,8,12,16}} ({esu:.3g} ESU, {t:.1f} s, "
                      f"FP64 C oracle, samples split over {cores} threads)",
            "single_core": {"value": esu1 / t1, "unit": "ESU/s", "cores": 1,
                            "sample": f"K=256, M=2, {s1} steps at each N ({esu1:.3g} ESU, {t1:.1f} s, one thread)"}}


def flops_per_esu_2d(N):
    """Algorithmic flops of one 2D element-sample update (FMA = 2 flops):
    the square n x n advected-basis system factored once (n^3/3 FMA), its
    4N face rows coupled through it (4N n^2 FMA) and the basis formed (n^2),
    n = N^2: 4.45e5 at N = 8."""
    n = N * N
    return 2 * (n ** 3 / 3 + 4 * N * n * n + n * n)


def _timed(fn):
    import torch

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fn()
    torch.cuda.synchronize()
    return time.perf_counter() - t0


def leg_2d(sl, stream, horizon=500, acc_samples=16):
    """Config 3 (64x64 elements, N=8, rotation drift): rates in FP32 and the
    mixed form (FP64 capacitance factor; M=1024) and FP64 (M=128) at two time
    steps, and FP32 and mixed against FP64 over the full 500-step horizon at
    the larger one.

    The stated dt (the Eq. 1d_timestep particle-gap bound, 6.93e-5) is not
    used: there the 2D step amplifies a perturbation ~12 % per step (x5.8e6
    over 120 steps, measured on the FP64 oracle), so no two implementations
    agree after a few hundred steps.  Half of it (3.465e-5) is stable; the
    edge-distance bound (1.618e-6) keeps every particle inside its element."""
    out = {"workload": "2D periodic [0,1]^2, 64x64 elements, N=8, rotation drift, D=0.005(1+0.3 sin 2pi x "
                       "sin 2pi y), Gaussian blob; dt: half the particle-gap bound (3.465e-5; the bound itself, "
                       "6.93e-5, is unstable in 2D) and the edge-distance bound (1.618e-6)"}
    for name, dt in (("half_node_gap_dt", I.DT_CFG3_HALF), ("edge_dt", I.DT_CFG3_EDGE)):
        leg = {"dt": dt}
        for mode, M, steps in (("fp32", 1024, 3), ("mixed", 1024, 3), ("fp64", 128, 2)):
            pb = I.config3(M=M, steps=steps, dt=dt)
            s = sl.Solver(pb, mode, stream=stream.cuda_stream)
            s.step(pb["dt"], 1)
            s.profile(True)
            s.step(pb["dt"], steps)
            ms, _ = s.profile_read()
            s.close()
            leg[mode] = {"value": 64 * 64 * M * steps / (ms * 1e-3), "unit": "ESU/s", "M": M, "steps": steps}
        ach = leg["fp32"]["value"] * flops_per_esu_2d(8) / 1e12
        leg["roofline_fp32"] = {"bound": "alu", "achieved": ach, "peak": PEAK_FP32_TFLOPS, "unit": "TFLOP/s",
                                "frac": ach / PEAK_FP32_TFLOPS, "flops_per_esu": flops_per_esu_2d(8),
                                "what": "the dense direct solve's flops (the method's work count) per second"}
        out[name] = leg
    # FP32 against FP64 over the whole horizon, same seeds
    pb = I.config3(M=acc_samples, steps=horizon, dt=I.DT_CFG3_HALF)
    means = {}
    for mode in ("fp64", "fp32", "mixed"):
        with sl.Solver(pb, mode, stream=stream.cuda_stream) as s:
            s.step()
            means[mode] = s.moments()[0]
    scale = np.abs(means["fp64"]).max()
    err = float(np.abs(means["fp32"] - means["fp64"]).max() / scale)
    err_mixed = float(np.abs(means["mixed"] - means["fp64"]).max() / scale)
    out["accuracy"] = {"dt": I.DT_CFG3_HALF, "steps": horizon, "M": acc_samples, "error_fp32_vs_fp64": err,
                       "error_mixed_vs_fp64": err_mixed, "tolerance": 1e-5, "met": max(err, err_mixed) <= 1e-5,
                       "what": "max |mean_mode - mean_fp64| / max |mean_fp64| after the full horizon"}
    out["summary"] = {"fp32_esu_per_s": {k: out[k]["fp32"]["value"] for k in ("half_node_gap_dt", "edge_dt")},
                      "mixed_esu_per_s": {k: out[k]["mixed"]["value"] for k in ("half_node_gap_dt", "edge_dt")},
                      "fp64_esu_per_s": {k: out[k]["fp64"]["value"] for k in ("half_node_gap_dt", "edge_dt")},
                      "fp32_frac": {k: out[k]["roofline_fp32"]["frac"] for k in ("half_node_gap_dt", "edge_dt")},
                      "error_fp32_vs_fp64_500_steps": err, "error_mixed_vs_fp64_500_steps": err_mixed}
    return out


def leg_batch(sl, stream, m_div=32):
    """Batched uneven instances (one graph launch per call, order classes on
    tuned parallel branches) vs the same instances stepped one by one:
    config 4 (all 512 drawn 2D instances, each with M/m_div samples, one
    step; the full configuration is m_div x 100 times this work), 32 1D
    draws of config 5, and 256 small 1D instances."""
    import torch

    out = {}
    draws = I.batch_instances(512)
    cfg4 = [dict(pb, M=max(8, pb["M"] // m_div)) for pb in draws]
    one_d = []
    rng = np.random.default_rng(45)
    for i in range(32):
        pb = I.config2(N=int(rng.integers(4, 17)), M=int(rng.integers(256, 2049)), K=int(rng.integers(64, 1025)))
        pb["seed"] = 7000 + i
        one_d.append(pb)
    small = I.small_instances_1d()
    # config 4 in its stated precision, FP32 bulk with the FP64 factor (the
    # mixed form), and in FP32; the 1D legs in FP32
    for name, pbs, steps, prec in (("config4_all_512", cfg4, 1, "mixed"), ("config4_all_512_fp32", cfg4, 1, "fp32"),
                                   ("config5_1d_mix", one_d, 20, "fp32"), ("small_1d_uneven", small, 20, "fp32")):
        for pb in pbs:  # half of each instance's particle bound (2D: edge distance)
            pb["dt"] = ("edge", 0.5) if pb["dim"] == 2 else ("node", 0.5)
        esu = sum(int(np.prod(pb["K"])) * pb["M"] for pb in pbs) * steps
        with sl.Batch(pbs, prec) as b:
            tune_ms = b.tune(1)
            grids, lanes = b.grids(), b.lanes()
            b.step(steps)  # capture
            t_batch = _timed(lambda: b.step(steps))
        solvers = [sl.Solver(pb, prec, stream=stream.cuda_stream) for pb in pbs]
        dts = [0.5 * (s.dt_edge if pb["dim"] == 2 else s.dt_max) for s, pb in zip(solvers, pbs)]
        for s, d in zip(solvers, dts):
            s.step(d, 1)

        def seq():
            for s, d in zip(solvers, dts):
                s.step(d, steps)

        t_seq = _timed(seq)
        for s in solvers:
            s.close()
        torch.cuda.synchronize()
        out[name] = {"instances": len(pbs), "steps": steps, "esu": esu, "precision": prec,
                     "batched": {"value": esu / t_batch, "unit": "ESU/s", "seconds": t_batch},
                     "one_by_one": {"value": esu / t_seq, "unit": "ESU/s", "seconds": t_seq},
                     "speedup": t_seq / t_batch, "tuned_grids_1d": grids, "tuned_branches": lanes,
                     "tune_ms": tune_ms}
    c4 = out["config4_all_512"]
    full = sum(int(np.prod(pb["K"])) * pb["M"] for pb in draws) * 100
    c4["what"] = (f"all 512 config-4 draws (K ~ U{{16..64}}, N ~ U{{4..12}}, constant or rotating drift) with "
                  f"M/{m_div} samples each, one step, FP32 remap with the capacitance matrix factored in FP64; "
                  f"the configuration as drawn (full M, 100 steps) is "
                  f"{full:.3g} ESU, {full / c4['esu']:.0f}x this")
    c4["full_config_extrapolated_s"] = full / c4["batched"]["value"]
    c4f = out["config4_all_512_fp32"]
    c4f["what"] = c4["what"].replace("FP32 remap with the capacitance matrix factored in FP64", "FP32")
    c4f["full_config_extrapolated_s"] = full / c4f["batched"]["value"]
    out["small_1d_uneven"]["what"] = ("256 instances, K ~ U{8..64}, N ~ U{4..8}, M ~ U{16..128}: each alone is "
                                      "far from filling the GPU, so one-by-one stepping is launch-bound")
    out["summary"] = {k: {"batched_esu_per_s": v["batched"]["value"], "speedup": v["speedup"],
                          "branches": v["tuned_branches"]}
                      for k, v in out.items() if isinstance(v, dict) and "batched" in v}
    out["summary"]["config4_full_extrapolated_s"] = {"mixed": c4["full_config_extrapolated_s"],
                                                     "fp32": c4f["full_config_extrapolated_s"]}
    return out


def _serve(sl, reqs, precision, duration, drain, max_active=0, keep=None):
    """Submits `reqs` at their arrival times to a server of `precision`,
    waits up to `drain` s after the window, and returns per-request records
    (completed, latency or censored latency, class) and the server stats.
    `keep`: indices whose means are returned for comparison."""
    srv = sl.Server(budget_bytes=64 << 30, slice_steps=5, heavy_slots=2, precision=precision, max_active=max_active)
    t0 = time.perf_counter()
    tickets = []
    for ta, pb in reqs:
        wait = t0 + ta - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        tickets.append(srv.submit(pb))
    deadline = t0 + duration + drain
    while time.perf_counter() < deadline:
        st = srv.stats()
        if st["queued"] == 0 and st["running"] == 0:
            break
        time.sleep(0.05)
    t_end = time.perf_counter()
    st = srv.stats()
    recs, kept = [], {}
    for i, (t, (ta, pb)) in enumerate(zip(tickets, reqs)):
        want = keep is not None and i in keep
        state, res = srv.poll(t, want=want)
        cls = "2d" if pb["dim"] == 2 else ("1d_cluster" if pb["K"][0] > 256 else "1d")
        if state == 2:
            ph = srv.timing(t)
            recs.append({"cls": cls, "done": True, "lat": ph[7], "phases": ph})
            if want:
                kept[i] = res[0]
        elif state < 0:  # refused by the solver (e.g. an order the precision does not support)
            recs.append({"cls": cls, "done": False, "failed": state})
        else:  # still queued or running: latency censored at the deadline
            recs.append({"cls": cls, "done": False, "lat": t_end - (t0 + ta)})
    srv.close()
    return recs, st, kept


def _latency_stats(recs):
    """p50/p99 over completed requests, and over all requests with the
    unfinished ones counted at their censored latency (a lower bound: where
    more than 1 % are unfinished, the censored p99 is itself a lower bound)."""
    done = np.array([r["lat"] for r in recs if r["done"]], dtype=float)
    every = np.array([r["lat"] for r in recs if "lat" in r], dtype=float)
    out = {"requests": len(recs), "completed": int(done.size),
           "refused": sum(1 for r in recs if "failed" in r),
           "served_fraction": float(done.size / max(len(recs), 1))}
    if done.size:
        out.update(p50_completed_s=float(np.percentile(done, 50)), p99_completed_s=float(np.percentile(done, 99)))
    if every.size:
        out.update(p50_censored_s=float(np.percentile(every, 50)), p99_censored_s=float(np.percentile(every, 99)),
                   p99_censored_is_lower_bound=bool(done.size < 0.99 * every.size))
    return out


def leg_serving(sl, duration=60.0, drain=10.0, fp64_duration=20.0, max_active=0):
    """Poisson arrivals (200/s) drawn like config 5, served with continuous
    batching, in FP32 (the served form) and, on the first `fp64_duration`
    seconds of the same stream, in plain FP64: latency percentiles with the
    unfinished requests counted as censored, the served fraction, the served
    rate, and the FP32 results against the FP64 ones for the requests both
    arms completed (equal accuracy: within the 1e-5 tolerance)."""
    reqs = I.serving_requests(rate=200.0, duration=duration, seed=5, steps=20)
    for _, pb in reqs:
        pb["dt"] = ("edge", 0.5) if pb["dim"] == 2 else ("node", 0.5)
    n64 = sum(1 for ta, _ in reqs if ta < fp64_duration)
    keep = set(range(n64))
    arms = {}
    kept = {}
    for prec, reqs_p, dur in (("fp64", reqs[:n64], fp64_duration), ("fp32", reqs, duration)):
        recs, st, kept[prec] = _serve(sl, reqs_p, prec, dur, drain, max_active, keep)
        by_class = {}
        for cls in ("1d", "1d_cluster", "2d"):
            sub = [r for r in recs if r["cls"] == cls]
            by_class[cls] = _latency_stats(sub)
            ph = np.array([r["phases"] for r in sub if r["done"]], dtype=float).reshape(-1, 9)
            if len(ph):
                by_class[cls]["p50_phases_s"] = {name: float(np.percentile(ph[:, i], 50)) for i, name in enumerate(
                    ("queued", "create_wait", "create", "running", "complete_wait", "moments", "release"))}
        arms[prec] = {"arrival_window_s": dur, "drain_s": drain, "offered_rate_per_s": len(reqs_p) / dur,
                      **_latency_stats(recs), "failed": st["failed"], "rejected": st["rejected"],
                      "served_rate_per_s": st["completed"] / max(st["span_s"], 1e-9),
                      "esu_per_s": st["esu_per_s"], "memory_peak_bytes": st["memory_peak"],
                      "light_slices": st["slices"], "scheduler_busy_s": st["sched_busy_s"],
                      "launch_max_s": st["launch_max_s"], "by_class": by_class}
    both = sorted(set(kept["fp32"]) & set(kept["fp64"]))
    errs = [float(np.abs(kept["fp32"][i] - kept["fp64"][i]).max() / max(np.abs(kept["fp64"][i]).max(), 1e-300))
            for i in both]
    out = {"fp32": arms["fp32"], "fp64": arms["fp64"],
           "equal_accuracy": {"requests_compared": len(both), "max_rel_error_fp32_vs_fp64": max(errs) if errs else None,
                              "tolerance": 1e-5, "met": bool(errs and max(errs) <= 1e-5),
                              "what": "served FP32 means against the same requests served in FP64 (max over nodes "
                                      "of |diff| / max |fp64 mean|)"},
           "config": "budget 64 GiB (reserved at creation), slice 5 steps, 2 heavy slots, heavy 2D launches "
                     "of ~2e10 flop with <= 2 queued, 20 steps per request, dt: half the particle-gap bound (1D), "
                     "half the edge-distance bound (2D), "
                     f"CUDA_DEVICE_MAX_CONNECTIONS={os.environ.get('CUDA_DEVICE_MAX_CONNECTIONS', '8')}",
           "note": "the offered 2D load exceeds the GPU's capacity: unfinished requests are counted at their "
                   "censored latency (deadline - arrival) in the *_censored_* percentiles"}
    out["summary"] = {p: {k: arms[p].get(k) for k in ("served_fraction", "p50_completed_s", "p99_completed_s",
                                                       "p99_censored_s", "esu_per_s")} for p in ("fp32", "fp64")}
    out["summary"]["equal_accuracy_max_err"] = out["equal_accuracy"]["max_rel_error_fp32_vs_fp64"]
    return out


def run_reference(args):
    """Reference arm: the FP64 CPU oracle timed on the host cores, each step a
    bounded sample of the workload."""
    _, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    ms = 2 * cores
    steps_per = 30
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for N in ORDERS:
            oracle.run(I.config2(N=N, M=ms, steps=steps_per), ns=ms, nthreads=cores, want_sums=True)
        if it >= args.warmup:
            times.append(time.perf_counter() - t0)
    esu = len(ORDERS) * K_ELEM * ms * steps_per
    value = esu / float(np.mean(times))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ESU/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": f"M={ms}, {steps_per} steps per order"},
            "cpu_baseline": {"value": value, "unit": "ESU/s", "cores": cores, "kind": "oracle",
                             "sample": f"K=256, M={ms}, {steps_per} steps at each N in {{4,8,12,16}} per step"},
            "e2e": {"value": value, "unit": "ESU/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _moments_bandwidth(sl, stream, reps=20):
    """HBM rate of the sample-moment kernels (Eq. averaged) on the headline
    state (K=256, N=16, M=4096, float-pair state): bytes = the state read
    once, the chunk partials written and read back, the two outputs
    written; time from CUDA events on the launching stream over `reps`
    calls."""
    import torch

    pb = I.config2(N=16)
    with sl.Solver(pb, "fp32", stream=stream.cuda_stream) as s:
        V = s.V
        d_mean = torch.empty(V, dtype=torch.float64, device="cuda")
        d_m2 = torch.empty_like(d_mean)
        for _ in range(3):
            s.moments_device(d_mean, d_m2)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            # hold the stream while the calls are queued, so that the events
            # time the kernels and not the host's launch rate
            torch.cuda._sleep(20_000_000)
            e0.record(stream)
            for _ in range(reps):
                s.moments_device(d_mean, d_m2)
            e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
    nc = -(-M_SAMPLES // 64)
    nbytes = M_SAMPLES * V * 8 + 2 * (2 * nc * V * 8) + 2 * V * 8
    gbs = nbytes / (ms * 1e-3) / 1e9
    peak = _measured_hbm()
    return {"kernel": "moments_partial_kernel + moments_final_kernel", "bytes_per_call": nbytes, "ms_per_call": ms,
            "achieved_gbs": gbs, "peak_gbs": peak, "frac": gbs / peak if peak else None,
            "peak_source": "measured copy bandwidth (hbm_gbs)" if peak else None,
            "workload": "K=256, N=16, M=4096 float-pair state (134 MB)"}


def _measured_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0  # fallback figure: one earlier GB300 copy measurement


def run_native(args):
    import torch

    dist, rank, world = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    import paper_2009_07340_gb300 as sl

    from paper_2009_07340_gb300 import build, shard

    build.build()
    stream = torch.cuda.Stream()
    sample0 = shard_sample0(rank, M_SAMPLES)
    prec = args.precision
    orders = ORDERS if not args.quick else (16,)
    sl_steps = SL_STEPS if not args.quick else 50

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---------------------------------------------------------------- device-resident timing
    solvers = {N: sl.Solver(I.config2(N=N), prec, stream=stream.cuda_stream, sample0=sample0) for N in orders}
    V = K_ELEM * 16
    d_mean = torch.zeros(V, dtype=torch.float64, device="cuda")
    d_m2 = torch.zeros(V, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    dt = I.DT_CFG2_HALF

    def one_step():
        for N in orders:
            s = solvers[N]
            s.step(dt, sl_steps)
            if dist is None:
                s.moments_device(d_mean, d_m2)
            else:  # every rank's chunk partials gathered in rank order, combined by the library
                shard.global_moments(s, M_SAMPLES * world, dist, stream=stream.cuda_stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_step()
    torch.cuda.synchronize()
    for s in solvers.values():
        s.profile_read()
        s.profile(True)
    barrier()
    torch.cuda.synchronize()
    clk = _clock_sampler() if rank == 0 else None
    step_ms = []
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            flush.fill_(1)  # evict L2 between timed steps (outside the events)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one_step()
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    barrier()
    clocks = _clock_summary(clk, local) if rank == 0 else None
    kern_ms, kern_launches, flops = 0.0, 0, 0.0
    for N, s in solvers.items():
        ms_, n_ = s.profile_read()
        s.profile(False)
        kern_ms += ms_
        kern_launches += n_
        flops += flops_per_esu_1d(N) * K_ELEM * M_SAMPLES * sl_steps * args.steps
    total_ms = max_over_ranks(float(np.sum(step_ms)), dist, device="cuda")
    esu_step = len(orders) * K_ELEM * M_SAMPLES * sl_steps
    value = whole_job_rate(esu_step * args.steps, world, total_ms * 1e-3)
    # launches per step: per order one Wiener kernel, one step kernel, two moment kernels
    gpu_launches = 4 * len(orders) * args.steps
    for s in solvers.values():
        s.close()

    line = None
    if rank == 0:
        fp32_like = prec in ("mixed", "fp32")
        peak = PEAK_FP32_TFLOPS if fp32_like else PEAK_FP64_TFLOPS
        achieved = flops / (kern_ms * 1e-3) / 1e12 if kern_ms > 0 else None
        captured = _captured_traffic() if prec == "fp32" else None
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak if achieved else None,
                    "traffic": float(np.mean([captured[N] for N in orders])) if captured else None,
                    "traffic_unit": "DRAM bytes per launch (ncu capture of this kernel version, mean over orders)",
                    # 8 bytes per node of state: an FP64 value or a float pair
                    "algorithmic_bytes_per_launch": float(np.mean([algorithmic_bytes_1d(
                        N, M_SAMPLES, K_ELEM, sl_steps, 8) for N in orders])),
                    "kernel": "sl1d_step_kernel<N,%s>" % prec,
                    "peak_source": "derived: 152 SM x %s x 2 flop x 2070 MHz" % ("128 FP32 lanes" if fp32_like
                                                                                 else "2 FP64 FMA units"),
                    "kernel_ms_per_launch": kern_ms / max(kern_launches, 1), "launches": kern_launches,
                    "flops_per_esu": {str(N): flops_per_esu_1d(N) for N in orders},
                    "flops_rule": "6N^2+8N per ESU: the reduced remap's 2N^2 + 3N(N+2) flops plus N(N+2) "
                                  "divisions counted as one flop each"}
        line = {"metric": METRIC, "value": value, "unit": "ESU/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"mixed": "f32 (f32-pair state, f64 factor, f64 moments)",
                          "fp32": "f32 (f32-pair state, f64 moments)", "fp64": "f64"}[prec],
                "data": "synthetic",
                "config": {"workload": WORKLOAD if not args.quick else "quick: N=16 only, 50 SL steps",
                           "precision": prec, "dt": dt, "tolerance_vs_fp64": 1e-5,
                           "l2": "flushed between timed steps (256 MiB write)",
                           "parallelism": f"samples sharded over {world} GPU(s)"
                                          + ("; moments: chunk partials gathered in rank order (NCCL) and "
                                             "combined by the library" if world > 1 else "")},
                "roofline": roofline, "gpu_launches": gpu_launches, "clocks": clocks}

    summary = {}
    # ---------------------------------------------------------------- accuracy and other precisions
    if rank == 0 and not args.no_secondary:
        rates, acc, ref_moments = {}, {}, {}
        # fresh 1000-step solves from phi0 in every mode; the FP64 moments are
        # the reference (the FP64 GPU path is pinned to the FP64 oracle)
        # at the workload's dt, and for N=16 also at the bound itself (2 dt)
        cases = [(N, 1.0) for N in orders] + ([(16, 2.0)] if 16 in orders else [])
        for mode in ("fp64", "mixed", "fp32"):
            tot_ms, esu = 0.0, 0
            for N, frac in cases:
                pb = I.config2(N=N, steps=sl_steps)
                pb["dt"] = frac * dt
                warm = sl.Solver(I.with_(pb, M=64), mode, stream=stream.cuda_stream)
                warm.step(pb["dt"], 2)
                warm.close()
                s = sl.Solver(pb, mode, stream=stream.cuda_stream)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(stream):
                    e0.record(stream)
                    s.step(pb["dt"], sl_steps)
                    e1.record(stream)
                e1.synchronize()
                if frac == 1.0:
                    tot_ms += e0.elapsed_time(e1)
                    esu += K_ELEM * M_SAMPLES * sl_steps
                mean, _ = s.moments()
                s.close()
                key = (N, frac)
                if mode == "fp64":
                    ref_moments[key] = mean
                else:
                    r = ref_moments[key]
                    acc.setdefault(frac, {}).setdefault(mode, {})[str(N)] = float(
                        np.abs(mean - r).max() / np.abs(r).max())
            rates[mode] = esu / (tot_ms * 1e-3)
        tol = 1e-5
        modes = {}
        for mode, what in (("fp32", "f32-pair state, FP32 capacitance factor (the headline mode)"),
                           ("mixed", "f32-pair state, FP64 capacitance factor (Gram/factor in FP64)"),
                           ("fp64", "all FP64")):
            m = {"esu_per_s": rates[mode], "what": what}
            if mode != "fp64":
                errs = acc[1.0][mode]
                m["error_vs_fp64_at_dt"] = errs
                m["tolerance_met_at_dt"] = bool(max(errs.values()) <= tol)
                if 2.0 in acc:
                    m["error_vs_fp64_at_node_gap_bound"] = acc[2.0][mode]
            modes[mode] = m
        line["precision_modes"] = {
            "dt": dt, "tolerance_vs_fp64": tol, **modes,
            "error_what": "max |mean - mean_fp64| / max |mean_fp64| after 1000 steps from phi0, same seeds",
            "node_gap_bound": {"dt": 2 * dt, "tolerance_met": False if 2.0 in acc else None,
                               "why": "at the N=16 particle-gap bound (Eq. 1d_timestep) the step itself amplifies "
                                      "a perturbation ~0.85% per step (x5000 over 1000 steps; measured on the FP64 "
                                      "oracle), so FP32 rounding grows to ~1e-2 there; the 1e-5 bar holds at the "
                                      "bench's dt, half the bound"}}
        summary["esu_per_s"] = {k: rates[k] for k in ("fp32", "mixed", "fp64")}
        summary["max_error_vs_fp64_at_dt"] = {k: max(acc[1.0][k].values()) for k in ("fp32", "mixed")}

    # ---------------------------------------------------------------- end to end through the C ABI
    if rank == 0 and not args.no_e2e:
        x_nodes = {}
        for N in orders:
            # initial nodal values, evaluated by the library itself once and
            # kept in pinned host memory as the step's input
            with sl.Solver(I.with_(I.config2(N=N), M=1), prec) as s0:
                x_nodes[N] = torch.from_numpy(s0.samples(0, 1)[0].ravel().copy()).pin_memory()
        e2e_times = []
        h2d = d2h = 0
        for it in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h2d = d2h = 0
            for N in orders:
                pb = I.config2(N=N)
                phi0 = x_nodes[N].numpy()
                s = sl.Solver(pb, prec, stream=stream.cuda_stream, phi0_nodal=phi0, sample0=sample0)
                s.step(dt, sl_steps)
                mean, m2 = s.moments()
                s.close()
                h2d += phi0.nbytes
                d2h += mean.nbytes + m2.nbytes
            t = time.perf_counter() - t0
            if it >= args.warmup:
                e2e_times.append(t)
        line["e2e"] = {"value": esu_step / float(np.mean(e2e_times)), "unit": "ESU/s",
                       "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                       "what": "sl_init (phi0 from pinned host memory) + sl_step + sl_moments (to host) + "
                               "sl_free per order, wall clock"}

    if rank == 0 and not args.no_extra:
        line["moments_hbm"] = _moments_bandwidth(sl, stream)
        summary["moments_hbm_frac"] = line["moments_hbm"]["frac"]
        line["config3_2d"] = leg_2d(sl, stream)
        line["batch"] = leg_batch(sl, stream)
        line["serving"] = leg_serving(sl, args.serve_seconds, fp64_duration=min(args.serve_fp64_seconds,
                                                                                 args.serve_seconds))
        summary["config3_2d"] = line["config3_2d"].get("summary")
        summary["batch"] = line["batch"].get("summary")
        summary["serving"] = line["serving"].get("summary")

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline(args.cpu_seconds)

    if rank == 0:
        # the compact summary goes last: it stays readable in the tail of a long line
        line["summary"] = summary
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["mixed", "fp32", "fp64"])
    ap.add_argument("--quick", action="store_true", help="N=16 only, 50 SL steps (profiling)")
    ap.add_argument("--no-secondary", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-extra", action="store_true", help="skip the 2D, batch and serving legs")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-fp64-seconds", type=float, default=20.0)
    args = ap.parse_args()
    if args.warmup < 3 and not args.quick:
        args.warmup = 3
    return run_reference(args) if args.impl == "reference" else run_native(args)


if __name__ == "__main__":
    sys.exit(main())
