"""Benchmark of the batched Hermite-Fourier split step.

Workload (one bench "step"): one batched solve of 4096 independent 1D GPE
instances of mixed grid size N ~ U{128,...,4096} (half-width 8 + N/64,
omega(t) = omega0 (1 + 0.3 sin t), omega0 ~ U[0.5,2], sigma ~ U[-1,20],
eps ~ U[0,0.1], V_I = cos(kx), k ~ U[1,4], Gaussian psi0 of width
1/sqrt(omega0) at x0 ~ U[-1,1]), 500 Strang steps of dt = 0.005 with the
commutator-free Magnus-4 + Theorem-2 harmonic flow, complex64 -- one
hfs_step(500) call, replayed from a captured CUDA graph.

Metric: grid-point-steps per second (sum over instances of N x time steps).
Between timed steps a 256 MiB buffer is written to flush L2 (outside the
per-step CUDA events).  ``e2e`` repeats the solve through the public C ABI
with host buffers: host->device copy of psi0 from pinned memory, the solve,
device->host copy of psi(T), all inside the timed region.

``--impl reference`` times the FP64 CPU oracle (the slow, plain
stage-by-stage implementation the tests compare with) on a bounded,
stratified sample of the same workload.

Multi-GPU (torchrun): every rank solves its own 4096-instance batch (seed
offset by the rank) with no data-path communication; value = all ranks'
grid-point-steps / max over ranks of the timed span ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "grid-point-steps/s"
COUNT, STEPS, DT = 4096, 500, 0.005
# tuned plans, keyed by GPU, precision, kernel-source hash, mode and batch
# (written by the autotuner on a miss; see hfs_autotune_cache)
PLAN_CACHE = os.path.join(ROOT, "paper_1007_3470_gb300", "tuned_plans.json")


def tune(solver, trial_steps):
    """Plans from the cache, or the search (recorded in the cache when the file
    is writable); returns (plans, how they were obtained)."""
    plans = solver.autotune(trial_steps, cache=PLAN_CACHE)
    return plans, {"cache": os.path.relpath(PLAN_CACHE, ROOT), "hit": solver.tune_cache_hit}


# DRAM bytes per launch of the fused step kernel (dram__bytes_read.sum +
# dram__bytes_write.sum from one ncu capture of the same command, summarised in
# profiles/), valid only while the kernel's sources hash to "src".
STEP1D_TRAFFIC = {"src": "88d5e6598e9904c5",
                  "batch_1d_4096x500_c64": 109323520 + 16402432,
                  "batch_1d_65536x1_streaming": (727424512 + 646248960 + 727406080 + 643721728) // 2}
STEP1D_SOURCES = ("hfs_step1d.cuh", "hfs_step1d.cu", "hfs_step1d_vicos.cu", "hfs_step1d_vix4.cu", "hfs_step1d_vinone.cu",
                  "hfs_step1d_wide.cu", "hfs_step1d_wide_vicos.cu", "hfs_step1d_wide_vix4.cu",
                  "hfs_step1d_wide_vinone.cu", "hfs_fft.cuh", "hfs_phase.cuh", "hfs_internal.cuh", "hfs_sched.h")


def step1d_traffic(workload: str):
    """Captured DRAM bytes per launch for this workload, or None when the
    kernel sources changed since the capture (or the workload was not captured)."""
    import hashlib
    h = hashlib.sha256()
    try:
        for f in STEP1D_SOURCES:
            with open(os.path.join(ROOT, "paper_1007_3470_gb300", "csrc", f), "rb") as fh:
                h.update(fh.read())
    except OSError:
        return None
    if h.hexdigest()[:16] != STEP1D_TRAFFIC["src"]:
        return None
    return STEP1D_TRAFFIC.get(workload)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def rank_seed(rank: int) -> int:
    """Each rank solves its own batch: the workload seed offset by the rank
    (instances are independent, so the data path needs no communication)."""
    from paper_1007_3470_gb300 import workloads as W
    return W.SEED + rank


def reduce_times_max(times, dist, device):
    """Max over ranks of each timing (the job is as slow as its slowest rank)."""
    import torch
    t = torch.tensor([float(v) for v in times], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def reduce_sum(value: float, dist, device) -> float:
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t[0])


def aggregate_value(gps_all_ranks: float, steps: int, total_ms: float) -> float:
    """Whole-job throughput: the grid-point-steps of all ranks per solve, times
    the timed solves, over the max-over-ranks timed span."""
    return gps_all_ranks * steps / (total_ms * 1e-3)


def algorithmic_counts(insts, steps):
    """Per solve: grid-point-steps, algorithmic flops and streaming bytes.

    flops per grid-point-step: 10 log2 N (forward + inverse FFT, radix-2
    count 5 N log2 N each) + 22 (two complex phase multiplies of 6 flops,
    the merged phase argument kappa x^2/2 + s (eps V_I + sigma |u|^2) with
    |u|^2 and 7 more, and the kinetic argument g k^2/2 with 3); the two
    sine/cosine pairs per point-step are not counted as flops."""
    pts = np.array([i.n[0] for i in insts], dtype=np.float64)
    gps = float(pts.sum() * steps)
    flops = float(np.sum(pts * (10.0 * np.log2(pts) + 22.0)) * steps)
    return gps, flops


def extra_measurements(hfs, W, torch):
    """Secondary measurements (not the headline): the 3D GPE step, the
    streaming mode of the batched step (one launch, one global round trip
    per time step), and single-instance vs batched solves at N = 256."""
    out = {}

    def kernel_ms(solver, nsteps, reps=2):
        hfs.hfs_set_profiling(solver.h, True)
        solver.step(nsteps)
        best = 1e30
        for _ in range(reps):
            solver.step(nsteps)
            best = min(best, hfs.hfs_last_step_kernel_ms(solver.h))
        return best

    # 3D, 128^3, sigma = 100, 200 Strang / Magnus-4 steps
    inst, psi0, steps = W.gpe_3d(n=128, h=0.005, steps=200)
    s3 = hfs.Solver([inst], dim=3, precision="c64", chunk_steps=steps)
    s3.set_schedule(inst.h, "strang", hfs.HFS_FLOW_CF4)
    s3.set_graphs(True)
    s3.set_psi(psi0.ravel())
    ms = kernel_ms(s3, steps)
    gps = 128 ** 3 * steps
    # algorithmic traffic: two global round trips of the complex64 state per
    # sub-stage (the z-pass and the plane pass), 32 B per grid-point-step
    peaks, _ = _peaks()
    hbm3 = gps * 32 / (ms * 1e-3) / 1e9
    out["gpe3d_128cube_200steps_c64"] = {"kernel_ms": ms, "grid_point_steps_per_s": gps / (ms * 1e-3),
                                         "hbm_equivalent_GBps_32B": hbm3,
                                         "hbm_equivalent_frac_of_measured": hbm3 / float(peaks.get("hbm_gbs", 6800.0)),
                                         "error": gpe3d_error(hfs, s3, inst, psi0, steps)}
    # the same with the norm projection (plain twiddles)
    s3.set_norm_projection(True)
    s3.set_time(0.0)
    s3.set_psi(psi0.ravel())
    ms_p = kernel_ms(s3, steps)
    out["gpe3d_128cube_200steps_c64_projected"] = {
        "kernel_ms": ms_p, "grid_point_steps_per_s": gps / (ms_p * 1e-3),
        "hbm_equivalent_frac_of_measured": gps * 32 / (ms_p * 1e-3) / 1e9 / float(peaks.get("hbm_gbs", 6800.0)),
        "error": gpe3d_error(hfs, s3, inst, psi0, steps)}
    s3.set_norm_projection(False)
    # the same with the z-transforms' radix-16 stages on the tensor cores
    s3.set_dft_engine(hfs.HFS_DFT_TENSOR_3XTF32)
    s3.set_time(0.0)
    s3.set_psi(psi0.ravel())
    ms_tc = kernel_ms(s3, steps)
    out["gpe3d_128cube_200steps_c64_tensor_dft"] = {
        "kernel_ms": ms_tc, "grid_point_steps_per_s": gps / (ms_tc * 1e-3),
        "dft_stages": "radix-16 z-pass stages as 3xTF32 tcgen05 matrix products",
        "error": gpe3d_error(hfs, s3, inst, psi0, steps)}
    # tensor-core stages with the norm projection (which removes their norm bias)
    s3.set_norm_projection(True)
    s3.set_time(0.0)
    s3.set_psi(psi0.ravel())
    ms_tcp = kernel_ms(s3, steps)
    out["gpe3d_128cube_200steps_c64_tensor_dft_projected"] = {
        "kernel_ms": ms_tcp, "grid_point_steps_per_s": gps / (ms_tcp * 1e-3),
        "error": gpe3d_error(hfs, s3, inst, psi0, steps)}
    s3.close()
    # streaming mode of the batched workload (one launch per time step)
    insts, psis, _ = W.batch_1d(count=COUNT, h=DT, steps=STEPS)
    ss = hfs.Solver(insts, precision="c64", chunk_steps=STEPS)
    ss.set_schedule(DT, "strang", hfs.HFS_FLOW_CF4)
    ss.set_norm_projection(True)
    ss.set_mode(hfs.HFS_MODE_STREAMING, 1)
    tune(ss, 8)
    ss.set_graphs(True)
    ss.set_psi(psis)
    ms = kernel_ms(ss, STEPS)
    gps = sum(i.n[0] for i in insts) * STEPS
    out["batch_streaming_1step_per_launch"] = {"kernel_ms": ms, "grid_point_steps_per_s": gps / (ms * 1e-3),
                                               "hbm_equivalent_GBps": gps * 16 / (ms * 1e-3) / 1e9}
    ss.close()
    # single instance vs batch at N = 256, 200 steps (T = 1)
    one, p1, _ = W.batch_1d(count=4096, sizes=(256,), h=DT, steps=200)
    s1 = hfs.Solver(one[:1], precision="c64", chunk_steps=200)
    s1.set_schedule(DT, "strang", hfs.HFS_FLOW_CF4)
    s1.set_graphs(True)
    s1.set_psi(p1[:1])
    ms1 = kernel_ms(s1, 200)
    s1.close()
    sb = hfs.Solver(one, precision="c64", chunk_steps=200)
    sb.set_schedule(DT, "strang", hfs.HFS_FLOW_CF4)
    sb.set_graphs(True)
    sb.set_psi(p1)
    msb = kernel_ms(sb, 200)
    sb.close()
    out["n256_T1_single_vs_batch"] = {"single_solves_per_s": 1e3 / ms1, "batch4096_solves_per_s": 4096e3 / msb}
    out["ho_vs_f_split"] = split_comparison(hfs, W)
    out["batch65536_streaming_hbm"] = hbm_streaming_measurement(hfs, W)
    out["surrogate_fno"] = surrogate_measurement()
    return out


def split_comparison(hfs, W):
    """HO split vs F split at equal FFT count (Sec. 4): the leap-frog BAB
    composition with both splittings on the autonomous problem mu = omega = 1,
    V_I = 0, psi0 = rho exp(-(x-1)^2/2), N = 1024, T = 10, in FP64 on the GPU;
    relative L2 error against the oracle's NI_5(8,4) HO-split solution at
    dt = 0.001.  FFT pairs per solve = T / dt for both splits."""
    from oracle import oracle as O
    T, out = 10.0, {}
    for sigma, dts in ((0.01, (0.04, 0.02, 0.01, 0.005)), (1.0, (0.04, 0.02, 0.01, 0.005)),
                       (100.0, (0.01, 0.005, 0.0025))):
        ref_inst, psi0 = W.split_comparison_1d(sigma, h=0.001)
        ref_inst.scheme = "ni5_84"
        ref = O.run(O.Problem(**ref_inst.as_dict()), psi0, int(round(T / 0.001)))
        rows = []
        for h in dts:
            row = {"dt": h, "fft_pairs": int(round(T / h))}
            for split, name in ((W.SPLIT_HO, "ho"), (W.SPLIT_FOURIER, "f")):
                inst, _ = W.split_comparison_1d(sigma, h=h, split=split)
                s = hfs.Solver([inst], precision="c128", chunk_steps=512)
                s.set_schedule(h, "strang", hfs.HFS_FLOW_LEMMA2, split=split)
                s.set_psi([psi0])
                s.step(int(round(T / h)))
                row["err_" + name] = O.rel_l2(s.get_psi(), ref)
                s.close()
            rows.append(row)
        out[f"sigma_{sigma:g}"] = rows
    return out


def unprojected_drift(hfs, insts, psis, steps):
    """Relative norm change of every instance of the batch over one solve with
    the norm projection off (device norms, FP64 accumulation): the FP32
    rounding drift, a zero-mean random walk (signed mean next to rms and max)."""
    s = hfs.Solver(insts, precision="c64", chunk_steps=steps)
    s.set_schedule(DT, "strang", hfs.HFS_FLOW_CF4)
    s.set_psi(psis)
    n0 = s.norm()
    s.step(steps)
    d = s.norm() / n0 - 1.0
    s.close()
    return {"max_abs": float(np.abs(d).max()), "rms": float(np.sqrt(np.mean(d * d))), "mean": float(d.mean()),
            "instances": len(insts)}


def gpe3d_error(hfs, s32, inst, psi0, steps):
    """psi(T) of the complex64 3D solve from psi0 against the same solve in
    FP64 on the device (the 128^3 grid is beyond the oracle; the FP64 path is
    pinned to the oracle at 32^3 and 64^3 by the GPU tests)."""
    s32.set_time(0.0)
    s32.set_psi(psi0.ravel())
    s32.step(steps)
    u32 = np.asarray(s32.get_psi()).astype(np.complex128)
    n32 = float(s32.norm()[0])
    s64 = hfs.Solver([inst], dim=3, precision="c128", chunk_steps=steps)
    s64.set_schedule(inst.h, "strang", hfs.HFS_FLOW_CF4)
    s64.set_psi(psi0.ravel())
    s64.step(steps)
    u64 = np.asarray(s64.get_psi())
    n64 = float(s64.norm()[0])
    s64.close()
    T = steps * inst.h
    err = float(np.linalg.norm(u32 - u64) / np.linalg.norm(u64))
    return {"rel_l2_vs_fp64_device": err, "bound": 1e-5 * max(T, 1.0), "within_bound": err <= 1e-5 * max(T, 1.0),
            "norm_drift_c64": abs(n32 - 1.0), "norm_drift_c128": abs(n64 - 1.0)}


def hbm_streaming_measurement(hfs, W, count: int = 65536, steps: int = 20):
    """The streaming mode on a batch whose state exceeds L2: 65536 instances
    of the same law (about 700 MB complex64), one launch per time step, so
    every launch reads and writes the whole state in HBM."""
    insts, psis, _ = W.batch_1d(count=count, seed=W.SEED + 65536, h=DT, steps=steps)
    pts = sum(i.n[0] for i in insts)
    s = hfs.Solver(insts, precision="c64", chunk_steps=steps)
    s.set_schedule(DT, "strang", hfs.HFS_FLOW_CF4)
    s.set_norm_projection(True)
    s.set_mode(hfs.HFS_MODE_STREAMING, 1)
    # plans per grid size measured in this mode (8 trial steps per candidate)
    tuned, _ = tune(s, 8)
    s.set_graphs(True)
    hfs.hfs_set_profiling(s.h, True)
    s.set_psi(psis)
    s.step(steps)
    best = 1e30
    for _ in range(2):
        s.step(steps)
        best = min(best, hfs.hfs_last_step_kernel_ms(s.h))
    st = s.status()
    # the result of one solve from psi0 against the FP64 oracle on two
    # instances of every grid size
    s.set_time(0.0)
    s.set_psi(psis)
    s.step(steps)
    out = s.split(s.get_psi())
    s.close()
    from oracle import oracle as O
    pick, seen = [], {}
    for i, inst in enumerate(insts):
        if seen.get(inst.n[0], 0) < 2:
            seen[inst.n[0]] = seen.get(inst.n[0], 0) + 1
            pick.append(i)
    refs = O.run_batch([O.Problem(**insts[i].as_dict()) for i in pick], [psis[i] for i in pick], steps)
    errs = [O.rel_l2(out[i], r) for i, r in zip(pick, refs)]
    bound = 1e-5 * max(steps * DT, 1.0)
    peaks, src = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    gbps = pts * steps * 16.0 / (best * 1e-3) / 1e9
    traffic = step1d_traffic("batch_1d_65536x1_streaming") if count == 65536 else None
    return {"instances": count, "points": pts, "state_MB": pts * 8 / 1e6, "time_steps": steps,
            "ms_per_launch": best / steps, "grid_point_steps_per_s": pts * steps / (best * 1e-3),
            "hbm_GBps_algorithmic": gbps, "hbm_frac_of_measured": gbps / hbm,
            "algorithmic_bytes_per_launch": pts * 16, "dram_bytes_per_launch": traffic, "plans": tuned,
            "status": st,
            "error": {"rel_l2_max": float(max(errs)), "bound": bound, "within_bound": bool(max(errs) <= bound),
                      "instances": len(pick), "vs": "FP64 oracle"}}


def surrogate_measurement():
    """The FNO surrogate of the N = 256, T = 1 family: 20000 training and 2000
    held-out solver trajectories, 30 epochs, held-out error distribution, and
    its inference throughput (batch 4096) against the plain solver at the
    surrogate's accuracy and at the reference step."""
    import time
    from paper_1007_3470_gb300 import surrogate as S
    from paper_1007_3470_gb300.fno import Fno, FnoConfig
    t0 = time.perf_counter()
    tr_i, tr_p, _ = S.family(20000, seed=101)
    te_i, te_p, _ = S.family(2000, seed=202)
    Xtr, Xte = S.features(tr_i, tr_p), S.features(te_i, te_p)
    Ytr, Yte = S.solve(tr_i, tr_p), S.solve(te_i, te_p)
    t1 = time.perf_counter()
    m = Fno(FnoConfig(), max_batch=4096, train=True, seed=7)
    S.train(m, Xtr, Ytr, epochs=30, batch=256, lr=2e-3)
    t2 = time.perf_counter()
    err = S.rel_errors(S.predict(m, Xte, 4096), Yte)
    med = float(np.median(err))
    bi, bp, _ = S.family(4096, seed=303)
    fno_rate = S.time_inference(m, S.features(bi, bp))
    m.close()
    dt, smed = S.equal_accuracy_solver(te_i, te_p, Yte, med)
    return {"train_samples": 20000, "heldout": 2000, "epochs": 30, "data_s": t1 - t0, "train_s": t2 - t1,
            "heldout_rel_l2": {"median": med, "p90": float(np.percentile(err, 90)), "max": float(err.max())},
            "fno_solves_per_s_batch4096": fno_rate,
            "solver_equal_accuracy": {"dt": dt, "median_rel_l2": smed,
                                      "solves_per_s_batch4096": S.time_solver(bi, bp, dt)},
            "solver_reference_dt_solves_per_s_batch4096": S.time_solver(bi, bp, S.DT)}


def run_native(args):
    import torch
    import torch.distributed as dist

    from paper_1007_3470_gb300 import hfs
    from paper_1007_3470_gb300 import workloads as W

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    COUNT_, STEPS_ = args.count, args.time_steps
    insts, psis, _ = W.batch_1d(count=COUNT_, seed=rank_seed(rank), h=DT, steps=STEPS_)
    gps, flops = algorithmic_counts(insts, STEPS_)
    solver = hfs.Solver(insts, precision="c64", chunk_steps=STEPS_)
    solver.set_schedule(DT, "strang", hfs.HFS_FLOW_CF4)
    solver.set_norm_projection(not args.no_projection)
    # candidates timed on full-length solves (shorter trials keep the phase
    # records in L2 and misjudge the plans)
    tuned, tuned_from = tune(solver, STEPS_) if args.autotune else (None, None)
    # each call computes the next call's phase records in a branch parallel to
    # its step kernel (every timed call does one call's schedule work)
    solver.set_schedule_reuse(not args.no_schedule_reuse)
    hfs.hfs_set_profiling(solver.h, True)
    solver.set_graphs(True)
    host0 = np.concatenate([p.astype(np.complex64) for p in psis])
    pinned_in = torch.from_numpy(host0.view(np.float32)).pin_memory()
    pinned_out = torch.empty_like(pinned_in).pin_memory()
    solver.set_psi(host0)
    stream = solver.stream
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def one():
        solver.step(STEPS_)

    for _ in range(args.warmup):
        one()
    stream.synchronize()
    # device-timed value: per-step CUDA events on the solver's stream, L2 flushed between steps
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    kern_ms = []
    with Clocks(local) as clk:
        t_wall0 = time.perf_counter()
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)
            evs[k][0].record(stream)
            one()
            evs[k][1].record(stream)
            # fused step kernel alone (events recorded by the library on the same stream)
            kern_ms.append(hfs.hfs_last_step_kernel_ms(solver.h))
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
    if ws > 1:
        dist.barrier()
    ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(ms)
    st = solver.status()
    # the dominant kernel: one resident launch per solve (all time steps on chip)
    step_ms = sum(kern_ms) / len(kern_ms)
    # end to end through the C ABI with host buffers
    e2e_ms = []
    for k in range(max(2, min(args.steps, 5))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # a solve of the batch from psi0, starting where the previous call
        # ended (a restart at one fixed time would let the schedule reuse
        # keep that call's records instead of computing the next call's)
        hfs.hfs_set_psi(solver.h, pinned_in.data_ptr(), False)
        solver.step(STEPS_)
        hfs.hfs_get_psi(solver.h, pinned_out.data_ptr(), False)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_step_ms = statistics.median(e2e_ms)
    # the result checked against the oracle: a solve of the batch from psi0 at t = 0
    hfs.hfs_set_time(solver.h, 0.0)
    hfs.hfs_set_psi(solver.h, pinned_in.data_ptr(), False)
    solver.step(STEPS_)
    hfs.hfs_get_psi(solver.h, pinned_out.data_ptr(), False)
    total_ms, e2e_step_ms = reduce_times_max([total_ms, e2e_step_ms], dist if ws > 1 else None, "cuda")
    gps_all = reduce_sum(gps, dist if ws > 1 else None, "cuda")
    value = aggregate_value(gps_all, args.steps, total_ms)
    peaks, src = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    # FP32 FMA peak: 152 SMs x 128 lanes x 2 flop x max SM clock
    alu_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12
    achieved_tflops = flops / (step_ms * 1e-3) / 1e12
    hbm_equiv = gps * 16.0 / (step_ms * 1e-3) / 1e9
    workload = f"batch_1d_{COUNT_}x{STEPS_}_c64"
    line = {
        "metric": METRIC, "value": value, "unit": "grid-point-steps/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64 (f32)", "data": "synthetic",
        "config": {"workload": workload, "instances": COUNT_, "time_steps": STEPS_,
                   "dt": DT, "grid_sizes": "128..4096 uniform", "composition": "strang", "ho_flow": "magnus4_cf+thm2",
                   "mode": "resident, graph-replayed", "l2": "flushed between steps (256 MiB write)",
                   "norm_projection": not args.no_projection,
                   "schedule": "FP64 phase records of the next call computed parallel to the step kernel"
                               if not args.no_schedule_reuse else "FP64 phase records computed in line",
                   "solves_per_s": ws * args.steps / (total_ms * 1e-3),
                   "plans": tuned, "plans_from": tuned_from},
        "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": alu_peak, "unit": "TFLOP/s",
                     "frac": achieved_tflops / alu_peak, "traffic": step1d_traffic(workload),
                     "traffic_note": "DRAM bytes per launch (ncu); the state stays on chip for all time "
                                     "steps, the rest is the FP32 phase records (no register spills)",
                     "peak_source": f"FP32 FMA: 152 SM x 128 lanes x 2 x {sm_max:.0f} MHz (sm_max_mhz {src})",
                     "hbm_equivalent_GBps": hbm_equiv, "hbm_equivalent_frac_of_measured": hbm_equiv / hbm},
        "e2e": {"value": gps_all / (e2e_step_ms * 1e-3), "unit": "grid-point-steps/s",
                "h2d_bytes_per_step": int(host0.nbytes), "d2h_bytes_per_step": int(host0.nbytes)},
        # per solve (one schedule chunk, resident): law_nodes (the batch shares the trap law),
        # stage_flow, records, step1d, advance_time
        "gpu_launches": 5 * args.steps,
        "kernel_ms_per_launch": step_ms,
        "clocks": clk.summary(),
        "status": st,
        "wall_s": t_wall,
    }
    if rank == 0 and not args.no_extras:
        line["extras"] = extra_measurements(hfs, W, torch)
        line["extras"]["norm_drift_without_projection"] = unprojected_drift(hfs, insts, psis, STEPS_)
    if rank == 0 and not args.no_cpu_baseline:
        # pinned_out holds psi(T) of the solve from psi0 at t = 0
        same = COUNT_ == COUNT and STEPS_ == STEPS and rank_seed(rank) == 20100703
        final = pinned_out.numpy().view(np.complex64) if same else None
        line["cpu_baseline"] = cpu_baseline(args.cpu_sample, final, [i.n[0] for i in insts])
        if final is not None:
            line["error"] = line["cpu_baseline"].pop("error")
    if rank == 0:
        print(json.dumps(line))
    solver.close()
    if ws > 1:
        dist.destroy_process_group()


def _stratified_sample(per_size: int, seed: int, with_index: bool = False):
    from paper_1007_3470_gb300 import workloads as W
    insts, psis, _ = W.batch_1d(count=COUNT, seed=seed, h=DT, steps=STEPS)
    pick, seen = [], {}
    for i, inst in enumerate(insts):
        n = inst.n[0]
        if seen.get(n, 0) < per_size:
            seen[n] = seen.get(n, 0) + 1
            pick.append(i)
    out = [insts[i] for i in pick], [psis[i] for i in pick]
    return (*out, pick) if with_index else out


def result_error(gpu_state: np.ndarray, sizes, pick, psis0, refs) -> dict:
    """Relative L2 error of the GPU's psi(T) against the oracle's on the
    sampled instances (gpu_state: the whole batch, concatenated), and the norm
    drift dx sum |psi|^2 (T) - (0) of the GPU result."""
    off = np.concatenate([[0], np.cumsum(sizes)])
    errs, drift = [], []
    for i, p0, r in zip(pick, psis0, refs):
        g = gpu_state[off[i]:off[i + 1]].astype(np.complex128)
        errs.append(np.linalg.norm(g - r) / np.linalg.norm(r))
        drift.append(abs(np.sum(np.abs(g) ** 2) - np.sum(np.abs(p0) ** 2)) / np.sum(np.abs(p0) ** 2))
    T = STEPS * DT
    bound, dbound = 1e-5 * max(T, 1.0), 1e-6
    return {"rel_l2_max": float(np.max(errs)), "rel_l2_median": float(np.median(errs)),
            "bound": bound, "norm_drift_bound": dbound,
            "within_bound": bool(np.max(errs) <= bound and np.max(drift) <= dbound),
            "norm_drift_max": float(np.max(drift)), "norm_drift_median": float(np.median(drift)),
            "instances": len(errs), "vs": "FP64 oracle"}


def cpu_baseline(per_size: int, gpu_state=None, sizes=None):
    """The FP64 oracle, as it stands, on a stratified sample of the workload
    (per_size instances of every grid size, all 500 steps), OpenMP over
    instances on every host core.  With the GPU's final state of the same
    batch, its results also give the error of that state (result_error)."""
    from oracle import oracle as O
    insts, psis, pick = _stratified_sample(per_size, 20100703, with_index=True)
    probs = [O.Problem(**i.as_dict()) for i in insts]
    cores = O.max_threads()
    t0 = time.perf_counter()
    refs = O.run_batch(probs, psis, STEPS, cores)
    dt = time.perf_counter() - t0
    gps = sum(i.n[0] for i in insts) * STEPS
    out = {"value": gps / dt, "unit": "grid-point-steps/s", "cores": cores, "kind": "oracle",
           "sample": f"{len(insts)} instances ({per_size} per grid size 128..4096) x {STEPS} steps, "
                     f"FP64 stage-by-stage oracle, {dt:.1f} s"}
    if gpu_state is not None:
        out["error"] = result_error(gpu_state, sizes, pick, psis, refs)
    return out


def run_case(args):
    """One secondary workload alone (for profiling): 3d | fno | hbm (streaming
    mode on a batch larger than L2)."""
    import torch
    from paper_1007_3470_gb300 import hfs
    from paper_1007_3470_gb300 import workloads as W
    torch.cuda.set_device(0)
    if args.case == "3d":
        inst, psi0, steps = W.gpe_3d(n=128, h=0.005, steps=args.time_steps)
        s3 = hfs.Solver([inst], dim=3, precision="c64", chunk_steps=steps)
        s3.set_schedule(inst.h, "strang", hfs.HFS_FLOW_CF4)
        if args.tensor_dft:
            s3.set_dft_engine(hfs.HFS_DFT_TENSOR_3XTF32)
        hfs.hfs_set_profiling(s3.h, True)
        s3.set_psi(psi0.ravel())
        for _ in range(args.warmup):
            s3.step(steps)
        ms = []
        for _ in range(args.steps):
            s3.step(steps)
            ms.append(hfs.hfs_last_step_kernel_ms(s3.h))
        s3.close()
        print(json.dumps({"case": "3d", "n": 128, "time_steps": steps, "tensor_dft": args.tensor_dft, "kernel_ms": ms,
                          "grid_point_steps_per_s": 128 ** 3 * steps / (min(ms) * 1e-3)}))
    elif args.case == "fno":
        from paper_1007_3470_gb300 import surrogate as S
        from paper_1007_3470_gb300.fno import Fno, FnoConfig
        bi, bp, _ = S.family(args.count, seed=303)
        X = S.features(bi, bp)
        Y = S.solve(bi, bp)
        m = Fno(FnoConfig(), max_batch=args.count, train=True, seed=7)
        if args.tcgen05_gemm:
            from paper_1007_3470_gb300.fno import HFS_FNO_GEMM_TCGEN05
            m.set_gemm_engine(HFS_FNO_GEMM_TCGEN05)
        xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
        torch.cuda.synchronize()
        for _ in range(args.warmup):
            m.train_step(xd, yd, 1e-3, want_loss=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            m.train_step(xd, yd, 1e-3, want_loss=False)
        m.stream.synchronize()
        dt = (time.perf_counter() - t0) / args.steps
        rate = S.time_inference(m, X)
        m.close()
        print(json.dumps({"case": "fno", "batch": args.count, "tcgen05_gemm": args.tcgen05_gemm, "train_step_ms": dt * 1e3,
                          "inference_samples_per_s": rate}))
    elif args.case == "hbm":
        print(json.dumps({"case": "hbm", **hbm_streaming_measurement(hfs, W, count=args.count,
                                                                     steps=args.time_steps)}))
    else:
        raise SystemExit(f"unknown case {args.case}")


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state; each step below is a full bounded sample
    insts, psis = _stratified_sample(args.ref_sample, 20100703)
    probs = [O.Problem(**i.as_dict()) for i in insts]
    cores = O.max_threads()
    gps = sum(i.n[0] for i in insts) * STEPS
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.run_batch(probs, psis, STEPS, cores)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = gps * args.steps / total
    line = {
        "metric": METRIC, "value": value, "unit": "grid-point-steps/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128 (f64)", "data": "synthetic",
        "config": {"workload": "batch_1d_4096x500_c64", "instances": COUNT, "time_steps": STEPS, "dt": DT,
                   "sample_per_step": f"{len(insts)} instances stratified over grid sizes"},
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": "grid-point-steps/s", "cores": cores, "kind": "oracle",
                         "sample": f"{len(insts)} instances ({args.ref_sample} per grid size) x {STEPS} steps per step"},
        "e2e": {"value": value, "unit": "grid-point-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--cpu-sample", type=int, default=320,
                    help="instances per grid size in the cpu_baseline oracle sample (about 15 s on 16 cores)")
    ap.add_argument("--ref-sample", type=int, default=48,
                    help="instances per grid size in each step of --impl reference (about 2 s on 16 cores)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the secondary measurements")
    ap.add_argument("--no-schedule-reuse", action="store_true",
                    help="compute each call's phase records in line before its step kernel")
    ap.add_argument("--no-projection", action="store_true",
                    help="run the headline solve without the norm projection")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="skip the per-grid-size plan autotuner")
    ap.add_argument("--count", type=int, default=COUNT, help="instances per batch (profiling cases use fewer)")
    ap.add_argument("--time-steps", type=int, default=STEPS, help="time steps per solve")
    ap.add_argument("--tcgen05-gemm", action="store_true",
                    help="case fno: the row-streaming GEMMs on the tcgen05 engine")
    ap.add_argument("--tensor-dft", action="store_true",
                    help="--case 3d: the z-transforms' radix-16 stages on the tensor cores")
    ap.add_argument("--case", choices=["3d", "fno", "hbm"], default=None,
                    help="run one secondary workload alone (profiling)")
    args = ap.parse_args()
    if args.case:
        from paper_1007_3470_gb300 import build as B
        B.build()
        run_case(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        from paper_1007_3470_gb300 import build as B
        B.build()
        run_native(args)


if __name__ == "__main__":
    main()
