"""Benchmark: one force evaluation of the angular-momentum-conserving FMM (tree build +
forces) on a Plummer sphere of N = 2^20 particles, p = 4, theta = 0.6, leaf size 32,
binary64 -- particles per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbfmm|reference]

One step = fmm_build + fmm_forces on device-resident inputs.  Each timed step is
bracketed by CUDA events on the library's stream; between steps a 512 MiB buffer is
rewritten to flush the 129 MB L2.  Under torchrun every rank works on its own GPU with no
collective on the data path (weak scaling): a single system runs as independent replicas,
and the batch workload is sharded -- a batch of n_sys x WORLD_SIZE systems split across the
ranks by a longest-processing-time partition, so each rank carries about one n_sys batch of
work.  Rank 0 prints one JSON line with the whole-job throughput (all ranks' particles over
the max-over-ranks time).  `--impl reference` times the CPU
oracle (the FP64 C reference this library is checked against) on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(workload="plummer-1m-conserving", N=1 << 20, seed=2, p=4, theta=0.6, leaf=32,
                variant="conserving", precision="fp64")
# further synthetic workloads (sizes and orders of the paper-shaped test set); the default
# line is plummer1m
WORKLOADS = {
    "plummer1m": WORKLOAD,
    "plummer4k": dict(workload="plummer-4096", N=4096, seed=1, p=2, theta=0.5, leaf=16, variant="conserving",
                      precision="fp64", gen="plummer"),
    "binary4m": dict(workload="binary-2x2m", N=1 << 22, seed=3, p=6, theta=0.7, leaf=32, variant="conserving",
                     precision="mixed", gen="binary"),
    "batch512": dict(workload="batch-512-systems", N=None, seed=1000, p=4, theta=0.6, leaf=32,
                     variant="conserving", precision="mixed", gen="batch", n_sys=512, autotune=True),
    "disk16m": dict(workload="disk-bulge-16m", N=1 << 24, seed=5, p=5, theta=0.7, leaf=32, variant="conserving",
                    precision="mixed", gen="disk", leapfrog=20),
}
METRIC = "particles/s, AM-conserving FMM force eval, N=1M p=4 θ=0.6; force err; |Σx×F|"
CPU_SAMPLE_N = 1 << 19          # oracle sample: same generator, p, theta, leaf; ~15 s of CPU
STAGES = ("build", "moments", "walk", "m2l", "l2l", "p2p", "l2p")


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock/throttle sampling in the background during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def algorithmic_flops(counts, tree_counts, p, variant):
    """Algorithmic FLOPs of the dominant stages (FMA = 2):
    P2P: 26 per unordered particle pair (difference 3, r^2 5, rsqrt 1, r^-3 2, the two
    mass factors 2, two accumulations 12, one comparison counted 1).
    M2L per mutual cell pair: contraction terms of both partners x 2 flops plus one
    derivative-tensor evaluation of ~6 C(p+3,3) flops."""
    c = tree_counts
    m2l, p2p = counts
    selfp = p2p[:, 0] == p2p[:, 1]
    n_pp = int(np.where(selfp, c[p2p[:, 0]] * (c[p2p[:, 0]] - 1) // 2, c[p2p[:, 0]] * c[p2p[:, 1]]).sum())
    comb = math.comb
    if variant == 1:
        per_m2l = 2 * 2 * 4 * comb(p - 1 + 6, 6) + 6 * comb(p + 2, 3)
    else:
        per_m2l = 2 * 2 * comb(p + 6, 6) + 6 * comb(p + 3, 3)
    return {"p2p": 26.0 * n_pp, "m2l": float(per_m2l) * len(m2l), "n_pp": n_pp, "n_m2l": len(m2l),
            "per_m2l_pair": per_m2l}


# DRAM bytes (read + write) per unit of the dominant binary64 kernels, from ncu captures of
# their DRAM counters at N = 2^19 (p = 4), scaled by the units of the timed launch: per mutual
# M2L pair for the M2L stage (the pair-tensor kernel plus m2l_con_t_k), per particle pair for
# p2p_k.  Traffic grows in proportion to these units (per-pair tensors and partials).
NCU_TRAFFIC_PER_UNIT = {("m2l_con_t_k", "fp64"): 555.0, ("p2p_k", "fp64"): 5.24}


def fp64_peak_tflops(sm_mhz: float) -> float:
    """binary64 FMA rate of a GB300 from unit counts: 152 SMs x 2 FP64 FMA per SM per clock
    x 2 flops (context for the measured rate)."""
    return 152 * 2 * 2 * sm_mhz * 1e6 / 1e12


def fp32_peak_tflops(sm_mhz: float) -> float:
    """binary32 FMA rate of a GB300 from unit counts: 152 SMs x 128 FP32 FMA per SM per clock
    x 2 flops (context for the measured rate)."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


# bytes per particle of the tree build (bounding cube .. sorted SoA): read x, y, z, m (32 B),
# write key and index (12 B), one read and write of (key, index) per radix pass (24 B x 8
# passes), write the sorted SoA (32 B); and the one-pass minimum (read 32 B, write key and
# index 12 B, write the sorted SoA 32 B)
BUILD_BYTES_PER_PARTICLE = 268
BUILD_BYTES_MIN_PER_PARTICLE = 76


def workload_config(W, world, n_total, n_systems, tune=None):
    """The "config" object of the JSON line (the same for the GPU arm and the reference arm)."""
    return {"workload": W["workload"], "N": n_total, "n_systems": n_systems,
            "p": W["p"], "theta": W["theta"], "leaf_size": W["leaf"],
            "variant": W["variant"], "precision": W["precision"],
            "parallelism": (f"lpt-shard{world}" if W.get("n_sys_total") else f"replicas{world}"),
            "autotune": tune, "l2": "flushed between timed steps (512 MiB write)"}


def run_gbfmm(args):
    import torch
    from paper_2107_07166_gb300 import fmm, shard, synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    W = dict(WORKLOADS[args.workload])
    if args.n:
        W["N"] = args.n
        W["workload"] = f"plummer-{args.n}-{args.variant}"
    if args.variant_set:
        W["variant"] = args.variant
    if args.precision_set or args.workload == "plummer1m":
        W["precision"] = args.precision
    args.precision = W["precision"]
    args.variant = W["variant"]
    gen = W.get("gen", "plummer")
    offsets = None
    if gen == "binary":
        x, m = synth.binary(W["N"] // 2, W["seed"], W["seed"] + 1)
    elif gen == "disk":
        x, m = synth.disk_bulge(W["N"], W["seed"])
    elif gen == "batch":
        if world > 1:
            # the units are systems: rank r takes its part of a batch of n_sys x world
            n_glob = W["n_sys"] * world
            sizes, _ = synth.batch_sizes(n_glob, W["seed"])
            mine = shard.lpt_partition(sizes, world)[rank]
            x, m, offsets = synth.batch_subset(n_glob, W["seed"], mine)
            W["n_sys_total"] = n_glob
        else:
            x, m, offsets = synth.batch(W["n_sys"], W["seed"])
        W["N"] = int(offsets[-1])
    else:
        x, m = synth.plummer(W["N"], W["seed"])
    N = W["N"]
    xd = torch.from_numpy(x).to(dev)
    md = torch.from_numpy(m).to(dev)
    acc = torch.empty((N, 3), dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(device=dev)
    prec = {"fp64": fmm.FP64, "df64": fmm.DF64, "mixed": fmm.MIXED}[args.precision]
    # measured FMA rate of the units the pair kernels run on (roofline denominator), untimed
    alu_peak = fmm.probe_fma_rate(local, fmm.MIXED if prec == fmm.MIXED else fmm.FP64)
    f = fmm.FMM(local, prec, stream)
    variant = fmm.CONSERVING if args.variant == "conserving" else fmm.STANDARD
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    # leaf size and M2L tile length chosen by the library's autotuner (untimed)
    tune = None
    if W.get("autotune") and not args.autotune:
        # the tuned values of the workload (leaf 32 with 64-entry M2L tiles on every run so
        # far), without the trial evaluations: for profiling runs
        W["leaf"] = 32
        f.set_tiles(64)
    if W.get("autotune") and args.autotune:
        leaves, chunks = (16, 24, 32, 48, 64), (16, 32, 64)
        with torch.cuda.stream(stream):
            bl, bc, tms = f.autotune(xd, md, W["p"], W["theta"], variant, leaf_sizes=leaves, m2l_chunks=chunks,
                                     offsets=offsets, reps=2)
        stream.synchronize()
        W["leaf"] = bl
        tune = {"leaf_sizes": list(leaves), "m2l_chunks": list(chunks), "best_leaf": bl, "best_m2l_chunk": bc,
                "best_ms": tms}

    def step():
        if offsets is not None:
            f.build_batch(xd, md, offsets, W["leaf"])
        else:
            f.build(xd, md, W["leaf"])
        f.forces(W["p"], W["theta"], variant, acc, None)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    stream.synchronize()

    # structure counts for the algorithmic work model (not timed)
    tree = f.get_tree()
    lists = f.get_lists()
    work = algorithmic_flops(lists, tree["count"].astype(np.int64), W["p"], variant)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    sampler = ClockSampler(local)
    barrier()
    sampler.start()
    step_ms, stage_ms = [], {s: [] for s in STAGES}
    l0 = fmm.kernel_launches()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        st = f.stage_times()
        for s in STAGES:
            stage_ms[s].append(st[s])
    launches = (fmm.kernel_launches() - l0) // max(args.steps, 1) * args.steps
    barrier()
    clocks = sampler.stop()

    # forces on the built tree (moments and lists kept): direct fmm_forces calls against
    # the same evaluation recorded once as a CUDA graph (fmm_forces_graph); untimed by the line
    graph = None
    if world == 1:
        out_d, out_g = torch.empty_like(acc), torch.empty_like(acc)

        def timed(fn, reps=5):
            ts_ = []
            for _ in range(reps):
                with torch.cuda.stream(stream):
                    flush.fill_(1)
                stream.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                e1.synchronize()
                ts_.append(e0.elapsed_time(e1))
            return statistics.mean(ts_)

        with torch.cuda.stream(stream):
            f.forces(W["p"], W["theta"], variant, out_d, None)
            f.forces_graph(W["p"], W["theta"], variant, out_g, None)  # records the graph
        stream.synchronize()
        k0 = fmm.kernel_launches()
        t_dir = timed(lambda: f.forces(W["p"], W["theta"], variant, out_d, None), reps=1)
        k_dir = fmm.kernel_launches() - k0
        t_dir, t_gr = [], []
        for _ in range(5):  # alternated, so that a clock change shows in both
            t_gr.append(timed(lambda: f.forces_graph(W["p"], W["theta"], variant, out_g, None), reps=1))
            t_dir.append(timed(lambda: f.forces(W["p"], W["theta"], variant, out_d, None), reps=1))
        t_dir, t_gr = statistics.mean(t_dir), statistics.mean(t_gr)
        graph = {"forces_direct_ms": t_dir, "forces_graph_ms": t_gr, "kernels_per_forces": k_dir,
                 "graph_launches_per_forces": 1, "bitwise_equal": bool(torch.equal(out_d, out_g))}
    t_step = sum(step_ms) / len(step_ms) / 1e3
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([t_step], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_step = float(t.item())
    n_total = N * world  # replicas
    if world > 1 and W.get("n_sys_total"):
        import torch.distributed as dist
        tn = torch.tensor([float(N)], dtype=torch.float64, device=dev)
        dist.all_reduce(tn, op=dist.ReduceOp.SUM)
        n_total = int(tn.item())
    value = n_total / t_step

    # end to end through the public API with host buffers (pinned), copies inside
    xh = torch.from_numpy(x).pin_memory()
    mh = torch.from_numpy(m).pin_memory()
    acch = torch.empty((N, 3), dtype=torch.float64).pin_memory()
    e2e_t = []
    for _ in range(max(2, min(args.steps, 5))):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        if offsets is not None:
            f.build_batch(xh, mh, offsets, W["leaf"])
        else:
            f.build(xh, mh, W["leaf"])
        f.forces(W["p"], W["theta"], variant, acch, None)
        torch.cuda.synchronize(dev)
        e2e_t.append(time.perf_counter() - t0)
    e2e_step = statistics.median(e2e_t)
    if world > 1:
        import torch.distributed as dist
        te = torch.tensor([e2e_step], dtype=torch.float64, device=dev)
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e_step = float(te.item())

    # accuracy and conservation of the timed configuration
    Fsum, Tsum = f.diagnostics()
    a = acc.cpu().numpy()
    err = {"vs_direct_sampled": sampled_direct_error(torch, dev, x, m, a, offsets=offsets)}
    if prec != fmm.FP64:     # the binary64 mode on the same input, untimed
        g = fmm.FMM(local, fmm.FP64, stream)
        ref = torch.empty_like(acc)
        with torch.cuda.stream(stream):
            if offsets is not None:
                g.build_batch(xd, md, offsets, W["leaf"])
            else:
                g.build(xd, md, W["leaf"])
            g.forces(W["p"], W["theta"], variant, ref, None)
        stream.synchronize()
        r = ref.cpu().numpy()
        err["vs_fp64_gpu"] = float(np.linalg.norm(a - r) / np.linalg.norm(r))
        pe = np.linalg.norm(a - r, axis=1) / np.maximum(np.linalg.norm(r, axis=1), 1e-300)
        err["vs_fp64_gpu_per_particle"] = {"median": float(np.median(pe)), "max": float(pe.max())}
        g.close()
    ts = float((m * np.linalg.norm(x, axis=1) * np.linalg.norm(a, axis=1)).sum())
    fsum = float((m * np.linalg.norm(a, axis=1)).sum())

    # momentum drift over leapfrog steps (the workload's drift run), untimed
    leap = None
    lf_steps = W.get("leapfrog", args.leapfrog) if args.leapfrog > 0 else 0
    if lf_steps > 0 and world == 1 and gen in ("plummer", "disk"):
        if gen == "disk":
            _, _, v0 = synth.disk_bulge(N, W["seed"], velocities=True)
        else:
            _, _, v0 = synth.plummer(N, W["seed"], velocities=True)
        xl = torch.from_numpy(x).to(dev)
        vl = torch.from_numpy(v0).to(dev)
        t0 = time.perf_counter()
        dg = f.leapfrog(xl, vl, md, W["leaf"], W["p"], W["theta"], variant, 1e-3, lf_steps)
        tl = time.perf_counter() - t0
        Pm, Lm = dg[:, :3], dg[:, 3:]
        pscale = float((m * np.linalg.norm(v0, axis=1)).sum())
        lscale = float((m * np.linalg.norm(x, axis=1) * np.linalg.norm(v0, axis=1)).sum())
        leap = {"steps": lf_steps, "dt": 1e-3, "seconds": tl,
                "max_dP_rel": float(np.abs(Pm - Pm[0]).max() / pscale),
                "max_dL_rel": float(np.abs(Lm - Lm[0]).max() / lscale),
                "norm": "|sum m v - initial| / sum m|v|, |sum m x x v - initial| / sum m|x||v|"}

    # the other variant on the same input and tree (same timing method): the cost of
    # realignment is the conserving time over the standard time
    variants = {}
    if args.modes and world == 1:
        other = fmm.STANDARD if variant == fmm.CONSERVING else fmm.CONSERVING
        out = torch.empty_like(acc)

        def sv():
            if offsets is not None:
                f.build_batch(xd, md, offsets, W["leaf"])
            else:
                f.build(xd, md, W["leaf"])
            f.forces(W["p"], W["theta"], other, out, None)

        with torch.cuda.stream(stream):
            for _ in range(3):
                sv()
        stream.synchronize()
        ts_ = []
        for _ in range(max(3, min(args.steps, 5))):
            with torch.cuda.stream(stream):
                flush.fill_(1)
            stream.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sv()
            e1.record(stream)
            e1.synchronize()
            ts_.append(e0.elapsed_time(e1))
        tm = statistics.mean(ts_)
        o = out.cpu().numpy()
        variants["standard" if other == fmm.STANDARD else "conserving"] = {
            "value": N / (tm / 1e3), "ms_per_step": tm,
            "force_err_rel_l2": {"vs_direct_sampled": sampled_direct_error(torch, dev, x, m, o, offsets=offsets)},
            "stage_ms": {k: round(v, 4) for k, v in f.stage_times().items()}}

    # accuracy-matched comparison: the realigned form costs accuracy at equal order, so it
    # is also timed one order higher (conserving at p + 1) against the standard form at p,
    # on the same input and tree, with the error of each against the direct sum
    matched = None
    if args.modes and world == 1 and W["p"] + 1 <= (fmm.MIXED_P_MAX if prec == fmm.MIXED else
                                                   (fmm.DF64_P_MAX if prec == fmm.DF64 else fmm.P_MAX)):
        out = torch.empty_like(acc)
        rows = {}
        for name, pp, vv in (("standard_p", W["p"], fmm.STANDARD), ("conserving_p", W["p"], fmm.CONSERVING),
                             ("conserving_p_plus_1", W["p"] + 1, fmm.CONSERVING)):
            def sv():
                if offsets is not None:
                    f.build_batch(xd, md, offsets, W["leaf"])
                else:
                    f.build(xd, md, W["leaf"])
                f.forces(pp, W["theta"], vv, out, None)

            with torch.cuda.stream(stream):
                for _ in range(3):
                    sv()
            stream.synchronize()
            ts_ = []
            for _ in range(max(3, min(args.steps, 5))):
                with torch.cuda.stream(stream):
                    flush.fill_(1)
                stream.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sv()
                e1.record(stream)
                e1.synchronize()
                ts_.append(e0.elapsed_time(e1))
            o = out.cpu().numpy()
            Fm, Tm = f.diagnostics()
            rows[name] = {"p": pp, "variant": "standard" if vv == fmm.STANDARD else "conserving",
                          "ms_per_step": statistics.mean(ts_),
                          "force_err_vs_direct_sampled": sampled_direct_error(torch, dev, x, m, o, offsets=offsets),
                          "net_torque_rel": float(np.linalg.norm(Tm) / float(
                              (m * np.linalg.norm(x, axis=1) * np.linalg.norm(o, axis=1)).sum()))}
        s0, s1 = rows["standard_p"], rows["conserving_p_plus_1"]
        matched = dict(rows, time_ratio_conserving_p_plus_1_over_standard_p=s1["ms_per_step"] / s0["ms_per_step"],
                       err_ratio_conserving_p_plus_1_over_standard_p=(s1["force_err_vs_direct_sampled"]
                                                                      / s0["force_err_vs_direct_sampled"]))

    # the fused schedule (no interaction lists; binary64) on the same input and variant
    schedules = None
    if args.modes and world == 1 and prec == fmm.FP64 and W["p"] <= 6:
        out = torch.empty_like(acc)
        f.set_schedule(fmm.SCHEDULE_FUSED)

        def sf():
            if offsets is not None:
                f.build_batch(xd, md, offsets, W["leaf"])
            else:
                f.build(xd, md, W["leaf"])
            f.forces(W["p"], W["theta"], variant, out, None)

        with torch.cuda.stream(stream):
            for _ in range(3):
                sf()
        stream.synchronize()
        ts_ = []
        for _ in range(max(3, min(args.steps, 5))):
            with torch.cuda.stream(stream):
                flush.fill_(1)
            stream.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sf()
            e1.record(stream)
            e1.synchronize()
            ts_.append(e0.elapsed_time(e1))
        o = out.cpu().numpy()
        schedules = {"fused": {"ms_per_step": statistics.mean(ts_), "value": N / (statistics.mean(ts_) / 1e3),
                               "force_err_vs_list_schedule": float(np.linalg.norm(o - a) / np.linalg.norm(a)),
                               "stage_ms": {k: round(v, 4) for k, v in f.stage_times().items()}}}
        f.set_schedule(fmm.SCHEDULE_LISTS)

    # the other arithmetic modes of the pair kernels on the same input (same timing method)
    modes = {}
    if args.modes and world == 1 and args.workload == "plummer1m" and not args.n:
        for name in ("fp64", "df64", "mixed"):
            if name == args.precision:
                continue
            pm = {"fp64": fmm.FP64, "df64": fmm.DF64, "mixed": fmm.MIXED}[name]
            h = fmm.FMM(local, pm, stream)
            out = torch.empty_like(acc)

            def st():
                h.build(xd, md, W["leaf"])
                h.forces(W["p"], W["theta"], variant, out, None)

            with torch.cuda.stream(stream):
                for _ in range(3):
                    st()
            stream.synchronize()
            ts_ = []
            for _ in range(max(3, min(args.steps, 5))):
                with torch.cuda.stream(stream):
                    flush.fill_(1)
                stream.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                st()
                e1.record(stream)
                e1.synchronize()
                ts_.append(e0.elapsed_time(e1))
            o = out.cpu().numpy()
            ref = a if args.precision == "fp64" else None
            if ref is None:
                g = fmm.FMM(local, fmm.FP64, stream)
                rr = torch.empty_like(acc)
                with torch.cuda.stream(stream):
                    g.build(xd, md, W["leaf"])
                    g.forces(W["p"], W["theta"], variant, rr, None)
                stream.synchronize()
                ref = rr.cpu().numpy()
                g.close()
            tm = statistics.mean(ts_)
            pe = np.linalg.norm(o - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-300)
            modes[name] = {"value": N / (tm / 1e3), "ms_per_step": tm,
                           "dtype": {"fp64": "f64", "df64": "f32x2", "mixed": "f32"}[name],
                           "force_err_vs_fp64_gpu": float(np.linalg.norm(o - ref) / np.linalg.norm(ref)),
                           "force_err_per_particle_vs_fp64_gpu": {"median": float(np.median(pe)),
                                                                  "max": float(pe.max())},
                           "stage_ms": {k: round(v, 4) for k, v in h.stage_times().items()}}
            h.close()

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return None

    stage_avg = {s: (statistics.mean(v) if v and v[0] >= 0 else None) for s, v in stage_ms.items()}
    # the dominant pair stage by its event time (the binary64 M2L stage is the pair-tensor
    # kernel, the contraction, the reduction, the source ids and the root-relative term; its
    # algorithmic flops are rated against the whole stage's time)
    dom = "m2l" if (stage_avg["m2l"] or 0) >= (stage_avg["p2p"] or 0) else "p2p"
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    nominal = fp32_peak_tflops(2070.0) if args.precision == "mixed" else fp64_peak_tflops(2070.0)
    peak = alu_peak or nominal
    unit_name = "binary32" if args.precision == "mixed" else "binary64"
    basis = (f"measured live: {unit_name} FMA-chain probe (fmm_probe_fma_rate, best of 3) = {alu_peak:.4g} TFLOP/s; "
             f"unit-count figure {nominal:.4g} TFLOP/s (152 SMs x "
             f"{'128 FFMA' if args.precision == 'mixed' else '2 DFMA'}/clk x 2 flops x 2070 MHz)"
             if alu_peak else f"{unit_name} unit-count figure (probe unavailable)")
    if args.precision == "df64":
        basis += "; the double-float kernels run on the binary32 units and are rated against the binary64 peak they replace"
    def stage_roofline(st):
        """roofline of one pair stage: algorithmic flops over its event time, ncu traffic"""
        achieved = work[st] / (stage_avg[st] / 1e3) / 1e12
        if st == "m2l":
            shared = args.precision == "fp64" and W["p"] <= 6  # binary64 M2L on shared pair tensors
            kname = ("m2l_con" if variant == 1 else "m2l_std") + ("_t_k" if shared else "_k")
        else:
            kname = "p2p_k" if args.precision != "mixed" else "p2p_ring_k"
        per_unit = NCU_TRAFFIC_PER_UNIT.get((kname, args.precision)) if W["p"] == 4 else None
        units = work["n_m2l"] if st == "m2l" else work["n_pp"]
        return {"bound": "alu", "achieved": round(achieved, 4), "peak": round(peak, 4), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4),
                "traffic": (round(per_unit * units) if per_unit else None),
                "traffic_basis": (("ncu dram bytes per unit at N=2^19 (m2l_ptensor_k + m2l_con_t_k, the M2L stage), "
                                   "scaled to this launch") if per_unit and st == "m2l" else
                                  ("ncu dram bytes per unit at N=2^19, scaled to this launch" if per_unit else None)),
                "kernel": kname,
                "peak_basis": basis, "sm_mhz_median": sm_mhz}

    roofline = stage_roofline(dom)
    # both pair stages, since their times are close: the algorithmic count of a particle pair
    # (26 flops, the reciprocal square root counted as one) is far below the binary64
    # instructions it takes, so the P2P line reads low while its binary64 pipe is busy
    roofline_stages = {st: stage_roofline(st) for st in ("m2l", "p2p") if stage_avg[st]}
    # the tree build (bounding cube .. r_max) against the measured HBM copy bandwidth, on the
    # byte model of the build above (and its one-pass minimum)
    hbm = measured_peaks().get("hbm_gbs")
    roofline_build = None
    if stage_avg["build"] and hbm:
        gbs = BUILD_BYTES_PER_PARTICLE * N / (stage_avg["build"] / 1e3) / 1e9
        roofline_build = {"bound": "hbm", "achieved": round(gbs, 2), "peak": hbm, "unit": "GB/s",
                          "frac": round(gbs / hbm, 4), "bytes_per_particle": BUILD_BYTES_PER_PARTICLE,
                          "achieved_min_model": round(BUILD_BYTES_MIN_PER_PARTICLE * N / (stage_avg["build"] / 1e3) / 1e9, 2),
                          "bytes_per_particle_min_model": BUILD_BYTES_MIN_PER_PARTICLE,
                          "stage_ms": stage_avg["build"], "peak_basis": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                          "note": "whole build stage (cube, keys, sort, gather, octree, COM, r_max) by CUDA events"}
    cpu = cpu_baseline() if (args.cpu_baseline and world == 1 and not args.n and args.workload == "plummer1m") else None
    rng = np.random.default_rng(0)
    line = {
        "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "df64": "f32x2", "mixed": "f32"}[args.precision],
        "data": {"plummer": "synthetic (seeded Plummer sphere)",
                 "binary": "synthetic (seeded binary of two Plummer spheres, 10 apart)",
                 "disk": "synthetic (seeded exponential disk + Hernquist bulge)",
                 "batch": "synthetic (seeded batch of Plummer/Hernquist systems, log-uniform sizes)"}[gen],
        "config": workload_config(W, world, n_total if W.get("n_sys_total") else N,
                                  W.get("n_sys_total") or (len(offsets) - 1 if offsets is not None else 1), tune),
        "stage_ms": {k: (round(v, 4) if v is not None else None) for k, v in stage_avg.items()},
        "work": {"n_m2l_pairs": work["n_m2l"], "n_p2p_particle_pairs": work["n_pp"],
                 "m2l_flops": work["m2l"], "p2p_flops": work["p2p"]},
        "force_err_rel_l2": err,
        "net_force_rel": float(np.linalg.norm(Fsum) / fsum), "net_torque_rel": float(np.linalg.norm(Tsum) / ts),
        "roofline": roofline,
        "roofline_stages": roofline_stages,
        "roofline_build": roofline_build,
        "accuracy_matched": matched,
        "schedules": schedules,
        "graph": graph,
        "variants": variants or None,
        "modes": modes or None,
        "leapfrog": leap,
        "e2e": {"value": n_total / e2e_step, "unit": "particles/s", "h2d_bytes_per_step": int(32 * N),
                "d2h_bytes_per_step": int(24 * N)},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return line


def sampled_direct_error(torch, dev, x, m, a, n_targets=400, offsets=None):
    """Relative L2 error of accelerations a (N x 3) against the direct sum (eq. jia) on
    n_targets sampled particles, evaluated with plain binary64 tensor operations.  With
    offsets (a batch of independent systems) each target sums over its own system only."""
    rng = np.random.default_rng(0)
    tg = np.sort(rng.choice(x.shape[0], n_targets, replace=False))
    X = torch.from_numpy(x).to(dev)
    M = torch.from_numpy(m).to(dev)
    ref = torch.zeros((n_targets, 3), dtype=torch.float64, device=dev)
    if offsets is not None:
        sys_of = np.searchsorted(offsets, tg, side="right") - 1
        for k, t in enumerate(tg):
            lo, hi = int(offsets[sys_of[k]]), int(offsets[sys_of[k] + 1])
            d = X[int(t)][None, :] - X[lo:hi]
            r2 = (d * d).sum(-1)
            inv3 = torch.where(r2 > 0, r2.rsqrt() ** 3, torch.zeros_like(r2))
            ref[k] = -(M[lo:hi, None] * d * inv3[:, None]).sum(0)
        ref = ref.cpu().numpy()
        return float(np.linalg.norm(a[tg] - ref) / np.linalg.norm(ref))
    ch = max(1, min(16, (1 << 25) // x.shape[0]))               # targets per chunk
    for i0 in range(0, n_targets, ch):
        t = torch.from_numpy(tg[i0:i0 + ch]).to(dev)
        d = X[t][:, None, :] - X[None, :, :]                      # (ch, N, 3)
        r2 = (d * d).sum(-1)
        inv3 = torch.where(r2 > 0, r2.rsqrt() ** 3, torch.zeros_like(r2))
        ref[i0:i0 + ch] = -(M[None, :, None] * d * inv3[..., None]).sum(1)
    ref = ref.cpu().numpy()
    return float(np.linalg.norm(a[tg] - ref) / np.linalg.norm(ref))


def oracle_sample_rate(n=CPU_SAMPLE_N):
    """The CPU oracle on a bounded sample of the workload (same generator, p, theta, leaf,
    variant; n particles): particles/s and seconds."""
    import oracle
    from paper_2107_07166_gb300 import synth
    W = WORKLOAD
    x, m = synth.plummer(n, W["seed"])
    oracle.build()
    t0 = time.perf_counter()
    oracle.run(x, m, W["leaf"], W["p"], W["theta"], 1, want_pot=False, want_internals=False)
    dt = time.perf_counter() - t0
    return n / dt, dt


def cpu_baseline():
    rate, dt = oracle_sample_rate()
    return {"value": rate, "unit": "particles/s", "cores": 1, "kind": "oracle",
            "sample": f"Plummer N={CPU_SAMPLE_N} (seed 2), p=4, theta=0.6, leaf 32, conserving, "
                      f"one build+forces, {dt:.1f} s single-threaded"}


# per-step sample of the reference arm: a quarter of the workload, so that a run of 20
# timed + 5 warm-up steps ends within a few minutes on one host core
REF_SAMPLE_N = 1 << 18


def workload_inputs(W, n=None, n_sys=None):
    """Seeded inputs of a workload (optionally a smaller sample of the same generator):
    x, m and the batch offsets (None for one system)."""
    from paper_2107_07166_gb300 import synth
    gen = W.get("gen", "plummer")
    N = n or W["N"]
    if gen == "binary":
        x, m = synth.binary(N // 2, W["seed"], W["seed"] + 1)
    elif gen == "disk":
        x, m = synth.disk_bulge(N, W["seed"])
    elif gen == "batch":
        x, m, off = synth.batch(n_sys or W["n_sys"], W["seed"])
        return x, m, off
    else:
        x, m = synth.plummer(N, W["seed"])
    return x, m, None


def oracle_extrapolated(W):
    """Oracle time of a workload too large to run in full on one host core.  The oracle
    (conserving, the workload's p, theta, leaf size) runs once on a sample of the same
    generator (N = 2^17, or 32 systems of a batch) with its own stage timers; each stage's
    time per unit (P2P per unordered particle pair, M2L per mutual pair, the walk per
    visited pair, the rest per particle with an N log N factor for the tree) is applied to
    the full workload's exact walk counts (oracle.counts: tree and walk only).  Returns a
    dict; the figure is an extrapolation, not a run of the full workload."""
    import oracle
    oracle.build()
    smp = dict(n_sys=32) if W.get("gen") == "batch" else dict(n=1 << 17)
    x, m, off = workload_inputs(W, **smp)
    bounds = [(0, x.shape[0])] if off is None else list(zip(off[:-1], off[1:]))
    st = dict(tree=0.0, moments=0.0, walk=0.0, m2l=0.0, l2l_l2p=0.0, p2p=0.0)
    cnt = np.zeros(4, dtype=np.int64)
    nlogn = 0.0
    for a, b in bounds:
        r = oracle.run(x[a:b], m[a:b], W["leaf"], W["p"], W["theta"], 1, want_pot=False, want_internals=False)
        for k, v in r.stage_seconds.items():
            st[k] += v
        cnt += np.array(oracle.counts(x[a:b], m[a:b], W["leaf"], W["theta"]))
        nlogn += (b - a) * math.log2(b - a)
    ns = x.shape[0]
    per = {"p2p_per_particle_pair": st["p2p"] / cnt[3], "m2l_per_pair": st["m2l"] / cnt[1],
           "walk_per_pair": st["walk"] / (cnt[1] + cnt[2]), "tree_per_nlogn": st["tree"] / nlogn,
           "moments_l2p_per_particle": (st["moments"] + st["l2l_l2p"]) / ns}
    x, m, off = workload_inputs(W)
    bounds = [(0, x.shape[0])] if off is None else list(zip(off[:-1], off[1:]))
    full = np.zeros(4, dtype=np.int64)
    nlogn_f = 0.0
    t0 = time.perf_counter()
    for a, b in bounds:
        full += np.array(oracle.counts(x[a:b], m[a:b], W["leaf"], W["theta"]))
        nlogn_f += (b - a) * math.log2(b - a)
    tc = time.perf_counter() - t0
    N = x.shape[0]
    parts = {"p2p": per["p2p_per_particle_pair"] * full[3], "m2l": per["m2l_per_pair"] * full[1],
             "walk": per["walk_per_pair"] * (full[1] + full[2]), "tree": per["tree_per_nlogn"] * nlogn_f,
             "moments_l2l_l2p": per["moments_l2p_per_particle"] * N}
    est = float(sum(parts.values()))
    return {"N": N, "extrapolated_seconds": est, "particles_per_s": N / est,
            "seconds_by_stage": {k: float(v) for k, v in parts.items()},
            "seconds_per_unit": {k: float(v) for k, v in per.items()},
            "full_counts": {"n_nodes": int(full[0]), "n_m2l_pairs": int(full[1]), "n_p2p_pairs": int(full[2]),
                            "n_particle_pairs": int(full[3])},
            "sample": {"N": ns, "seconds_by_stage": st, "n_particle_pairs": int(cnt[3]), "n_m2l_pairs": int(cnt[1])},
            "count_walk_seconds": tc}


def run_reference(args):
    """The oracle as it stands, single-threaded on the host, on this workload's config:
    every step is one build + forces of a bounded sample (REF_SAMPLE_N particles of the
    same generator, p, theta, leaf size and variant); value = sample particles / step time."""
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    if args.workload != "plummer1m" and (WORKLOADS[args.workload].get("gen") == "batch"
                                         or (WORKLOADS[args.workload]["N"] or 0) > (1 << 19)):
        # the large workloads: extrapolated from timed samples and exact walk counts
        W = dict(WORKLOADS[args.workload])
        ex = oracle_extrapolated(W)
        line = {"metric": METRIC, "value": ex["particles_per_s"], "unit": "particles/s", "n_gpus": world,
                "impl": "reference", "kind": "oracle, extrapolated", "dtype": "f64",
                "config": workload_config(W, world, ex["N"], W.get("n_sys", 1)), "extrapolation": ex,
                "cpu_baseline": {"value": ex["particles_per_s"], "unit": "particles/s", "cores": 1, "kind": "oracle",
                                 "sample": "one timed sample of the same generator (stage timers per unit) "
                                           "applied to the full workload's walk counts (extrapolated)"}}
        print(json.dumps(line))
        return line
    for _ in range(max(0, args.warmup)):
        oracle_sample_rate(REF_SAMPLE_N)
    times = []
    for _ in range(max(1, args.steps)):
        _, dt = oracle_sample_rate(REF_SAMPLE_N)
        times.append(dt)
    t = statistics.mean(times)
    rate = REF_SAMPLE_N / t
    W = dict(WORKLOAD)
    line = {
        "metric": METRIC, "value": rate, "unit": "particles/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Plummer sphere)", "impl": "reference",
        "config": workload_config(W, world, W["N"], 1),
        "sample": {"N": REF_SAMPLE_N, "of_N": W["N"],
                   "note": "each step times the oracle on this bounded sample of the configured workload"},
        "cpu_baseline": {"value": rate, "unit": "particles/s", "cores": 1, "kind": "oracle",
                         "sample": f"Plummer N={REF_SAMPLE_N} per step (bounded sample of the N=2^20 workload, "
                                   "same seed, p, theta, leaf size, variant), single-threaded FP64 C oracle"},
        "e2e": {"value": rate, "unit": "particles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return line


def run_two_shapes(args):
    """Synthetic stand-in for the paper's two-shape test (Fig. 2): two irregular clusters of
    4000 particles at COM distance d, each alone in one child of the root (leaf size 4000,
    theta = 0.999), so that the walk emits exactly one mutual M2L between them and evaluates
    each cluster's own forces directly.  The deviation from the full direct sum is then the
    error of the approximated inter-shape force, reported relative to that force (L2 over
    all particles), with the net force and torque of the result."""
    import torch
    from paper_2107_07166_gb300 import fmm, synth
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    n_each, seed = 4000, 7
    forms = [("order0-standard", 1, fmm.STANDARD), ("order0-realigned", 1, fmm.CONSERVING),
             ("order0-realigned-literal", 1, fmm.CONSERVING_PAPER0), ("order1-standard", 2, fmm.STANDARD),
             ("order1-realigned", 2, fmm.CONSERVING)]
    prec = {"fp64": fmm.FP64, "df64": fmm.DF64, "mixed": fmm.MIXED}[args.precision]
    f = fmm.FMM(0, prec, torch.cuda.current_stream())
    rows = []
    for d in (4.0, 8.0, 16.0, 32.0, 64.0):
        x, m = synth.clusters_pair(n_each, seed, d)
        N = x.shape[0]
        X = torch.from_numpy(x).to(dev)
        M = torch.from_numpy(m).to(dev)
        side = torch.cat([torch.zeros(n_each, dtype=torch.bool), torch.ones(n_each, dtype=torch.bool)]).to(dev)
        full = torch.zeros((N, 3), dtype=torch.float64, device=dev)
        inter = torch.zeros((N, 3), dtype=torch.float64, device=dev)
        for i0 in range(0, N, 512):
            dd = X[i0:i0 + 512, None, :] - X[None, :, :]
            r2 = (dd * dd).sum(-1)
            inv3 = torch.where(r2 > 0, r2.rsqrt() ** 3, torch.zeros_like(r2))
            w = M[None, :] * inv3
            full[i0:i0 + 512] = -(w[..., None] * dd).sum(1)
            other = (side[i0:i0 + 512, None] != side[None, :]).to(torch.float64)
            inter[i0:i0 + 512] = -((w * other)[..., None] * dd).sum(1)
        xm = (M[:, None] * X)
        fs = float((M * inter.norm(dim=1)).sum())
        ts = float((M * X.norm(dim=1) * inter.norm(dim=1)).sum())
        row = {"d": d}
        for name, p, variant in forms:
            acc = torch.empty((N, 3), dtype=torch.float64, device=dev)
            f.build(X, M, n_each)
            f.forces(p, 0.999, variant, acc, None)
            cnt = f.counts()
            F = (M[:, None] * acc).sum(0)
            T = torch.cross(X, acc, dim=1).mul(M[:, None]).sum(0)
            row[name] = {"err": float((acc - full).norm() / inter.norm()),
                         "net_force_rel": float(F.norm()) / fs, "net_torque_rel": float(T.norm()) / ts,
                         "n_m2l": int(cnt["n_m2l"])}
        del xm
        rows.append(row)
    f.close()
    line = {"study": "two-shapes", "n_each": n_each, "seed": seed, "theta": 0.999, "leaf_size": n_each,
            "precision": args.precision, "rows": rows,
            "note": "error of the approximated inter-shape force relative to that force, L2 over both shapes"}
    print(json.dumps(line))
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbfmm", choices=["gbfmm", "reference"])
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--n", type=int, default=0, help="override N (profiling of a smaller case)")
    ap.add_argument("--workload", default="plummer1m", choices=sorted(WORKLOADS),
                    help="plummer1m (default line) or another synthetic workload")
    ap.add_argument("--variant", default=None, choices=["conserving", "standard"])
    ap.add_argument("--precision", default=None, choices=["fp64", "df64", "mixed"],
                    help="arithmetic of the pair kernels (M2L, P2P)")
    ap.add_argument("--leapfrog", type=int, default=100, help="KDK steps of the momentum-drift run (0: skip)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="batch workload: take the tuned leaf size and M2L tile (32, 64) without timing trials")
    ap.add_argument("--no-modes", dest="modes", action="store_false",
                    help="skip timing the other arithmetic modes on the same input")
    ap.add_argument("--study", default=None, choices=["two-shapes"],
                    help="run a study instead of the benchmark (one JSON line)")
    args = ap.parse_args()
    args.variant_set = args.variant is not None
    args.precision_set = args.precision is not None
    args.variant = args.variant or "conserving"
    args.precision = args.precision or "fp64"
    if args.impl == "reference":
        run_reference(args)
        return
    if args.study == "two-shapes":
        run_two_shapes(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    run_gbfmm(args)


if __name__ == "__main__":
    main()
