#!/usr/bin/env python3
"""Throughput of the RCB tree pipeline (build + neighbour search + gravity) on GB300.

One step = rebuild the tree from device-resident particles (Sec. 2.1 build and the per-sink
walk), neighbour search (Sec. 2.3) and gravity (Sec. 2.4).  The headline workload is the
uniform-density unit sphere with N = 4,194,304 particles, log-uniform masses over a 10x range,
h for ~50 neighbours, N_ll = 12, theta = 0.7, mixed form; the FP64 form is timed on the same
tree and reported beside it with the mixed form's error against it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --gpus N > 1 (launched by torchrun) every rank runs an independent replica on its own GPU
(the path has no exchange step: replicas only); value = particles processed by all ranks / the
slowest rank's time.  --impl reference times the CPU oracle on the host cores instead.
Prints one JSON line on rank 0.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mparticles/s (RCB build+neighbours+gravity) at N=4M, mixed vs FP64 at stated err"
UNIT = "Mparticles/s"
N_LL = 12
FLOPS_PER_PAIR = 38        # float32 flops of one kernel-softened near-field pair, Eq. 10 with its potential (FMA = 2, MUFU = 1)
FLOPS_PER_PAIR_NEWTON = 24  # the same pair on its Newtonian branch (q >= 2), the form most pairs take
# DRAM bytes of one near-kernel launch at the headline workload: dram__bytes_read.sum +
# dram__bytes_write.sum of one ncu capture at N = 2,097,152 (1,088,807,680 B for 1,038,400,525
# pairs) scaled by the pair count to N = 4,194,304 (2,065,548,119 pairs).  Valid only for the
# source it was taken on; any later change of gravity.cu reports null.
NEAR_TRAFFIC = {"bytes": 2165816177, "gravity_cu_sha1": "5fba030d72bbabd0aae346047f31157e9a41dfb4"}
SMS = 152
FP32_LANES = 128           # FP32 lanes per SM
L2_FLUSH_BYTES = 256 << 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=4194304)
    p.add_argument("--kind", default="sphere")
    p.add_argument("--mass", default="loguniform10")
    p.add_argument("--theta", type=float, default=0.7)
    p.add_argument("--split", choices=["mass", "number", "median"], default="mass",
                   help="cut of the headline tree (Sec. 2.1.3): centre of mass, centre of number, median")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-sample-sinks", type=int, default=256)
    p.add_argument("--direct-targets", type=int, default=4000,
                   help="targets of the oracle's direct sum for accuracy_vs_direct")
    p.add_argument("--headline-only", action="store_true",
                   help="time only the headline step (no FP64 form, accuracy, e2e or CPU legs); for profiling")
    p.add_argument("--presort", choices=["none", "morton"], default="none",
                   help="permute the inputs into Morton order on the host before anything is timed "
                        "(the A/B of a caller that keeps its particles in that order)")
    p.add_argument("--table1", action="store_true",
                   help="instead of the step: the scan of the mean ll-cell occupancy of Sec. 3.2.1 (Table 1)")
    return p.parse_args()


def workload_name(a):
    kinds = {"sphere": "uniform-density unit sphere", "plummer": "Plummer sphere", "cube": "uniform unit cube"}
    return (f"{kinds.get(a.kind, a.kind)}, N={a.n}, {a.mass} masses, h for ~50 neighbours, N_ll={N_LL}, "
            f"theta={a.theta}")


def bench_config(a, world):
    """The `config` object of the JSON line (both arms)."""
    cfg = {"workload": workload_name(a), "N": a.n, "theta": a.theta, "n_ll": N_LL, "form": "mixed", "split": a.split,
           "parallelism": f"replicas x{world}",
           "l2": "inputs (164 MB) exceed L2 and a 256 MB buffer is written between timed steps"}
    if a.presort != "none":
        cfg["presort"] = a.presort
    return cfg


def device_presort_ms(xt, mt, ht, reps=10):
    """What the Morton presort would cost inside a step: keys, a device sort (torch) and the
    gathers of x, m and h, timed with CUDA events (median of reps; the step itself does not
    include it)."""
    import torch

    def presort():
        lo, hi = xt.min(0).values, xt.max(0).values
        q = ((xt - lo) / torch.where(hi > lo, hi - lo, torch.ones_like(hi)) * (2 ** 21 - 1)).to(torch.int64)

        def spread(v):
            v = v & 0x1fffff
            for sh, mask in ((32, 0x1f00000000ffff), (16, 0x1f0000ff0000ff), (8, 0x100f00f00f00f00f),
                             (4, 0x10c30c30c30c30c3), (2, 0x1249249249249249)):
                v = (v | (v << sh)) & mask
            return v

        key = spread(q[:, 0]) | (spread(q[:, 1]) << 1) | (spread(q[:, 2]) << 2)
        p = torch.argsort(key)
        return xt[p], mt[p], ht[p]

    for _ in range(3):
        presort()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        presort()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def morton_order(x):
    """Permutation that sorts the particles by their 63-bit Morton key (21 bits per axis of the
    inputs' bounding box); used only to lay the inputs out in that order before timing."""
    import numpy as np
    lo, hi = x.min(0), x.max(0)
    q = ((x - lo) / np.where(hi > lo, hi - lo, 1.0) * (2 ** 21 - 1)).astype(np.uint64)

    def spread(v):
        v = v & np.uint64(0x1fffff)
        for sh, mask in ((32, 0x1f00000000ffff), (16, 0x1f0000ff0000ff), (8, 0x100f00f00f00f00f),
                         (4, 0x10c30c30c30c30c3), (2, 0x1249249249249249)):
            v = (v | (v << np.uint64(sh))) & np.uint64(mask)
        return v

    key = spread(q[:, 0]) | (spread(q[:, 1]) << np.uint64(1)) | (spread(q[:, 2]) << np.uint64(2))
    return np.argsort(key, kind="stable")


def max_over_ranks(value, dist, device):
    """The largest of every rank's value (the slowest replica's time); value itself on one rank."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, n, ms):
    """Mparticles/s of the whole job: every replica processes n particles per step of ms."""
    return world * n / (ms * 1e-3) / 1e6


# ------------------------------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(device_index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                rows.append({"sm": float(parts[1]), "max": float(parts[2]), "util": float(parts[4]),
                             "hw": parts[6], "hwt": parts[7], "swt": parts[8], "pcap": parts[9]})
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [r for r in rows if r["util"] > 0] or rows
        reasons = set()
        for r in load:
            for k, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                            ("pcap", "sw_power_cap")):
                if r[k].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in load), "sm_max_mhz": max(r["max"] for r in rows),
                "samples_under_load": len(load), "reasons": sorted(reasons)}


# ------------------------------------------------------------------------------------------ CPU oracle
def oracle_sample_run(x, m, h, theta, n_sinks, seed=7, tree=None):
    """The oracle as it stands on the host cores: the full build (or the tree given), then walk +
    neighbours + gravity for a seeded sample of sinks.  Returns (t_build, t_sample, details, the
    sampled particles' original indices, their oracle accelerations, the tree)."""
    import numpy as np

    import oracle
    t0 = time.perf_counter()
    T = tree if tree is not None else oracle.OracleTree(x, m, h, n_ll=N_LL)
    t_build = time.perf_counter() - t0
    nd = T.nodes()
    leaf0 = 1 << T.L
    live = np.flatnonzero(nd["count"][leaf0:] > 0)
    rng = np.random.default_rng(seed)
    sinks = np.sort(rng.choice(live, min(n_sinks, len(live)), replace=False))
    n_part = int(nd["count"][leaf0 + sinks].sum())
    t0 = time.perf_counter()
    T.walk(theta, sinks)
    T.neighbours()
    acc, _ = T.gravity()
    t_sample = time.perf_counter() - t0
    perm = T.perm()
    parts = np.concatenate([perm[nd["first"][leaf0 + j]:nd["first"][leaf0 + j] + nd["count"][leaf0 + j]] for j in sinks])
    return t_build, t_sample, {"sample_particles": n_part, "sample_sinks": int(len(sinks))}, parts, acc[parts], T


def run_reference(a, rank, world):
    """The reference arm: the CPU oracle as it stands, on the host cores.  The tree is built once
    (timed); every step then runs the walk, neighbour search and gravity for a fresh seeded sample
    of sinks (timed).  A step's time is that sample's time plus the build's measured cost for the
    sample's particles (build time x sample particles / N); the value is the sample's particles over
    that time, so both describe work that ran.  The full-N step the same per-particle costs give is
    reported on its own (extrapolated_full_n_ms)."""
    if rank != 0:
        return
    import numpy as np

    import oracle
    import synth
    x, m, h = synth.make_particles(a.kind, a.n, synth.seed_for(3, 0), a.mass)
    if a.presort == "morton":
        perm = morton_order(x)
        x, m, h = (np.ascontiguousarray(v[perm]) for v in (x, m, h))
    oracle.build()
    t0 = time.perf_counter()
    T = oracle.OracleTree(x, m, h, n_ll=N_LL)
    t_build = time.perf_counter() - t0
    steps_ms, parts = [], []
    det = None
    for i in range(a.warmup + a.steps):
        _, t_sample, det, _, _, _ = oracle_sample_run(x, m, h, a.theta, a.cpu_sample_sinks, seed=100 + i, tree=T)
        n_part = det["sample_particles"]
        if i >= a.warmup:
            steps_ms.append((t_sample + t_build * n_part / a.n) * 1e3)
            parts.append(n_part)
    ms = statistics.mean(steps_ms)
    value = statistics.mean(parts) / (ms * 1e-3) / 1e6
    sample = (f"oracle tree built once ({t_build:.2f} s for N={a.n}); per step walk+neighbours+gravity for "
              f"{det['sample_sinks']} random sinks (~{int(statistics.mean(parts))} particles), plus the build's "
              f"measured cost for those particles")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(a, world),
            "build_s": t_build,
            "extrapolated_full_n_ms": ms * a.n / statistics.mean(parts),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def rel_err_stats(a_gpu, a_ref):
    """RMS, 99.9th percentile and maximum of |a - a_ref| / |a_ref| over the rows given."""
    import numpy as np
    e = np.linalg.norm(a_gpu - a_ref, axis=1) / np.linalg.norm(a_ref, axis=1)
    return {"n": int(e.size), "rms": float(np.sqrt(np.mean(e * e))), "p99.9": float(np.percentile(e, 99.9)),
            "max": float(e.max())}


# ------------------------------------------------------------------------------------------ GPU
def idx_total_bytes(idx):
    return idx.numel() * idx.element_size()


def memory_leg(rcb, a, xt, mt, ht):
    """Device bytes per particle of each stage of the step, on a fresh tree (the library allocates
    through torch's caching allocator, so torch's counters see every buffer): held after the call
    and the peak during it, above what was held before.  The step's own outputs (accelerations,
    potentials, CSR offsets and rows) are reported apart from the library's buffers."""
    import torch
    n = a.n

    def held():
        torch.cuda.synchronize()
        return torch.cuda.memory_allocated()

    base = held()
    torch.cuda.reset_peak_memory_stats()
    tree = rcb.RCBTree(xt, mt, ht, n_ll=N_LL, theta=a.theta, precision="mixed", split=a.split)
    after_build = held()
    peak_build = torch.cuda.max_memory_allocated()
    torch.cuda.reset_peak_memory_stats()
    acc, pot, off, idx = tree.gravity_neighbours()
    after_gn = held()
    peak_gn = torch.cuda.max_memory_allocated()
    outputs = sum(t.numel() * t.element_size() for t in (acc, pot, off, idx))
    info = tree.info()
    tree.free()
    del acc, pot, off, idx, tree
    return {
        "unit": "B per particle",
        "inputs": sum(t.numel() * t.element_size() for t in (xt, mt, ht)) / n,
        "build_held": (after_build - base) / n,
        "build_peak": (peak_build - base) / n,
        "gravity_neighbours_library_held": (after_gn - after_build - outputs) / n,
        "gravity_neighbours_peak": (peak_gn - after_build) / n,
        "outputs": outputs / n,
        "build_list_slots": info["nsinks"] * (info["cap_near"] + info["cap_far"]) * 4 / n,
        "lists_entries_per_particle": {"near": info["near_total"] / n, "far": info["far_total"] / n},
        "note": ("fresh tree after the timed region; build_held = tree arrays and the per-sink near/far "
                 "list slots (build_list_slots: nsinks x (near + far capacity) int32, each capacity the "
                 "longest list plus a margin); gravity_neighbours_library_held = far coefficients, the "
                 "staged neighbour rows and their scratch; outputs = acc + pot (float64) and the CSR "
                 "(int64 offsets, int32 rows)"),
    }


def split_variant_leg(rcb, a, split, xt, mt, ht, flush, acc_ref):
    """A tree cut by another rule of Sec. 2.1.3 on the same input: construction, walk and gravity
    times by the library's stage events, its list sizes, and its force difference from acc_ref
    (the centre-of-mass tree's accelerations)."""
    import torch
    vt = rcb.RCBTree(xt, mt, ht, n_ll=N_LL, theta=a.theta, precision="mixed", timing=True, split=split)
    try:
        b_ms, w_ms, g_ms = [], [], []
        for _ in range(3):
            flush.zero_()
            torch.cuda.synchronize()
            vt.rebuild(xt, mt, ht)
            st = vt.stage_times()
            b_ms.append(st["build"])
            w_ms.append(st["walk"])
            flush.zero_()
            torch.cuda.synchronize()
            acc_v, _ = vt.gravity()
            st = vt.stage_times()
            g_ms.append(st["far"] + st["near"])
        dv = torch.linalg.norm(acc_v - acc_ref, dim=1) / torch.linalg.norm(acc_ref, dim=1)
        vinfo = vt.info()
        sample = dv[:: max(1, dv.numel() // 1000000)].float()
        return {"construction_ms": statistics.mean(b_ms) - statistics.mean(w_ms), "walk_ms": statistics.mean(w_ms),
                "gravity_ms": statistics.mean(g_ms), "near_pairs": int(vinfo["near_pairs"]),
                "far_total": int(vinfo["far_total"]),
                "rms_rel_diff_vs_mass_split": float(torch.sqrt(torch.mean(dv * dv))),
                "p999_rel_diff_vs_mass_split": float(torch.quantile(sample, 0.999))}
    finally:
        vt.free()


def extra_legs(a, world, dist, tree, x, m, h, xt, mt, ht, flush, stream, step, barrier, ms, stage_ms):
    """FP64 form on the same tree, the mixed form's error against it, and the end-to-end leg."""
    import numpy as np
    import torch

    import paper_1108_0028_gb300 as rcb

    # FP64 form on the same tree (gravity only differs), and the mixed form's error against it
    acc_m, pot_m = tree.gravity()
    tree.set_precision("fp64")
    acc_d, pot_d = tree.gravity()
    f64_grav = []
    for _ in range(3):
        flush.zero_()
        torch.cuda.synchronize()
        tree.gravity()
        st = tree.stage_times()
        f64_grav.append(st["far"] + st["near"])
    tree.set_precision("mixed")
    torch.cuda.synchronize()
    e = (torch.linalg.norm(acc_m - acc_d, dim=1) / torch.linalg.norm(acc_d, dim=1)).cpu().numpy()
    ep = (torch.abs(pot_m - pot_d) / torch.abs(pot_d)).cpu().numpy()
    t_fp64 = ms - (stage_ms["far"] + stage_ms["near"]) + statistics.mean(f64_grav)
    fp64 = {"value": job_throughput(world, a.n, t_fp64), "unit": UNIT, "ms_per_step": t_fp64,
            "gravity_ms": statistics.mean(f64_grav)}
    accuracy = {"reference": "FP64 GPU form on the same tree (parity of the FP64 form with the FP64 oracle is "
                             "tested separately: RMS 1e-15)",
                "rms": float(np.sqrt(np.mean(e * e))), "p99.9": float(np.percentile(e, 99.9)),
                "max": float(e.max()), "pot_rms": float(np.sqrt(np.mean(ep * ep)))}
    forces = {"mixed": acc_m.cpu().numpy(), "fp64": acc_d.cpu().numpy()}

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    xh, mh, hh = (torch.from_numpy(v).pin_memory() for v in (x, m, h))
    xd, md, hd = torch.empty_like(xt), torch.empty_like(mt), torch.empty_like(ht)
    off0, idx0, acc0, pot0 = step()
    offh = torch.empty(off0.shape, dtype=off0.dtype).pin_memory()
    idxh = torch.empty(idx0.shape, dtype=idx0.dtype).pin_memory()
    acch = torch.empty(acc0.shape, dtype=acc0.dtype).pin_memory()
    poth = torch.empty(pot0.shape, dtype=pot0.dtype).pin_memory()
    e2e_ms = []
    for _ in range(max(3, a.steps // 2)):
        flush.zero_()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        xd.copy_(xh, non_blocking=True)
        md.copy_(mh, non_blocking=True)
        hd.copy_(hh, non_blocking=True)
        tree.rebuild(xd, md, hd)
        acc, pot, off, idx = tree.gravity_neighbours()
        offh.copy_(off, non_blocking=True)
        idxh[:idx.numel()].copy_(idx, non_blocking=True)
        acch.copy_(acc, non_blocking=True)
        poth.copy_(pot, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    ems_seq = max_over_ranks(statistics.mean(e2e_ms), dist, xt.device)
    # The same steps as a time loop runs them: two input and two output buffers, so that step
    # k + 1's inputs are copied in while step k computes and step k's results are copied out
    # while step k + 1 computes (compute, input copies and output copies on three streams,
    # ordered by events).  Every step still copies its inputs in and its results out inside the
    # timed region, which ends when the last results are on the host.
    S, Cin, Cout = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    xin = [(torch.empty_like(xt), torch.empty_like(mt), torch.empty_like(ht)) for _ in range(2)]
    # results on the device and on the host, two of each, allocated once
    outd = [(torch.empty_like(off0), torch.empty(max(idx0.numel(), 1) + (1 << 20), dtype=idx0.dtype, device=xt.device),
             torch.empty_like(acc0), torch.empty_like(pot0)) for _ in range(2)]
    outh = [tuple(torch.empty(d_.shape, dtype=d_.dtype).pin_memory() for d_ in o) for o in outd]
    in_ev = [torch.cuda.Event(), torch.cuda.Event()]
    out_free = [torch.cuda.Event(), torch.cuda.Event()]  # a buffer's copy to the host has finished
    del off0, idx0, acc0, pot0

    def copy_in(b):
        with torch.cuda.stream(Cin):
            for d_, h_ in zip(xin[b], (xh, mh, hh)):
                d_.copy_(h_, non_blocking=True)
            in_ev[b].record(Cin)

    K = max(3, a.steps // 2)
    flush.zero_()
    copy_in(0)
    for b in range(2):
        out_free[b].record(Cout)
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(S)
    nidx = 0
    for k in range(K):
        b = k % 2
        offd, idxd, accd, potd = outd[b]
        S.wait_event(in_ev[b])
        tree.rebuild(*xin[b], stream=S)
        if k + 1 < K:
            copy_in(1 - b)  # the other buffer's build finished before this one began
        S.wait_event(out_free[b])
        rcb.rcb_gravity_neighbours(tree.handle, accd, potd, offd, S)
        st_, nidx = rcb.rcb_neighbours(tree.handle, offd, idxd, idxd.numel(), S)
        if st_ != 0:
            raise RuntimeError(f"rcb_neighbours failed: {st_}")
        done = torch.cuda.Event()
        done.record(S)
        Cout.wait_event(done)
        with torch.cuda.stream(Cout):
            for h_, d_, n_ in zip(outh[b], outd[b], (offd.numel(), nidx, accd.numel(), potd.numel())):
                h_.view(-1)[:n_].copy_(d_.view(-1)[:n_], non_blocking=True)
            out_free[b].record(Cout)
    last = torch.cuda.Event()
    last.record(Cout)
    S.wait_event(last)
    e1.record(S)
    torch.cuda.synchronize()
    idx = outd[0][1][:nidx]
    ems = max_over_ranks(e0.elapsed_time(e1) / K, dist, xt.device)
    h2d = (x.nbytes + m.nbytes + h.nbytes)
    d2h = offh.numel() * 8 + idx_total_bytes(idx) + acch.numel() * 8 + poth.numel() * 8
    e2e = {"value": job_throughput(world, a.n, ems), "unit": UNIT, "ms_per_step": ems,
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "pipelined_steps": K,
           "sequential": {"value": job_throughput(world, a.n, ems_seq), "ms_per_step": ems_seq,
                          "note": "one step at a time: copy in, compute, copy out, no overlap"}}
    idx0 = idx
    # per stage (Sec. 2.1-2.2 build with the walk; Sec. 2.3 neighbours alone; Sec. 2.4 gravity
    # alone; and the fused pass the step uses), each timed by the library's stage events
    def staged(fn, keys, reps=5):
        out = []
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize()
            fn()
            st = tree.stage_times()
            out.append(sum(st[k] for k in keys))
        return statistics.mean(out)

    build_ms = staged(lambda: tree.rebuild(xt, mt, ht), ["build"])
    walk_ms = staged(lambda: tree.rebuild(xt, mt, ht), ["walk"])
    nb_ms = staged(lambda: (tree.refit(xt, mt), tree.neighbours()), ["nb_count", "nb_fill", "nb_sort"])
    grav_ms = staged(lambda: tree.gravity(), ["far", "near"])
    fused_ms = staged(lambda: (tree.refit(xt, mt), tree.gravity_neighbours()),
                      ["far", "near", "nb_count", "nb_fill", "nb_sort"])
    # backward (the VJP of the forces through the frozen tree, Sec. 2.4 differentiated): the
    # adjoint of loss = sum |a|^2 on the current tree, in the mixed form
    tree.rebuild(xt, mt, ht)
    acc_b, _ = tree.gravity()
    g_acc = 2.0 * acc_b
    tree.gravity_backward(g_acc)
    bwd_ms = staged(lambda: tree.gravity_backward(g_acc), ["backward"])
    # the first backward after a build also transposes the near lists: time it on a fresh build
    bwd_first = []
    for _ in range(3):
        tree.rebuild(xt, mt, ht)
        tree.gravity()
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tree.gravity_backward(g_acc)
        e1.record(stream)
        torch.cuda.synchronize()
        bwd_first.append(e0.elapsed_time(e1))
    bwd_first_ms = statistics.mean(bwd_first)
    # tree update (Sec. 2.1.8): integrity check, refit and a new walk, when every particle is
    # still in its ll-cell; positions displaced by 1e-12 (alternating with the originals)
    gen = torch.Generator(device=xt.device)
    gen.manual_seed(5)
    xj = xt + 1e-12 * torch.randn(xt.shape, dtype=xt.dtype, device=xt.device, generator=gen)
    tree.rebuild(xt, mt, ht)
    upd = []
    for i in range(5):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rebuilt = tree.update(xj if i % 2 == 0 else xt, mt, ht, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if rebuilt:
            raise RuntimeError("tree update rebuilt although no particle left its ll-cell")
        upd.append(e0.elapsed_time(e1))
    update_ms = statistics.mean(upd)
    # SPH density over the neighbour CSR of the built tree (the first consumer of the lists)
    tree.rebuild(xt, mt, ht)
    off_d, idx_d = tree.neighbours()
    dens = []
    for _ in range(5):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tree.density(off_d, idx_d, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        dens.append(e0.elapsed_time(e1))
    density_ms = statistics.mean(dens)
    del off_d, idx_d
    # MAC-only near lists (the Sec. 2.5 variant): gravity alone on such a tree, its near pairs and
    # its force difference from the conservative lists of the headline tree
    tree.rebuild(xt, mt, ht)
    acc_std, _ = tree.gravity()
    acc_std = acc_std.clone()
    near_pairs_std = tree.info()["near_pairs"]
    mac_tree = rcb.RCBTree(xt, mt, ht, n_ll=N_LL, theta=a.theta, precision="mixed", timing=True,
                           mac_only=True)
    mac_ms = []
    for _ in range(5):
        flush.zero_()
        torch.cuda.synchronize()
        acc_mac, _ = mac_tree.gravity()
        st = mac_tree.stage_times()
        mac_ms.append(st["far"] + st["near"])
    dmac = torch.linalg.norm(acc_mac - acc_std, dim=1) / torch.linalg.norm(acc_std, dim=1)
    mac_info = mac_tree.info()
    mac_only = {"ms": statistics.mean(mac_ms), "mparticles_s": job_throughput(world, a.n, statistics.mean(mac_ms)),
                "near_pairs": mac_info["near_pairs"], "near_pairs_conservative": near_pairs_std,
                "rms_rel_diff_vs_conservative": float(torch.sqrt(torch.mean(dmac * dmac))),
                "path": "rcb_gravity on a tree built with RCB_FLAG_MAC_ONLY (near lists from the MAC alone)"}
    mac_tree.free()
    del acc_mac, dmac
    # the split variants of Sec. 2.1.3 on the same input (centre of number, median position):
    # construction, walk and gravity by the library's stage events, list sizes, and the force
    # difference from the centre-of-mass tree
    std_info = tree.info()
    split_variants = {"mass": {"near_pairs": near_pairs_std, "far_total": std_info["far_total"]}}
    for split in ("number", "median"):
        try:
            split_variants[split] = split_variant_leg(rcb, a, split, xt, mt, ht, flush, acc_std)
        except (KeyError, TypeError, ValueError, rcb.RCBError) as e:  # a report of this leg only, not of the step
            # a CUDA error leaves the context unusable: every later number would be invalid, so it
            # ends the run instead of being reported as this leg's failure
            if isinstance(e, rcb.RCBError) and e.status == rcb.RCB_ERR_CUDA:
                raise
            torch.cuda.synchronize()  # raises if the context holds a sticky error
            split_variants[split] = {"error": repr(e)}
    del acc_std
    L = tree.info()["L"]
    build_bytes = a.n * (72 * L + 56)  # every level reads and writes 36 B per particle, h gathered once
    per_stage = {
        "build": {"ms": build_ms, "mparticles_s": job_throughput(world, a.n, build_ms),
                  "algorithmic_bytes": build_bytes, "achieved_gbs": build_bytes / (build_ms * 1e-3) / 1e9,
                  "path": "rcb_build: tree construction and the walk that writes the interaction lists"},
        "construction": {"ms": build_ms - walk_ms, "mparticles_s": job_throughput(world, a.n, build_ms - walk_ms),
                         "algorithmic_bytes": build_bytes,
                         "achieved_gbs": build_bytes / ((build_ms - walk_ms) * 1e-3) / 1e9,
                         "path": "presort, level passes, subtrees, leaf moments, bottom-up (rcb_build less the walk)"},
        "walk": {"ms": walk_ms, "mparticles_s": job_throughput(world, a.n, walk_ms),
                 "path": "per-sink walk writing near and far lists"},
        "neighbours": {"ms": nb_ms, "mparticles_s": job_throughput(world, a.n, nb_ms), "path": "rcb_neighbours alone"},
        "gravity": {"ms": grav_ms, "mparticles_s": job_throughput(world, a.n, grav_ms), "path": "rcb_gravity alone"},
        "neighbours_gravity_fused": {"ms": fused_ms, "mparticles_s": job_throughput(world, a.n, fused_ms),
                                     "path": "rcb_gravity_neighbours + compaction (the step's path)"},
        "gravity_mac_only": mac_only,
        "split_variants": split_variants,
        "density": {"ms": density_ms, "mparticles_s": job_throughput(world, a.n, density_ms),
                    "path": "rcb_density over the CSR of rcb_neighbours (cubic spline, support 2h)"},
        "update": {"ms": update_ms, "mparticles_s": job_throughput(world, a.n, update_ms),
                   "path": "rcb_update: integrity check, refit, new walk (no particle left its ll-cell)"},
        "gravity_backward": {"ms": bwd_ms, "mparticles_s": job_throughput(world, a.n, bwd_ms),
                             "path": "rcb_gravity_backward on the built tree (lists already transposed)"},
        "gravity_backward_first": {"ms": bwd_first_ms, "setup_ms": bwd_first_ms - bwd_ms,
                                   "path": "the first rcb_gravity_backward after a build, transposition of the near "
                                           "lists included (setup_ms: its excess over a later call)"},
    }
    return fp64, accuracy, e2e, int(idx0.numel()), per_stage, forces


def run_ours(a, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_1108_0028_gb300 as rcb
    import synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    rcb.lib()
    x, m, h = synth.make_particles(a.kind, a.n, synth.seed_for(3, 0), a.mass)
    if a.presort == "morton":
        perm = morton_order(x)
        x, m, h = (np.ascontiguousarray(v[perm]) for v in (x, m, h))
    xt = torch.from_numpy(x).to(dev)
    mt = torch.from_numpy(m).to(dev)
    ht = torch.from_numpy(h).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    presort_ms = None
    if a.presort == "morton":
        presort_ms = device_presort_ms(xt, mt, ht)
    tree = rcb.RCBTree(xt, mt, ht, n_ll=N_LL, theta=a.theta, precision="mixed", timing=True, split=a.split)

    def step():
        tree.rebuild(xt, mt, ht)
        acc, pot, off, idx = tree.gravity_neighbours()
        return off, idx, acc, pot

    for _ in range(a.warmup):
        step()
    barrier()
    sampler = ClockSampler(local_rank) if rank == 0 else None
    launches0 = tree.info()["launches"]
    step_ms, stages = [], []
    for _ in range(a.steps):
        flush.zero_()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        stages.append(tree.stage_times())
    barrier()
    launches = tree.info()["launches"] - launches0
    ms = max_over_ranks(statistics.mean(step_ms), dist, dev)
    value = job_throughput(world, a.n, ms)
    stage_ms = {k: statistics.mean(s[k] for s in stages) for k in stages[0]}
    info = tree.info()

    fp64 = accuracy = e2e = per_stage = forces = None
    idx_total = None
    alu = None
    if not a.headline_only:
        fp64, accuracy, e2e, idx_total, per_stage, forces = extra_legs(a, world, dist, tree, x, m, h, xt, mt, ht, flush,
                                                                       stream, step, barrier, ms, stage_ms)
        alu = rcb.alu_rates(SMS)
    clocks = sampler.stop() if sampler else None
    tree.free()
    del tree
    memory = memory_leg(rcb, a, xt, mt, ht)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    # roofline of the dominant kernel: the near field (float32 ALU)
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    peak = SMS * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
    near_s = stage_ms["near"] * 1e-3
    achieved = info["near_pairs"] * FLOPS_PER_PAIR / near_s / 1e12
    traffic = None
    try:
        import hashlib
        src = os.path.join(ROOT, "paper_1108_0028_gb300", "csrc", "gravity.cu")
        if hashlib.sha1(open(src, "rb").read()).hexdigest() == NEAR_TRAFFIC["gravity_cu_sha1"] and \
                (a.n, a.kind, a.mass, a.theta) == (4194304, "sphere", "loguniform10", 0.7):
            traffic = NEAR_TRAFFIC["bytes"]
    except OSError:
        pass
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_unit": "B per launch", "kernel": "k_near_mixed",
                "frac_newtonian_count": achieved * FLOPS_PER_PAIR_NEWTON / FLOPS_PER_PAIR / peak,
                "basis": f"{info['near_pairs']} near pairs x {FLOPS_PER_PAIR} FP32 flops (one kernel-softened pair of "
                         f"Eq. 10; frac_newtonian_count counts {FLOPS_PER_PAIR_NEWTON}, the Newtonian branch; the "
                         f"neighbour tests fused into the same kernel are not counted) / near-kernel event time; "
                         f"peak = {SMS} SMs x {FP32_LANES} FP32 lanes x 2 x median SM clock under load "
                         f"({sm_mhz:.0f} MHz)"}
    # build: algorithmic bytes of the build kernels over their event time, against measured HBM
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    if per_stage:
        for k in ("build", "construction"):
            per_stage[k]["hbm_peak_gbs"] = hbm
            per_stage[k]["frac"] = per_stage[k]["achieved_gbs"] / hbm
    cpu = None
    acc_vs_oracle = acc_vs_direct = None
    if not a.no_cpu_baseline and not a.headline_only and world == 1:
        import numpy as np

        import oracle
        oracle.build()
        t_build, t_sample, det, parts, acc_o, _ = oracle_sample_run(x, m, h, a.theta, a.cpu_sample_sinks)
        t_step = t_build + t_sample * a.n / det["sample_particles"]
        cpu = {"value": a.n / t_step / 1e6, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
               "sample": (f"full-N build ({t_build:.2f} s), then walk+neighbours+gravity for "
                          f"{det['sample_sinks']} random sinks ({det['sample_particles']} particles, "
                          f"{t_sample:.2f} s); value = N over the build plus the sample's time scaled to N")}
        # accuracy against the truth (Sec. 3.1): the oracle's own tree forces for the sampled sinks'
        # particles, and the direct kernel-softened sum for a seeded sample of targets
        acc_vs_oracle = {k: rel_err_stats(v[parts], acc_o) for k, v in forces.items()}
        acc_vs_oracle["sample"] = f"{det['sample_particles']} particles of {det['sample_sinks']} random sinks"
        tg = np.sort(np.random.default_rng(11).choice(a.n, min(a.direct_targets, a.n), replace=False))
        t0 = time.perf_counter()
        acc_dir, _ = oracle.direct(x, m, h, tg)
        acc_vs_direct = {k: rel_err_stats(v[tg], acc_dir) for k, v in forces.items()}
        acc_vs_direct["sample"] = (f"{len(tg)} seeded random targets, oracle direct sum over all N "
                                   f"({time.perf_counter() - t0:.1f} s on {oracle.num_threads()} cores)")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "mixed: f32 near/far tensors, f64 build + Taylor coefficients; int64/int128 tree keys",
        "data": "synthetic",
        "config": bench_config(a, world),
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "stages_ms": stage_ms,
        "per_stage": per_stage,
        "fp64": fp64,
        "accuracy_mixed_vs_fp64": accuracy,
        "accuracy_vs_oracle": acc_vs_oracle,
        "accuracy_vs_direct": acc_vs_direct,
        "fp32_peak_measured": None if alu is None else dict(alu, note="alu_rate probe (peak/alu_rate.cu): best of "
                                                            "three runs; the roofline peak above is the nominal "
                                                            "SMs x lanes x 2 x clock"),
        "tree": {k: info[k] for k in ("L", "nsinks", "near_total", "far_total", "reach_total", "near_pairs",
                                        "candidate_pairs", "walk_fp64_decisions", "smem_subtrees")},
        "neighbours_total": idx_total,
        "memory": memory,
        "presort_device_ms": presort_ms,
        "hbm_peak_gbs": hbm,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_table1(a):
    """The scan of Sec. 3.2.1 (Table 1) on the GPU: for each mean ll-cell occupancy N_ll, the tree
    depth, the stage times of the build (construction and walk), of rcb_neighbours alone and of
    rcb_gravity alone (near and far field), and the share of particles whose acceleration is within
    1 % of the direct sum.  Input as in the table: a uniform sphere of 500,000 particles with h for
    105 neighbours, theta = 0.7 (mixed form; seeded random positions stand in for the Sobol set).
    Times are medians of library stage events over 5 repetitions after one warm-up."""
    import numpy as np
    import torch

    import oracle
    import paper_1108_0028_gb300 as rcb
    import synth
    n = 500000
    x, m, h = synth.make_particles("sphere", n, synth.seed_for(3, 7), "equal", n_neigh=105.0)
    dev = torch.device("cuda", 0)
    xt, mt, ht = (torch.from_numpy(v).to(dev) for v in (x, m, h))
    oracle.build()
    tg = np.sort(np.random.default_rng(11).choice(n, 4000, replace=False))
    acc_dir, _ = oracle.direct(x, m, h, tg)
    rows = []
    for nll in (1, 3, 6, 12, 24, 48, 64, 128):
        tree = rcb.RCBTree(xt, mt, ht, n_ll=nll, theta=0.7, precision="mixed", timing=True)
        rec = {k: [] for k in ("construction", "walk", "neighbours", "near", "far", "gravity")}
        for r in range(6):
            tree.rebuild(xt, mt, ht)
            st_b = tree.stage_times()
            _, idx = tree.neighbours()
            st_n = tree.stage_times()
            acc, _ = tree.gravity()
            st_g = tree.stage_times()
            if r == 0:
                continue
            rec["construction"].append(st_b["build"] - st_b["walk"])
            rec["walk"].append(st_b["walk"])
            rec["neighbours"].append(st_n["nb_count"] + st_n["nb_fill"])
            rec["near"].append(st_g["near"])
            rec["far"].append(st_g["far"])
            rec["gravity"].append(st_g["near"] + st_g["far"])
        info = tree.info()
        e = rel_err_stats(acc.cpu().numpy()[tg], acc_dir)
        ev = np.linalg.norm(acc.cpu().numpy()[tg] - acc_dir, axis=1) / np.linalg.norm(acc_dir, axis=1)
        rows.append({"n_ll": nll, "L": info["L"], "p_below_1pct": float(np.mean(ev < 0.01)),
                     "mean_rel_err": float(ev.mean()), "rms_rel_err": e["rms"],
                     "ms": {k: float(statistics.median(v)) for k, v in rec.items()},
                     "neighbours_per_particle": idx.numel() / n, "near_pairs": info["near_pairs"],
                     "far_per_particle": info["far_total"] / n})
        tree.free()
    print(json.dumps({"table1": rows, "N": n, "theta": 0.7, "form": "mixed", "n_neigh_target": 105,
                      "reference": "oracle direct sum at 4000 seeded targets"}), flush=True)


def main():
    a = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if a.table1:
        run_table1(a)
        return
    if a.impl == "reference":
        run_reference(a, rank, world)
    else:
        run_ours(a, rank, world, local_rank)


if __name__ == "__main__":
    main()
