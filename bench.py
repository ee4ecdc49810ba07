#!/usr/bin/env python3
"""Benchmark: group-shared Barnes-Hut force evaluation with persistent lists
(Sec. 4.2) on a synthetic planetary ring, one JSON line on stdout.

A step is one kick-drift-kick leapfrog step of the whole path: keys, sort,
octree, moments, groups and the tree walk on list-constructing steps (every
4th force evaluation), the moment refresh otherwise, the force kernel, the
FP64 contact pass and the update.  Default workload: the large ring, 2^26
particles, theta 0.4, quadrupole, FP32 group-relative forces, FP64 positions
and updates.

  value    interactions/s over the timed steps (all ranks), device-timed with
           CUDA events; particle-steps/s beside it
  e2e      the same through bh_step_host with pinned host buffers, the
           host<->device copies of every step inside the timed region
  roofline the force kernel against the FP32 peak (152 SMs x 128 lanes x 2
           flops x 2070 MHz), achieved = counted interactions x FP32 flops
           per interaction of the kernel source / event-timed kernel time
  cpu_baseline  the CPU FP64 oracle (host cores) on a ring sector of the same
           surface density

--impl reference runs the oracle as the reference arm.  Under torchrun each
rank runs an independent replica (weak scaling); with --shard the patches
workload instead splits one set of 64 patches across the ranks by the LPT
rule on estimated cost (strong scaling; no data-path collective).  Rank 0
prints; value sums the ranks' interactions over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# FP32 flops per interaction of the force kernel (FFMA/FFMA2 lane = 2,
# FADD/FMUL = 1; rsqrt not counted): particle-particle with the two-float
# separation 24 (23 without softening, where the + eps^2 is not issued),
# particle-particle with a far list particle (single-float separation) 18
# (17 without softening: its r^2 chain adds eps^2 = 0, not counted),
# particle-cell with quadrupole 48 (a = (M R^2 - 5/2 (d.q) / R^2) d / R^5
# + q / R^5: 3 FADD, 3 FFMA for R^2, FMUL R^-2, 9 for q, 3 for d.q, 2 FMUL
# for R^-5, FMUL + FMUL + FFMA for the coefficient, 6 FFMA), monopole only 18.
FLOPS_PP, FLOPS_PP_NO_EPS, FLOPS_PC2, FLOPS_PC1 = 24, 23, 48, 18
FLOPS_PP_FAR, FLOPS_PP_FAR_NO_EPS = 18, 17
# The plain FP64 kernel (absolute coordinates, rsqrt not counted): pp 18
# (3 sub, r^2 5, + eps^2 1, 3 mul, 3 FMA), pc with quadrupole 53, monopole 21.
FLOPS64_PP, FLOPS64_PC2, FLOPS64_PC1 = 18, 53, 21
# The paper's convention (Sec. 5.1): 49 per particle-particle, 31 per particle-cell.
PAPER_PP, PAPER_PC = 49, 31
FP32_LANES, SM_MAX_MHZ = 128, 2070.0
NUM_SMS = 152  # replaced by the device's multiprocessor count when a GPU is present
HBM_FALLBACK_GBS = 6800.0  # the profiling recipe's fallback copy bandwidth

# Algorithmic HBM bytes of the HBM-bound stages (per particle; per node where
# stated), for their GB/s against the measured copy bandwidth:
#  keys      x, y, z read for the root box and again for the keys, key + index
#            written (24 + 24 + 12); the cylindrical frame first reads x, y and
#            writes phi, r (+32)
#  sort      8 passes of 8 bits, each reading and writing key + index (8 x 24)
#  permute   index read, 8 particle arrays read and written (4 + 8 x 16)
#  moments   x, y, z, m (FP64 path) or the hi/lo float4 pair (FP32 path) read
#            per particle; per node its record written and read once more by
#            its parent (FP64: 2 x 80; FP32: 2 x 48 + 4)
#  split     x, y, z, m read, two float4 written (32 + 32)
#  update    per step: kick-drift reads a, v, x and writes v, x (72 + 48), the
#            closing kick reads a, v and writes v (48 + 24)
STAGE_BYTES = {"keys": 60, "keys_cyl_extra": 32, "sort": 192, "permute": 132, "split": 64, "update": 192}
MOMENT_BYTES = {0: (32, 160), 1: (32, 100)}  # precision -> (per particle, per node)


def fp32_peak_tflops(mhz: float) -> float:
    return NUM_SMS * FP32_LANES * 2 * mhz * 1e6 / 1e12


def hbm_peak():
    """Measured copy bandwidth (GB/s) from MEASURED_PEAKS.json, else the
    recipe's fallback; (value, basis)."""
    try:
        v = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
        return v, "measured (MEASURED_PEAKS.json copy bandwidth)"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback (profiling recipe)"


def stage_rates(stage_ms: dict, stage_calls: dict, steps: int, n: int, n_nodes: int, key_frame: int,
                precision: int, peak_gbs: float) -> dict:
    """Per stage: ms per step, and for the HBM-bound stages GB/s from the
    algorithmic bytes per call and the fraction of the copy bandwidth."""
    out = {}
    for st, ms in stage_ms.items():
        calls = stage_calls.get(st, 0)
        if not calls:
            continue
        rec = {"ms_per_step": ms / steps, "calls": calls}
        per_call = None
        if st == "keys":
            per_call = n * (STAGE_BYTES["keys"] + (STAGE_BYTES["keys_cyl_extra"] if key_frame == 1 else 0))
        elif st in ("sort", "permute", "split"):
            per_call = n * STAGE_BYTES[st]
        elif st == "update":  # two kernels per step, half the step's bytes per call on average
            per_call = n * STAGE_BYTES["update"] / 2
        elif st == "moments":
            bp, bn = MOMENT_BYTES[precision]
            per_call = n * bp + n_nodes * bn
        if per_call is not None:
            gbs = per_call * calls / (ms * 1e-3) / 1e9
            rec.update({"gb_per_s": gbs, "frac_of_hbm": gbs / peak_gbs, "bytes_per_call": per_call})
        out[st] = rec
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ring64m_fp32")
    ap.add_argument("--n", type=int, default=None, help="override the particle count")
    ap.add_argument("--sector-of", type=int, default=None,
                    help="with --n: a ring sector of n particles at the surface density of a ring of this many "
                         "(a small case whose lists look like the large ring's, for profiling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-error", action="store_true")
    ap.add_argument("--autotune", action="store_true", help="run the library autotuner before timing")
    ap.add_argument("--no-autotune", action="store_true", help="keep the workload's preset launch settings")
    ap.add_argument("--key-frame", type=int, default=None, choices=[0, 1],
                    help="tree frame: 0 Cartesian, 1 cylindrical (default: the workload's)")
    ap.add_argument("--n-g", type=int, default=None, help="override the group size limit")
    ap.add_argument("--n-leaf", type=int, default=None, help="override the leaf size limit")
    ap.add_argument("--tune", default="", help="launch settings to apply, e.g. chunk=64,order_window=8192")
    ap.add_argument("--shard", action="store_true",
                    help="patches workload under torchrun: split one set of patches across the ranks (LPT on "
                         "estimated cost, strong scaling) instead of one set per rank")
    return ap.parse_args()


def rank_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def max_over_ranks(x: float, device="cpu") -> float:
    """The largest x over all ranks (timing: the job takes as long as its
    slowest replica); x itself when not distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device="cpu") -> float:
    """The sum of x over all ranks (work done by the whole job); x itself
    when not distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard_patches(sizes, rank: int, world: int):
    """Patch indices this rank steps when one set of patches is split across
    the ranks, and the load imbalance (largest / mean estimated cost)."""
    from paper_1907_02289_gb300 import shard
    costs = [shard.patch_cost(int(s)) for s in sizes]
    parts = shard.lpt_assign(costs, world)
    if any(not p for p in parts):
        raise SystemExit(f"--shard: {len(sizes)} patches cannot give every one of {world} ranks a patch")
    return parts[rank], shard.imbalance(costs, parts)


def replica_seed(base_seed: int, rank: int) -> int:
    """Seed of rank's replica: every rank steps its own, different ring."""
    return base_seed + 1000 * rank


class Clocks:
    """nvidia-smi clock/throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [v.strip() for v in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# Sources whose change invalidates a recorded traffic figure: the force
# kernel and the list expansion (which fixes the order the kernel reads).
TRAFFIC_SOURCES = ("force32.cu", "force_common.cuh", "walk.cu")


def recorded_traffic(kernel: str, workload: str, n: int, key_frame: int, tuning: dict, path: str | None = None):
    """DRAM bytes per launch of the force kernel from the committed ncu
    captures (one record per launch setting captured), if one was taken on
    this workload (size, frame, n_g and launch settings) with the kernel
    source as it is now (else None)."""
    import hashlib
    path = path or os.path.join(ROOT, "profiles", "traffic.json")
    try:
        recs = json.load(open(path))[kernel]
    except (OSError, KeyError, ValueError):
        return None
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_1907_02289_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    for rec in recs if isinstance(recs, list) else [recs]:
        if (rec.get("source_sha256") != h.hexdigest() or rec.get("workload") != workload or rec.get("N") != n
                or rec.get("key_frame") != key_frame):
            continue
        if any(rec.get("tuning", {}).get(k) != tuning.get(k) for k in ("n_g", "chunk", "warps", "sched",
                                                                        "order_window", "order_by_cost")):
            continue
        return rec["bytes_per_launch"]
    return None


def oracle_sector(n_sector: int, full_n: int, prm: dict, seed: int = 77):
    """A ring sector with the surface density of the full ring (same
    workload, bounded sample) for the CPU oracle."""
    from paper_1907_02289_gb300 import synth
    return synth.ring(n_sector, seed, phi_max=2 * math.pi * n_sector / full_n)


def cpu_oracle_rate(P: dict, prm: dict):
    """One oracle force evaluation with list construction; interactions/s."""
    import numpy as np

    import oracle as orc
    op = orc.Params(**{k: v for k, v in prm.items() if k in orc.Params.__dataclass_fields__})
    t0 = time.perf_counter()
    S = orc.rebuild(P, op)
    orc.accel(S, op)
    dt = time.perf_counter() - t0
    t = S.tree
    ni = t["end"][S.groups].astype(np.int64) - t["begin"][S.groups]
    leafn = t["end"].astype(np.int64) - t["begin"]
    nj = np.add.reduceat(leafn[S.lists["P"]], S.lists["pp_off"][:-1]) if len(S.lists["P"]) else np.zeros(len(ni))
    inter = int((ni * nj).sum() + (ni * np.diff(S.lists["pc_off"])).sum())
    return inter / dt, inter, dt, orc.num_threads()


def run_reference(args):
    rank, _, world = rank_info()
    if rank != 0:
        return
    from paper_1907_02289_gb300 import synth

    import numpy as np

    import oracle as orc
    pr = synth.PRESETS[args.workload]
    # the patches have the surface density of the 2^20 ring
    full_n = args.n or pr["n"] or (1 << 20)
    prm = dict(pr["params"])
    n_s = min(full_n, 1 << 18)
    P = oracle_sector(n_s, full_n, prm)
    op = orc.Params(**{k: v for k, v in prm.items() if k in orc.Params.__dataclass_fields__})
    # KDK steps of the oracle on the sector, lists rebuilt every rebuild_every
    S = orc.rebuild(P, op)
    a = orc.accel(S, op)
    k = 1
    inter_tot, t_tot = 0, 0.0

    def count(S):
        t = S.tree
        ni = t["end"][S.groups].astype(np.int64) - t["begin"][S.groups]
        leafn = t["end"].astype(np.int64) - t["begin"]
        nj = np.add.reduceat(leafn[S.lists["P"]], S.lists["pp_off"][:-1])
        return int((ni * nj).sum() + (ni * np.diff(S.lists["pc_off"])).sum())

    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        Q = S.P
        for ci, c in enumerate("xyz"):
            Q["v" + c] = Q["v" + c] + 0.5 * op.dt * a[:, ci]
        for c in "xyz":
            Q[c] = Q[c] + op.dt * Q["v" + c]
        if k % op.rebuild_every == 0:
            S = orc.rebuild(Q, op)
        else:
            orc.refresh(S, op)
        a = orc.accel(S, op)
        for ci, c in enumerate("xyz"):
            S.P["v" + c] = S.P["v" + c] + 0.5 * op.dt * a[:, ci]
        k += 1
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            inter_tot += count(S)
            t_tot += dt
    value = inter_tot / t_tot
    sample = f"ring sector of {n_s} particles at the surface density of the {full_n}-particle ring"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "interactions/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "N": n_s, "sample_of_N": full_n},
            "particle_steps_per_s": n_s * args.steps / t_tot,
            "cpu_baseline": {"value": value, "unit": "interactions/s", "cores": orc.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "interactions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


METRIC = "interactions/s and particle-steps/s per GB300 at stated force error; % FP32 peak"


def run_ours(args):
    import numpy as np
    import torch

    from paper_1907_02289_gb300 import _build, bh, synth
    global NUM_SMS
    rank, local, world = rank_info()
    _build.build()
    torch.cuda.set_device(local)
    NUM_SMS = torch.cuda.get_device_properties(local).multi_processor_count
    # measured FMA-loop peaks of this device (roofline context for the FP32
    # kernel, the roofline denominator of the FP64 kernel)
    peak32_measured = bh.bh_measure_peak(bh.BH_PEAK_FP32)
    peak64_measured = bh.bh_measure_peak(bh.BH_PEAK_FP64)
    hbm_gbs, hbm_basis = hbm_peak()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pr = synth.PRESETS[args.workload]
    prm = dict(pr["params"])
    if args.key_frame is not None:
        prm["key_frame"] = args.key_frame
    if args.n_g is not None:
        prm["n_g"] = args.n_g
    if args.n_leaf is not None:
        prm["n_leaf"] = args.n_leaf
    offsets = None
    sharded = args.shard and pr["kind"] == "patches"
    shard_info = None
    if args.shard and not sharded:
        raise SystemExit("--shard applies to the patches workload only")
    if pr["kind"] == "patches":
        if sharded:  # one set of patches for the whole job, LPT-split across the ranks
            parts, sizes = synth.patches(seed=pr["seed"])
            mine, imb = shard_patches(sizes, rank, world)
            shard_info = {"patches_this_rank": len(mine), "patches_total": len(sizes),
                          "estimated_cost_imbalance": imb}
            parts, sizes = [parts[i] for i in mine], [sizes[i] for i in mine]
        else:
            parts, sizes = synth.patches(seed=replica_seed(pr["seed"], rank))
        P = {f: np.concatenate([q[f] for q in parts]) for f in synth.FIELDS}
        offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        n = int(offsets[-1])
    else:
        n = args.n or pr["n"]
        if args.sector_of and pr["kind"] == "ring":
            P = synth.ring(n, replica_seed(pr["seed"], rank), phi_max=2 * math.pi * n / args.sector_of)
        else:
            P = synth.ring(n, replica_seed(pr["seed"], rank)) if pr["kind"] == "ring" else synth.make(args.workload, n)[0]
    stream = torch.cuda.current_stream()

    ctx = bh.Context(offsets=offsets, **prm)
    D = bh.Particles(P)
    tuning = None
    if (pr.get("autotune") and not args.no_autotune) or args.autotune:
        # autotuned launch settings and n_g (the batched configuration also
        # issues its list-reusing steps as CUDA graphs)
        tuned_ms = ctx.bh_autotune(D)
        if pr["kind"] == "patches":
            ctx.bh_set_tuning(graph=1)
        tuning = dict(ctx.bh_get_tuning(), autotuned_step_ms=tuned_ms)
        prm["n_g"] = tuning["n_g"]
    if args.tune:
        ctx.bh_set_tuning(**{k: int(v) for k, v in (kv.split("=") for kv in args.tune.split(","))})
        tuning = dict(ctx.bh_get_tuning(), **({"autotuned_step_ms": tuning["autotuned_step_ms"]} if tuning else {}))
    # initial evaluation + warm-up steps (evaluations 0..W); timed steps then
    # start on a list-constructing evaluation when W = 3 and rebuild_every = 4
    ctx.bh_step(D, args.warmup)
    ctx.bh_sync()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    clocks = Clocks(local)
    ctx.bh_set_timing(True)
    ctx.bh_get_timing(reset=True)
    c0 = ctx.bh_get_counters()
    inter = pp = pc = pp_far = refined = 0
    barrier()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        ctx.bh_step(D, 1)
        c = ctx.bh_get_counters()
        pp += c["n_pp"]
        pc += c["n_pc"]
        pp_far += c["n_pp_far"]
        refined += c["n_refined"]
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    c_stage = ctx.bh_get_counters()  # after the synchronisation: every stage event is complete
    sizes = ctx.bh_get_sizes()
    force_ms, force_launches = ctx.bh_get_timing(reset=True)
    stages = stage_rates(c_stage["stage_ms"], c_stage["stage_calls"], args.steps, n, sizes["n_nodes"],
                         prm.get("key_frame", 0), prm["precision"], hbm_gbs)
    free_b, total_b = torch.cuda.mem_get_info()
    mem_used_gb = (total_b - free_b) / 1e9  # device memory in use after the timed steps (all holders)
    balance = None
    if ctx.bh_get_tuning()["sched"] != bh.BH_SCHED_GRID and prm["precision"] == 1:
        try:
            balance = ctx.bh_get_balance()
        except bh.BHError:
            balance = None
    ctx.bh_set_timing(False)
    c1 = ctx.bh_get_counters()
    launches = c1["n_launches"] - c0["n_launches"]
    inter = pp + pc
    elapsed = max_over_ranks(elapsed, "cuda")
    # work of the whole job: every rank's own (sharded patches differ per
    # rank; replicas are alike, so this is world x one rank's)
    job_inter = sum_over_ranks(inter, "cuda")
    job_n = sum_over_ranks(n, "cuda")
    job_paper_flops = sum_over_ranks(pp * PAPER_PP + pc * PAPER_PC, "cuda")
    value = job_inter / elapsed
    if prm["precision"] == 1:
        flops_pc = FLOPS_PC2 if prm["order"] >= 2 else FLOPS_PC1
        flops_pp = FLOPS_PP_NO_EPS if prm["eps"] == 0.0 else FLOPS_PP
        flops_far = FLOPS_PP_FAR_NO_EPS if prm["eps"] == 0.0 else FLOPS_PP_FAR
    else:
        flops_pc = FLOPS64_PC2 if prm["order"] >= 2 else FLOPS64_PC1
        flops_pp = flops_far = FLOPS64_PP
    flops = (pp - pp_far) * flops_pp + pp_far * flops_far + pc * flops_pc
    # force launches timed by the library (graph-captured steps are not timed
    # per launch): mean flops of an evaluation / mean time of a timed launch
    achieved = (flops / args.steps) / (force_ms / force_launches / 1e3) / 1e12 if force_ms > 0 else None
    f32 = prm["precision"] == 1
    peak = fp32_peak_tflops(SM_MAX_MHZ) if f32 else peak64_measured
    roofline = {"kernel": "k_force32" if f32 else "k_force64", "bound": "alu" if f32 else "fp64",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak if achieved else None,
                "traffic": recorded_traffic("k_force32", args.workload, n, prm.get("key_frame", 0),
                                            ctx.bh_get_tuning()) if prm["precision"] == 1 else None,
                "peak_basis": (f"{NUM_SMS} SMs (device attribute) x 128 FP32 lanes x 2 flops x 2070 MHz (max SM "
                               f"clock); measured FMA-loop peak of this device {peak32_measured:.2f} TFLOP/s")
                if f32 else "measured FMA-loop FP64 peak of this device (bh_measure_peak)",
                "peak_measured_fma": peak32_measured if f32 else peak64_measured,
                "frac_of_measured_fma": (achieved / (peak32_measured if f32 else peak64_measured)) if achieved else None,
                "flops_per_interaction": {"pp": flops_pp, "pp_far": flops_far, "pc": flops_pc},
                "kernel_ms_per_launch": force_ms / max(force_launches, 1), "launches": force_launches}
    if clk.get("sm_mhz") and f32:
        roofline["peak_at_median_clock"] = fp32_peak_tflops(clk["sm_mhz"])
        roofline["frac_at_median_clock"] = achieved / roofline["peak_at_median_clock"] if achieved else None

    # force error of this path against the plain FP64 GPU path on the same lists
    err = fp64 = None
    if not args.no_error and prm["precision"] == 1:
        Pnow = D.numpy()
        ctxe = bh.Context(offsets=offsets, **dict(prm, precision=0))
        De = bh.Particles(Pnow)
        ctxe.bh_build_tree(De)
        ctxe.bh_make_lists()
        ctxe.bh_set_timing(True)
        ctxe.bh_compute_forces(De, bh.BH_FORCE_TREE_ONLY)
        ms64, _ = ctxe.bh_get_timing(reset=True)
        ce = ctxe.bh_get_counters()
        ctx32 = bh.Context(offsets=offsets, **prm)
        D32 = bh.Particles(De.numpy())
        ctx32.bh_build_tree(D32)
        ctx32.bh_make_lists()
        ctx32.bh_compute_forces(D32, bh.BH_FORCE_TREE_ONLY)
        ctxe.bh_sync()
        ctx32.bh_sync()
        a64 = torch.stack([De.t["ax"], De.t["ay"], De.t["az"]], 1)
        a32 = torch.stack([D32.t["ax"], D32.t["ay"], D32.t["az"]], 1)
        r = torch.linalg.norm(a64, dim=1)
        rel = (torch.linalg.norm(a32 - a64, dim=1) / r).cpu().numpy()
        rn = r.cpu().numpy()
        dn = torch.linalg.norm(a32 - a64, dim=1).cpu().numpy()
        ok = rn >= 1e-2 * np.median(rn)
        rmsn_all = dn / np.sqrt(np.mean(rn * rn))
        gate = 1e-5
        above = rel > gate
        worst_ok = float(rel[ok].max())
        near_rms = float(rmsn_all[~ok].max()) if (~ok).any() else 0.0
        passed = bool(worst_ok <= gate and near_rms <= gate)
        c32 = ctx32.bh_get_counters()
        err = {"reference": "plain FP64 GPU path on the same lists (itself within 1e-12 of the CPU oracle)",
               "gate": gate,
               "gate_used": "max relative error over particles with |a| >= 1e-2 x median; the near-cancelling "
                            "rest (|a| < 1e-2 x median) in the rms-normalised form |da| / rms|a|",
               "max_rel_excl_near_cancelling": worst_ok, "near_cancelling": int((~ok).sum()),
               "max_rms_normalised_near_cancelling": near_rms, "gate_passed": passed,
               "max_rel": float(rel.max()), "max_rms_normalised": float(rmsn_all.max()),
               "p99_9_rel": float(np.percentile(rel, 99.9)), "median_rel": float(np.median(rel)),
               "n_above_gate_excl_near_cancelling": int((above & ok).sum()), "n_above_gate": int(above.sum()),
               "refined_particles": c32["n_refined"]}
        # the plain FP64 kernel on the same particles and lists, for the ratio
        rate64 = (ce["n_pp"] + ce["n_pc"]) / (ms64 / 1e3)
        rate32 = (pp + pc) / args.steps / (force_ms / force_launches / 1e3)
        # the FP32 path's rate with its refinement pass counted (the part that
        # brings the ill-conditioned particles to the gate)
        refine_ms = stages.get("refine", {}).get("ms_per_step", 0.0)
        rate32r = (pp + pc) / args.steps / ((force_ms / force_launches + refine_ms) / 1e3)
        fp64 = {"kernel": "k_force64", "kernel_ms": ms64, "interactions_per_s": rate64,
                "fp32_kernel_interactions_per_s": rate32, "fp32_with_refinement_interactions_per_s": rate32r,
                "fp32_over_fp64": rate32r / rate64}
        for x in (ctxe, ctx32):
            x.close()
        del De, D32

    e2e = None
    if not args.no_e2e:
        ctxh = bh.Context(offsets=offsets, **prm)
        if tuning:
            ctxh.bh_set_tuning(**{k: v for k, v in tuning.items() if k != "autotuned_step_ms"})
        H = bh.HostParticles(P, pinned=True)
        ctxh.bh_step_host(H, args.warmup)
        ctxh.bh_set_timing(False)
        ppe = pce = 0
        cb0 = ctxh.bh_get_counters()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctxh.bh_step_host(H, 1)
            c = ctxh.bh_get_counters()
            ppe += c["n_pp"]
            pce += c["n_pc"]
        barrier()
        te = time.perf_counter() - t0
        te = max_over_ranks(te, "cuda")
        cb1 = ctxh.bh_get_counters()
        # bytes the library copied per step (ids, and masses on the way back,
        # only on list-constructing steps: the others leave them unchanged)
        e2e = {"value": sum_over_ranks(ppe + pce, "cuda") / te, "unit": "interactions/s",
               "h2d_bytes_per_step": (cb1["n_h2d_bytes"] - cb0["n_h2d_bytes"]) / args.steps,
               "d2h_bytes_per_step": (cb1["n_d2h_bytes"] - cb0["n_d2h_bytes"]) / args.steps,
               "particle_steps_per_s": job_n * args.steps / te, "api": "bh_step_host (pinned host buffers)"}
        ctxh.close()

    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        if pr["kind"] == "cube":  # small enough for the whole set, plus the direct sum
            import oracle as orc
            rate, inter_s, dt_s, cores = cpu_oracle_rate(P, prm)
            op = orc.Params(**{k: v for k, v in prm.items() if k in orc.Params.__dataclass_fields__})
            t0 = time.perf_counter()
            orc.direct(P, op)
            t_direct = time.perf_counter() - t0
            what = (f"one list-constructing force evaluation of the whole {n}-particle set; direct sum "
                    f"{n * (n - 1) / t_direct:.3e} pairs/s")
        elif offsets is None:
            n_s = min(n, 1 << 21)
            rate, inter_s, dt_s, cores = cpu_oracle_rate(oracle_sector(n_s, n, prm), prm)
            what = (f"one list-constructing force evaluation of a {n_s}-particle ring sector at the surface "
                    f"density of the {n}-particle ring")
        else:  # the first patches, about 2^20 particles
            k = int(np.searchsorted(offsets, 1 << 20)) or 1
            k = min(k, len(offsets) - 1)
            sub = {f: P[f][:offsets[k]] for f in synth.FIELDS}
            inter_s = dt_s = 0.0
            for q in range(k):
                part = {f: sub[f][offsets[q]:offsets[q + 1]] for f in synth.FIELDS}
                _, i_q, t_q, cores = cpu_oracle_rate(part, prm)
                inter_s += i_q
                dt_s += t_q
            rate = inter_s / dt_s
            inter_s = int(inter_s)
            what = f"one list-constructing force evaluation of each of the first {k} patches ({int(offsets[k])} particles)"
        cpu = {"value": rate, "unit": "interactions/s", "cores": cores, "kind": "oracle",
               "sample": f"{what} ({inter_s} interactions, {dt_s:.1f} s)"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "interactions/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
                "scaling": "strong" if sharded else "weak", "vs_baseline": None, "dtype": "f32" if prm["precision"] == 1 else "f64",
                "data": "synthetic",
                "config": {"workload": args.workload, "N": n,
                           **({"sector_of_N": args.sector_of} if args.sector_of else {}),
                           "theta": prm["theta"], "n_g": prm["n_g"],
                           "n_leaf": prm["n_leaf"],
                           "key_frame": "cylindrical (phi, r, z)" if prm.get("key_frame", 0) == 1 else "Cartesian",
                           "order": prm["order"], "rebuild_every": prm["rebuild_every"],
                           "precision": "FP32 group-relative forces, FP64 positions/velocities/updates"
                           if prm["precision"] == 1 else "FP64",
                           "l2": "inputs larger than L2 (particle arrays %.1f GB)" % (n * 88 / 1e9),
                           "parallelism": ("patches split across ranks (LPT)" if sharded and world > 1
                                           else "replicas" if world > 1 else "single GPU"),
                           **({"shard_rank0": shard_info} if shard_info else {}),
                           **({"patches": len(offsets) - 1} if offsets is not None else {}),
                           **({"tuning": tuning} if tuning else {})},
                "particle_steps_per_s": job_n * args.steps / elapsed,
                "interactions_per_step": inter / args.steps,
                "refined_particles_per_step": refined / args.steps,
                "stages": stages, "hbm_peak_gbs": hbm_gbs, "hbm_peak_basis": hbm_basis,
                "pp_pc_per_step": [pp / args.steps, pc / args.steps],
                "pp_far_per_step": pp_far / args.steps,
                ("pct_fp32_peak" if f32 else "pct_fp64_peak"): 100 * roofline["frac"] if roofline["frac"] else None,
                "flops_per_s_paper_convention": job_paper_flops / elapsed,
                "force_error": err, "fp64_path": fp64, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk, "device_memory_used_gb": mem_used_gb,
                **({"load_balance_busy_fraction": balance} if balance is not None else {})}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
