"""Benchmark of the S_N source-iteration solve (cell-direction-group updates/s).

Default workload: the batched cone-beam form -- 96^3 voxels of 1/3 cm (the
32 cm water-cylinder phantom with bone and air inserts), 19 groups, S8
(80 directions), P3, 32 CT source positions on a 50 cm circle -- with an FP32
sweep, the scatter-source contraction and the Eq. 3 moments on the tensor cores
(split BF16, FP32 accumulation; the fastest form measured) and FP64 scalar
flux, residual and balance. One step = one full dts_solve of the batch (ray
trace, first-collision source, every group's source iteration to tol,
downscatter), inputs already resident in HBM. Beside it: the FP64 plain form on
one source of the same workload ("FP32-batched vs FP64 plain", and the 1e-4
relative L2 gate), the CUDA-core FP32 form on the same batch, the end-to-end
rate through the C ABI with host buffers, and the CPU oracle on a sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun one ring of 32 N source positions is partitioned over the N
ranks (32 per GPU, weak scaling, no collective on the data path); rank 0
gathers the per-source results on the host and prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-direction-group updates/s, FP32-batched vs FP64 plain, at 1e-4 rel L2"
UNIT = "updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch96", choices=["batch96", "hetero64", "precision128"])
    ap.add_argument("--sources", type=int, default=32)
    ap.add_argument("--voxels", type=int, default=96,
                    help="batch96 only: the phantom at N^3 voxels (profiling cases; the benchmark is 96)")
    ap.add_argument("--groups", type=int, default=19, help="batch96 only: energy groups (19)")
    ap.add_argument("--tol", type=float, default=None)
    ap.add_argument("--max-iters", type=int, default=None)
    ap.add_argument("--tile", default="auto", help="tx,ty,tz or 'auto' (dts_tune_tile)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 plain comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the CUDA-core FP32 comparison")
    ap.add_argument("--precision", default="auto", choices=["auto", "fp32", "splitbf16", "tf32"],
                    help="arithmetic of the FP32-batched form's scatter-source contraction")
    ap.add_argument("--split", type=int, default=4,
                    help="solve each GPU's sources as this many problems on their own streams "
                         "(dts_solve_many: one part's moment kernels beside another's sweep); 1 = one problem")
    ap.add_argument("--loop", default="host", choices=["host", "device"],
                    help="host: one host round trip per source iteration (the kernels the launch-list "
                         "profile covers); device: a group's source iterations as one CUDA-graph launch "
                         "with the convergence decisions on the device (dts_set_device_loop)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def make_workload(args, rank=0):
    """The rank's share of the workload. batch96: one ring of sources x world
    CT source positions (2 pi k / n on the 50 cm circle), partitioned over the
    ranks (rank r solves positions r, r + world, ...), so every GPU solves
    `sources` independent projections of one scan; one GPU solves the ring of
    `sources` positions."""
    from paper_1910_11335_b300 import inputs, shard
    if args.workload == "batch96":
        if getattr(args, "voxels", 96) == 96 and getattr(args, "groups", 19) == 19:
            w = inputs.batch_96(args.sources)
        else:
            w = inputs.cone_beam(args.voxels, args.groups, 8, 3, args.sources, seed_index=1, tol=1e-6,
                                 name=f"cone{args.voxels}_s8p3_{args.groups}g_x{args.sources}")
        world = dist_env()[2]
        if world > 1:
            ring = inputs.ring_sources(w.sources[0].spectrum, args.sources * world)
            w.sources = [ring[k] for k in shard.partition(len(ring), world, rank)]
        return w
    if args.workload == "hetero64":
        return inputs.hetero_64()
    return inputs.precision_128()


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "of measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "of fallback"


def cpu_info():
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def cpu_sample(w, threads):
    """The oracle, as it stands, on a bounded sample of the workload: source 0,
    group 0, one source iteration (ray trace, first-collision source and one
    full sweep of all directions) on `threads` host threads."""
    import oracle
    from paper_1910_11335_b300.inputs import first_groups, with_sources
    t = first_groups(with_sources(w, [0]), 1)
    t0 = time.perf_counter()
    oracle.solve(t, 0, tol=0.0, max_iters=1, n_threads=threads)
    dt = time.perf_counter() - t0
    return t.n_voxels * t.n_dirs / dt, dt


def oracle_threads():
    """Threads the oracle can use: it runs the eight octants of a sweep in parallel."""
    return min(8, os.cpu_count() or 1)


def run_reference(args):
    rank, local, world = dist_env()
    if rank != 0:
        return
    w = make_workload(args)
    threads = oracle_threads()
    vals = []
    for i in range(args.warmup + args.steps):
        v, dt = cpu_sample(w, threads)
        if i >= args.warmup:
            vals.append(v)
    value = statistics.mean(vals)
    sample = (f"{w.name}: source 0, group 0, 1 source iteration "
              f"({w.n_voxels * w.n_dirs:.3e} updates) per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "ms_per_step": 1e3 * w.n_voxels * w.n_dirs / value, "dtype": "f64",
            "data": "synthetic", "scaling": "weak", "vs_baseline": None,
            "config": {"workload": w.name, "voxels": [w.nx, w.ny, w.nz], "groups": w.n_groups,
                       "directions": w.n_dirs, "legendre_order": w.legendre_order, "sources_per_gpu": w.batch,
                       "tol": args.tol if args.tol is not None else w.tol,
                       "oracle": "plain FP64 C, gcc -O2, OpenMP over octants"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample, **cpu_info()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# Per-kernel constants measured with ncu on a small case (48^3, 32 sources, S8 P3, 2 groups, 8 x 4 x 4
# tiles; profiles/k_sweep_batch_cone48_s8p3_x32.md, profiles/k_moments_q_cone48_s8p3_x32.md), used while
# the kernel's source block is the one that was profiled (its SHA-256), else reported null:
#   inst_per_update    warp instructions issued per cell-direction update (smsp__inst_executed.sum);
#                      the Q-input sweep's is the benchmark phantom's at 96^3 over all 19 groups (3
#                      sources, 2 iterations per group, every sweep launch of the solve:
#                      profiles/k_sweep_batch_cone96_s8p3_x3_19g.md)
#   dram_over_design   dram__bytes_read.sum + dram__bytes_write.sum over the design's bytes per update
#   fma_pipe           sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active / 100
# The DRAM ratios are a 48^3 case's; at 96^3 the tile-to-tile faces, which make most of the sweep's
# excess, are the same bytes per update and only their L2 hit rate can differ.
MEASURED = {
    "k_sweep_batch (Q input)": {"inst_per_update": 1.883, "dram_over_design": 1.279, "fma_pipe": 0.1904,
                                "block": "sweep"},
    "k_sweep_batch": {"inst_per_update": 2.819, "dram_over_design": 1.147, "fma_pipe": 0.2485, "block": "sweep"},
    "k_moments_q": {"inst_per_update": 0.554, "dram_over_design": 0.999, "fma_pipe": 0.1423,
                    "tensor_pipe": 0.0566, "block": "tc"},
    "k_reduce_psi": {"inst_per_update": 0.603, "dram_over_design": 1.016, "fma_pipe": 0.4854, "block": "reduce_psi"},
}
# SHA-256 of each measured kernel's source block: a source change invalidates the constants until the
# kernel is measured again
MEASURED_SHA256 = {
    "sweep": "029fa16a9443c7f5e4c5e10fb17f40199f112cbda85c39ef7e7d7351d173c72e",
    "tc": "bdd8c508c979144689f27e53fd314ae70370ecb493640dde9540a83e7c281b44",
    "reduce_psi": "0b3b2d49fb436c16e2769deb7cac4deaf371d47eaf48a506616ba083c66c6e69",
}


def kernel_block_sha256(block):
    """SHA-256 of the source of a profiled kernel: the batched sweep's block of
    dts_kernels.cuh, the tensor-core file, or the angular-flux moment kernel's block."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1910_11335_b300", "csrc")
    if block == "tc":
        src = open(os.path.join(csrc, "dts_tc.cuh")).read()
    else:
        src = open(os.path.join(csrc, "dts_kernels.cuh")).read()
        a, b = {"sweep": ("// A3 + A4, batched form (FP32)", "// Error-free FP32 accumulation"),
                "reduce_psi": ("// Eq. 3 and its higher moments from the angular fluxes",
                               "// per source: residual")}[block]
        src = src[src.index(a):src.index(b)]
    return hashlib.sha256(src.encode()).hexdigest()


def measured(kernel):
    m = MEASURED.get(kernel)
    if m and kernel_block_sha256(m["block"]) == MEASURED_SHA256[m["block"]]:
        return m
    return None


def roofline(stats, ms_step, steps, K, ndo, tc, peaks, which, n_sm):
    """The dominant kernel's roofline and the HBM accounting of the iteration.

    The wavefront sweep takes most of a step. It moves per update (design of the
    tensor-core forms, which materialise the per-direction source) the Q it
    reads (4 B) and the angular flux it writes (4 B) plus sigma_t shared by the
    octant's directions; the fused CUDA-core form reads the K source moments per
    (cell, octant) instead of Q. It is bound by instruction issue and latency,
    not by HBM, so its roofline is the SM issue rate: achieved = measured warp
    instructions per update x updates per second of sweep time (CUDA events
    around the sweep graph), peak = 4 warp instructions per cycle per SM x SMs x
    maximum SM clock. The HBM fractions are reported beside it: on the method's
    algorithmic minimum (2K+1) x 4 / N_d bytes per update (read K source moments
    and sigma_t, write K moments per cell; faces and fluxes on chip), on the
    design's bytes, and on the DRAM bytes ncu measured; the moment kernel
    (Eq. 3 + scatter-source contraction), which is HBM-bound, gets its own."""
    updates = sum(s["updates"] for s in stats)
    sweep_s = sum(s["sweep_ms"] for s in stats) / 1e3
    red_s = sum(s["reduce_ms"] for s in stats) / 1e3
    n_launch = sum(s["sweep_launches"] for s in stats)
    ups = updates / sweep_s
    hbm = peaks["hbm_gbs"]
    bpu_alg = (2 * K + 1) * 4.0 / (8 * ndo)
    bpu_sweep = 8.0 + 4.0 / ndo if tc else (K + 1) * 4.0 / ndo + 4.0
    # moment kernel: psi read, Q written (tensor-core forms) or T written, F read, scalar flux in and out
    bpu_mom = (4.0 + 4.0 if tc else 4.0 + K * 4.0 / (8 * ndo)) + K * 4.0 / (8 * ndo) + 16.0 / (8 * ndo)
    kname = "k_sweep_batch (Q input)" if tc else "k_sweep_batch"
    meas = measured(kname)
    mom = measured("k_moments_q" if tc else "k_reduce_psi")
    peak_inst = 4.0 * n_sm * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e9   # G warp instructions / s
    out = {"bound": "alu", "unit": "Ginst/s", "peak": peak_inst, "kernel": kname,
           "peak_source": f"4 warp instructions per cycle x {n_sm} SMs x {peaks.get('sm_max_mhz', 2032.0):.0f} MHz",
           "achieved": None, "frac": None, "traffic": None,
           "sweep_updates_per_s": ups, "sweep_share_of_step": sweep_s * 1e3 / (ms_step * steps)}
    if meas:
        out["achieved"] = meas["inst_per_update"] * ups / 1e9
        out["frac"] = out["achieved"] / peak_inst
        # per launch, like the timing: the average launch's design bytes times the measured ratio
        out["traffic"] = meas["dram_over_design"] * bpu_sweep * updates / n_launch
        out["fma_pipe_utilization"] = meas["fma_pipe"]
        out["inst_per_update"] = meas["inst_per_update"]
    out["hbm"] = {
        "peak_gbs": hbm, "peak_source": which,
        "algorithmic_bytes_per_update": bpu_alg,
        "frac_algorithmic": ups * bpu_alg / 1e9 / hbm,
        "sweep_design_bytes_per_update": bpu_sweep,
        "sweep_frac_design": ups * bpu_sweep / 1e9 / hbm,
        "sweep_frac_dram_measured": (ups * bpu_sweep * meas["dram_over_design"] / 1e9 / hbm) if meas else None,
        "moment_kernel": "k_moments_q" if tc else "k_reduce_psi",
        "moment_bytes_per_update": bpu_mom,
        "moment_frac_design": updates / red_s * bpu_mom / 1e9 / hbm,
        "iteration_frac_dram_measured": (
            (updates * bpu_sweep * meas["dram_over_design"] + updates * bpu_mom * mom["dram_over_design"])
            / (sweep_s + red_s) / 1e9 / hbm) if (meas and mom) else None,
    }
    return out


def aggregate(ms: float, updates: float, world: int, device=None):
    """Whole-job numbers over ranks: the slowest rank's time and the sum of
    every rank's updates (weak scaling: each rank solves its own batch)."""
    if world <= 1:
        return ms, float(updates)
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([float(updates)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(u[0])


class Parts:
    """The workload's sources as consecutive runs (dts.source_parts), each one
    problem on its own stream, solved together by dts_solve_many; with one run,
    one problem on the given stream solved by dts_solve."""

    def __init__(self, w, prec, tol, args, dts, dev, stream, torch, split=None, loop=None):
        self.dts = dts
        device_loop = (args.loop if loop is None else loop) == "device"
        self.runs = dts.source_parts(w.batch, args.split if split is None else split, w.sn_order)
        tile = tuple(int(x) for x in args.tile.split(","))
        self.streams = [stream] if len(self.runs) == 1 else [torch.cuda.Stream(dev) for _ in self.runs]
        self.probs = [dts.problem_from_workload(w, precision=prec, tol=tol, max_iters=args.max_iters or 1000,
                                                tile=tile, device=dev, stream=st.cuda_stream, sources=run,
                                                device_loop=device_loop)
                      for run, st in zip(self.runs, self.streams)]

    def solve(self):
        """One solve of every source; the parts' stats merged into one dict."""
        if len(self.probs) == 1:
            sts = [self.probs[0].solve(allow_not_converged=True)]
        else:
            sts = self.dts.solve_many(self.probs, allow_not_converged=True)
        d = [x.as_dict() for x in sts]
        out = {k: sum(x[k] for x in d) for k in ("updates", "sweeps", "launches", "sweep_launches",
                                                  "sweep_ms", "reduce_ms")}
        out.update(max_residual=max(x["max_residual"] for x in d), solve_ms=max(x["solve_ms"] for x in d),
                   converged=min(x["converged"] for x in d), tile_x=d[0]["tile_x"], tile_y=d[0]["tile_y"],
                   tile_z=d[0]["tile_z"])
        return out

    def locate(self, k):
        """(problem, member) of source k."""
        for p, run in zip(self.probs, self.runs):
            if k in run:
                return p, run.index(k)
        raise IndexError(k)

    def fluence(self, k, comp, out=None):
        p, b = self.locate(k)
        return p.fluence(b, comp, out=out)

    def close(self):
        for p in self.probs:
            p.close()


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1910_11335_b300 import build, dts, shard
    build.build()
    rank, local, world = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    w = make_workload(args, rank)
    fp32 = args.workload != "hetero64"
    # auto: the fastest measured form of this workload, the split-BF16 tensor-core contraction
    prec = {"auto": dts.PREC_FP32_SPLITBF16, "fp32": dts.PREC_FP32, "splitbf16": dts.PREC_FP32_SPLITBF16,
            "tf32": dts.PREC_FP32_TF32}[args.precision] if fp32 else dts.PREC_FP64
    tc = prec in (dts.PREC_FP32_SPLITBF16, dts.PREC_FP32_TF32)
    tol = args.tol if args.tol is not None else w.tol
    tuned = None
    if args.tile == "auto":
        tile, tuned = dts.tune_tile(w, precision=prec, device=local)
        args.tile = ",".join(str(x) for x in tile)
    parts = Parts(w, prec, tol, args, dts, local, stream, torch)

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        parts.solve()
    torch.cuda.synchronize(dev)
    barrier()
    clocks = Clocks(local)
    clocks.start()
    stats = []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        stats.append(parts.solve())
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    updates = sum(s["updates"] for s in stats)
    ms, updates = aggregate(ms, updates, world, dev)
    value = updates / (ms / 1e3)

    K, ndo = (w.legendre_order + 1) ** 2, w.n_dirs // 8
    peaks, which = measured_peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    ms_rank = ev0.elapsed_time(ev1)

    # the ranks' per-source results gathered to rank 0 on the host (untimed; no device collective)
    gathered = None
    if world > 1:
        mine = shard.partition(args.sources * world, world, rank)
        local_res = {k: float(parts.fluence(i, dts.TOTAL).sum()) for i, k in enumerate(mine)}
        res = shard.gather_to_root(local_res, world, rank)
        gathered = len(res) if res is not None else None

    extra = {}
    if rank == 0 and fp32 and not args.no_fp64:
        extra = fp64_plain(w, parts, dts, local, stream, tol=1e-8)
    if rank == 0 and fp32 and tc and not args.no_compare:
        extra["cuda_core_fp32"] = cuda_core_form(w, tol, args, dts, local, stream)
    split = [len(r) for r in parts.runs]
    parts.close()
    # The dominant kernel's own launch times. With several parts the parts' sweeps and moment
    # kernels overlap, so a part's CUDA-event sweep time is shared with other kernels; the sweep's
    # rate is taken from one more solve of the same sources as one problem (after the timed
    # region; CUDA events around its sweep graphs on its stream), and the sweep's instruction
    # rate over the timed steps is reported beside it.
    if len(split) > 1:
        # host loop: its CUDA events time the sweep and moment graphs apart
        solo = Parts(w, prec, tol, args, dts, local, stream, torch, split=1, loop="host")
        solo.solve()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        solo_st = solo.solve()
        torch.cuda.synchronize(dev)
        solo_ms = (time.perf_counter() - t0) * 1e3
        solo.close()
    elif args.loop == "host":
        solo_st, solo_ms = stats[-1], ms_rank / args.steps
    else:   # the device-resident loop times no phases: one more solve with the host loop
        solo = Parts(w, prec, tol, args, dts, local, stream, torch, split=1, loop="host")
        solo.solve()
        torch.cuda.synchronize(dev)
        solo_st = solo.solve()
        solo_ms = solo_st["solve_ms"]
        solo.close()
    roof = roofline([solo_st], solo_st["solve_ms"], 1, K, ndo, tc, peaks, which, n_sm)
    if len(split) == 1 and args.loop == "host":
        roof["measured_on"] = "the timed steps"
    else:
        roof["measured_on"] = (f"one untimed solve of the same {w.batch} sources as one problem with the "
                               f"host-driven loop ({solo_ms:.0f} ms; the timed steps run {len(split)} "
                               f"part(s) with the {args.loop} loop)")
    if roof.get("inst_per_update"):
        over = roof["inst_per_update"] * sum(s["updates"] for s in stats) / (ms_rank / 1e3) / 1e9
        roof["achieved_over_timed_steps"] = over
        roof["frac_over_timed_steps"] = over / roof["peak"]
    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(w, prec, tol, args, dts, local, stream, torch, world, dev)
    cpu = None
    if rank == 0 and not args.no_cpu:
        threads = oracle_threads()
        v1, dt1 = cpu_sample(w, 1)
        vn, dtn = cpu_sample(w, threads)
        cpu = {"value": vn, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{w.name}: source 0, group 0, one source iteration "
                         f"({w.n_voxels * w.n_dirs:.3e} updates; {dtn:.1f} s on {threads} threads, "
                         f"{dt1:.1f} s on 1)",
               "single_thread": v1, **cpu_info()}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if fp32 else "f64",
            "data": "synthetic",
            "config": {"workload": w.name, "voxels": [w.nx, w.ny, w.nz], "groups": w.n_groups,
                       "directions": w.n_dirs, "legendre_order": w.legendre_order,
                       "sources_per_gpu": w.batch, "tol": tol,
                       "precision": {dts.PREC_FP32: "fp32 sweep and contraction (CUDA cores), fp64 accumulation",
                                     dts.PREC_FP32_SPLITBF16: "fp32 sweep, split-bf16 tensor-core contractions "
                                                              "(fp32 accumulate), fp64 accumulation",
                                     dts.PREC_FP32_TF32: "fp32 sweep, split-tf32 tensor-core scatter-source "
                                                         "contraction, fp64 accumulation",
                                     dts.PREC_FP64: "fp64"}[prec],
                       "tile": [stats[0]["tile_x"], stats[0]["tile_y"], stats[0]["tile_z"]],
                       "tile_choice": "dts_tune_tile" if tuned else "given",
                       "split": split,
                       "parallelism": f"x{world}: one ring of {args.sources * world} source positions "
                                      f"partitioned over the GPUs, no data-path collective",
                       "l2": "inputs larger than L2 (device state of tens of GB per step)"},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(sum(s["launches"] for s in stats)),
            "clocks": clk,
            "solve": {"sweeps_per_step": stats[0]["sweeps"], "updates_per_step": stats[0]["updates"],
                      "max_residual": stats[-1]["max_residual"], "converged": stats[-1]["converged"],
                      "loop": args.loop,
                      # the device-resident loop has no per-phase events (its stats carry 0)
                      "sweep_ms_per_step": (sum(s["sweep_ms"] for s in stats) / args.steps
                                            if args.loop == "host" else None),
                      "reduce_ms_per_step": (sum(s["reduce_ms"] for s in stats) / args.steps
                                             if args.loop == "host" else None)},
        }
        if gathered is not None:
            line["gathered_sources"] = gathered
        line.update(extra)
        if extra.get("fp64_plain"):
            line["fp32_batched_over_fp64_plain"] = value / extra["fp64_plain"]["value"]
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def cuda_core_form(w, tol, args, dts, dev, stream):
    """The same batch solved once (after a warm-up) in the CUDA-core FP32 form,
    for the comparison with the tensor-core form: updates/s and the relative L2
    difference of source 0's total fluence."""
    import copy
    import torch
    tile, _ = dts.tune_tile(w, precision=dts.PREC_FP32, device=dev)
    a = copy.copy(args)
    a.tile = ",".join(str(x) for x in tile)
    q = Parts(w, dts.PREC_FP32, tol, a, dts, dev, stream, torch)
    q.solve()
    torch.cuda.synchronize(dev)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    st = q.solve()
    t1.record(stream)
    torch.cuda.synchronize(dev)
    ms = t0.elapsed_time(t1)
    out = {"value": st["updates"] / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "tile": list(tile),
           "split": [len(r) for r in q.runs], "sweep_ms": st["sweep_ms"], "reduce_ms": st["reduce_ms"]}
    q.close()
    return out


def fp64_plain(w, p32, dts, dev, stream, tol):
    """FP64 plain GPU form on source 0 of the same workload; returns its
    updates/s and the FP32-batched error against it (relative L2 of the total
    scalar fluence over all groups)."""
    import torch
    from paper_1910_11335_b300 import inputs  # noqa: F401
    tile, _ = dts.tune_tile(w, precision=dts.PREC_FP64, batch=1, device=dev)
    q = dts.problem_from_workload(w, precision=dts.PREC_FP64, tol=tol, max_iters=1000, tile=tile,
                                  device=dev, stream=stream.cuda_stream, sources=[0])
    q.solve(allow_not_converged=True)
    torch.cuda.synchronize(dev)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    st = q.solve(allow_not_converged=True)
    t1.record(stream)
    torch.cuda.synchronize(dev)
    ms = t0.elapsed_time(t1)
    a = p32.fluence(0, dts.TOTAL)   # source 0 of the FP32 batch
    b = q.fluence(0, dts.TOTAL)
    err = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    errs_g = [float(np.linalg.norm(a[g] - b[g]) / np.linalg.norm(b[g])) for g in range(w.n_groups)]
    K, ndo = (w.legendre_order + 1) ** 2, w.n_dirs // 8
    v = st.updates / (ms / 1e3)
    q.close()
    return {"fp64_plain": {"value": v, "unit": UNIT, "sources": 1, "converged": st.converged,
                           "tile": list(tile),
                           "sweeps": st.sweeps, "ms": ms,
                           # the method's algorithmic bytes in FP64: (2K+1) 8 / N_d per update
                           "sweep_achieved_gbs_algorithmic": st.updates * (2 * K + 1) * 8.0 / (8 * ndo) / 1e9
                           / (st.sweep_ms / 1e3)},
            "fp32_batched_over_fp64_plain": None,
            "rel_l2_fp32_vs_fp64": err, "rel_l2_fp32_vs_fp64_max_group": max(errs_g)}


def end_to_end(w, prec, tol, args, dts, dev, stream, torch, world=1, device=None):
    """Same metric through the C ABI with HOST buffers: every step uploads the
    materials and sources from pinned host memory and solves; the total scalar
    fluence of every source lands in pinned host memory during the solve, each
    group's as soon as the group is done (dts_set_host_output), and the solve
    returns when the last group's copy has landed."""
    steps = max(1, min(args.steps, 2))
    G, V, B = w.n_groups, w.n_voxels, w.batch
    mat = torch.from_numpy(w.mat_id.reshape(-1).astype(np.int32)).pin_memory().numpy()
    st_h = torch.from_numpy(np.ascontiguousarray(w.sigma_t)).pin_memory().numpy()
    ss_h = torch.from_numpy(np.ascontiguousarray(w.sigma_s)).pin_memory().numpy()
    parts = Parts(w, prec, tol, args, dts, dev, stream, torch)

    def host_array(n):   # page-locked when the host allows it (the copies then overlap the solve)
        try:
            return torch.empty(n, dtype=torch.float64).pin_memory().numpy()
        except RuntimeError:
            return np.empty(n)

    outs = [host_array(len(run) * G * V) for run in parts.runs]
    for p, out in zip(parts.probs, outs):
        p.set_host_output(dts.TOTAL, out)
    parts.solve()
    torch.cuda.synchronize(dev)
    h2d = len(parts.probs) * (mat.nbytes + st_h.nbytes + ss_h.nbytes) + B * (8 * 7 + 8 * G)
    d2h = B * G * V * 8
    updates = 0
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        for p, run in zip(parts.probs, parts.runs):
            p.set_materials(st_h, ss_h, mat)
            for b, k in enumerate(run):
                p.set_source(b, w.sources[k])
        st = parts.solve()
        updates += st["updates"]
    dt = time.perf_counter() - t0
    parts.close()
    # whole job, as for the device-timed value: the slowest rank's time, every rank's updates and bytes
    ms, total = aggregate(dt * 1e3, updates, world, device)
    return {"value": total / (ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d) * world,
            "d2h_bytes_per_step": int(d2h) * world, "steps": steps}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
