"""Benchmark of the S_N source-iteration solve (cell-direction-group updates/s).

Default workload: the batched cone-beam form -- 96^3 voxels of 1/3 cm (the
32 cm water-cylinder phantom with bone and air inserts), 19 groups, S8
(80 directions), P3, 32 CT source positions on a 50 cm circle -- solved in FP32
(sweep, contraction and octant partials) with FP64 accumulation, residual and
balance. One step = one full dts_solve of the batch (ray trace, first-collision
source, every group's source iteration to tol, downscatter), inputs already
resident in HBM. The FP64 plain form runs one source of the same workload for
the "FP32-batched vs FP64 plain" comparison and the 1e-4 relative L2 gate.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank solves its own batch of 32 source positions (weak
scaling; no collective on the data path) and rank 0 prints one JSON line.
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
    ap.add_argument("--tol", type=float, default=None)
    ap.add_argument("--max-iters", type=int, default=None)
    ap.add_argument("--tile", default="auto", help="tx,ty,tz or 'auto' (dts_tune_tile)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 plain comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--precision", default="auto", choices=["auto", "fp32", "splitbf16", "tf32"],
                    help="arithmetic of the FP32-batched form's scatter-source contraction")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def make_workload(args, rank=0):
    from paper_1910_11335_b300 import inputs
    if args.workload == "batch96":
        w = inputs.batch_96(args.sources)
        if rank:
            # rank r rotates its ring by r/world of one source spacing
            world = dist_env()[2]
            w.sources = inputs.ring_sources(w.sources[0].spectrum, args.sources)
            rot = 2 * math.pi * rank / (world * args.sources)
            for s in w.sources:
                x, y, z = s.pos
                c, sn = math.cos(rot), math.sin(rot)
                s.pos = (c * x - sn * y, sn * x + c * y, z)
                s.axis = (-s.pos[0] / 50.0, -s.pos[1] / 50.0, 0.0)
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
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "of fallback"


def direct_output(tile, fp32, K, ndo):
    """Whether the library's batched kernel writes angular fluxes (N_d per cell)
    instead of 8 K octant moment partials: FP32 batched tiles with 8 K > N_d."""
    return sweep_kernel_name(tile, fp32) == "k_sweep_batch" and 8 * K > 8 * ndo   # 8 K > N_d


def sweep_bytes_per_update(K, ndo, rsz, psi=False):
    """Algorithmic bytes of the sweep kernel per cell-direction update: per
    (cell, octant) it reads K source moments and sigma_t, shared by the
    octant's ndo directions; it writes K octant moment partials per (cell,
    octant), or in the direct-output form one angular flux per update."""
    if psi:
        return (K + 1) * rsz / ndo + rsz
    return (2 * K + 1) * rsz / ndo


def cpu_sample(w, seconds_hint=True):
    """The oracle, as it stands, on a bounded sample of the workload: source 0,
    group 0, one source iteration (ray trace, first-collision source and one
    full sweep of all directions)."""
    import oracle
    from paper_1910_11335_b300.inputs import first_groups, with_sources
    t = first_groups(with_sources(w, [0]), 1)
    threads = min(8, os.cpu_count() or 1)
    t0 = time.perf_counter()
    oracle.solve(t, 0, tol=0.0, max_iters=1, n_threads=threads)
    dt = time.perf_counter() - t0
    u = t.n_voxels * t.n_dirs
    return u / dt, threads, dt


def run_reference(args):
    rank, local, world = dist_env()
    if rank != 0:
        return
    w = make_workload(args)
    vals = []
    for i in range(args.warmup + args.steps):
        v, threads, dt = cpu_sample(w)
        if i >= args.warmup:
            vals.append(v)
    value = statistics.mean(vals)
    sample = (f"{w.name}: source 0, group 0, 1 source iteration "
              f"({w.n_voxels * w.n_dirs:.3e} updates) per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "ms_per_step": 1e3 * w.n_voxels * w.n_dirs / value, "dtype": "f64",
            "data": "synthetic", "scaling": "weak", "vs_baseline": None,
            "config": {"workload": w.name, "oracle": "plain FP64 C, gcc -O2, OpenMP over octants"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# DRAM bytes of the sweep kernel from one ncu capture at full size
# (profiles/k_sweep_batch_batch96_s8p3.md: dram__bytes_read.sum + dram__bytes_write.sum of three
# mid-sweep launches over their algorithmic bytes). The ratio is only used while the batched kernel's
# source is the one that was profiled; any change to it makes "traffic" null until it is re-measured.
MEASURED_TRAFFIC = {
    ("k_sweep_batch", "batch96_s8p3_19g_x32", (8, 4, 4)): {
        "dram_over_algorithmic": 1.33,
        "source_sha256": "f53287b3d101fe2b58b18602fd4d49ee50f1132d46e9cc1f42b2468f8087e835",
    },
}


def batched_kernel_sha256():
    """Hash of the batched sweep kernel's source block (what the traffic ratio was measured on)."""
    import hashlib
    src = open(os.path.join(ROOT, "paper_1910_11335_b300", "csrc", "dts_kernels.cuh")).read()
    a = src.index("// A3 + A4, batched form (FP32)")
    b = src.index("// Translation units that only launch the sweep define DTS_SWEEP_KERNEL_ONLY so")
    return hashlib.sha256(src[a:b].encode()).hexdigest()


def sweep_kernel_name(tile, fp32):
    """The sweep kernel the library launches for a tile shape."""
    if fp32 and tuple(tile) in ((8, 4, 4), (4, 4, 4)):
        return "k_sweep_batch"
    if tile[1] * tile[2] == 32 and tile[1] in (4, 8):
        return "k_sweep_lines"
    return "k_sweep_stage"


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


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1910_11335_b300 import build, dts
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
    tol = args.tol if args.tol is not None else w.tol
    tuned = None
    if args.tile == "auto":
        tile, tuned = dts.tune_tile(w, precision=prec, device=local)
        args.tile = ",".join(str(x) for x in tile)
    tile = tuple(int(x) for x in args.tile.split(","))
    p = dts.problem_from_workload(w, precision=prec, tol=tol, max_iters=args.max_iters or 1000,
                                  tile=tile, device=local, stream=stream.cuda_stream)

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        p.solve(allow_not_converged=True)
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
        st = p.solve(allow_not_converged=True)
        stats.append(st.as_dict())
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    updates = sum(s["updates"] for s in stats)
    ms, updates = aggregate(ms, updates, world, dev)
    value = updates / (ms / 1e3)

    # roofline of the dominant kernel (the wavefront sweep), timed live by
    # CUDA events recorded around its launches inside the iteration graph
    K, ndo = (w.legendre_order + 1) ** 2, w.n_dirs // 8
    rsz = 4 if fp32 else 8
    sweep_ms = sum(s["sweep_ms"] for s in stats)
    psi = direct_output(tile, fp32, K, ndo)
    bpu = sweep_bytes_per_update(K, ndo, rsz, psi)
    peaks, which = measured_peaks()
    achieved = (sum(s["updates"] for s in stats) * bpu / 1e9) / (sweep_ms / 1e3)
    traffic = None
    kname = sweep_kernel_name(tile, fp32)
    meas = MEASURED_TRAFFIC.get((kname, w.name, tuple(tile)))
    n_launch = sum(s["sweep_launches"] for s in stats)
    if meas and n_launch and batched_kernel_sha256() == meas["source_sha256"]:
        # per launch, like "achieved": the average launch's algorithmic bytes times the measured ratio
        traffic = meas["dram_over_algorithmic"] * bpu * sum(s["updates"] for s in stats) / n_launch
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "kernel": sweep_kernel_name(tile, fp32), "peak_source": which,
                "sweep_share_of_step": sweep_ms / ms if ms else None,
                "bytes_per_update": bpu,
                "sweep_output": "angular fluxes" if psi else "octant moment partials"}

    extra = {}
    if rank == 0 and fp32 and not args.no_fp64:
        extra = fp64_plain(w, p, dts, local, stream, tol=1e-8)
    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(w, prec, tol, args, dts, local, stream, torch)
    cpu = None
    if rank == 0 and not args.no_cpu:
        v, threads, dt = cpu_sample(w)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{w.name}: source 0, group 0, one source iteration "
                         f"({w.n_voxels * w.n_dirs:.3e} updates, {dt:.1f} s)"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if fp32 else "f64",
            "data": "synthetic",
            "config": {"workload": w.name, "voxels": [w.nx, w.ny, w.nz], "groups": w.n_groups,
                       "directions": w.n_dirs, "legendre_order": w.legendre_order,
                       "sources_per_gpu": w.batch, "tol": tol,
                       "precision": "fp32 sweep/contraction, fp64 accumulation" if fp32 else "fp64",
                       "tile": [stats[0]["tile_x"], stats[0]["tile_y"], stats[0]["tile_z"]],
                       "tile_choice": "dts_tune_tile" if tuned else "given",
                       "parallelism": f"weak x{world}, independent source batches",
                       "l2": "inputs larger than L2 (device state of tens of GB per step)"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(sum(s["launches"] for s in stats)),
            "clocks": clk,
            "solve": {"sweeps_per_step": stats[0]["sweeps"], "updates_per_step": stats[0]["updates"],
                      "max_residual": stats[-1]["max_residual"], "converged": stats[-1]["converged"],
                      "sweep_ms_per_step": sweep_ms / args.steps,
                      "reduce_ms_per_step": sum(s["reduce_ms"] for s in stats) / args.steps},
        }
        line.update(extra)
        if extra.get("fp64_plain"):
            line["fp32_batched_over_fp64_plain"] = value / extra["fp64_plain"]["value"]
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


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
    a = p32.fluence(0, dts.TOTAL)
    b = q.fluence(0, dts.TOTAL)
    err = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    errs_g = [float(np.linalg.norm(a[g] - b[g]) / np.linalg.norm(b[g])) for g in range(w.n_groups)]
    K, ndo = (w.legendre_order + 1) ** 2, w.n_dirs // 8
    v = st.updates / (ms / 1e3)
    q.close()
    return {"fp64_plain": {"value": v, "unit": UNIT, "sources": 1, "converged": st.converged,
                           "tile": list(tile),
                           "sweeps": st.sweeps, "ms": ms,
                           "sweep_achieved_gbs": st.updates * sweep_bytes_per_update(K, ndo, 8) / 1e9
                           / (st.sweep_ms / 1e3)},
            "fp32_batched_over_fp64_plain": None,
            "rel_l2_fp32_vs_fp64": err, "rel_l2_fp32_vs_fp64_max_group": max(errs_g)}


def end_to_end(w, prec, tol, args, dts, dev, stream, torch):
    """Same metric through the C ABI with HOST buffers: every step uploads the
    materials and sources from pinned host memory, solves, and reads the total
    scalar fluence of every source back into pinned host memory."""
    steps = max(1, min(args.steps, 2))
    G, V, B = w.n_groups, w.n_voxels, w.batch
    mat = torch.from_numpy(w.mat_id.reshape(-1).astype(np.int32)).pin_memory().numpy()
    st_h = torch.from_numpy(np.ascontiguousarray(w.sigma_t)).pin_memory().numpy()
    ss_h = torch.from_numpy(np.ascontiguousarray(w.sigma_s)).pin_memory().numpy()
    out = torch.empty(G * V, dtype=torch.float64).pin_memory().numpy()
    tile = tuple(int(x) for x in args.tile.split(","))
    p = dts.problem_from_workload(w, precision=prec, tol=tol, max_iters=args.max_iters or 1000,
                                  tile=tile, device=dev, stream=stream.cuda_stream)
    p.solve(allow_not_converged=True)
    torch.cuda.synchronize(dev)
    h2d = mat.nbytes + st_h.nbytes + ss_h.nbytes + B * (8 * 7 + 8 * G)
    d2h = B * G * V * 8
    updates = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        p.set_materials(st_h, ss_h, mat)
        for b, s in enumerate(w.sources):
            p.set_source(b, s)
        st = p.solve(allow_not_converged=True)
        updates += st.updates
        for b in range(B):
            p.fluence(b, dts.TOTAL, out=out)
    dt = time.perf_counter() - t0
    p.close()
    return {"value": updates / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": steps}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
