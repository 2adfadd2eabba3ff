"""Write the full-size, converged oracle references of the parity tests.

    python tests/golden/make_fullsize.py [hetero64] [precision128] [batch96]

Calls only the FP64 CPU oracle (oracle/) and the seeded input generators; no
value here comes from the CUDA path. At these sizes the oracle runs for tens of
minutes per configuration, far longer than a GPU test may take, so each run is
stored once as a compact reference: for every solved (source, group)

  - the total and collided scalar fluence at a fixed seeded sample of voxels,
  - the full-field sum, sum of squares and maximum of both,
  - the oracle's iteration count and final residual.

The GPU tests (tests/test_gpu_fullsize.py) compare the library's converged
fluence with these: the per-group maximum error over the samples normalised by
the full-field maximum, the relative L2 error over the samples, and the
full-field sums.

Runs (source iteration to the stated tolerance, all threads the oracle uses):
  hetero64     64^3 S8 P3, 19 groups, one source, tol 1e-12
  precision128 128^3 S8 P3, groups 0..4 of 19, one source, tol 1e-10
               (downscatter only: the first groups are exact without the rest)
  batch96      96^3 S8 P3, source 0 with all 19 groups and sources 8, 16, 24
               with groups 0..5, tol 1e-10
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1910_11335_b300 import inputs  # noqa: E402

N_SAMPLES = 4096
SAMPLE_SEED = 1910_11335


def sample_voxels(n_voxels: int) -> np.ndarray:
    rng = np.random.default_rng(SAMPLE_SEED)
    return np.sort(rng.choice(n_voxels, size=N_SAMPLES, replace=False)).astype(np.int64)


def reference(w, source, n_groups, tol, threads):
    """One oracle solve of `source` over the first n_groups groups."""
    sub = inputs.first_groups(inputs.with_sources(w, [source]), n_groups)
    t0 = time.perf_counter()
    r = oracle.solve(sub, 0, tol=tol, max_iters=5000, n_threads=threads)
    dt = time.perf_counter() - t0
    idx = sample_voxels(w.n_voxels)
    col, tot = r.collided, r.total
    out = {
        "idx": idx,
        "collided_samples": col[:, idx].copy(),
        "total_samples": tot[:, idx].copy(),
        "collided_sum": col.sum(axis=1), "collided_sumsq": (col * col).sum(axis=1),
        "collided_max": np.abs(col).max(axis=1),
        "total_sum": tot.sum(axis=1), "total_sumsq": (tot * tot).sum(axis=1),
        "total_max": np.abs(tot).max(axis=1),
        "iters": r.iters.copy(), "resid": r.resid.copy(),
        "tol": np.float64(tol), "source": np.int64(source), "n_groups": np.int64(n_groups),
        "oracle_seconds": np.float64(dt), "threads": np.int64(threads),
    }
    return out


def write(name, runs):
    path = os.path.join(HERE, f"fullsize_{name}.npz")
    flat = {}
    for i, run in enumerate(runs):
        for k, v in run.items():
            flat[f"r{i}_{k}"] = v
    flat["n_runs"] = np.int64(len(runs))
    np.savez_compressed(path, **flat)
    print(f"wrote {path}", flush=True)


def main(argv):
    which = argv or ["hetero64", "precision128", "batch96"]
    threads = min(8, os.cpu_count() or 1)
    oracle.build()
    if "hetero64" in which:
        w = inputs.hetero_64()
        write("hetero64", [reference(w, 0, w.n_groups, 1e-12, threads)])
    if "precision128" in which:
        w = inputs.precision_128()
        write("precision128", [reference(w, 0, 5, 1e-10, threads)])
    if "batch96" in which:
        w = inputs.batch_96()
        runs = [reference(w, 0, w.n_groups, 1e-10, threads)]
        for s in (8, 16, 24):
            runs.append(reference(w, s, 6, 1e-10, threads))
        write("batch96", runs)


if __name__ == "__main__":
    main(sys.argv[1:])
