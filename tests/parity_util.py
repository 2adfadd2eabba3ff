"""Helpers shared by the GPU parity tests (metrics and workload edits)."""
from __future__ import annotations

import numpy as np

#: FP64 path vs FP64 oracle, normalised max error per group at equal iteration counts
TOL_FP64 = 1e-10
#: reduced-precision forms vs FP64 oracle, relative L2 of the scalar fluence
TOL_FP32_L2 = 1e-4


def rel_max(a, b):
    """max |a - b| / max |b| (per-group normalised maximum error)."""
    a, b = np.asarray(a), np.asarray(b)
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / den) if den > 0 else float(np.max(np.abs(a)))


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / den) if den > 0 else float(np.linalg.norm(a))


from paper_1910_11335_b300.inputs import first_groups, with_sources  # noqa: E402,F401
