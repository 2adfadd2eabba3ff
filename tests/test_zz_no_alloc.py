"""dts_sweep_once_noalloc, the entry point for callers that cannot allocate
device memory (a fixed caller-managed pool, or a host that forbids further
cudaMalloc/cudaFree), checked against the solver's ordinary entry point.

One source iteration of a one-group problem with a volumetric source is
exactly one sweep of T = (q, 0, ..., 0): dts_solve with max_iters = 1 and
keep_moments gives its moments, and the no-allocation call must give the same.
Several calls run back to back, so contents left in the shared scratch array
by one call must not leak into the next. This file is collected last.
"""
import numpy as np
import pytest

from paper_1910_11335_b300 import dts, inputs
from parity_util import TOL_FP64, rel_max

pytestmark = pytest.mark.gpu


def _solver_moments(w):
    p = dts.problem_from_workload(w, tol=0.0, max_iters=1, keep_moments=True)
    p.solve()
    m = p.moments(0, 0)
    p.close()
    return m


def _noalloc_moments(w):
    import torch
    K, V = (w.legendre_order + 1) ** 2, w.n_voxels
    src = torch.zeros((K, V), dtype=torch.float64, device="cuda")
    src[0] = torch.from_numpy(w.sources[0].q[0]).cuda()
    sig = torch.from_numpy(np.ascontiguousarray(w.sigma_t[w.mat_id.reshape(-1), 0])).cuda()
    phi = torch.full((K, V), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    dts.sweep_once_noalloc(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.sn_order, w.legendre_order,
                           src, sig, phi, stream.cuda_stream)
    stream.synchronize()
    return phi.cpu().numpy()


def test_noalloc_sweep_matches_solver_on_calls_in_a_row():
    a = inputs.random_volumetric(13, 9, 7, n_groups=1, sn_order=8, legendre_order=3,
                                 seed_index=1301, thin=False)
    b = inputs.random_volumetric(6, 11, 5, n_groups=1, sn_order=4, legendre_order=1,
                                 seed_index=1302, thin=False)
    for w in (a, a, b, a):   # a repeated shape reuses the tables; a new shape uploads its own
        ref = _solver_moments(w)
        got = _noalloc_moments(w)
        assert np.all(np.isfinite(got))
        for k in range(ref.shape[0]):
            assert rel_max(got[k], ref[k]) <= TOL_FP64, (w.name, k)


def test_noalloc_rejects_grids_beyond_the_scratch_size():
    import torch
    n = 64                                     # 64^3 voxels at P3 need ~300 MB of scratch
    t = torch.zeros(16 * n ** 3, dtype=torch.float64, device="cuda")
    s = torch.ones(n ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(dts.DTSError) as e:
        dts.sweep_once_noalloc(n, n, n, 1.0, 1.0, 1.0, 8, 3, t, s, t)
    assert e.value.status == dts.DTS_ERR_INVALID_ARG
    assert "scratch" in str(e.value)
