"""Parity of the CUDA solver (through the C ABI) with the FP64 CPU oracle on
the same seeded inputs.

FP64 form: normalised max error <= 1e-10 per group at equal iteration counts.
FP32 form: relative L2 error <= 1e-4 per group against the converged oracle.
"""
import math

import numpy as np
import pytest

from paper_1910_11335_b300 import dts, inputs
from parity_util import TOL_FP32_L2, TOL_FP64, first_groups, rel_l2, rel_max, with_sources

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1910_11335_b300 import build
    build.build()


def _gpu(w, **kw):
    p = dts.problem_from_workload(w, **kw)
    st = p.solve(allow_not_converged=True)
    return p, st


# --------------------------------------------------------------------------- #
def test_plain16_fp64_converged(ora):
    w = inputs.plain_16()
    r = ora.solve(w, n_threads=8)
    p, st = _gpu(w)
    assert st.converged == 1
    assert p.iterations()[0, 0] == r.iters[0]
    assert rel_max(p.fluence(0, dts.COLLIDED)[0], r.collided[0]) <= TOL_FP64
    assert np.all(p.fluence(0, dts.UNCOLLIDED) == 0.0)
    assert st.updates == r.iters[0] * w.n_voxels * 24


CASES = [
    # dims,        N, L, G, tile,      batch
    ((13, 11, 9), 4, 1, 3, (8, 8, 8), 1),
    ((10, 9, 8), 8, 3, 3, (4, 4, 4), 2),
    ((7, 12, 5), 6, 2, 2, (3, 5, 2), 1),
    ((9, 9, 9), 2, 0, 2, (1, 1, 1), 1),
    ((17, 6, 11), 8, 1, 2, (8, 4, 8), 3),
    # warp-synchronous line kernel (32 x-lines per tile): both line layouts,
    # odd and long x extents, ragged tails in every axis
    ((13, 11, 9), 8, 3, 3, (8, 4, 8), 2),
    ((10, 9, 17), 6, 2, 2, (5, 8, 4), 1),
    ((21, 7, 6), 4, 1, 2, (16, 4, 8), 1),
    ((6, 5, 9), 2, 0, 2, (3, 4, 8), 1),
    ((40, 12, 10), 8, 3, 2, (32, 8, 4), 1),
]


@pytest.mark.parametrize("dims,N,L,G,tile,B", CASES)
def test_cone_fp64_moments(ora, dims, N, L, G, tile, B):
    w = inputs.small_cone(*dims, n_groups=G, sn_order=N, legendre_order=L, n_sources=B)
    iters = 5
    p, st = _gpu(w, tol=0.0, max_iters=iters, tile=tile, keep_moments=True)
    assert (st.tile_x, st.tile_y, st.tile_z) == tile
    assert np.all(p.iterations() == iters)
    for b in range(B):
        r = ora.solve(w, b, tol=0.0, max_iters=iters, n_threads=8)
        assert rel_max(p.fluence(b, dts.UNCOLLIDED), r.phi_u) <= 1e-13
        for g in range(G):
            m = p.moments(b, g)
            for k in range(m.shape[0]):
                assert rel_max(m[k], r.phi_c[g, k]) <= TOL_FP64, (b, g, k)


def test_volumetric_thick_fp64_with_fixup(ora):
    w = inputs.random_volumetric(11, 7, 5, n_groups=3, sn_order=4, legendre_order=1,
                                 seed_index=77, thin=False)
    r = ora.solve(w, tol=0.0, max_iters=30, n_threads=8)
    assert np.all(r.fixups > 0)
    p, st = _gpu(w, tol=0.0, max_iters=30, tile=(4, 4, 4))
    col = p.fluence(0, dts.COLLIDED)
    for g in range(3):
        assert rel_max(col[g], r.collided[g]) <= TOL_FP64
    # particle balance of the last sweep: source = absorption + leakage
    bal = p.balance()[0]
    for g in range(3):
        assert abs(bal[g, 0] - bal[g, 1] - bal[g, 2]) <= 1e-12 * bal[g, 0]
        assert abs(bal[g, 2] - r.leak[g]) <= 1e-10 * r.leak[g]


def test_converged_iteration_counts_match(ora):
    w = inputs.small_cone(12, 10, 14, n_groups=3, sn_order=6, legendre_order=1, tol=1e-9)
    r = ora.solve(w, n_threads=8)
    p, st = _gpu(w)
    assert st.converged == 1
    assert np.array_equal(p.iterations()[0], r.iters)
    tot = p.fluence(0, dts.TOTAL)
    for g in range(3):
        assert rel_max(tot[g], r.total[g]) <= TOL_FP64


def test_fp32_form_relative_l2(ora):
    w = inputs.small_cone(16, 16, 16, n_groups=4, sn_order=8, legendre_order=3, n_sources=2)
    p, st = _gpu(w, precision=dts.PREC_FP32, tol=1e-6, max_iters=500)
    for b in range(2):
        r = ora.solve(w, b, tol=1e-11, max_iters=500, n_threads=8)
        col = p.fluence(b, dts.COLLIDED)
        tot = p.fluence(b, dts.TOTAL)
        for g in range(4):
            assert rel_l2(col[g], r.collided[g]) <= TOL_FP32_L2, (b, g)
            assert rel_l2(tot[g], r.total[g]) <= TOL_FP32_L2
        assert rel_l2(col, r.collided) <= TOL_FP32_L2


BATCH_CASES = [
    # dims,       N, L, G, batch  (FP32, 8x4x4 tiles: lanes = source x direction pairs)
    ((13, 11, 9), 8, 3, 3, 4),     # 3 sources x 10 directions per warp, ragged group
    ((10, 9, 17), 6, 1, 2, 7),     # 5 x 6
    ((9, 14, 6), 4, 2, 2, 11),     # 10 x 3
    ((7, 6, 9), 2, 0, 2, 33),      # 32 x 1
]


@pytest.mark.parametrize("dims,N,L,G,B", BATCH_CASES)
def test_batched_fp32_kernel(ora, dims, N, L, G, B):
    w = inputs.small_cone(*dims, n_groups=G, sn_order=N, legendre_order=L, n_sources=B)
    p, st = _gpu(w, precision=dts.PREC_FP32, tol=0.0, max_iters=5, tile=(8, 4, 4))
    assert (st.tile_x, st.tile_y, st.tile_z) == (8, 4, 4)
    for b in sorted({0, B // 2, B - 1}):
        r = ora.solve(w, b, tol=0.0, max_iters=5, n_threads=8)
        col = p.fluence(b, dts.COLLIDED)
        for g in range(G):
            assert rel_l2(col[g], r.collided[g]) <= TOL_FP32_L2, (b, g)
    bal = p.balance()
    for b in range(B):
        for g in range(G):
            assert abs(bal[b, g, 0] - bal[b, g, 1] - bal[b, g, 2]) <= 1e-5 * bal[b, g, 0]


@pytest.mark.parametrize("tile", [(8, 4, 4), (4, 4, 4)])
def test_batched_direct_output_moments(ora, tile):
    """S8 P3 batches take the direct angular-flux output of the batched kernel
    (N_d = 80 fluxes per cell instead of 8 x 16 octant partials); every Legendre
    moment, not only the scalar flux, is formed from them and pushed into the
    lower groups."""
    w = inputs.small_cone(11, 9, 10, n_groups=3, sn_order=8, legendre_order=3, n_sources=5)
    p, st = _gpu(w, precision=dts.PREC_FP32, tol=0.0, max_iters=4, tile=tile, keep_moments=True)
    assert (st.tile_x, st.tile_y, st.tile_z) == tile
    for b in (0, 4):
        r = ora.solve(w, b, tol=0.0, max_iters=4, n_threads=8)
        for g in range(w.n_groups):
            m = p.moments(b, g)
            assert rel_l2(m, r.phi_c[g]) <= TOL_FP32_L2, (b, g)
            assert rel_l2(m[0], r.collided[g]) <= TOL_FP32_L2, (b, g)


def test_batched_fp32_sources_converging_at_different_counts(ora):
    w = inputs.small_cone(16, 15, 14, n_groups=3, sn_order=8, legendre_order=3, n_sources=8)
    # members 4..7: volumetric sources in air, water and bone regions, which
    # converge at other iteration counts than the cone beams
    rng = np.random.default_rng(4)
    mat = w.mat_id.reshape(-1)
    for b, m in zip(range(4, 8), (0, 1, 2, 1)):
        q = np.zeros((3, w.n_voxels))
        idx = np.flatnonzero(mat == m)
        q[:, rng.choice(idx, min(20, idx.size), replace=False)] = 1.0
        w.sources[b] = inputs.Source(kind=0, q=q)
    p, st = _gpu(w, precision=dts.PREC_FP32, tol=1e-6, max_iters=500, tile=(8, 4, 4))
    assert (st.tile_x, st.tile_y, st.tile_z) == (8, 4, 4)
    its = p.iterations()
    assert len(set(its[:, 0])) > 1          # the batch members stop at different iterations
    for b in (0, 3, 4, 5, 6, 7):
        r = ora.solve(w, b, tol=1e-11, max_iters=500, n_threads=8)
        tot = p.fluence(b, dts.TOTAL)
        for g in range(3):
            assert rel_l2(tot[g], r.total[g]) <= TOL_FP32_L2, (b, g)


def test_fp64_is_deterministic():
    w = inputs.small_cone(10, 9, 8, n_groups=2, sn_order=8, legendre_order=3)
    a, _ = _gpu(w, tol=0.0, max_iters=4)
    b, _ = _gpu(w, tol=0.0, max_iters=4)
    assert np.array_equal(a.fluence(0, dts.TOTAL), b.fluence(0, dts.TOTAL))


@pytest.mark.parametrize("dims,tile", [((1, 1, 1), (0, 0, 0)), ((1, 7, 1), (0, 0, 0)),
                                       ((2, 1, 3), (2, 2, 2)), ((5, 4, 3), (16, 16, 1))])
def test_degenerate_grids(ora, dims, tile):
    w = inputs.random_volumetric(*dims, n_groups=2, sn_order=4, legendre_order=1,
                                 seed_index=900 + sum(dims), thin=False)
    r = ora.solve(w, tol=0.0, max_iters=6)
    p, _ = _gpu(w, tol=0.0, max_iters=6, tile=tile)
    col = p.fluence(0, dts.COLLIDED)
    for g in range(2):
        assert rel_max(col[g], r.collided[g]) <= TOL_FP64


def test_device_output_into_torch_tensor(ora):
    import torch
    w = inputs.small_cone(9, 8, 7, n_groups=2, sn_order=4, legendre_order=1)
    stream = torch.cuda.current_stream().cuda_stream
    p = dts.problem_from_workload(w, tol=0.0, max_iters=3, stream=stream)
    p.solve()
    out = torch.empty(w.n_groups * w.n_voxels, dtype=torch.float64, device="cuda")
    p.fluence(0, dts.TOTAL, out=out)
    torch.cuda.current_stream().synchronize()
    r = ora.solve(w, tol=0.0, max_iters=3)
    assert rel_max(out.cpu().numpy().reshape(2, -1), r.total) <= TOL_FP64


def test_status_codes():
    w = inputs.small_cone(6, 5, 4, n_groups=2, sn_order=4, legendre_order=1)
    p = dts.Problem(nx=6, ny=5, nz=4, dx=1.0, dy=1.0, dz=1.0, n_groups=2, sn_order=4,
                    legendre_order=1, batch=1)
    with pytest.raises(dts.DTSError) as e:
        p.solve()
    assert e.value.status == dts.DTS_ERR_STATE
    bad = w.sigma_s.copy()
    bad[1, 0, 1, 0] = 0.1                                   # upscatter
    with pytest.raises(dts.DTSError) as e:
        p.set_materials(w.sigma_t, bad, w.mat_id.reshape(-1))
    assert e.value.status == dts.DTS_ERR_INVALID_ARG
    with pytest.raises(dts.DTSError):
        p.set_materials(-w.sigma_t, w.sigma_s, w.mat_id.reshape(-1))
    with pytest.raises(dts.DTSError):
        p.set_materials(w.sigma_t, w.sigma_s, np.full(w.n_voxels, 99, dtype=np.int32))
    p.set_materials(w.sigma_t, w.sigma_s, w.mat_id.reshape(-1))
    with pytest.raises(dts.DTSError) as e:
        p.set_source(1, w.sources[0])
    assert e.value.status == dts.DTS_ERR_INVALID_ARG
    with pytest.raises(dts.DTSError):
        p.set_source(0, inputs.Source(kind=1, pos=(0, -50, 0), axis=(0, 0, 0), half_angle=0.3,
                                      spectrum=np.ones(2)))
    with pytest.raises(dts.DTSError) as e:
        p.fluence(0)
    assert e.value.status == dts.DTS_ERR_STATE
    with pytest.raises(dts.DTSError) as e:
        dts.Problem(nx=8, ny=8, nz=8, dx=1, dy=1, dz=1, sn_order=8, legendre_order=3,
                    tile=(16, 16, 16))
    assert e.value.status == dts.DTS_ERR_INVALID_ARG
    with pytest.raises(dts.DTSError):
        dts.Problem(nx=0, ny=8, nz=8, dx=1, dy=1, dz=1)
    with pytest.raises(dts.DTSError):
        dts.Problem(nx=8, ny=8, nz=8, dx=1, dy=1, dz=1, sn_order=5)
    q = dts.problem_from_workload(w, tol=1e-14, max_iters=2)
    with pytest.raises(dts.DTSError) as e:
        q.solve()
    assert e.value.status == dts.DTS_ERR_NOT_CONVERGED
    st = q.solve(allow_not_converged=True)
    assert st.converged == 0 and st.sweeps == 2 * 2 and q.iterations().max() == 2


# --------------------------------------------------------------------------- #
# full-size workloads in the launch configuration the benchmark uses; the
# oracle reproduces the highest groups exactly (downscatter only)
# --------------------------------------------------------------------------- #
def test_full_size_hetero64_fp64(ora):
    w = inputs.hetero_64()
    p, st = _gpu(w, tol=0.0, max_iters=2)
    r = ora.solve(first_groups(w, 2), tol=0.0, max_iters=2, n_threads=8)
    col = p.fluence(0, dts.COLLIDED)
    for g in range(2):
        assert rel_max(col[g], r.collided[g]) <= TOL_FP64
    unc = p.fluence(0, dts.UNCOLLIDED)
    rng = np.random.default_rng(5)
    for v in rng.integers(0, w.n_voxels, size=64):
        pu, _ = ora.uncollided_voxel(w, w.sources[0], int(v))
        assert np.allclose(unc[:, v], pu, rtol=1e-12, atol=0)


def test_full_size_batch96_fp32(ora):
    w = inputs.batch_96()
    p, st = _gpu(w, precision=dts.PREC_FP32, tol=0.0, max_iters=2)
    assert st.sweeps == 32 * 19 * 2
    for b in (0, 17):
        r = ora.solve(first_groups(with_sources(w, [b]), 2), tol=0.0, max_iters=2, n_threads=8)
        col = p.fluence(b, dts.COLLIDED)
        unc = p.fluence(b, dts.UNCOLLIDED)
        for g in range(2):
            assert rel_l2(col[g], r.collided[g]) <= TOL_FP32_L2, (b, g)
            assert rel_max(unc[g], r.phi_u[g]) <= 1e-12
        rng = np.random.default_rng(b)
        for v in rng.integers(0, w.n_voxels, size=32):
            pu, _ = ora.uncollided_voxel(w, w.sources[b], int(v))
            assert np.allclose(unc[:, v], pu, rtol=1e-12, atol=0)


def test_full_size_precision128_fp32_vs_fp64(ora):
    # the 128^3 reduced-precision configuration at full size, each form converged to its own tolerance:
    # FP32 against the FP64 form on the GPU (which the tests above hold to the oracle), and the
    # uncollided fluence of both against the oracle on sampled voxels
    w = inputs.precision_128()
    p32, st32 = _gpu(w, precision=dts.PREC_FP32, tile=(8, 4, 4))
    assert st32.converged == 1
    p64, st64 = _gpu(w, precision=dts.PREC_FP64, tol=1e-8, tile=(8, 8, 8))
    assert st64.converged == 1
    a, b = p32.fluence(0, dts.TOTAL), p64.fluence(0, dts.TOTAL)
    assert rel_l2(a, b) <= TOL_FP32_L2
    for g in range(w.n_groups):
        assert rel_l2(a[g], b[g]) <= TOL_FP32_L2, g
    u32, u64 = p32.fluence(0, dts.UNCOLLIDED), p64.fluence(0, dts.UNCOLLIDED)
    rng = np.random.default_rng(128)
    for v in rng.integers(0, w.n_voxels, size=24):
        pu, _ = ora.uncollided_voxel(w, w.sources[0], int(v))
        assert np.allclose(u64[:, v], pu, rtol=1e-12, atol=0)
        assert np.allclose(u32[:, v], pu, rtol=1e-12, atol=0)


@pytest.mark.parametrize("tile", [(8, 4, 4), (4, 4, 4)])
def test_batched_fp32_with_density_scales(ora, tile):
    # per-voxel density scales on sigma_t and sigma_s (CT-derived densities): the FP32 forms round
    # sigma_s * scale_s once per (cell, l, group) in the downscatter push and the first-collision source
    import copy
    w = copy.copy(inputs.small_cone(10, 9, 8, n_groups=3, sn_order=8, legendre_order=3, n_sources=3))
    rng = np.random.default_rng(11)
    w.scale_t = rng.uniform(0.6, 1.4, size=w.mat_id.shape)
    w.scale_s = w.scale_t * rng.uniform(0.9, 1.1, size=w.mat_id.shape)
    p = dts.problem_from_workload(w, precision=dts.PREC_FP32, tol=0.0, max_iters=4, tile=tile)
    p.solve(allow_not_converged=True)
    for b in range(3):
        r = ora.solve(w, b, tol=0.0, max_iters=4, n_threads=8)
        assert rel_max(p.fluence(b, dts.UNCOLLIDED), r.phi_u) <= 1e-12
        col = p.fluence(b, dts.COLLIDED)
        for g in range(w.n_groups):
            assert rel_l2(col[g], r.collided[g]) <= TOL_FP32_L2, (b, g)


@pytest.mark.parametrize("prec", [dts.PREC_FP32, dts.PREC_FP32_SPLITBF16], ids=["fp32", "splitbf16"])
def test_fp32_batched_is_reproducible_including_leakage(prec):
    # every (source, octant, tile) sweep writes its own leakage slot, summed per source in a fixed
    # order, so the balance terms -- not only the fluence -- repeat bit for bit
    w = inputs.small_cone(12, 10, 9, n_groups=2, sn_order=8, legendre_order=3, n_sources=4)
    runs = []
    for _ in range(2):
        p = dts.problem_from_workload(w, precision=prec, tol=0.0, max_iters=4, tile=(8, 4, 4))
        p.solve(allow_not_converged=True)
        runs.append((p.fluence(1, dts.TOTAL), p.balance()))
        p.close()
    assert np.array_equal(runs[0][0], runs[1][0])
    assert np.array_equal(runs[0][1], runs[1][1])
    assert np.all(runs[0][1][:, :, 2] > 0.0)      # leakage present in every (source, group)
