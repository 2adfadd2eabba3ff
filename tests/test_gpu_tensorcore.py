"""Parity of the tensor-core forms (DTS_PREC_FP32_SPLITBF16, DTS_PREC_FP32_TF32)
with the FP64 CPU oracle, through the C ABI.

In these forms the scatter-source contraction of Eq. 2, Q_n = sum_k M[n][k] T_k,
runs on the tensor cores (tcgen05) once per source iteration and the sweep reads
the materialised Q; the gate is the reduced-precision one: relative L2 error of
the scalar fluence (and of every Legendre moment) <= 1e-4 per group.
"""
import numpy as np
import pytest

from paper_1910_11335_b300 import dts, inputs
from parity_util import TOL_FP32_L2, rel_l2, rel_max

pytestmark = pytest.mark.gpu

TC = [dts.PREC_FP32_SPLITBF16, dts.PREC_FP32_TF32]
TC_IDS = ["splitbf16", "tf32"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1910_11335_b300 import build
    build.build()


CASES = [
    # dims,       N, L, G, batch   ragged 8x4x4 tiles in every axis
    ((13, 11, 9), 8, 3, 3, 4),     # S8 P3: 80 directions (N = 80), 16 moments
    ((10, 9, 17), 6, 1, 2, 7),     # S6 P1: 48 directions, 4 moments padded to 16
    ((9, 14, 6), 4, 2, 2, 11),     # S4 P2: 24 directions padded to 32, 9 moments
    ((7, 6, 9), 2, 0, 2, 33),      # S2 P0: 8 directions padded to 16, one moment
]


@pytest.mark.parametrize("prec", TC, ids=TC_IDS)
@pytest.mark.parametrize("dims,N,L,G,B", CASES)
def test_tensorcore_moments_vs_oracle(ora, prec, dims, N, L, G, B):
    w = inputs.small_cone(*dims, n_groups=G, sn_order=N, legendre_order=L, n_sources=B)
    p = dts.problem_from_workload(w, precision=prec, tol=0.0, max_iters=5, keep_moments=True)
    st = p.solve(allow_not_converged=True)
    assert (st.tile_x, st.tile_y, st.tile_z) == (8, 4, 4)
    assert st.sweeps == B * G * 5
    for b in sorted({0, B // 2, B - 1}):
        r = ora.solve(w, b, tol=0.0, max_iters=5, n_threads=8)
        assert rel_max(p.fluence(b, dts.UNCOLLIDED), r.phi_u) <= 1e-12
        for g in range(G):
            m = p.moments(b, g)
            assert rel_l2(m[0], r.collided[g]) <= TOL_FP32_L2, (b, g)
            assert rel_l2(m, r.phi_c[g]) <= TOL_FP32_L2, (b, g)
    bal = p.balance()
    for b in range(B):
        for g in range(G):
            assert abs(bal[b, g, 0] - bal[b, g, 1] - bal[b, g, 2]) <= 1e-5 * bal[b, g, 0]


@pytest.mark.parametrize("prec", TC, ids=TC_IDS)
def test_tensorcore_converged_vs_oracle(ora, prec):
    w = inputs.small_cone(16, 16, 16, n_groups=4, sn_order=8, legendre_order=3, n_sources=2)
    p = dts.problem_from_workload(w, precision=prec, tol=1e-6, max_iters=500)
    st = p.solve()
    assert st.converged == 1
    for b in range(2):
        r = ora.solve(w, b, tol=1e-11, max_iters=500, n_threads=8)
        tot, col = p.fluence(b, dts.TOTAL), p.fluence(b, dts.COLLIDED)
        for g in range(4):
            assert rel_l2(col[g], r.collided[g]) <= TOL_FP32_L2, (b, g)
            assert rel_l2(tot[g], r.total[g]) <= TOL_FP32_L2, (b, g)
        assert rel_l2(col, r.collided) <= TOL_FP32_L2


@pytest.mark.parametrize("prec", TC, ids=TC_IDS)
def test_tensorcore_sources_converging_at_different_counts(ora, prec):
    w = inputs.small_cone(16, 15, 14, n_groups=3, sn_order=8, legendre_order=3, n_sources=8)
    rng = np.random.default_rng(4)
    mat = w.mat_id.reshape(-1)
    for b, m in zip(range(4, 8), (0, 1, 2, 1)):
        q = np.zeros((3, w.n_voxels))
        idx = np.flatnonzero(mat == m)
        q[:, rng.choice(idx, min(20, idx.size), replace=False)] = 1.0
        w.sources[b] = inputs.Source(kind=0, q=q)
    p = dts.problem_from_workload(w, precision=prec, tol=1e-6, max_iters=500)
    p.solve()
    its = p.iterations()
    assert len(set(its[:, 0])) > 1      # inactive members' items are skipped by the moment kernel
    for b in (0, 3, 4, 7):
        r = ora.solve(w, b, tol=1e-11, max_iters=500, n_threads=8)
        tot = p.fluence(b, dts.TOTAL)
        for g in range(3):
            assert rel_l2(tot[g], r.total[g]) <= TOL_FP32_L2, (b, g)


@pytest.mark.parametrize("prec", TC, ids=TC_IDS)
def test_tensorcore_matches_cuda_core_form(prec):
    """The tensor-core contraction changes only the rounding of Q: the scalar
    fluence stays within the reduced-precision gate of the CUDA-core FP32 form."""
    w = inputs.small_cone(12, 13, 11, n_groups=3, sn_order=8, legendre_order=3, n_sources=3)
    a = dts.problem_from_workload(w, precision=prec, tol=0.0, max_iters=6)
    a.solve(allow_not_converged=True)
    c = dts.problem_from_workload(w, precision=dts.PREC_FP32, tol=0.0, max_iters=6, tile=(8, 4, 4))
    c.solve(allow_not_converged=True)
    for b in range(3):
        assert rel_l2(a.fluence(b, dts.COLLIDED), c.fluence(b, dts.COLLIDED)) <= TOL_FP32_L2


def test_tensorcore_forms_need_the_8x4x4_tile():
    for prec in TC:
        with pytest.raises(dts.DTSError) as e:
            dts.Problem(nx=8, ny=8, nz=8, dx=1, dy=1, dz=1, sn_order=8, legendre_order=3,
                        precision=prec, tile=(8, 4, 8))
        assert e.value.status == dts.DTS_ERR_INVALID_ARG
