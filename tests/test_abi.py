"""The C-ABI library without a GPU: it loads, exports every symbol include/dts.h
declares, and its host-side helpers agree with the oracle's independent
implementations (no device work)."""
import os
import re

import numpy as np
import pytest

from paper_1910_11335_b300 import dts

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1910_11335_b300 import build
    build.build()
    return dts.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "dts.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dts_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(dts.EXPORTS) == names


def test_version_and_status_strings(lib):
    assert lib.dts_version() == 1
    assert lib.dts_status_string(0) == b"DTS_OK"
    assert lib.dts_status_string(5) == b"DTS_ERR_NOT_CONVERGED"


@pytest.mark.parametrize("N", [2, 4, 6, 8])
def test_quadrature_matches_oracle(lib, ora, N):
    a = dts.quadrature(N)
    b = ora.quadrature(N)
    for x, y in zip(a, b):
        assert np.max(np.abs(x - y)) < 1e-14


@pytest.mark.parametrize("N,L", [(2, 0), (4, 1), (6, 2), (8, 3)])
def test_moment_tables_match_oracle(lib, ora, N, L):
    D, M = dts.moment_tables(N, L)
    _, Do, Mo = ora.sh_tables(N, L)
    assert np.max(np.abs(D - Do)) < 1e-14
    assert np.max(np.abs(M - Mo)) < 1e-15


def test_subsweep_size_matches_oracle(lib, ora):
    for dims in [(1, 1, 1), (5, 5, 5), (3, 7, 2), (8, 1, 6), (12, 12, 12)]:
        for S in range(sum(dims) - 2):
            assert dts.subsweep_size(*dims, S) == ora.subsweep_size(*dims, S)
    assert dts.subsweep_size(5, 5, 5, 13) == 0      # beyond the last sub-sweep


def test_invalid_arguments_rejected_on_host(lib):
    with pytest.raises(dts.DTSError) as e:
        dts.quadrature(5)
    assert e.value.status == dts.DTS_ERR_INVALID_ARG
    with pytest.raises(dts.DTSError):
        dts.moment_tables(4, 4)
    # entry points on a problem reject a NULL problem before any device work
    for rc in (lib.dts_set_device_loop(None, 1), lib.dts_debug_poison_wait(None, 1),
               lib.dts_set_iteration_callback(None, dts.IterationFn(), None)):
        assert rc == dts.DTS_ERR_INVALID_ARG


def test_create_without_usable_device_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(dts.DTSError) as e:
        dts.Problem(nx=4, ny=4, nz=4, dx=1.0, dy=1.0, dz=1.0)
    assert e.value.status in (dts.DTS_ERR_CUDA, dts.DTS_ERR_INVALID_ARG)


class _FakeCudaTensor:
    """Just enough of a CUDA tensor for the binding's argument checks (no device needed)."""

    def __init__(self, n, dtype=None):
        import torch
        self.is_cuda = True
        self.dtype = dtype or torch.float64
        self._n = n
        self.device = type("D", (), {"index": 0})()

    def is_contiguous(self):
        return True

    def numel(self):
        return self._n

    def data_ptr(self):   # pragma: no cover - reaching it would be the failure
        raise AssertionError("the binding must reject the call before touching device memory")


def test_noalloc_binding_rejects_short_or_wrong_tensors_before_any_launch():
    import torch
    n, K = 5, 4                                # 5^3 voxels at P1
    V = n ** 3
    good_src, sig = _FakeCudaTensor(K * V), _FakeCudaTensor(V)
    for src, st, phi, what in ((good_src, sig, _FakeCudaTensor(K * V - 1), "phi"),
                               (_FakeCudaTensor(K * V - 1), sig, _FakeCudaTensor(K * V), "src_moments"),
                               (good_src, _FakeCudaTensor(V - 1), _FakeCudaTensor(K * V), "sigma_t"),
                               (good_src, sig, _FakeCudaTensor(K * V, torch.float32), "phi")):
        with pytest.raises(ValueError, match=what):
            dts.sweep_once_noalloc(n, n, n, 1.0, 1.0, 1.0, 4, 1, src, st, phi)
