"""Python binding of the C ABI in include/dts.h (argument marshalling only).

Every step of the solve runs in libdts.so (CUDA, sm_103a). There is no CPU
fallback: if the library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
from typing import Optional

import numpy as np

from . import inputs

_PKG = os.path.dirname(os.path.abspath(__file__))
#: DTS_DEBUG_BOUNDS=1 in the environment loads the bounds-checked build instead
DEBUG_BOUNDS = os.environ.get("DTS_DEBUG_BOUNDS", "") == "1"
LIB_PATH = os.path.join(_PKG, "libdts_debug.so" if DEBUG_BOUNDS else "libdts.so")

DTS_OK, DTS_ERR_INVALID_ARG, DTS_ERR_STATE, DTS_ERR_OOM, DTS_ERR_CUDA, DTS_ERR_NOT_CONVERGED, \
    DTS_ERR_TIMEOUT, DTS_ERR_INTERNAL = range(8)
PREC_FP64, PREC_FP32, PREC_FP32_SPLITBF16, PREC_FP32_TF32 = 0, 1, 2, 3
UNCOLLIDED, COLLIDED, TOTAL = 0, 1, 2

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class ProblemDesc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double),
                ("n_groups", C.c_int), ("sn_order", C.c_int), ("legendre_order", C.c_int),
                ("batch", C.c_int), ("precision", C.c_int), ("tol", C.c_double),
                ("max_iters", C.c_int), ("cuda_stream", C.c_void_p), ("device", C.c_int),
                ("tile_x", C.c_int), ("tile_y", C.c_int), ("tile_z", C.c_int),
                ("keep_moments", C.c_int)]


class SourceDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("q", _dp), ("pos", C.c_double * 3), ("axis", C.c_double * 3),
                ("half_angle", C.c_double), ("spectrum", _dp), ("aperture", C.c_int),
                ("normal", C.c_double * 3), ("half_azimuth", C.c_double), ("half_polar", C.c_double)]


class SolveStats(C.Structure):
    _fields_ = [("updates", C.c_int64), ("sweeps", C.c_int64), ("max_residual", C.c_double),
                ("solve_ms", C.c_double), ("sweep_ms", C.c_double), ("reduce_ms", C.c_double),
                ("launches", C.c_int64), ("converged", C.c_int),
                ("tile_x", C.c_int), ("tile_y", C.c_int), ("tile_z", C.c_int),
                ("sweep_launches", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


#: dts_iteration_fn: (user, group, iteration, residuals[batch], batch)
IterationFn = C.CFUNCTYPE(None, C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_double), C.c_int)


class DTSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status


_lib = None

#: every function include/dts.h declares
EXPORTS = ("dts_create_problem", "dts_set_materials", "dts_set_source", "dts_solve",
           "dts_get_scalar_fluence", "dts_get_moments", "dts_get_iterations", "dts_get_residuals",
           "dts_get_balance", "dts_last_error", "dts_destroy_problem", "dts_status_string",
           "dts_version", "dts_quadrature", "dts_moment_tables", "dts_subsweep_size",
           "dts_sweep_once_noalloc", "dts_solve_adjoint", "dts_get_adjoint_iterations",
           "dts_tune_tile", "dts_set_source_cones", "dts_get_dose", "dts_debug_fail_allocation",
           "dts_solve_many", "dts_tune_cache_file", "dts_set_iteration_callback",
           "dts_debug_bounds_selftest", "dts_set_initial_guess", "dts_debug_poison_wait",
           "dts_set_host_output", "dts_set_device_loop")


def lib():
    """Load libdts.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_1910_11335_b300.build`"
                           + (" --debug-bounds" if DEBUG_BOUNDS else ""))
    L = C.CDLL(LIB_PATH)
    pp = C.POINTER(C.c_void_p)
    sig = {
        "dts_create_problem": ([C.POINTER(ProblemDesc), pp], C.c_int),
        "dts_set_materials": ([C.c_void_p, C.c_int, _dp, _dp, _ip, _dp, _dp], C.c_int),
        "dts_set_source": ([C.c_void_p, C.c_int, C.POINTER(SourceDesc)], C.c_int),
        "dts_set_source_cones": ([C.c_void_p, C.c_int, C.c_int, C.POINTER(SourceDesc)], C.c_int),
        "dts_get_dose": ([C.c_void_p, C.c_int, C.c_int, _dp, _dp, C.c_void_p, C.c_size_t, C.c_int], C.c_int),
        "dts_solve": ([C.c_void_p, C.POINTER(SolveStats)], C.c_int),
        "dts_solve_many": ([C.POINTER(C.c_void_p), C.c_int, C.POINTER(SolveStats)], C.c_int),
        "dts_get_scalar_fluence": ([C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_size_t, C.c_int], C.c_int),
        "dts_get_moments": ([C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_size_t, C.c_int], C.c_int),
        "dts_get_iterations": ([C.c_void_p, _ip, C.c_size_t], C.c_int),
        "dts_get_residuals": ([C.c_void_p, _dp, C.c_size_t], C.c_int),
        "dts_get_balance": ([C.c_void_p, _dp, C.c_size_t], C.c_int),
        "dts_last_error": ([C.c_void_p], C.c_char_p),
        "dts_destroy_problem": ([C.c_void_p], None),
        "dts_status_string": ([C.c_int], C.c_char_p),
        "dts_version": ([], C.c_int),
        "dts_debug_fail_allocation": ([C.c_int], None),
        "dts_quadrature": ([C.c_int, _dp, _dp, _dp, _dp, C.POINTER(C.c_int)], C.c_int),
        "dts_moment_tables": ([C.c_int, C.c_int, _dp, _dp], C.c_int),
        "dts_subsweep_size": ([C.c_int, C.c_int, C.c_int, C.c_int], C.c_longlong),
        "dts_tune_tile": ([C.POINTER(ProblemDesc), C.POINTER(C.c_double)], C.c_int),
        "dts_tune_cache_file": ([C.c_char_p], C.c_int),
        "dts_debug_bounds_selftest": ([C.c_int, C.POINTER(C.c_int)], C.c_int),
        "dts_set_initial_guess": ([C.c_void_p, C.c_int, _dp, C.c_size_t, C.c_int], C.c_int),
        "dts_debug_poison_wait": ([C.c_void_p, C.c_int], C.c_int),
        "dts_set_host_output": ([C.c_void_p, C.c_int, C.c_void_p, C.c_size_t], C.c_int),
        "dts_set_iteration_callback": ([C.c_void_p, IterationFn, C.c_void_p], C.c_int),
        "dts_set_device_loop": ([C.c_void_p, C.c_int], C.c_int),
        "dts_solve_adjoint": ([C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.c_int], C.c_int),
        "dts_get_adjoint_iterations": ([C.c_void_p, _ip, C.c_size_t], C.c_int),
        "dts_sweep_once_noalloc": ([C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                    C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _status_name(s: int) -> str:
    try:
        return lib().dts_status_string(s).decode()
    except Exception:  # pragma: no cover
        return f"status {s}"


def _check(status: int, handle=None):
    if status != DTS_OK:
        msg = lib().dts_last_error(handle).decode()
        raise DTSError(status, msg)


def _dptr(a: Optional[np.ndarray]):
    return C.cast(None, _dp) if a is None else a.ctypes.data_as(_dp)


# ------------------------------------------------------------------ host helpers
def quadrature(sn_order: int):
    mu, eta, xi, w = (np.zeros(80) for _ in range(4))
    n = C.c_int(0)
    _check(lib().dts_quadrature(sn_order, _dptr(mu), _dptr(eta), _dptr(xi), _dptr(w), C.byref(n)))
    k = n.value
    return mu[:k].copy(), eta[:k].copy(), xi[:k].copy(), w[:k].copy()


def moment_tables(sn_order: int, legendre_order: int):
    """(D[K][nd], M[nd][K]) as the solver uses them."""
    nd, K = sn_order * (sn_order + 2), (legendre_order + 1) ** 2
    D, M = np.zeros((K, nd)), np.zeros((nd, K))
    _check(lib().dts_moment_tables(sn_order, legendre_order, _dptr(D), _dptr(M)))
    return D, M


def subsweep_size(nx, ny, nz, S) -> int:
    return int(lib().dts_subsweep_size(nx, ny, nz, S))


def sweep_once_noalloc(nx, ny, nz, dx, dy, dz, sn_order, legendre_order, src_moments, sigma_t,
                       phi, stream=None):
    """One FP64 source iteration (sweep + moments) of one group using only the
    library's fixed device scratch array, for callers that must not allocate.
    src_moments [K][V], sigma_t [V] and phi [K][V] are contiguous float64 CUDA
    tensors on the current device; work is enqueued on `stream` (a
    cudaStream_t handle or None). Raises ValueError before any device work
    when a tensor is not such a tensor or is too short."""
    import torch
    K, V = (legendre_order + 1) ** 2, nx * ny * nz
    need = {"src_moments": K * V, "sigma_t": V, "phi": K * V}
    tensors = {"src_moments": src_moments, "sigma_t": sigma_t, "phi": phi}
    for name, t in tensors.items():
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != torch.float64:
            raise ValueError(f"{name} must be float64, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.numel() < need[name]:
            raise ValueError(f"{name} holds {t.numel()} elements, needs {need[name]}")
    cur = torch.cuda.current_device()
    for name, t in tensors.items():
        if t.device.index != cur:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{cur}")
    _check(lib().dts_sweep_once_noalloc(nx, ny, nz, dx, dy, dz, sn_order, legendre_order,
                                        C.c_void_p(src_moments.data_ptr()),
                                        C.c_void_p(sigma_t.data_ptr()), C.c_void_p(phi.data_ptr()),
                                        stream))


def debug_bounds_selftest(plant: bool):
    """dts_debug_bounds_selftest: (is_debug_build, status, message)."""
    flag = C.c_int(-1)
    st = lib().dts_debug_bounds_selftest(int(bool(plant)), C.byref(flag))
    return flag.value == 1, st, lib().dts_last_error(None).decode()


def debug_fail_allocation(after: int):
    """Test hook: the device allocation after `after` more successful ones fails once as
    out-of-memory (DTS_ERR_OOM); a negative value disarms it."""
    lib().dts_debug_fail_allocation(int(after))


def tune_cache_file(path: Optional[str]):
    """Name the tile tuner's cache file for this process (None turns it off;
    until called, the DTS_TUNE_CACHE environment variable names it)."""
    _check(lib().dts_tune_cache_file(None if path is None else os.fsencode(path)))


def tune_tile(w: inputs.Workload, precision=PREC_FP64, batch=None, device=0):
    """Tile chosen by dts_tune_tile for workload w's shape: ((tx, ty, tz), probe updates/s)."""
    d = ProblemDesc(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.x0, w.y0, w.z0, w.n_groups, w.sn_order,
                    w.legendre_order, batch or w.batch, precision, 0.0, 2, None, device, 0, 0, 0, 0)
    best = C.c_double(0.0)
    _check(lib().dts_tune_tile(C.byref(d), C.byref(best)))
    return (d.tile_x, d.tile_y, d.tile_z), best.value


# ------------------------------------------------------------------ problems
class Problem:
    """A solver instance on one GPU (wraps dts_problem)."""

    def __init__(self, *, nx, ny, nz, dx, dy, dz, x0=0.0, y0=0.0, z0=0.0, n_groups=1,
                 sn_order=4, legendre_order=0, batch=1, precision=PREC_FP64, tol=1e-8,
                 max_iters=1000, device=0, stream=None, tile=(0, 0, 0), keep_moments=False):
        d = ProblemDesc(nx, ny, nz, dx, dy, dz, x0, y0, z0, n_groups, sn_order, legendre_order,
                        batch, precision, tol, max_iters, stream, device, tile[0], tile[1],
                        tile[2], int(keep_moments))
        h = C.c_void_p()
        _check(lib().dts_create_problem(C.byref(d), C.byref(h)))
        self._h = h
        self.desc = d
        self.V = nx * ny * nz
        self.G, self.B = n_groups, batch
        self.K = (legendre_order + 1) ** 2
        self.nd = sn_order * (sn_order + 2)

    # context manager / lifetime
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().dts_destroy_problem(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # inputs
    def set_materials(self, sigma_t, sigma_s, mat_id, scale_t=None, scale_s=None):
        st = np.ascontiguousarray(sigma_t, dtype=np.float64)
        ss = np.ascontiguousarray(sigma_s, dtype=np.float64)
        mi = np.ascontiguousarray(mat_id, dtype=np.int32)
        a = None if scale_t is None else np.ascontiguousarray(scale_t, dtype=np.float64)
        b = None if scale_s is None else np.ascontiguousarray(scale_s, dtype=np.float64)
        _check(lib().dts_set_materials(self._h, st.shape[0], _dptr(st), _dptr(ss),
                                       mi.ctypes.data_as(_ip), _dptr(a), _dptr(b)), self._h)

    def set_source(self, b: int, src: inputs.Source):
        if src.kind == 2:   # several cone beams summed into one source
            specs = [np.ascontiguousarray(c.spectrum, dtype=np.float64) for c in src.cones]
            arr = (SourceDesc * len(src.cones))()
            for i, (c, sp) in enumerate(zip(src.cones, specs)):
                arr[i] = SourceDesc(c.kind, None, (C.c_double * 3)(*c.pos), (C.c_double * 3)(*c.axis),
                                    c.half_angle, _dptr(sp), c.aperture, (C.c_double * 3)(*c.normal),
                                    c.half_azimuth, c.half_polar)
            _check(lib().dts_set_source_cones(self._h, b, len(src.cones), arr), self._h)
            return
        q = None if src.q is None else np.ascontiguousarray(src.q, dtype=np.float64)
        sp = None if src.spectrum is None else np.ascontiguousarray(src.spectrum, dtype=np.float64)
        s = SourceDesc(src.kind, _dptr(q), (C.c_double * 3)(*src.pos),
                       (C.c_double * 3)(*src.axis), src.half_angle, _dptr(sp), src.aperture,
                       (C.c_double * 3)(*src.normal), src.half_azimuth, src.half_polar)
        _check(lib().dts_set_source(self._h, b, C.byref(s)), self._h)

    def set_host_output(self, comp: int, host):
        """Stream component comp of every member's scalar fluence into host (a
        C-contiguous float64 array of B*G*V values, page-locked for overlap) group
        by group during later solves; None turns it off (dts_set_host_output)."""
        if host is None:
            self._host_out = None
            _check(lib().dts_set_host_output(self._h, comp, None, 0), self._h)
            return
        if not (isinstance(host, np.ndarray) and host.dtype == np.float64 and host.flags.c_contiguous):
            raise ValueError("host must be a C-contiguous float64 numpy array")
        self._host_out = host   # kept alive while the library writes into it
        _check(lib().dts_set_host_output(self._h, comp, host.ctypes.data_as(C.c_void_p), host.size), self._h)

    def set_initial_guess(self, b: int, moments):
        """Start member b's source iteration in every group from moments [G][K][V]
        (as moments() returns per group); None clears it (dts_set_initial_guess)."""
        if moments is None:
            _check(lib().dts_set_initial_guess(self._h, b, None, 0, 0), self._h)
            return
        m = np.ascontiguousarray(moments, dtype=np.float64).reshape(-1)
        _check(lib().dts_set_initial_guess(self._h, b, _dptr(m), m.size, 0), self._h)

    def debug_poison_wait(self, on: bool, sweep: bool = False):
        """Make the tensor-core moment kernel's flux-stage waits (or, with
        sweep=True, the sweep's face-copy waits) run out (their bound ends them;
        the solve returns DTS_ERR_TIMEOUT), or stop doing so."""
        _check(lib().dts_debug_poison_wait(self._h, (2 if sweep else 1) if on else 0), self._h)

    def on_iteration(self, fn):
        """Call fn(group, iteration, residuals) after every source iteration of a
        solve (residuals: numpy array [batch], NaN for members already stopped);
        None turns it off (dts_set_iteration_callback)."""
        if fn is None:
            self._iter_cb = None
            _check(lib().dts_set_iteration_callback(self._h, C.cast(None, IterationFn), None), self._h)
            return

        def tramp(_user, g, it, res, n):
            fn(g, it, np.ctypeslib.as_array(res, shape=(n,)).copy())

        self._iter_cb = IterationFn(tramp)   # kept alive with the problem
        _check(lib().dts_set_iteration_callback(self._h, self._iter_cb, None), self._h)

    def set_device_loop(self, on: bool):
        """Run each group's source iterations as one CUDA-graph launch with the
        convergence decisions made on the device (dts_set_device_loop)."""
        _check(lib().dts_set_device_loop(self._h, int(bool(on))), self._h)

    # solve
    def solve(self, allow_not_converged: bool = False) -> SolveStats:
        st = SolveStats()
        rc = lib().dts_solve(self._h, C.byref(st))
        if rc == DTS_ERR_NOT_CONVERGED and allow_not_converged:
            return st
        _check(rc, self._h)
        return st

    # outputs
    def fluence(self, b: int = 0, comp: int = TOTAL, out=None):
        """Scalar fluence [G][V] of batch member b: a numpy array, or written
        into `out` (a contiguous float64 CUDA tensor) on the problem's stream."""
        n = self.G * self.V
        if out is not None and hasattr(out, "data_ptr") and getattr(out, "is_cuda", False):
            assert out.dtype.itemsize == 8 and out.is_contiguous() and out.numel() >= n
            _check(lib().dts_get_scalar_fluence(self._h, b, comp, C.c_void_p(out.data_ptr()), n, 1),
                   self._h)
            return out
        host = np.empty(n) if out is None else out
        _check(lib().dts_get_scalar_fluence(self._h, b, comp, host.ctypes.data_as(C.c_void_p), n, 0),
               self._h)
        return host.reshape(self.G, self.V)

    def dose(self, b: int, mu_en_rho, energy_mev, comp: int = TOTAL):
        """Absorbed dose per source particle (Gy) [V] from fluence component comp."""
        mu = np.ascontiguousarray(mu_en_rho, dtype=np.float64)
        e = np.ascontiguousarray(energy_mev, dtype=np.float64)
        out = np.empty(self.V)
        _check(lib().dts_get_dose(self._h, b, comp, mu.ctypes.data_as(_dp), e.ctypes.data_as(_dp),
                                  out.ctypes.data_as(C.c_void_p), out.size, 0), self._h)
        return out

    def moments(self, b: int, g: int):
        out = np.empty(self.K * self.V)
        _check(lib().dts_get_moments(self._h, b, g, out.ctypes.data_as(C.c_void_p), out.size, 0),
               self._h)
        return out.reshape(self.K, self.V)

    def iterations(self):
        out = np.zeros(self.B * self.G, dtype=np.int32)
        _check(lib().dts_get_iterations(self._h, out.ctypes.data_as(_ip), out.size), self._h)
        return out.reshape(self.B, self.G)

    def residuals(self):
        out = np.zeros(self.B * self.G)
        _check(lib().dts_get_residuals(self._h, _dptr(out), out.size), self._h)
        return out.reshape(self.B, self.G)

    def adjoint(self, b: int, dL_dphi, with_sigma_t: bool = False):
        """Discrete adjoint of the last (FP64, keep_moments) solve of batch
        member b. dL_dphi [G][V] is dL/d(total scalar fluence). Returns
        (dL/dscale_t [V], dL/dscale_s [V][, dL/dsigma_t^g [G][V]]) as numpy
        arrays, or writes into CUDA tensors when dL_dphi is one."""
        if hasattr(dL_dphi, "is_cuda") and dL_dphi.is_cuda:
            import torch
            a = dL_dphi.contiguous().to(torch.float64)
            gt = torch.empty(self.V, dtype=torch.float64, device=a.device)
            gs = torch.empty_like(gt)
            gg = torch.empty(self.G * self.V, dtype=torch.float64, device=a.device) if with_sigma_t else None
            _check(lib().dts_solve_adjoint(self._h, b, C.c_void_p(a.data_ptr()), C.c_void_p(gt.data_ptr()),
                                           C.c_void_p(gs.data_ptr()),
                                           C.c_void_p(gg.data_ptr()) if gg is not None else None, 1),
                   self._h)
            return (gt, gs, gg.view(self.G, self.V)) if with_sigma_t else (gt, gs)
        a = np.ascontiguousarray(dL_dphi, dtype=np.float64).reshape(-1)
        assert a.size == self.G * self.V
        gt, gs = np.zeros(self.V), np.zeros(self.V)
        gg = np.zeros(self.G * self.V) if with_sigma_t else None
        _check(lib().dts_solve_adjoint(self._h, b, a.ctypes.data_as(C.c_void_p), gt.ctypes.data_as(C.c_void_p),
                                       gs.ctypes.data_as(C.c_void_p),
                                       gg.ctypes.data_as(C.c_void_p) if gg is not None else None, 0),
               self._h)
        return (gt, gs, gg.reshape(self.G, self.V)) if with_sigma_t else (gt, gs)

    def adjoint_iterations(self):
        out = np.zeros(self.G, dtype=np.int32)
        _check(lib().dts_get_adjoint_iterations(self._h, out.ctypes.data_as(_ip), out.size), self._h)
        return out

    def balance(self):
        out = np.zeros(self.B * self.G * 3)
        _check(lib().dts_get_balance(self._h, _dptr(out), out.size), self._h)
        return out.reshape(self.B, self.G, 3)


def solve_many(problems, allow_not_converged: bool = False):
    """Solve several problems together (dts_solve_many): disjoint source sets,
    each problem on its own stream, with one problem's moment kernels running
    beside another's sweep. Returns one SolveStats per problem."""
    n = len(problems)
    hs = (C.c_void_p * n)(*[p._h for p in problems])
    st = (SolveStats * n)()
    rc = lib().dts_solve_many(hs, n, st)
    if not (rc == DTS_ERR_NOT_CONVERGED and allow_not_converged):
        _check(rc, None)
    return list(st)


def source_parts(n_sources: int, parts: int, sn_order: int):
    """Split source indices 0..n_sources-1 into `parts` consecutive runs for
    solve_many. The batched sweep packs 32 // (N(N+2)/8) sources into a warp
    (3 for S8), so every run but the last is a whole number of warps: the runs
    together need as many warps per tile as one batch of all the sources."""
    ndo = sn_order * (sn_order + 2) // 8
    gran = max(1, 32 // ndo)
    parts = max(1, min(parts, n_sources))
    warps = -(-n_sources // gran)
    if warps < parts:
        gran, warps = 1, n_sources
    base, extra = divmod(warps, parts)
    sizes = [(base + (1 if k >= parts - extra else 0)) * gran for k in range(parts - 1)]
    sizes.append(n_sources - sum(sizes))
    out, s0 = [], 0
    for n in sizes:
        out.append(list(range(s0, s0 + n)))
        s0 += n
    return out


def problem_from_workload(w: inputs.Workload, precision=PREC_FP64, tol=None, max_iters=None,
                          tile=(0, 0, 0), keep_moments=False, device=0, stream=None,
                          sources=None, device_loop=False) -> Problem:
    """Create a Problem for workload w and upload its materials and sources
    (all of w.sources, or the subset `sources`)."""
    srcs = w.sources if sources is None else [w.sources[i] for i in sources]
    p = Problem(nx=w.nx, ny=w.ny, nz=w.nz, dx=w.dx, dy=w.dy, dz=w.dz, x0=w.x0, y0=w.y0, z0=w.z0,
                n_groups=w.n_groups, sn_order=w.sn_order, legendre_order=w.legendre_order,
                batch=len(srcs), precision=precision, tol=w.tol if tol is None else tol,
                max_iters=w.max_iters if max_iters is None else max_iters, device=device,
                stream=stream, tile=tile, keep_moments=keep_moments)
    p.set_materials(w.sigma_t, w.sigma_s, w.mat_id.reshape(-1),
                    None if w.scale_t is None else w.scale_t.reshape(-1),
                    None if w.scale_s is None else w.scale_s.reshape(-1))
    for b, s in enumerate(srcs):
        p.set_source(b, s)
    if device_loop:
        p.set_device_loop(True)
    return p
