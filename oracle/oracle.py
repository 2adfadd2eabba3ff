"""ctypes wrapper around the C oracle (oracle/dts_oracle.c).

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline). Builds the shared
object with gcc on first use. Every function here marshals arguments only; the
arithmetic is in the C file.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "dts_oracle.c")
LIB = os.path.join(HERE, "libdts_oracle.so")

_lib = None
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_lp = C.POINTER(C.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2, no fast-math, OpenMP over octants)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c99", "-Wall",
               "-Wno-unused-variable", SRC, "-o", LIB + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(LIB + ".tmp", LIB)
    return LIB


class _Problem(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double),
                ("G", C.c_int), ("N", C.c_int), ("L", C.c_int), ("n_mat", C.c_int),
                ("sigma_t", _dp), ("sigma_s", _dp), ("mat", _ip),
                ("scale_t", _dp), ("scale_s", _dp),
                ("tol", C.c_double), ("max_iters", C.c_int), ("n_threads", C.c_int),
                ("fixup", C.c_int)]


class _Source(C.Structure):
    _fields_ = [("kind", C.c_int), ("q", _dp), ("pos", C.c_double * 3),
                ("axis", C.c_double * 3), ("half_angle", C.c_double), ("spectrum", _dp),
                ("n_cones", C.c_int), ("cone_geo", _dp), ("cone_spec", _dp),
                ("aperture", C.c_int), ("normal", C.c_double * 3), ("half_azimuth", C.c_double),
                ("half_polar", C.c_double)]


class _Result(C.Structure):
    _fields_ = [("phi_u", _dp), ("phi_c", _dp), ("iters", _ip), ("resid", _dp),
                ("src", _dp), ("absorb", _dp), ("leak", _dp), ("fixups", _lp)]


def load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        lib.ora_quadrature.argtypes = [C.c_int, _dp, _dp, _dp, _dp]
        lib.ora_quadrature.restype = C.c_int
        lib.ora_real_sh.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double]
        lib.ora_real_sh.restype = C.c_double
        lib.ora_assoc_legendre.argtypes = [C.c_int, C.c_int, C.c_double]
        lib.ora_assoc_legendre.restype = C.c_double
        lib.ora_subsweep_size.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int]
        lib.ora_subsweep_size.restype = C.c_long
        lib.ora_subsweep_cells.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _ip]
        lib.ora_subsweep_cells.restype = C.c_long
        lib.ora_dd_cell.argtypes = [C.c_double, C.c_double, _dp, _dp, _dp, C.POINTER(C.c_int)]
        lib.ora_dd_cell.restype = C.c_double
        lib.ora_sweep_dir.argtypes = [C.POINTER(_Problem), _dp, C.c_double, C.c_double, C.c_double,
                                      _dp, C.c_double, _dp, _dp, _lp]
        lib.ora_sweep_dir.restype = None
        lib.ora_uncollided_voxel.argtypes = [C.POINTER(_Problem), C.POINTER(_Source), C.c_int, _dp, _dp]
        lib.ora_uncollided_voxel.restype = C.c_int
        lib.ora_solve.argtypes = [C.POINTER(_Problem), C.POINTER(_Source), C.POINTER(_Result)]
        lib.ora_solve.restype = C.c_int
        lib.ora_has_openmp.restype = C.c_int
        lib.ora_adjoint.argtypes = [C.POINTER(_Problem), C.POINTER(_Source), _dp, _dp, _dp, _dp]
        lib.ora_adjoint.restype = C.c_int
        _lib = lib
    return _lib


def _ptr(a: Optional[np.ndarray], t=_dp):
    if a is None:
        return C.cast(None, t)
    return a.ctypes.data_as(t)


def quadrature(N: int):
    """Level-symmetric S_N set: (mu, eta, xi, w), octant-major."""
    lib = load()
    mu, eta, xi, w = (np.zeros(80) for _ in range(4))
    nd = lib.ora_quadrature(N, _ptr(mu), _ptr(eta), _ptr(xi), _ptr(w))
    if nd < 0:
        raise ValueError(f"unsupported S_N order {N}")
    return mu[:nd].copy(), eta[:nd].copy(), xi[:nd].copy(), w[:nd].copy()


def real_sh(l: int, m: int, mu: float, eta: float, xi: float) -> float:
    return load().ora_real_sh(l, m, mu, eta, xi)


def sh_tables(N: int, L: int):
    """Y[K][nd], D = w Y (moments), M = (2l+1)/(4 pi) Y (source), K = (L+1)^2."""
    mu, eta, xi, w = quadrature(N)
    K = (L + 1) ** 2
    Y = np.zeros((K, len(w)))
    ls = np.zeros(K, dtype=int)
    for l in range(L + 1):
        for m in range(-l, l + 1):
            k = l * l + l + m
            ls[k] = l
            for n in range(len(w)):
                Y[k, n] = real_sh(l, m, mu[n], eta[n], xi[n])
    D = Y * w[None, :]
    M = ((2 * ls + 1) / (4 * np.pi))[:, None] * Y
    return Y, D, M.T.copy()


def subsweep_size(nx, ny, nz, S) -> int:
    return int(load().ora_subsweep_size(nx, ny, nz, S))


def subsweep_cells(nx, ny, nz, S) -> np.ndarray:
    lib = load()
    n = lib.ora_subsweep_cells(nx, ny, nz, S, C.cast(None, _ip))
    out = np.zeros((max(n, 1), 3), dtype=np.int32)
    lib.ora_subsweep_cells(nx, ny, nz, S, _ptr(out, _ip))
    return out[:n]


def dd_cell(q, sig, a, psi_in):
    a = np.ascontiguousarray(a, dtype=np.float64)
    pin = np.ascontiguousarray(psi_in, dtype=np.float64)
    out = np.zeros(3)
    nf = C.c_int(0)
    psi = load().ora_dd_cell(q, sig, _ptr(a), _ptr(pin), _ptr(out), C.byref(nf))
    return psi, out, nf.value


def _problem(w, tol=None, max_iters=None, n_threads=1, keep=None, fixup=True):
    keep = [] if keep is None else keep
    sig_t = np.ascontiguousarray(w.sigma_t, dtype=np.float64)
    sig_s = np.ascontiguousarray(w.sigma_s, dtype=np.float64)
    mat = np.ascontiguousarray(w.mat_id, dtype=np.int32)
    st = None if w.scale_t is None else np.ascontiguousarray(w.scale_t, dtype=np.float64)
    ss = None if w.scale_s is None else np.ascontiguousarray(w.scale_s, dtype=np.float64)
    keep += [sig_t, sig_s, mat, st, ss]
    p = _Problem(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.x0, w.y0, w.z0,
                 w.n_groups, w.sn_order, w.legendre_order, sig_t.shape[0],
                 _ptr(sig_t), _ptr(sig_s), _ptr(mat, _ip), _ptr(st), _ptr(ss),
                 w.tol if tol is None else tol,
                 w.max_iters if max_iters is None else max_iters, n_threads, int(bool(fixup)))
    return p, keep


def _source(src, keep):
    q = None if src.q is None else np.ascontiguousarray(src.q, dtype=np.float64)
    spec = None if src.spectrum is None else np.ascontiguousarray(src.spectrum, dtype=np.float64)
    geo = cspec = None
    n = 0
    if src.kind == 2:
        n = len(src.cones)
        geo = np.ascontiguousarray([[*c.pos, *c.axis, c.half_angle, c.aperture, *c.normal, c.half_azimuth,
                                     c.half_polar] for c in src.cones], dtype=np.float64)
        cspec = np.ascontiguousarray([c.spectrum for c in src.cones], dtype=np.float64)
    keep += [q, spec, geo, cspec]
    s = _Source(src.kind, _ptr(q), (C.c_double * 3)(*src.pos), (C.c_double * 3)(*src.axis),
                src.half_angle, _ptr(spec), n, _ptr(geo), _ptr(cspec), src.aperture,
                (C.c_double * 3)(*src.normal), src.half_azimuth, src.half_polar)
    return s


def sweep_dir(w, sigt, omega, Q, inflow=0.0, fixup=True):
    """One upwind sweep of direction omega with angular source Q[V] and a
    uniform boundary inflow. Returns (psi[V], leakage, fixup count)."""
    p, keep = _problem(w, fixup=fixup)
    sigt = np.ascontiguousarray(sigt, dtype=np.float64).ravel()
    Q = np.ascontiguousarray(Q, dtype=np.float64).ravel()
    psi = np.zeros(w.n_voxels)
    leak = C.c_double(0.0)
    nf = C.c_int64(0)
    load().ora_sweep_dir(C.byref(p), _ptr(sigt), omega[0], omega[1], omega[2], _ptr(Q), inflow,
                         _ptr(psi), C.byref(leak), C.byref(nf))
    return psi, leak.value, nf.value


def uncollided_voxel(w, src, v: int):
    """(phi_u[G], Omega_u[3]) at voxel v for a kind-1 source."""
    p, keep = _problem(w)
    s = _source(src, keep)
    pg = np.zeros(w.n_groups)
    om = np.zeros(3)
    if load().ora_uncollided_voxel(C.byref(p), C.byref(s), int(v), _ptr(pg), _ptr(om)) != 0:
        raise MemoryError
    return pg, om


@dataclasses.dataclass
class OracleResult:
    phi_u: np.ndarray      # [G][V]
    phi_c: np.ndarray      # [G][K][V]
    iters: np.ndarray      # [G]
    resid: np.ndarray      # [G]
    src: np.ndarray        # [G]
    absorb: np.ndarray     # [G]
    leak: np.ndarray       # [G]
    fixups: np.ndarray     # [G]

    @property
    def collided(self):
        return self.phi_c[:, 0, :]

    @property
    def total(self):
        return self.phi_u + self.phi_c[:, 0, :]


def solve(w, source_index: int = 0, tol=None, max_iters=None, n_threads=1,
          fixup=True) -> OracleResult:
    """Full source-iteration solve of batch member `source_index`.
    fixup=False switches the negative-flux fixup off (plain diamond difference,
    a linear scheme), which only the dense direct-solve pins use."""
    p, keep = _problem(w, tol, max_iters, n_threads, fixup=fixup)
    s = _source(w.sources[source_index], keep)
    G, V, K = w.n_groups, w.n_voxels, (w.legendre_order + 1) ** 2
    r = OracleResult(np.zeros((G, V)), np.zeros((G, K, V)), np.zeros(G, dtype=np.int32),
                     np.zeros(G), np.zeros(G), np.zeros(G), np.zeros(G), np.zeros(G, dtype=np.int64))
    cres = _Result(_ptr(r.phi_u), _ptr(r.phi_c), _ptr(r.iters, _ip), _ptr(r.resid), _ptr(r.src),
                   _ptr(r.absorb), _ptr(r.leak), _ptr(r.fixups, _lp))
    rc = load().ora_solve(C.byref(p), C.byref(s), C.byref(cres))
    if rc != 0:
        raise RuntimeError(f"oracle solve failed ({rc})")
    return r


def adjoint(w, dL_dphi, source_index: int = 0, tol=None, max_iters=None, n_threads=1):
    """Gradient of L = sum a * phi_total (a = dL_dphi [G][V]) with respect to the
    per-voxel multipliers of sigma_t and sigma_s, by the discrete adjoint of the
    converged solve. Returns (dL/dscale_t [V], dL/dscale_s [V], dL/dsigma_t^g [G][V])."""
    p, keep = _problem(w, tol, max_iters, n_threads)
    s = _source(w.sources[source_index], keep)
    a = np.ascontiguousarray(dL_dphi, dtype=np.float64).reshape(w.n_groups, w.n_voxels)
    gt, gs = np.zeros(w.n_voxels), np.zeros(w.n_voxels)
    gg = np.zeros((w.n_groups, w.n_voxels))
    if load().ora_adjoint(C.byref(p), C.byref(s), _ptr(a), _ptr(gt), _ptr(gs), _ptr(gg)) != 0:
        raise RuntimeError("oracle adjoint failed")
    return gt, gs, gg


def solve_workload(w, **kw):
    return [solve(w, b, **kw) for b in range(w.batch)]


def n_threads_available() -> int:
    return int(load().ora_has_openmp())


MEV_PER_G_TO_GY = 1.602176634e-10   # 1 MeV/g in J/kg (elementary charge x 1e6 J/MeV / 1e-3 kg)


def dose(phi, mat, mu_en_rho, energy_mev):
    """Absorbed dose per source particle (Gy) from the scalar fluence phi[G][V]
    (photons/cm^2 per source particle): the post-processing module's
    fluence-to-dose conversion (Sec. II.C), in the collision-kerma form
    D(v) = c sum_g phi_g(v) E_g (mu_en/rho)_g(mat(v)), c = 1 MeV/g in Gy, since
    the method transports no electrons (Sec. IV). Plain numpy, one term per
    group in group order."""
    phi = np.asarray(phi, dtype=np.float64)
    mat = np.asarray(mat).reshape(-1)
    out = np.zeros(phi.shape[1])
    for g in range(phi.shape[0]):
        out += phi[g] * energy_mev[g] * mu_en_rho[mat, g]
    return MEV_PER_G_TO_GY * out
