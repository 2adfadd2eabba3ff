"""Seeded synthetic workloads for the S_N source-iteration solve.

This module produces INPUT DATA only: voxel phantoms (material ids), multigroup
cross-section tables, source descriptions and spectra. It performs none of the
transport method's arithmetic (no quadrature, no ray tracing, no sweeps), so
both the CUDA library and the CPU oracle can be fed from it without sharing any
solver code.

The paper's own workloads (Sec. II.E: a water cylinder in a voxel box, NJOY/ENDF
multigroup libraries, point and cone-beam X-ray sources with a kVp spectrum,
16-cone CT rings) cannot be reproduced here: the cross-section libraries, the
CT images and MCNP are not available. The generators below are stand-ins with
the same structure: a water cylinder with bone-like and air-like inserts,
downscatter-only group transfer matrices with Legendre moments, mean free paths
anchored on the values quoted in Sec. II.E (13.9 mm at 20 keV, 60.6 mm at
100 keV), a cone-beam point source 50 cm from the phantom centre and a
120 kVp-like spectrum.

Every generator is seeded with ``numpy.random.Generator(PCG64(SEED_BASE + i))``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

SEED_BASE = 1910_11335

#: material indices used by the cylinder phantoms
MAT_AIR, MAT_WATER = 0, 1
N_BONE = 4


@dataclasses.dataclass
class Source:
    """One source description (one batch member).

    kind 0: isotropic volumetric source ``q[G][V]`` in photons/cm^3 (total over
    4 pi). kind 1: point source at ``pos`` collimated to a cone around ``axis``
    with half-angle ``half_angle`` (radians; >= pi means isotropic), emitting
    ``spectrum[g]`` photons per source particle into group g; with
    ``aperture`` 1 the beam is a fan instead: the azimuthal angle subtended in
    the plane normal to ``normal`` is 2 ``half_azimuth`` and the polar angle out
    of that plane 2 ``half_polar``. kind 2: the sum of the kind-1 sources in
    ``cones`` (several cone or fan beams at once).
    """
    kind: int
    q: Optional[np.ndarray] = None
    pos: tuple = (0.0, 0.0, 0.0)
    axis: tuple = (0.0, 1.0, 0.0)
    half_angle: float = math.pi
    spectrum: Optional[np.ndarray] = None
    cones: Optional[list] = None
    aperture: int = 0
    normal: tuple = (0.0, 0.0, 1.0)
    half_azimuth: float = 0.0
    half_polar: float = 0.0


@dataclasses.dataclass
class Workload:
    """A complete problem description (geometry, materials, sources, options)."""
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    x0: float
    y0: float
    z0: float
    n_groups: int
    sn_order: int
    legendre_order: int
    sigma_t: np.ndarray          # [n_mat][G]
    sigma_s: np.ndarray          # [n_mat][L+1][G_from][G_to]
    mat_id: np.ndarray           # [nz][ny][nx] int32, x fastest
    sources: List[Source]
    tol: float = 1e-8
    max_iters: int = 1000
    group_energy_kev: Optional[np.ndarray] = None
    scale_t: Optional[np.ndarray] = None   # [nz][ny][nx] or None
    scale_s: Optional[np.ndarray] = None

    @property
    def n_voxels(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_mat(self) -> int:
        return int(self.sigma_t.shape[0])

    @property
    def n_dirs(self) -> int:
        return self.sn_order * (self.sn_order + 2)

    @property
    def batch(self) -> int:
        return len(self.sources)


def rng_for(index: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + index))


# --------------------------------------------------------------------------- #
# cross sections
# --------------------------------------------------------------------------- #
def group_structure(n_groups: int, e_hi: float = 120.0, e_lo: float = 25.0):
    """Equal-width groups from e_hi down to e_lo keV; group 0 is the highest energy."""
    edges = np.linspace(e_hi, e_lo, n_groups + 1)
    mids = 0.5 * (edges[:-1] + edges[1:])
    return edges, mids


def water_like_xs(rng: np.random.Generator, n_groups: int, legendre_order: int):
    """Synthetic water-like multigroup data.

    sigma_t is log-linear in energy (hence in group index) through the two
    mean-free-path anchors of Sec. II.E, each jittered by x(1 + 0.05 U[-1,1]).
    The scattering ratio falls linearly from 0.95 (group 0) to 0.55 (last
    group). Group transfer is downscatter only: a fraction p_0 = 0.6 stays in
    the group and 0.4 goes geometrically (ratio 1/2) to the next <= 4 groups,
    renormalised where fewer groups remain; the last group scatters only into
    itself. Legendre moments follow Henyey-Greenstein: sigma_{s,l} = gbar^l
    sigma_{s,0} with gbar = 0.25 +- 0.05.
    Returns (sigma_t[G], sigma_s[L+1][G][G], group mid energies).
    """
    _, mids = group_structure(n_groups)
    s20 = (10.0 / 13.9) * (1.0 + 0.05 * rng.uniform(-1.0, 1.0))   # 1/mfp, 1/cm
    s100 = (10.0 / 60.6) * (1.0 + 0.05 * rng.uniform(-1.0, 1.0))
    slope = (math.log(s100) - math.log(s20)) / (100.0 - 20.0)
    sig_t = np.exp(math.log(s20) + slope * (mids - 20.0))
    c = np.linspace(0.95, 0.55, n_groups) if n_groups > 1 else np.array([0.95])
    gbar = 0.25 + 0.05 * rng.uniform(-1.0, 1.0)
    p_tail = 0.4 * np.array([1.0, 0.5, 0.25, 0.125]) / 1.875
    p = np.concatenate([[0.6], p_tail])
    sig_s0 = np.zeros((n_groups, n_groups))
    for gf in range(n_groups):
        span = min(len(p), n_groups - gf)
        pp = p[:span] / p[:span].sum()
        for j in range(span):
            sig_s0[gf, gf + j] = c[gf] * sig_t[gf] * pp[j]
    sig_s = np.stack([sig_s0 * gbar ** l for l in range(legendre_order + 1)])
    return sig_t, sig_s, mids


def cylinder_materials(rng: np.random.Generator, n_groups: int, legendre_order: int):
    """Material table: air, water and N_BONE bone-like materials.

    Bone i scales water sigma_t by m_i ~ U[1.5, 3] and water sigma_s by
    0.7 m_i (a lower scattering ratio). Air is 1e-3 x water.
    """
    sig_t_w, sig_s_w, mids = water_like_xs(rng, n_groups, legendre_order)
    mult = rng.uniform(1.5, 3.0, size=N_BONE)
    n_mat = 2 + N_BONE
    sig_t = np.zeros((n_mat, n_groups))
    sig_s = np.zeros((n_mat, legendre_order + 1, n_groups, n_groups))
    sig_t[MAT_AIR], sig_s[MAT_AIR] = 1e-3 * sig_t_w, 1e-3 * sig_s_w
    sig_t[MAT_WATER], sig_s[MAT_WATER] = sig_t_w, sig_s_w
    for i, m in enumerate(mult):
        sig_t[2 + i] = m * sig_t_w
        sig_s[2 + i] = 0.7 * m * sig_s_w
    return sig_t, sig_s, mids, mult


# --------------------------------------------------------------------------- #
# phantom
# --------------------------------------------------------------------------- #
def sphere_inserts(rng: np.random.Generator, radius_cyl=14.0, half_height=16.0,
                   n_bone=N_BONE, n_air=2):
    """Non-overlapping spheres inside the cylinder (rejection sampling).

    Returns a list of (cx, cy, cz, r, material) with material 2+i for bone i
    and MAT_AIR for air inserts.
    """
    spheres = []
    mats = [2 + i for i in range(n_bone)] + [MAT_AIR] * n_air
    for mat in mats:
        for _ in range(100000):
            r = rng.uniform(1.5, 4.0)
            cx, cy = rng.uniform(-radius_cyl, radius_cyl, size=2)
            cz = rng.uniform(-half_height, half_height)
            if math.hypot(cx, cy) + r > radius_cyl or abs(cz) + r > half_height:
                continue
            if any(math.dist((cx, cy, cz), s[:3]) < r + s[3] for s in spheres):
                continue
            spheres.append((cx, cy, cz, r, mat))
            break
        else:  # pragma: no cover - geometry always admits 6 small spheres
            raise RuntimeError("could not place sphere")
    return spheres


def cylinder_phantom(n: int, spheres, box_half=16.0, radius_cyl=14.0):
    """Material ids of an n^3 voxelisation of the 32 cm box (membership by voxel centre)."""
    h = 2.0 * box_half / n
    c = -box_half + (np.arange(n) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    mat = np.full((n, n, n), MAT_AIR, dtype=np.int32)
    mat[x * x + y * y <= radius_cyl * radius_cyl] = MAT_WATER
    for (cx, cy, cz, r, m) in spheres:
        inside = (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2 <= r * r
        mat[inside] = m
    return mat, h


def kvp_spectrum(rng: np.random.Generator, mids: np.ndarray):
    """120 kVp-like spectrum: seeded piecewise-linear histogram, normalised to sum 1.

    Knots: 25 keV (r x peak, r ~ U[0.2,0.4]), a jittered knot on the rising
    side, the peak (U[55,65] keV), a jittered knot on the falling side, and
    zero at 120 keV.
    """
    e_peak = rng.uniform(55.0, 65.0)
    r_low = rng.uniform(0.2, 0.4)
    e1 = 0.5 * (25.0 + e_peak) + rng.uniform(-3.0, 3.0)
    v1 = 0.5 * (r_low + 1.0) * (1.0 + 0.1 * rng.uniform(-1.0, 1.0))
    e3 = 0.5 * (e_peak + 120.0) + rng.uniform(-3.0, 3.0)
    v3 = 0.5 * (1.0 + 0.1 * rng.uniform(-1.0, 1.0))
    ke = np.array([25.0, e1, e_peak, e3, 120.0])
    kv = np.array([r_low, v1, 1.0, v3, 0.0])
    s = np.clip(np.interp(mids, ke, kv), 0.0, None)
    return s / s.sum()


def ring_sources(spectrum, n_sources: int, distance=50.0, half_angle=math.radians(15.0)):
    """Cone-beam point sources on a circle in the central z-plane, aimed at the centre.

    Source k sits at angle 2 pi k / n; k = 0 is on the -y axis.
    """
    out = []
    for k in range(n_sources):
        a = 2.0 * math.pi * k / n_sources
        pos = (distance * math.sin(a), -distance * math.cos(a), 0.0)
        axis = (-pos[0] / distance, -pos[1] / distance, 0.0)
        out.append(Source(kind=1, pos=pos, axis=axis, half_angle=half_angle,
                          spectrum=np.asarray(spectrum, dtype=np.float64)))
    return out


# --------------------------------------------------------------------------- #
# the five workloads
# --------------------------------------------------------------------------- #
def plain_16(tol: float = 1e-8) -> Workload:
    """Plain FP64 S_N: 16^3 x 1 cm, S4, one group, sigma_t 0.2, sigma_s 0.18, P0,
    isotropic volumetric source 1.0 in the central 4^3 voxels, vacuum boundaries."""
    n = 16
    q = np.zeros((1, n, n, n))
    q[0, 6:10, 6:10, 6:10] = 1.0
    return Workload(
        name="plain16_s4p0_1g", nx=n, ny=n, nz=n, dx=1.0, dy=1.0, dz=1.0,
        x0=0.0, y0=0.0, z0=0.0, n_groups=1, sn_order=4, legendre_order=0,
        sigma_t=np.array([[0.2]]), sigma_s=np.array([[[[0.18]]]]),
        mat_id=np.zeros((n, n, n), dtype=np.int32),
        sources=[Source(kind=0, q=q.reshape(1, -1))], tol=tol)


def cone_beam(n: int = 64, n_groups: int = 19, sn_order: int = 8, legendre_order: int = 3,
              n_sources: int = 1, seed_index: int = 1, tol: float = 1e-8,
              name: Optional[str] = None) -> Workload:
    """Heterogeneous cone-beam phantom: water cylinder (r = 14 cm) in a 32 cm box,
    4 bone and 2 air spherical inserts, point source(s) 50 cm from the centre
    with a 30-degree (full apex angle) cone and a 120 kVp-like spectrum.

    The geometry, cross sections and spectrum are drawn from seed_index, so
    different grid resolutions of the same seed describe the same object.
    """
    rng = rng_for(seed_index)
    sig_t, sig_s, mids, _ = cylinder_materials(rng, n_groups, legendre_order)
    spheres = sphere_inserts(rng)
    spectrum = kvp_spectrum(rng, mids)
    mat, h = cylinder_phantom(n, spheres)
    return Workload(
        name=name or f"cone{n}_s{sn_order}p{legendre_order}_{n_groups}g_b{n_sources}",
        nx=n, ny=n, nz=n, dx=h, dy=h, dz=h, x0=-16.0, y0=-16.0, z0=-16.0,
        n_groups=n_groups, sn_order=sn_order, legendre_order=legendre_order,
        sigma_t=sig_t, sigma_s=sig_s, mat_id=mat,
        sources=ring_sources(spectrum, n_sources), tol=tol, group_energy_kev=mids)


def hetero_64() -> Workload:
    """64^3 x 0.5 cm, 19 groups, S8, P3, one cone-beam source; FP64 to 1e-8."""
    return cone_beam(64, 19, 8, 3, 1, seed_index=1, tol=1e-8, name="hetero64_s8p3_19g")


def precision_128() -> Workload:
    """The same phantom at 128^3 x 0.25 cm, 19 groups, S8, P3 (reduced-precision form)."""
    return cone_beam(128, 19, 8, 3, 1, seed_index=1, tol=1e-6, name="precision128_s8p3_19g")


def adjoint_64() -> Workload:
    """64^3, 8 groups over 25-120 keV, S6, P1 (differentiation form)."""
    return cone_beam(64, 8, 6, 1, 1, seed_index=3, tol=1e-8, name="adjoint64_s6p1_8g")


def batch_96(n_sources: int = 32) -> Workload:
    """The same phantom at 96^3 x 1/3 cm, 19 groups, S8, P3, 32 CT source positions."""
    return cone_beam(96, 19, 8, 3, n_sources, seed_index=1, tol=1e-6,
                     name=f"batch96_s8p3_19g_x{n_sources}")


def small_cone(nx: int, ny: int, nz: int, n_groups: int = 3, sn_order: int = 4,
               legendre_order: int = 1, n_sources: int = 1, seed_index: int = 1,
               tol: float = 1e-10) -> Workload:
    """A coarse, possibly non-cubic voxelisation of the cone-beam phantom for
    parity tests at sizes the oracle finishes in seconds (ragged tiles, thick
    cells that trigger the negative-flux fixup)."""
    rng = rng_for(seed_index)
    sig_t, sig_s, mids, _ = cylinder_materials(rng, n_groups, legendre_order)
    spheres = sphere_inserts(rng)
    spectrum = kvp_spectrum(rng, mids)
    dims = (nz, ny, nx)
    hs = [32.0 / d for d in dims]
    cz, cy, cx = [-16.0 + (np.arange(d) + 0.5) * h for d, h in zip(dims, hs)]
    z, y, x = np.meshgrid(cz, cy, cx, indexing="ij")
    mat = np.full(dims, MAT_AIR, dtype=np.int32)
    mat[x * x + y * y <= 14.0 ** 2] = MAT_WATER
    for (sx, sy, sz, r, m) in spheres:
        mat[(x - sx) ** 2 + (y - sy) ** 2 + (z - sz) ** 2 <= r * r] = m
    return Workload(
        name=f"small{nx}x{ny}x{nz}_s{sn_order}p{legendre_order}_{n_groups}g_b{n_sources}",
        nx=nx, ny=ny, nz=nz, dx=hs[2], dy=hs[1], dz=hs[0], x0=-16.0, y0=-16.0, z0=-16.0,
        n_groups=n_groups, sn_order=sn_order, legendre_order=legendre_order,
        sigma_t=sig_t, sigma_s=sig_s, mat_id=mat,
        sources=ring_sources(spectrum, n_sources), tol=tol, group_energy_kev=mids)


def random_volumetric(nx, ny, nz, n_groups=2, sn_order=2, legendre_order=1, n_mat=3,
                      seed_index=100, h=(0.5, 0.6, 0.7), thin=True) -> Workload:
    """Small random heterogeneous problem with a seeded non-negative volumetric
    source (for dense direct-solve and balance checks). ``thin`` keeps cells
    optically thin so the negative-flux fixup never fires."""
    rng = rng_for(seed_index)
    scale = 0.3 if thin else 3.0
    sig_t = rng.uniform(0.5, 1.0, size=(n_mat, n_groups)) * scale
    sig_s = np.zeros((n_mat, legendre_order + 1, n_groups, n_groups))
    for m in range(n_mat):
        for gf in range(n_groups):
            c = rng.uniform(0.3, 0.9)
            share = rng.uniform(0.2, 1.0, size=n_groups - gf)
            share /= share.sum()
            g = rng.uniform(0.1, 0.3)
            for j, sh in enumerate(share):
                for l in range(legendre_order + 1):
                    sig_s[m, l, gf, gf + j] = c * sig_t[m, gf] * sh * g ** l
    mat = rng.integers(0, n_mat, size=(nz, ny, nx), dtype=np.int32)
    q = rng.uniform(0.0, 1.0, size=(n_groups, nz * ny * nx))
    return Workload(
        name=f"rand{nx}x{ny}x{nz}_s{sn_order}p{legendre_order}_{n_groups}g",
        nx=nx, ny=ny, nz=nz, dx=h[0], dy=h[1], dz=h[2], x0=0.0, y0=0.0, z0=0.0,
        n_groups=n_groups, sn_order=sn_order, legendre_order=legendre_order,
        sigma_t=sig_t, sigma_s=sig_s, mat_id=mat, sources=[Source(kind=0, q=q)], tol=1e-13)


def detector_layout(w: Workload, bin_size: int = 2):
    """Detector plane behind the phantom (the far y layer, source on the -y side),
    binned bin_size x bin_size voxels in (x, z). Returns pixel index per voxel of
    that layer ([nz][nx], -1 outside) and the pixel count."""
    px = np.arange(w.nx) // bin_size
    pz = np.arange(w.nz) // bin_size
    npx, npz = (w.nx + bin_size - 1) // bin_size, (w.nz + bin_size - 1) // bin_size
    pix = pz[:, None] * npx + px[None, :]
    return pix.astype(np.int64), npx * npz


def detector_target_noise(n_pixels: int, seed_index: int = 3) -> np.ndarray:
    """Seeded multiplicative noise 1 + 0.05 N(0,1) for the detector target image."""
    rng = rng_for(1000 + seed_index)
    return 1.0 + 0.05 * rng.standard_normal(n_pixels)


def first_groups(w: Workload, n_groups: int) -> Workload:
    """The same problem restricted to its first n_groups (highest energies).
    With downscatter only, groups 0..n-1 do not depend on later groups, so a
    solve of the truncated problem reproduces them."""
    import copy
    t = copy.copy(w)
    t.n_groups = n_groups
    t.sigma_t = np.ascontiguousarray(w.sigma_t[:, :n_groups])
    t.sigma_s = np.ascontiguousarray(w.sigma_s[:, :, :n_groups, :n_groups])
    srcs = []
    for s in w.sources:
        s2 = copy.copy(s)
        if s.q is not None:
            s2.q = np.ascontiguousarray(s.q[:n_groups])
        if s.spectrum is not None:
            s2.spectrum = np.ascontiguousarray(s.spectrum[:n_groups])
        srcs.append(s2)
    t.sources = srcs
    if w.group_energy_kev is not None:
        t.group_energy_kev = w.group_energy_kev[:n_groups]
    return t


def dose_coefficients(w: Workload, seed_index: int = 7):
    """Seeded synthetic mass energy-absorption coefficients mu_en/rho [n_mat][G]
    (cm^2/g) and group energies E [G] (MeV) for the fluence-to-dose
    post-processing (no measured data is present): a power law
    a (E / 60 keV)^-p per material with p ~ U[1.5, 2.5] (photo-absorption
    falling with energy) flattening to a floor of 0.02 cm^2/g; bone-like
    materials get a ~ U[2, 4] x water, air ~ water."""
    rng = rng_for(seed_index)
    n_mat = w.sigma_t.shape[0]
    e_kev = np.asarray(w.group_energy_kev if w.group_energy_kev is not None
                       else np.linspace(120.0, 25.0, w.n_groups), dtype=np.float64)
    a = np.empty(n_mat)
    a[:] = rng.uniform(0.03, 0.05)                 # water at 60 keV
    a[MAT_AIR] = a[MAT_WATER] * rng.uniform(0.9, 1.0)
    a[2:] = a[MAT_WATER] * rng.uniform(2.0, 4.0, size=n_mat - 2)
    p = rng.uniform(1.5, 2.5, size=n_mat)
    mu = a[:, None] * (e_kev[None, :] / 60.0) ** (-p[:, None]) + 0.02
    return mu, e_kev / 1000.0


def fan_sources(spectrum, n_sources: int, distance=50.0, half_azimuth=math.radians(20.0),
                half_polar=math.radians(4.0)):
    """Fan-beam point sources on a circle in the central z-plane, aimed at the
    centre, fan plane normal to z (the rotation axis of a CT gantry)."""
    out = ring_sources(spectrum, n_sources, distance)
    for s in out:
        s.aperture, s.normal = 1, (0.0, 0.0, 1.0)
        s.half_azimuth, s.half_polar = half_azimuth, half_polar
    return out


def combined_fans(w: Workload, n_fans: int = 16, **kw) -> Workload:
    """The same problem with one source made of n_fans fan beams on a ring
    (multi-fan CT arrangement), each with source 0's spectrum."""
    import copy
    t = copy.copy(w)
    t.sources = [Source(kind=2, cones=fan_sources(w.sources[0].spectrum, n_fans, **kw))]
    t.name = f"{w.name}_fans{n_fans}"
    return t


def combined_cones(w: Workload, n_cones: int = 16, distance=50.0, half_angle=math.radians(15.0)) -> Workload:
    """The same problem with one source made of n_cones cone beams on a ring (the
    paper's CT mode of several cones at once), each with source 0's spectrum."""
    import copy
    t = copy.copy(w)
    cones = ring_sources(w.sources[0].spectrum, n_cones, distance, half_angle)
    t.sources = [Source(kind=2, cones=cones)]
    t.name = f"{w.name}_cones{n_cones}"
    return t


def with_sources(w: Workload, idx) -> Workload:
    """The same problem with the batch restricted to sources idx."""
    import copy
    t = copy.copy(w)
    t.sources = [w.sources[i] for i in idx]
    return t


WORKLOADS = {
    "plain16": plain_16,
    "hetero64": hetero_64,
    "precision128": precision_128,
    "adjoint64": adjoint_64,
    "batch96": batch_96,
}
