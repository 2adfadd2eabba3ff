"""Fan-beam sources in the oracle (point source with a fan aperture: azimuthal
angle 2 half_azimuth in the fan plane, polar angle 2 half_polar out of it),
pinned by limits and symmetry rather than by the beam test itself."""
import copy
import math

import numpy as np

from paper_1910_11335_b300 import inputs


def _homogeneous(n=10, G=2):
    w = inputs.small_cone(n, n, n, n_groups=G, sn_order=2, legendre_order=0)
    w = copy.copy(w)
    w.mat_id = np.full_like(w.mat_id, inputs.MAT_WATER)
    return w


def _one(w, src):
    t = copy.copy(w)
    t.sources = [src]
    return t


def test_fan_open_to_the_sphere_is_an_isotropic_point_source(ora):
    w = _homogeneous()
    spec = w.sources[0].spectrum
    iso = inputs.Source(kind=1, pos=(0.0, -50.0, 0.0), axis=(0.0, 1.0, 0.0), half_angle=math.pi, spectrum=spec)
    fan = inputs.Source(kind=1, pos=(0.0, -50.0, 0.0), axis=(0.0, 1.0, 0.0), spectrum=spec, aperture=1,
                        normal=(0.0, 0.0, 1.0), half_azimuth=math.pi, half_polar=math.pi / 2)
    a = ora.solve(_one(w, iso), 0, tol=0.0, max_iters=1, n_threads=4).phi_u
    b = ora.solve(_one(w, fan), 0, tol=0.0, max_iters=1, n_threads=4).phi_u
    assert np.array_equal(a, b)


def test_fan_is_mirror_symmetric(ora):
    w = _homogeneous()
    fan = inputs.fan_sources(w.sources[0].spectrum, 1, half_azimuth=math.radians(9.0),
                             half_polar=math.radians(7.0))[0]
    u = ora.solve(_one(w, fan), 0, tol=0.0, max_iters=1, n_threads=4).phi_u
    u = u.reshape(w.n_groups, w.nz, w.ny, w.nx)
    assert u.max() > 0 and (u == 0).any()              # a beam, not the whole box
    assert np.allclose(u, u[:, ::-1, :, :], rtol=1e-12, atol=0)   # z -> -z (fan plane z = 0)
    assert np.allclose(u, u[:, :, :, ::-1], rtol=1e-12, atol=0)   # x -> -x (central ray on x = 0)


def test_fan_lit_voxels_match_the_enclosing_cone(ora):
    # a fan inside a cone of half-angle acos(cos(ha) cos(hp)) lights a subset of its voxels, with the
    # same uncollided values there (same point source, same ray)
    w = _homogeneous()
    ha, hp = math.radians(8.0), math.radians(5.0)
    fan = inputs.fan_sources(w.sources[0].spectrum, 1, half_azimuth=ha, half_polar=hp)[0]
    cone = inputs.ring_sources(w.sources[0].spectrum, 1, half_angle=math.acos(math.cos(ha) * math.cos(hp)) + 1e-9)[0]
    f = ora.solve(_one(w, fan), 0, tol=0.0, max_iters=1, n_threads=4).phi_u
    c = ora.solve(_one(w, cone), 0, tol=0.0, max_iters=1, n_threads=4).phi_u
    lit = f > 0
    assert lit.any() and (c[~lit] > 0).any()
    assert np.array_equal(f[lit], c[lit])


def _centres(w):
    z, y, x = np.meshgrid(w.z0 + (np.arange(w.nz) + 0.5) * w.dz, w.y0 + (np.arange(w.ny) + 0.5) * w.dy,
                          w.x0 + (np.arange(w.nx) + 0.5) * w.dx, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()])


def _lit_by_angles(w, k, n, ha, hp, vertical=False, distance=50.0):
    # independent of the projection form: rotate the voxel centres so that source k of a ring of n sits on
    # the -y axis looking along +y, then read elevation and azimuth off spherical coordinates
    a = 2.0 * math.pi * k / n
    rot = np.array([[math.cos(a), math.sin(a), 0.0], [-math.sin(a), math.cos(a), 0.0], [0.0, 0.0, 1.0]])
    x, y, z = rot @ _centres(w)
    y = y + distance
    if vertical:                     # fan plane normal to x: swap the roles of x and z
        x, z = z, x
    r = np.sqrt(x * x + y * y + z * z)
    elev, azim = np.arcsin(z / r), np.arctan2(x, y)
    inside = (np.abs(elev) <= hp) & (np.abs(azim) <= ha)
    margin = np.minimum(np.abs(np.abs(elev) - hp), np.abs(np.abs(azim) - ha))
    return inside, margin > 1e-9


def test_fan_cut_matches_spherical_angles(ora):
    w = _homogeneous(12, G=1)
    spec = w.sources[0].spectrum
    ha, hp = math.radians(11.0), math.radians(6.0)
    for k, n in ((0, 1), (1, 3), (5, 7)):
        fan = inputs.fan_sources(spec, n, half_azimuth=ha, half_polar=hp)[k]
        u = ora.solve(_one(w, fan), 0, tol=0.0, max_iters=1, n_threads=4).phi_u[0]
        inside, clear = _lit_by_angles(w, k, n, ha, hp)
        assert inside.any() and (~inside).any()
        assert np.array_equal(u[clear] > 0, inside[clear]), (k, n)
    # a vertical fan, its normal given off-perpendicular to the axis (only the part orthogonal to it counts)
    fan = inputs.fan_sources(spec, 1, half_azimuth=ha, half_polar=hp)[0]
    fan.normal = (1.0, 0.7, 0.0)
    u = ora.solve(_one(w, fan), 0, tol=0.0, max_iters=1, n_threads=4).phi_u[0]
    inside, clear = _lit_by_angles(w, 0, 1, ha, hp, vertical=True)
    assert inside.any()
    assert np.array_equal(u[clear] > 0, inside[clear])
