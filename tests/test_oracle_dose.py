"""Fluence-to-dose post-processing in the oracle (collision-kerma form) against
closed forms and the SI definition of the conversion constant."""
import numpy as np

from paper_1910_11335_b300 import inputs


def test_conversion_constant_is_one_mev_per_gram(ora):
    e_charge = 1.602176634e-19            # C (exact SI value): 1 eV = e J
    assert abs(ora.MEV_PER_G_TO_GY - e_charge * 1e6 / 1e-3) <= 1e-15 * ora.MEV_PER_G_TO_GY


def test_dose_closed_form_one_group_one_material(ora):
    V = 10
    phi = np.full((1, V), 3.0e-4)          # photons/cm^2 per source particle
    mat = np.zeros(V, dtype=np.int32)
    mu = np.array([[0.0265]])              # cm^2/g
    e = np.array([0.1])                    # MeV
    d = ora.dose(phi, mat, mu, e)
    assert np.allclose(d, 3.0e-4 * 0.1 * 0.0265 * 1.602176634e-10, rtol=1e-15, atol=0)


def test_dose_per_material_and_group(ora):
    # two materials, two groups, one voxel each: every (group, material) term by hand
    phi = np.array([[1.0, 2.0], [4.0, 8.0]])
    mat = np.array([1, 0], dtype=np.int32)
    mu = np.array([[0.5, 0.25], [3.0, 1.0]])
    e = np.array([0.08, 0.03])
    d = ora.dose(phi, mat, mu, e) / ora.MEV_PER_G_TO_GY
    assert np.allclose(d, [1.0 * 0.08 * 3.0 + 4.0 * 0.03 * 1.0, 2.0 * 0.08 * 0.5 + 8.0 * 0.03 * 0.25],
                       rtol=1e-15, atol=0)


def test_synthetic_coefficients_are_plausible():
    w = inputs.small_cone(6, 5, 4, n_groups=5)
    mu, e = inputs.dose_coefficients(w)
    assert mu.shape == (w.sigma_t.shape[0], 5) and e.shape == (5,)
    assert np.all(mu > 0)
    order = np.argsort(e)
    assert np.all(np.diff(mu[:, order], axis=1) < 0)      # falls with energy
    assert np.all(mu[2:] > mu[inputs.MAT_WATER])           # bone-like above water
