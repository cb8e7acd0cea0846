"""Pins of the oracle's thermal initial state against what the fluctuation-dissipation
balance fixes: every mode of every site an independent normal of variance
rho0 kT b_k / cs2 (the variance the amplitude of Eq. 10 maintains), and a state the
dynamics keep stationary."""
import numpy as np

from oracle import rflbm_oracle as o


def test_zero_temperature_gives_the_rest_state():
    f = o.thermal_state(0.0, 7, np.arange(100), rho0=1.3)
    assert np.array_equal(f, o.rest_state(100, 1.3))


def test_mode_statistics_of_the_draw():
    kT, rho0, m_sites = 2e-4, 1.1, 200_000
    f = o.thermal_state(kT, 3, np.arange(m_sites), rho0=rho0)
    m = o.moments(f - o.rest_state(m_sites, rho0))
    theory = o.fdt_mode_variance(rho0, kT)
    var = m.var(axis=1)
    assert np.all(np.abs(var / theory - 1.0) < 0.015), var / theory
    # zero means, no correlation between modes
    assert np.all(np.abs(m.mean(axis=1)) < 5.0 * np.sqrt(theory / m_sites))
    corr = np.corrcoef(m)
    assert np.max(np.abs(corr - np.eye(27))) < 0.015
    # independent draws for different seeds, replicas and sites
    g = o.thermal_state(kT, 4, np.arange(10), rho0=rho0)
    h = o.thermal_state(kT, 3, np.arange(10), rho0=rho0, replica=1)
    assert not np.allclose(g, f[:, :10]) and not np.allclose(h, f[:, :10])


def _normalised_variances(f, n_sites, kT):
    m = o.moments(f - o.rest_state(n_sites))
    return (m.var(axis=1) / o.fdt_mode_variance(1.0, kT))


def test_dynamics_keep_the_thermal_state_stationary():
    """Five Reg-FLBM steps from the thermal state leave every mode at the FDT variance."""
    L, kT, tau = 12, 1e-4, 0.8
    shape, n = (L, L, L), L ** 3
    f = o.thermal_state(kT, 11, np.arange(n))
    assert abs(_normalised_variances(f, n, kT).mean() - 1.0) < 0.02
    f = o.run(f, shape, tau, kT, 11, 5)
    v = _normalised_variances(f, n, kT)
    assert abs(v.mean() - 1.0) < 0.02 and np.all(np.abs(v - 1.0) < 0.15), v
