"""Pins of the oracle's time step against what the physics fixes: conservation,
streaming direction, fixed points, the regularisation itself, the Taylor-Green viscous
decay at nu = cs2 (tau - 1/2) (Sec. II.A) and the fluctuation-dissipation variances the
noise amplitude of Eq. 10 is built to sustain."""
import numpy as np
import pytest

from oracle import rflbm_oracle as o
from paper_2507_08820_gb300 import workloads as W


def _random_state(shape, seed, du=0.05, amp=1e-3):
    n = int(np.prod(shape))
    rho, u = W.random_fields(*shape, seed=seed, drho=0.05, du=du)
    return o.equilibrium_state(rho, u) + W.population_perturbation(n, seed + 1, amp)


def test_stream_moves_each_population_by_its_velocity_with_periodic_wrap():
    shape = (5, 4, 3)
    nx, ny, nz = shape
    c = o.velocities()
    for x0, y0, z0 in ((0, 0, 0), (4, 3, 2), (2, 1, 1)):
        f = np.zeros((27, nx * ny * nz))
        s0 = x0 + nx * (y0 + ny * z0)
        f[:, s0] = np.arange(1, 28)
        g = o.stream(f, shape)
        for i in range(27):
            x, y, z = (x0 + c[i, 0]) % nx, (y0 + c[i, 1]) % ny, (z0 + c[i, 2]) % nz
            s = x + nx * (y + ny * z)
            assert g[i, s] == i + 1 and np.count_nonzero(g[i]) == 1


@pytest.mark.parametrize("model", ["reg", "bgk"])
def test_collision_conserves_mass_and_momentum_per_site(model):
    f = _random_state((4, 3, 5), seed=10)
    sites = np.arange(f.shape[1])
    fs = o.collide(f, 0.7, 1e-4, seed=3, step=5, sites=sites, model=model)
    assert np.allclose(o.density(fs), o.density(f), rtol=1e-14, atol=0)
    assert np.allclose(o.momentum(fs), o.momentum(f), rtol=0, atol=1e-15)


@pytest.mark.parametrize("model,omega_g", [("reg", 1.0), ("reg", 0.8), ("bgk", 1.0)])
def test_global_mass_and_momentum_conserved_over_steps(model, omega_g):
    shape = (6, 5, 4)
    f = _random_state(shape, seed=20)
    m0, j0 = f.sum(), o.momentum(f).sum(axis=1)
    f = o.run(f, shape, 0.6, 1e-3, seed=9, steps=5, model=model, omega_g=omega_g)
    assert abs(f.sum() - m0) / m0 < 1e-13
    assert np.allclose(o.momentum(f).sum(axis=1), j0, rtol=0, atol=1e-12)


def test_rest_state_is_stationary_without_noise():
    shape = (4, 4, 4)
    f0 = o.rest_state(64, rho0=1.3)
    f = o.run(f0, shape, 0.8, 0.0, seed=1, steps=3)
    assert np.allclose(f, f0, rtol=1e-15, atol=0)


def test_uniform_flow_is_a_fixed_point_without_noise():
    shape = (3, 4, 5)
    n = 60
    rho = np.full(n, 1.1)
    u = np.tile(np.array([[0.05], [-0.03], [0.02]]), (1, n))
    f0 = o.equilibrium_state(rho, u)
    f = o.run(f0, shape, 0.55, 0.0, seed=1, steps=4)
    assert np.allclose(f, f0, rtol=0, atol=1e-15)


@pytest.mark.parametrize("model", ["reg", "bgk"])
def test_unit_relaxation_returns_the_equilibrium(model):
    """omega = 1 without noise: f* = f^(0) for both models (Eqs. 12, 25)."""
    f = _random_state((3, 3, 3), seed=30)
    fs = o.collide(f, 1.0, 0.0, 1, 0, np.arange(27), model=model)
    rho, u, _ = o.macroscopic(f)
    assert np.allclose(fs, o.hermite_equilibrium(rho, u), rtol=0, atol=1e-15)


def test_regularisation_keeps_only_equilibrium_ghosts_and_relaxes_stress():
    """Reg-FLBM with omega_g = 1 and no noise: post-collision ghost moments are the
    equilibrium ones rho u^p u^q u^r (the raw ghost non-equilibrium is discarded), the
    stress modes relax as a_0 + (1 - omega)(m - a_0), conserved moments are kept."""
    tau = 0.7
    f = _random_state((3, 3, 3), seed=40, amp=5e-3)
    rho, u, _ = o.macroscopic(f)
    fs = o.collide(f, tau, 0.0, 1, 0, np.arange(27))
    m, ms = o.moments(f), o.moments(fs)
    for k, seq in enumerate(o.MODE_SEQ):
        p, q, r = (seq.count(a) for a in "xyz")
        a0 = rho * u[0] ** p * u[1] ** q * u[2] ** r
        if k < 4:
            want = m[k]
        elif k < 10:
            want = a0 + (1 - 1 / tau) * (m[k] - a0)
        else:
            want = a0
        assert np.allclose(ms[k], want, rtol=0, atol=1e-15), k
    # and the raw ghost non-equilibrium of the input was far from zero
    a0g = np.array([rho * u[0] ** s.count("x") * u[1] ** s.count("y") * u[2] ** s.count("z")
                    for s in o.MODE_SEQ[10:]])
    assert np.abs(m[10:] - a0g).max() > 1e-3


def test_noise_enters_only_non_conserved_modes_with_eq10_amplitude():
    """The difference between a noisy and a noiseless collision has zero mass and
    momentum and, in mode k >= 4, equals phi_k r_k with the normals drawn for the site
    and rho the local density."""
    tau, kT, seed, step = 0.9, 2e-4, 11, 7
    f = _random_state((3, 2, 2), seed=50)
    sites = np.arange(12)
    d = (o.collide(f, tau, kT, seed, step, sites)
         - o.collide(f, tau, 0.0, seed, step, sites))
    dm = o.moments(d)
    assert np.allclose(dm[:4], 0, atol=1e-16)
    r = o.normals(seed, step, sites)
    rho, b, w = o.density(f), o.norms(), 1.0 / tau
    for k in range(4, 27):
        om = w if k < 10 else 1.0
        phi = np.sqrt(rho * kT * om * (2 - om) * b[k] * 3.0)
        assert np.allclose(dm[k], phi * r[k - 4], rtol=1e-12, atol=1e-17), k


def _tg_rate(L, tau, steps=600, fit_from=100):
    shape = (L, L, 1)
    rho, u = W.taylor_green_fields(L, L, 1, u0=0.01)
    f = o.equilibrium_state(rho, u)
    x, y, _ = W.site_coords(L, L, 1)
    k = 2 * np.pi / L
    prof = -np.cos(k * x) * np.sin(k * y)
    amp = []
    for t in range(steps):
        ux = o.momentum(f)[0] / o.density(f)
        amp.append((ux * prof).sum() / (prof * prof).sum())
        f = o.step(f, shape, tau, 0.0, 1, t)
    slope = np.polyfit(np.arange(fit_from, steps), np.log(amp[fit_from:]), 1)[0]
    return -slope, 2 * o.CS2 * (tau - 0.5) * k * k


@pytest.mark.slow
@pytest.mark.parametrize("tau", [0.6, 0.8])
def test_taylor_green_decays_at_the_bgk_viscosity(tau):
    """Without noise the vortex amplitude decays as exp(-2 nu k^2 t) with
    nu = cs2 (tau - 1/2) (Sec. II.A): fitted rate within 1% on a 32x32 periodic box."""
    rate, theory = _tg_rate(32, tau)
    assert abs(rate / theory - 1) < 0.01, (rate, theory)


def _equilibrium_run(model, tau, kT, L=8, burn=250, samples=1000, seed=7):
    shape = (L, L, L)
    n = L ** 3
    f = o.rest_state(n)
    E = o.basis()
    acc = np.zeros(27)
    sk = np.zeros((4, L, L, L))
    for t in range(burn + samples):
        f = o.step(f, shape, tau, kT, seed, t, model=model)
        if t >= burn:
            m = E @ f
            m[0] -= 1.0
            acc += (m * m).mean(axis=1)
            for a in range(4):
                F = np.fft.fftn(m[a].reshape(L, L, L))
                sk[a] += (F * np.conj(F)).real / n
    return acc / samples, sk / samples


@pytest.mark.slow
@pytest.mark.parametrize("model", ["reg", "bgk"])
def test_fluctuation_dissipation_mode_variances_and_flat_structure_factor(model):
    """At equilibrium every mode of every site fluctuates with variance
    rho0 kT b_k / cs2 (the detailed-balance amplitude of Eq. 10), conserved modes times
    (1 - 1/N) because the k = 0 Fourier mode is frozen; the static structure factors of
    rho and j are flat, S(k) = rho0 kT / cs2 and rho0 kT, at every k != 0."""
    kT = 1e-4
    var, sk = _equilibrium_run(model, tau=0.8, kT=kT)
    n = 8 ** 3
    theory = o.fdt_mode_variance(1.0, kT)
    theory[:4] *= 1.0 - 1.0 / n
    assert np.all(np.abs(var / theory - 1) < 0.015), var / theory
    s_theory = np.array([kT / o.CS2, kT, kT, kT])
    for a in range(4):
        s = sk[a].ravel()[1:]          # drop k = 0
        assert abs(s.mean() / s_theory[a] - 1) < 0.02
        # low and high |k| halves are both flat
        kk = np.fft.fftfreq(8)
        kmag = np.sqrt(sum(np.meshgrid(kk, kk, kk, indexing="ij")[i] ** 2 for i in range(3)))
        kmag = kmag.ravel()[1:]
        lo, hi = s[kmag < np.median(kmag)], s[kmag >= np.median(kmag)]
        assert abs(lo.mean() / s_theory[a] - 1) < 0.04
        assert abs(hi.mean() / s_theory[a] - 1) < 0.04


def test_advection_direction_of_a_density_pulse():
    """A density pulse in a uniform flow splits into two sound pulses moving at
    u - cs and u + cs; their mass centroid therefore moves at u (sign of Eq. 8)."""
    L, u0, steps = 96, 0.1, 30
    shape = (L, 1, 1)
    x = np.arange(L)
    rho = 1.0 + 1e-4 * np.exp(-((x - 48.0) ** 2) / 8.0)
    u = np.zeros((3, L))
    u[0] = u0
    f = o.equilibrium_state(rho, u)
    f = o.run(f, shape, 0.8, 0.0, seed=1, steps=steps)
    d = o.density(f) - 1.0
    centroid = (x * d).sum() / d.sum()
    assert abs(centroid - (48.0 + u0 * steps)) < 0.15, centroid
