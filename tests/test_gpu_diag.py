"""Equilibrium statistics and hydrodynamics of the CUDA path at the paper's scale.

1. The diagnostics themselves (per-mode sums, structure factors) against the oracle's
   moments and numpy's FFT on the same state.
2. The thermal-equilibrium configuration on a periodic 128^3 box, tau in {0.6, 0.8, 1.0}
   x kT in {1e-5, 1e-4, 1e-3}, rest start, 2e4 steps: every Table II mode fluctuates per
   site with variance rho0 kT b_k / cs2 (the fluctuation-dissipation amplitude of Eq. 10),
   and the static structure factors of rho, rho u and Pi are flat at rho0 kT / cs2,
   rho0 kT, 2 rho0 kT cs2 and rho0 kT cs2 (Sec. III); tolerance 2 %.
3. Without noise, the Taylor-Green vortex on the 128^3 box (u0 = 0.02, k = 2 pi / 128)
   decays at 2 nu k^2 with nu = cs2 (tau - 1/2) (Sec. II.A); tolerance 1 %.
"""
import numpy as np
import pytest

from oracle import rflbm_oracle as o
from paper_2507_08820_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_08820_gb300 import build
    build.build()
    from paper_2507_08820_gb300 import rflbm
    return rflbm


def _shells_numpy(field, shape, nshell):
    """Shell sums of |F|^2 / N, shell = round(|k| L / 2 pi), L = max edge (full spectrum)."""
    nx, ny, nz = shape
    F = np.fft.fftn(field.reshape(nz, ny, nx))
    S = (F * np.conj(F)).real / field.size
    fz = np.fft.fftfreq(nz)[:, None, None]
    fy = np.fft.fftfreq(ny)[None, :, None]
    fx = np.fft.fftfreq(nx)[None, None, :]
    shell = np.rint(max(shape) * np.sqrt(fx ** 2 + fy ** 2 + fz ** 2)).astype(int)
    s = np.bincount(shell.ravel(), weights=S.ravel(), minlength=nshell)[:nshell]
    c = np.bincount(shell.ravel(), minlength=nshell)[:nshell].astype(float)
    return s, c


def test_diagnostics_match_oracle_on_the_same_state(R):
    shape = (12, 10, 8)
    n = int(np.prod(shape))
    rho, u = W.random_fields(*shape, seed=41, drho=0.02, du=0.02)
    f0 = o.equilibrium_state(rho, u) + W.population_perturbation(n, 42, 1e-3)
    box = R.Box(*shape, tau=0.8)
    R.rflbm_set_populations(box.h, np.ascontiguousarray(f0))
    f = box.populations()
    s1, s2 = R.rflbm_mode_sums(box.h)
    m = o.moments(f)
    m[0] -= 1.0
    assert np.allclose(s1, m.sum(axis=1), rtol=0, atol=1e-6 * np.abs(m).sum(axis=1).max())
    assert np.allclose(s2, (m * m).sum(axis=1), rtol=1e-5, atol=1e-12)
    r, j, pi = o.macroscopic(f)
    fields = [r - 1.0, j[0] * r, j[1] * r, j[2] * r, *pi]
    ns = R.rflbm_shell_count(box.h)
    for k, phi in enumerate(fields):
        got_s, got_c = R.rflbm_structure_factor(box.h, k, ns)
        want_s, want_c = _shells_numpy(phi, shape, ns)
        assert np.array_equal(got_c, want_c), k
        assert np.allclose(got_s, want_s, rtol=1e-5, atol=1e-6 * want_s.max()), k
    box.close()


B = np.array([1, 1 / 3, 1 / 3, 1 / 3, 2 / 9, 2 / 9, 2 / 9, 1 / 9, 1 / 9, 1 / 9] + [2 / 27] * 6
             + [1 / 27] + [4 / 81] * 3 + [2 / 81] * 3 + [4 / 243] * 3 + [8 / 729])


@pytest.mark.parametrize("kT", [1e-5, 1e-4, 1e-3])
@pytest.mark.parametrize("tau", [0.6, 0.8, 1.0])
def test_fluctuation_dissipation_at_128cubed(R, tau, kT):
    L, burn, every, total = 128, 3000, 100, 20000
    n = L ** 3
    box = R.Box(L, L, L, tau=tau, kT=kT, seed=1)
    R.rflbm_init_rest(box.h)
    R.rflbm_step(box.h, burn)
    ns = R.rflbm_shell_count(box.h)
    var = np.zeros(27)
    S = np.zeros((10, ns))
    count = None
    snaps = 0
    for _ in range(burn, total, every):
        R.rflbm_step(box.h, every)
        s1, s2 = R.rflbm_mode_sums(box.h)
        var += s2 / n - (s1 / n) ** 2
        for k in range(10):
            s, count = R.rflbm_structure_factor(box.h, k, ns)
            S[k] += s
        snaps += 1
    box.close()
    var /= snaps
    S /= snaps
    # per-site mode variances: rho0 kT b_k / cs2, conserved modes times (1 - 1/N)
    theory = 3.0 * kT * B
    theory[:4] *= 1.0 - 1.0 / n
    assert np.all(np.abs(var / theory - 1.0) < 0.02), var / theory
    # structure factors, scored over the shells 4 <= |n| <= 32 in three bands
    s_theory = np.array([3 * kT, kT, kT, kT, 2 * kT / 3, 2 * kT / 3, 2 * kT / 3,
                         kT / 3, kT / 3, kT / 3])
    shell = np.arange(ns)
    for lo, hi in ((4, 8), (8, 16), (16, 33)):
        band = (shell >= lo) & (shell < hi)
        er = S[:, band].sum(axis=1) / count[band].sum() / s_theory
        assert np.all(np.abs(er - 1.0) < 0.02), (lo, hi, er)


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.0])
def test_taylor_green_decay_at_128cubed(R, tau):
    L = 128
    n = L ** 3
    rho, u = W.taylor_green_fields(L, L, L, u0=0.02)
    box = R.Box(L, L, L, tau=tau, kT=0.0)
    R.rflbm_init_field(box.h, rho, np.ascontiguousarray(u))
    x, y, _ = W.site_coords(L, L, L)
    k = 2 * np.pi / L
    prof = -np.cos(k * x) * np.sin(k * y)
    uu = np.empty((3, n))
    ts, amps = [], []
    for t in range(0, 3001, 100):
        if t:
            R.rflbm_step(box.h, 100)
        R.rflbm_moments(box.h, None, uu, None)
        ts.append(t)
        amps.append((uu[0] * prof).sum() / (prof * prof).sum())
    box.close()
    rate = -np.polyfit(ts[2:], np.log(amps[2:]), 1)[0]
    theory = 2.0 * o.CS2 * (tau - 0.5) * k * k
    assert abs(rate / theory - 1.0) < 0.01, (rate, theory)
