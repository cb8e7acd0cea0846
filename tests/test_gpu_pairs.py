"""The two-site form of the TMA step kernels (two adjacent sites per thread, packed f32x2
arithmetic), ping-pong and AA: where it runs, and that it computes every site bit for bit
like the one-site general gather kernels (and, in test_gpu_aa.py, like the one-site AA
kernels of the float32 fluctuating step)."""
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


def _state(shape, seed=21):
    n = int(np.prod(shape))
    rho, u = W.random_fields(*shape, seed=seed, drho=0.02, du=0.03)
    return np.ascontiguousarray(o.equilibrium_state(rho, u) + W.population_perturbation(n, seed + 1, 2e-4))


@pytest.mark.parametrize("kw,pairs", [
    (dict(kT=1e-4), 1), (dict(kT=0.0), 2), (dict(kT=1e-4, storage=1), 2), (dict(kT=0.0, storage=1), 2),
    (dict(kT=1e-4, storage=2), 2), (dict(kT=0.0, storage=2), 2), (dict(kT=1e-4, model=1), 1),
    (dict(kT=0.0, model=1, storage=1), 1), (dict(kT=0.0, omega_g=0.7), 1), (dict(kT=1e-4, phi_rho=1), 1),
    (dict(kT=0.0, phi_rho=1), 2), (dict(kT=0.0, pattern=1), 2), (dict(kT=1e-4, storage=1, pattern=1), 2),
    (dict(kT=1e-4, pattern=1), 1), (dict(kT=1e-4, model=1, storage=2, pattern=1), 1),
    (dict(kT=0.0, kernel=1), 1), (dict(kT=1e-4, storage=1, kernel=1), 1),
    (dict(kT=0.0, kernel=1, pattern=1), 1),
])
def test_sites_per_thread(R, kw, pairs):
    box = R.Box(128, 3, 2, tau=0.8, **kw)
    assert R.rflbm_step_sites_per_thread(box.h) == pairs
    box.close()


@pytest.mark.parametrize("nx,odd_pairs", [(128, 1), (256, 2)])
def test_float32_fluctuating_aa_odd_steps(R, nx, odd_pairs):
    """The odd AA steps of the float32 fluctuating step run two sites per thread where
    they store straight to the neighbours (rows of several segments), one where a segment
    is a whole row; the even steps one."""
    box = R.Box(nx, 3, 2, tau=0.8, kT=1e-4, pattern=1)
    R.rflbm_init_rest(box.h)
    assert R.rflbm_step_sites_per_thread(box.h) == 1
    R.rflbm_step(box.h, 1)
    assert R.rflbm_step_sites_per_thread(box.h) == odd_pairs
    R.rflbm_step(box.h, 1)
    assert R.rflbm_step_sites_per_thread(box.h) == 1
    box.close()


# the last four with ragged last segments in ping-pong (16-bit storage: 104 and 200; 100 and
# 300 are no whole 16-byte units there and run the gather kernel on both sides)
SHAPES = [(32, 5, 4), (64, 6, 5), (96, 4, 3), (128, 3, 3), (192, 3, 2), (256, 3, 2), (160, 3, 2),
          (100, 5, 4), (104, 4, 3), (200, 3, 2), (300, 2, 2)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("kw", [dict(kT=0.0), dict(kT=1e-4, storage=1), dict(kT=0.0, storage=1),
                                dict(kT=3e-4, storage=2), dict(kT=0.0, storage=2), dict(kT=1e-4)])
@pytest.mark.parametrize("pattern", [0, 1])
def test_two_site_form_matches_the_gather_kernel_bitwise(R, shape, kw, pattern):
    """Ping-pong and AA (whose odd steps store whole rows where a segment is a row, else
    straight to the neighbours), after 1, 2, 4 and 7 steps (both AA parities)."""
    f0 = _state(shape, seed=7)
    out = []
    for kernel in (R.RFLBM_KERNEL_TMA, R.RFLBM_KERNEL_GATHER):
        box = R.Box(*shape, tau=0.7, seed=3, kernel=kernel, pattern=pattern, **kw)
        if kernel == R.RFLBM_KERNEL_GATHER:
            assert R.rflbm_step_sites_per_thread(box.h) == 1
        R.rflbm_set_populations(box.h, f0)
        R.rflbm_set_step(box.h, 5)
        snaps = []
        for steps in (1, 1, 2, 3):
            R.rflbm_step(box.h, steps)
            f = np.empty((27, box.n), np.float32)
            R.rflbm_get_populations_f32(box.h, f)
            snaps.append(f)
        out.append(snaps)
        box.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b), float(np.max(np.abs(a - b)))
