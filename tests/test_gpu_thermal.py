"""The thermal initial state on the GPU: the same draw as the oracle's, the fluctuation-
dissipation variances of every mode at once, kept by the dynamics, and thermalised low-k
shells where a start from rest would need long runs (small viscosity)."""
import numpy as np
import pytest

from oracle import rflbm_oracle as o

pytestmark = pytest.mark.gpu
POP_RTOL = 1e-5
U = {1: 2.0 ** -11, 2: 2.0 ** -8}


@pytest.fixture(scope="module")
def R():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_08820_gb300 import build
    build.build()
    from paper_2507_08820_gb300 import rflbm
    return rflbm


@pytest.mark.parametrize("shape,kernel", [((13, 6, 5), 0), ((64, 6, 5), 2)])
@pytest.mark.parametrize("storage", [0, 1, 2])
@pytest.mark.parametrize("pattern", [0, 1])
def test_thermal_state_matches_the_oracle(R, shape, kernel, storage, pattern):
    n = int(np.prod(shape))
    kT, seed, replica = 3e-4, 12345678901, 2
    box = R.Box(*shape, tau=0.8, kT=kT, seed=seed, replica=replica, kernel=kernel, storage=storage,
                pattern=pattern)
    R.rflbm_init_thermal(box.h)
    got = box.populations()
    assert R.rflbm_get_step(box.h) == 0
    box.close()
    want = o.thermal_state(kT, seed, np.arange(n), replica=replica)
    w = o.weights()[:, None]
    if storage == 0:
        assert np.max(np.abs(got - want) / np.maximum(np.abs(want), w)) < POP_RTOL
    else:
        bound = 1.05 * U[storage] * np.abs(want - w) + 1e-6 * w
        assert np.all(np.abs(got - want) <= bound)


def _mode_variances(R, box, n):
    s1, s2 = R.rflbm_mode_sums(box.h)
    return s2 / n - (s1 / n) ** 2


@pytest.mark.parametrize("pattern", [0, 1])
def test_thermal_state_has_and_keeps_the_fdt_variances(R, pattern):
    L, kT = 64, 1e-4
    n = L ** 3
    theory = o.fdt_mode_variance(1.0, kT)
    box = R.Box(L, L, L, tau=0.8, kT=kT, seed=4, pattern=pattern)
    R.rflbm_init_thermal(box.h)
    v0 = _mode_variances(R, box, n) / theory
    R.rflbm_step(box.h, 1000)
    v1 = _mode_variances(R, box, n) / theory
    box.close()
    assert np.all(np.abs(v0 - 1.0) < 0.01), v0
    assert np.all(np.abs(v1 - 1.0) < 0.015), v1


def _low_k_ratio(R, box, field, theory, lo=1, hi=4):
    ns = R.rflbm_shell_count(box.h)
    s, count = R.rflbm_structure_factor(box.h, field, ns)
    return s[lo:hi].sum() / count[lo:hi].sum() / theory


def test_low_k_shells_start_thermalised(R):
    """At tau = 0.51 (nu = 1/300) the transverse momentum of the lowest shells relaxes over
    ~10^4 steps: from rest it is far below rho0 kT after 200 steps, from the thermal state it
    is at rho0 kT from the start."""
    L, kT, tau = 64, 1e-4, 0.51
    ratios = {}
    for start in ("rest", "thermal"):
        acc = 0.0
        box = R.Box(L, L, L, tau=tau, kT=kT, seed=8)
        (R.rflbm_init_rest if start == "rest" else R.rflbm_init_thermal)(box.h)
        R.rflbm_step(box.h, 200)
        for k in (1, 2, 3):  # rho u_x, rho u_y, rho u_z
            acc += _low_k_ratio(R, box, k, kT) / 3.0
        box.close()
        ratios[start] = acc
    assert ratios["rest"] < 0.6, ratios
    assert abs(ratios["thermal"] - 1.0) < 0.1, ratios
