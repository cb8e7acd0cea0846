"""The back transform of Eq. 11 on the tensor cores against the float32 FMA form of the step
kernels (include/rflbm_testing.h): both against f_i = w_i sum_k e_ki M_k in FP64, with
e_ki = h_p(c_x) h_q(c_y) h_r(c_z), h = (1, c, c^2 - 1/3) (Table II) and the lattice weights of
Table I. The FMA form is float32-exact to a few units in the last place; the MMA form carries
the moments as a bfloat16 high part plus a bfloat16 remainder (about 16 significant bits)."""
import itertools

import numpy as np
import pytest

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


def _reference(M):
    h = lambda p, c: (1.0, float(c), c * c - 1.0 / 3.0)[p]  # noqa: E731
    W = {-1: 1.0 / 6.0, 0: 2.0 / 3.0, 1: 1.0 / 6.0}
    f = np.zeros_like(M, dtype=np.float64)
    for i, (a, b, c) in enumerate(itertools.product((-1, 0, 1), repeat=3)):
        w = W[a] * W[b] * W[c]
        for k, (p, q, r) in enumerate(itertools.product(range(3), repeat=3)):
            f[i] += w * h(p, a) * h(q, b) * h(r, c) * M[k]
    return f


def test_mma_back_transform_matches_the_fma_form(R):
    g = np.random.default_rng(5)
    n = 128 * 48
    M = g.normal(0.0, 1.0, (27, n)).astype(np.float32) * np.float32(1e-2)
    M[0] += np.float32(0.05)
    want = _reference(M.astype(np.float64))
    scale = np.max(np.abs(want))
    f_fma = R.rflbm_testing_backtransform(0, M)
    f_mma = R.rflbm_testing_backtransform(1, M)
    err_fma = np.max(np.abs(f_fma - want)) / scale
    err_mma = np.max(np.abs(f_mma - want)) / scale
    assert err_fma < 1e-6, err_fma
    # the high part alone (8 significant bits) would miss by about 2^-9
    assert err_mma < 1e-4, err_mma


def test_both_forms_time(R):
    for method in (0, 1):
        assert R.rflbm_testing_backtransform_time(method, 152 * 4, 4) > 0.0


def test_noise_draw_alone_times(R):
    assert R.rflbm_testing_noise_time(1 << 20) > 0.0


def _raw_moments(f):
    """m_pqr = sum_i f_i c_x^p c_y^q c_z^r for the ten exponent triples of order <= 2, in FP64."""
    exps = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (0, 2, 0), (0, 0, 2),
            (1, 1, 0), (1, 0, 1), (0, 1, 1)]
    m = np.zeros((10, f.shape[1]))
    for i, (a, b, c) in enumerate(itertools.product((-1, 0, 1), repeat=3)):
        for k, (p, q, r) in enumerate(exps):
            m[k] += float(a) ** p * float(b) ** q * float(c) ** r * f[i]
    return m


def test_mma_forward_projection_is_exact_for_float16_populations(R):
    """Populations that are float16 values (as 16-bit storage gives them): the tensor-core
    projection with float16 operands and float32 accumulation equals the FP64 moments within
    float32 accumulation, and so does the FMA form."""
    g = np.random.default_rng(7)
    n = 128 * 40
    f = (g.normal(0.0, 1e-2, (27, n)) + 1.0 / 27.0).astype(np.float16).astype(np.float32)
    want = _raw_moments(f.astype(np.float64))
    scale = np.max(np.abs(want))
    for method in (0, 1):
        got = R.rflbm_testing_forward(method, f)
        err = np.max(np.abs(got - want)) / scale
        assert err < 2e-6, (method, err)


def test_forward_forms_time(R):
    for method in (0, 1):
        assert R.rflbm_testing_forward_time(method, 152 * 4, 4) > 0.0
