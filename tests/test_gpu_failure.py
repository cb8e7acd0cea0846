"""Failure detection on the GPU without a fault: a step whose copy barrier is made to wait
for bytes that never arrive (testing hook) gives up after its bounded wait, the host sees
RFLBM_ETIMEOUT, and the context and the handle stay usable."""
import time

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


@pytest.mark.parametrize("nx,kw,pre_steps,pairs", [
    (32, dict(kT=1e-4), 0, 1),                      # one-site ping-pong step, one CTA
    (32, dict(kT=1e-4, storage=1), 0, 2),           # two-site ping-pong step
    (32, dict(kT=1e-4, pattern=1), 0, 1),           # AA even step
    (32, dict(kT=1e-4, pattern=1), 1, 1),           # AA odd step, whole-row stores
    (32, dict(kT=0.0, storage=1, pattern=1), 0, 2),  # two-site AA even step
    (256, dict(kT=1e-4, pattern=1), 1, 2),          # two-site AA odd step, direct stores
])
def test_expired_copy_wait_reports_timeout_and_recovers(R, nx, kw, pre_steps, pairs):
    box = R.Box(nx, 1, 1, tau=0.8, seed=3, **kw)
    assert R.rflbm_step_path(box.h)[0] == R.RFLBM_KERNEL_TMA
    R.rflbm_init_rest(box.h)
    R.rflbm_step(box.h, pre_steps)
    assert R.rflbm_step_sites_per_thread(box.h) == pairs
    R.rflbm_testing_expect_extra_bytes(box.h, 16)
    t0 = time.time()
    R.rflbm_step(box.h, 1)
    with pytest.raises(R.RflbmError) as e:
        R.rflbm_synchronize(box.h)
    assert e.value.status == R.RFLBM_ETIMEOUT
    assert time.time() - t0 < 60.0
    # the flag is cleared by the report; normal steps work again on a re-initialised state
    R.rflbm_testing_expect_extra_bytes(box.h, 0)
    R.rflbm_init_rest(box.h)
    R.rflbm_step(box.h, 5)
    R.rflbm_synchronize(box.h)
    st, status = R.rflbm_stats(box.h)
    assert status == R.RFLBM_OK and abs(st.mass - nx) < 1e-5 * nx
    f = box.populations()
    assert np.all(np.isfinite(f))
    with pytest.raises(R.RflbmError):
        R.rflbm_testing_expect_extra_bytes(box.h, 1 << 21)
    box.close()
