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


def test_expired_copy_wait_reports_timeout_and_recovers(R):
    box = R.Box(32, 1, 1, tau=0.8, kT=1e-4, seed=3)  # one CTA of 32 sites
    assert R.rflbm_step_path(box.h) == (R.RFLBM_KERNEL_TMA, 32)
    R.rflbm_init_rest(box.h)
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
    assert status == R.RFLBM_OK and abs(st.mass - 32.0) < 1e-5
    f = box.populations()
    assert np.all(np.isfinite(f))
    with pytest.raises(R.RflbmError):
        R.rflbm_testing_expect_extra_bytes(box.h, 1 << 21)
    box.close()
