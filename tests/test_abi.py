"""The C ABI library builds, loads and exports every function include/rflbm.h declares;
host-side validation works without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "rflbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rflbm_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2507_08820_gb300 import build
    return ctypes.CDLL(build.build())


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name


def test_binding_wraps_every_declared_symbol(lib):
    from paper_2507_08820_gb300 import rflbm as R
    for name in _declared():
        assert callable(getattr(R, name)), name


def test_config_validation_without_gpu(lib):
    from paper_2507_08820_gb300 import rflbm as R
    cfg = R.rflbm_config_default()
    assert (cfg.nx, cfg.ny, cfg.nz, cfg.tau, cfg.omega_g) == (32, 32, 32, 0.8, 1.0)
    # 27 planes of 32768 floats
    assert R.rflbm_buffer_bytes(cfg) == 27 * 32768 * 4
    cfg.nx = 5  # plane stride rounded up to 64 elements
    assert R.rflbm_buffer_bytes(cfg) == 27 * ((5 * 32 * 32 + 63) // 64 * 64) * 4
    for field, bad in (("tau", 0.5), ("kT", -1.0), ("rho0", 0.0), ("omega_g", 2.0),
                       ("nx", 0), ("model", 7), ("storage", 9)):
        c = R.rflbm_config_default()
        setattr(c, field, bad)
        with pytest.raises(R.RflbmError) as e:
            R.rflbm_buffer_bytes(c)
        assert e.value.status == R.RFLBM_EINVAL
    c = R.rflbm_config_default()
    c.nx = c.ny = c.nz = 1300  # 2.2e9 sites > 2^31 - 1
    with pytest.raises(R.RflbmError):
        R.rflbm_buffer_bytes(c)


def test_null_handle_is_rejected(lib):
    from paper_2507_08820_gb300 import rflbm as R
    with pytest.raises(R.RflbmError) as e:
        R.rflbm_step(None, 1)
    assert e.value.status == R.RFLBM_EINVAL
    assert "NULL" in R.rflbm_last_error()
