"""The C ABI library builds, loads and exports every function include/rflbm.h declares;
host-side validation works without a GPU."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for header in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        text = re.sub(r"/\*.*?\*/", "", open(header).read(), flags=re.S)
        names.update(re.findall(r"\b(rflbm_\w+)\s*\(", text))
    return sorted(names)


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


def test_config_struct_mirror_matches_the_library(lib):
    from paper_2507_08820_gb300 import rflbm as R
    assert R.rflbm_config_size() == ctypes.sizeof(R.rflbm_config_t)
    cfg = R.rflbm_config_default()
    assert (cfg.pattern, cfg.kernel, cfg.device) == (R.RFLBM_PATTERN_PINGPONG, R.RFLBM_KERNEL_AUTO, -1)


def test_aa_pattern_validation_without_gpu(lib):
    from paper_2507_08820_gb300 import rflbm as R
    cfg = R.rflbm_config_default()
    cfg.pattern = R.RFLBM_PATTERN_AA
    for storage in (R.RFLBM_STORE_F32, R.RFLBM_STORE_F16, R.RFLBM_STORE_BF16):
        cfg.storage = storage
        assert R.rflbm_buffer_bytes(cfg) == 27 * 32768 * (4 if storage == 0 else 2)
    cfg.storage = R.RFLBM_STORE_F32
    for field, bad in (("pattern", 2), ("omega_g", 0.8), ("phi_rho", R.RFLBM_PHI_RHO0)):
        c = R.rflbm_config_default()
        c.pattern = R.RFLBM_PATTERN_AA
        setattr(c, field, bad)
        with pytest.raises(R.RflbmError) as e:
            R.rflbm_buffer_bytes(c)
        assert e.value.status == R.RFLBM_EINVAL
    # BGK relaxes every mode at omega_h: omega_g does not enter, and AA accepts it
    c = R.rflbm_config_default()
    c.pattern, c.model, c.omega_g = R.RFLBM_PATTERN_AA, R.RFLBM_MODEL_BGK, 0.8
    assert R.rflbm_buffer_bytes(c) > 0


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


def test_binding_rejects_wrong_dtype_and_short_buffers_before_any_launch(lib):
    """A tensor of the wrong element type, or one shorter than the call touches, raises
    ValueError in the binding: no pointer reaches a kernel that would run past the end of
    the allocation."""
    import numpy as np
    torch = pytest.importorskip("torch")
    from paper_2507_08820_gb300 import rflbm as R
    with pytest.raises(ValueError):
        R._ptr(torch.zeros(64, dtype=torch.float16), np.float32)
    with pytest.raises(ValueError):
        R._ptr(torch.zeros(64, dtype=torch.float32), np.float64)
    with pytest.raises(ValueError):
        R._ptr(torch.zeros(26, dtype=torch.float32), np.float32, 27)
    with pytest.raises(ValueError):
        R._ptr(np.zeros(26, dtype=np.float64), np.float64, 27)
    with pytest.raises(ValueError):
        R._ptr(np.zeros(27, dtype=np.float32), np.float64, 27)
    assert R._ptr(np.zeros(27), np.float64, 27)[1] == 0
    assert R._ptr(torch.zeros(27, dtype=torch.float64), np.float64, 27)[1] == 0
    # the allocation-free diagnostics: float16 populations, or fewer than 27 n values
    with pytest.raises(ValueError):
        R.rflbm_stats_f32_noalloc(torch.zeros(27 * 10, dtype=torch.float16), 10)
    with pytest.raises(ValueError):
        R.rflbm_stats_f32_noalloc(torch.zeros(27 * 10 - 1, dtype=torch.float32), 10)


def test_batch_create_validates_before_touching_the_device(lib):
    """An ensemble with no replicas, an unknown storage format, a non-positive rho0, a tile
    size outside {-1 (rule), 0 (autotuned), 96, 128, 192, 256, 512} or an invalid replica is
    refused with RFLBM_EINVAL before any CUDA call, so the check runs without a GPU."""
    from paper_2507_08820_gb300 import rflbm as R
    good = dict(nx=16, ny=16, nz=16, tau=0.8, kT=1e-4, seed=1)
    cases = [([], {}), ([good], dict(storage=9)), ([good], dict(rho0=0.0)),
             ([good], dict(tile=100)), ([good], dict(tile=-2)), ([good], dict(tile=64)),
             ([good, dict(good, tau=0.5)], {}), ([dict(good, nx=0)], {}),
             ([dict(good, kT=-1.0)], {})]
    for reps, kw in cases:
        with pytest.raises(R.RflbmError) as e:
            R.rflbm_batch_create(reps, **kw)
        assert e.value.status == R.RFLBM_EINVAL, (reps, kw)
        assert R.rflbm_last_error(), (reps, kw)


def test_slab_config_validation_without_gpu(lib):
    """A z-slab (nz_global > 0) holds its nz rows between two ghost rows, so its buffers are
    sized for nx ny (nz + 2) sites; rows outside the decomposed box, z0 without a slab, a
    negative nz_global and a decomposed box of 2^31 sites or more are refused."""
    from paper_2507_08820_gb300 import rflbm as R

    def cfg(**kw):
        c = R.rflbm_config_default()
        for k, v in kw.items():
            setattr(c, k, v)
        return c

    whole = R.rflbm_buffer_bytes(cfg(nx=32, ny=32, nz=34))
    assert R.rflbm_buffer_bytes(cfg(nx=32, ny=32, nz=32, z0=0, nz_global=64)) == whole
    assert R.rflbm_buffer_bytes(cfg(nx=32, ny=32, nz=32, z0=32, nz_global=64)) == whole
    assert R.rflbm_buffer_bytes(cfg(nx=32, ny=32, nz=1, z0=63, nz_global=64)) == \
        R.rflbm_buffer_bytes(cfg(nx=32, ny=32, nz=3))
    for bad in (dict(z0=1), dict(nz_global=-1), dict(z0=-1, nz_global=64),
                dict(z0=33, nz_global=64), dict(nz=65, nz_global=64),
                dict(nx=1300, ny=1300, nz=2, nz_global=1300)):
        with pytest.raises(R.RflbmError) as e:
            R.rflbm_buffer_bytes(cfg(**{"nx": 32, "ny": 32, "nz": 32, **bad}))
        assert e.value.status == R.RFLBM_EINVAL, bad
