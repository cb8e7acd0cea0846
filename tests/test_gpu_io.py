"""Population import and export through the ABI from every kind of memory: pageable host
memory (through the staging buffer), page-locked host memory (read and written in place by
the conversion kernels) and device memory, in both streaming patterns."""
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


def _f32_state(shape, seed):
    n = int(np.prod(shape))
    rho, u = W.random_fields(*shape, seed=seed, drho=0.02, du=0.03)
    f = o.equilibrium_state(rho, u) + W.population_perturbation(n, seed + 1, 2e-4)
    return np.ascontiguousarray(f.astype(np.float32))


@pytest.mark.parametrize("shape", [(13, 6, 5), (64, 6, 5)])
@pytest.mark.parametrize("where", ["pageable", "pinned", "device"])
@pytest.mark.parametrize("pattern", [0, 1])
def test_float32_import_and_export(R, shape, where, pattern):
    import torch
    f32 = _f32_state(shape, 3)
    src = {"pageable": lambda a: a, "pinned": lambda a: torch.from_numpy(a).pin_memory(),
           "device": lambda a: torch.from_numpy(a).cuda()}[where](f32)
    box = R.Box(*shape, tau=0.8, kT=1e-4, pattern=pattern)
    R.rflbm_set_populations_f32(box.h, src)
    got = box.populations()  # float64 export
    # the float32 shift g = f - w rho0 rounds once; back in float64 within 1 ulp of f
    assert np.allclose(got, f32.astype(np.float64), rtol=2.5e-7, atol=0)
    out_pinned = torch.empty(f32.shape, dtype=torch.float32).pin_memory()
    out_pageable = np.empty_like(f32)
    R.rflbm_get_populations_f32(box.h, out_pinned)
    R.rflbm_get_populations_f32(box.h, out_pageable)
    box.close()
    assert np.array_equal(out_pinned.numpy(), out_pageable)
    assert np.allclose(out_pageable, f32, rtol=2.5e-7, atol=0)
