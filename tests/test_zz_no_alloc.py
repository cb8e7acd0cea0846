"""The allocation-free diagnostics entry point, rflbm_stats_f32_noalloc.

It serves callers that cannot allocate device memory when they want these numbers (their
framework has already reserved the device memory for its own pool, or they run as a hook
between the steps of another solver): it reduces caller-owned float32 populations with a
fixed scratch area in the library's static device memory. Here it must agree with
rflbm_stats, which uses scratch allocated with its handle, on two different states in
consecutive calls, within the tests' relative tolerance of 1e-5; repeated calls must leave
the device's free memory unchanged; and a site of negative density must count as unstable
in both reductions.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
RTOL = 1e-5


@pytest.fixture(scope="module")
def R():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_08820_gb300 import build
    build.build()
    from paper_2507_08820_gb300 import rflbm
    return rflbm


def _agree(a, b):
    assert a.nonfinite == b.nonfinite == 0
    assert abs(a.mass - b.mass) <= RTOL * abs(b.mass)
    scale = np.max(np.abs(np.array(b.momentum)))
    assert np.max(np.abs(np.array(a.momentum) - np.array(b.momentum))) <= RTOL * scale
    assert abs(a.max_speed - b.max_speed) <= RTOL * b.max_speed


def _box_state(R, shape):
    n = int(np.prod(shape))
    g = np.random.default_rng(3)
    rho = 1.0 + 0.01 * g.uniform(-1, 1, n)
    u = np.empty((3, n))
    u[0], u[1], u[2] = 0.02, -0.01, 0.005
    u += 0.005 * g.uniform(-1, 1, (3, n))
    box = R.Box(*shape, tau=0.8, kT=1e-4, seed=4)
    R.rflbm_init_field(box.h, rho, np.ascontiguousarray(u))
    return box, n


def test_noalloc_stats_match_handle_stats_on_two_calls(R):
    import torch
    shape = (64, 48, 40)  # 122880 sites: eight partial sums of the fixed scratch
    box, n = _box_state(R, shape)
    f = torch.empty((27, n), dtype=torch.float32, device="cuda")
    for steps in (2, 3):  # two consecutive calls on two different states
        R.rflbm_step(box.h, steps)
        ref, status = R.rflbm_stats(box.h)
        assert status == R.RFLBM_OK
        R.rflbm_get_populations_f32(box.h, f)
        torch.cuda.synchronize()
        got, status = R.rflbm_stats_f32_noalloc(f, n)
        assert status == R.RFLBM_OK
        _agree(got, ref)
    box.close()


def test_noalloc_stats_leave_free_device_memory_unchanged(R):
    """The property the entry point exists for: after a first call, further calls do not
    change the CUDA driver's count of free device memory (which also sees allocations made
    outside PyTorch's caching allocator)."""
    import torch
    shape = (32, 32, 32)
    box, n = _box_state(R, shape)
    f = torch.empty((27, n), dtype=torch.float32, device="cuda")
    R.rflbm_get_populations_f32(box.h, f)
    torch.cuda.synchronize()
    R.rflbm_stats_f32_noalloc(f, n)
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        got, status = R.rflbm_stats_f32_noalloc(f, n)
        assert status == R.RFLBM_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    box.close()


def test_non_positive_density_site_counts_as_unstable(R):
    """A finite site whose 27 populations sum to a negative density is reported as
    unstable by both reductions, and its |j| / rho does not enter max_speed."""
    import torch
    shape = (32, 8, 8)
    box, n = _box_state(R, shape)
    fh = box.populations()
    fh[:, 77] = 0.0
    fh[0, 77] = -1e-3  # rho = -1e-3 with momentum 2e-3 along x
    fh[1, 77] = 1e-3
    fh[2, 77] = -1e-3
    R.rflbm_set_populations(box.h, np.ascontiguousarray(fh))
    ref, status = R.rflbm_stats(box.h)
    assert status == R.RFLBM_EUNSTABLE and ref.nonfinite == 1
    assert ref.max_speed < 1.0
    f = torch.tensor(fh, dtype=torch.float32, device="cuda").contiguous()
    got, status = R.rflbm_stats_f32_noalloc(f, n)
    assert status == R.RFLBM_EUNSTABLE and got.nonfinite == 1
    assert got.max_speed < 1.0
    box.close()


def test_noalloc_stats_reject_sizes_beyond_the_scratch(R):
    import torch
    f = torch.zeros(27, dtype=torch.float32, device="cuda")
    with pytest.raises(R.RflbmError) as e:
        R.rflbm_stats_f32_noalloc(f, R.RFLBM_STATS_NOALLOC_MAX_SITES + 1)
    assert e.value.status == R.RFLBM_EINVAL
    assert "capacity" in R.rflbm_last_error()
