"""The AA streaming pattern: one population buffer updated in place.

An AA step runs the same per-site arithmetic on the same inputs with the same Philox
counters as a ping-pong step, so the two patterns give bit-identical populations, state
images and diagnostics after every number of steps (both parities of the in-place layout).
The AA path is also compared with the FP64 oracle directly, and checkpoints move between
the two patterns.
"""
import numpy as np
import pytest

from oracle import rflbm_oracle as o
from paper_2507_08820_gb300 import workloads as W

pytestmark = pytest.mark.gpu
POP_RTOL = 1e-5


@pytest.fixture(scope="module")
def R():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_08820_gb300 import build
    build.build()
    from paper_2507_08820_gb300 import rflbm
    return rflbm


def _state(shape, seed=21, du=0.03):
    n = int(np.prod(shape))
    rho, u = W.random_fields(*shape, seed=seed, drho=0.02, du=du)
    return np.ascontiguousarray(o.equilibrium_state(rho, u) + W.population_perturbation(n, seed + 1, 2e-4))


def _rel(got, want, rho0=1.0):
    w = o.weights()[:, None] * rho0
    return float(np.max(np.abs(got - want) / np.maximum(np.abs(want), w)))


def _snapshot(R, box):
    f = np.empty((27, box.n), np.float32)
    R.rflbm_get_populations_f32(box.h, f)
    img = np.empty(R.rflbm_state_bytes(box.h), np.uint8)
    R.rflbm_save_state(box.h, img)
    return f, img


def _pair(R, shape, kernel, storage, f0, **kw):
    boxes = []
    for pattern in (R.RFLBM_PATTERN_PINGPONG, R.RFLBM_PATTERN_AA):
        box = R.Box(*shape, kernel=kernel, storage=storage, pattern=pattern, **kw)
        R.rflbm_set_populations(box.h, f0)
        boxes.append(box)
    return boxes


CASES = [((13, 6, 5), 0), ((64, 6, 5), 2), ((128, 4, 3), 2), ((96, 5, 4), 2), ((256, 3, 4), 2),
         ((224, 3, 2), 2), ((288, 2, 3), 2), ((576, 2, 2), 2), ((160, 3, 2), 2),
         ((192, 2, 3), 2), ((32, 3, 3), 1)]
MODELS = [dict(kT=1e-4), dict(kT=0.0), dict(model=1, kT=1e-4), dict(model=1, kT=0.0)]


@pytest.mark.parametrize("storage", [0, 1, 2])
@pytest.mark.parametrize("shape,kernel", CASES)
@pytest.mark.parametrize("variant", MODELS)
def test_aa_matches_pingpong_bitwise(R, shape, kernel, storage, variant):
    f0 = _state(shape)
    pp, aa = _pair(R, shape, kernel, storage, f0, tau=0.7, seed=5, **variant)
    assert R.rflbm_step_path(aa.h) == R.rflbm_step_path(pp.h)
    done = 0
    for target in (1, 2, 3, 5, 8):
        R.rflbm_step(pp.h, target - done)
        R.rflbm_step(aa.h, target - done)
        done = target
        (fp, ip), (fa, ia) = _snapshot(R, pp), _snapshot(R, aa)
        assert np.array_equal(fa, fp), (target, float(np.max(np.abs(fa - fp))))
        assert np.array_equal(ia, ip), target
    pp.close()
    aa.close()


@pytest.mark.parametrize("shape,kernel", [((13, 6, 5), 0), ((64, 6, 5), 2), ((96, 4, 3), 2)])
@pytest.mark.parametrize("steps", [1, 2, 3])
def test_aa_against_oracle(R, shape, kernel, steps):
    f0 = _state(shape, seed=41)
    box = R.Box(*shape, tau=0.8, kT=1e-4, seed=7, kernel=kernel, pattern=R.RFLBM_PATTERN_AA)
    R.rflbm_set_populations(box.h, f0)
    start = box.populations()  # f0 rounded to float32 storage
    R.rflbm_set_step(box.h, 11)
    R.rflbm_step(box.h, steps)
    got = box.populations()
    box.close()
    want = o.run(start, shape, 0.8, 1e-4, 7, steps, t0=11)
    assert _rel(got, want) < POP_RTOL


@pytest.mark.parametrize("shape,kernel", [((13, 6, 5), 0), ((64, 6, 5), 2)])
@pytest.mark.parametrize("split", [3, 4])
@pytest.mark.parametrize("storage", [0, 1])
def test_checkpoints_move_between_patterns(R, shape, kernel, split, storage):
    """A state image saved after an odd (flipped layout) or even (natural layout) number of
    AA steps resumes in either pattern bit-identically to an uninterrupted run."""
    f0 = _state(shape, seed=51)
    kw = dict(tau=0.75, kT=1e-4, seed=13, kernel=kernel, storage=storage)
    ref = R.Box(*shape, pattern=R.RFLBM_PATTERN_PINGPONG, **kw)
    R.rflbm_set_populations(ref.h, f0)
    R.rflbm_step(ref.h, 7)
    want, want_img = _snapshot(R, ref)
    ref.close()
    aa = R.Box(*shape, pattern=R.RFLBM_PATTERN_AA, **kw)
    R.rflbm_set_populations(aa.h, f0)
    R.rflbm_step(aa.h, split)
    img = np.empty(R.rflbm_state_bytes(aa.h), np.uint8)
    R.rflbm_save_state(aa.h, img)
    aa.close()
    for pattern in (R.RFLBM_PATTERN_PINGPONG, R.RFLBM_PATTERN_AA):
        box = R.Box(*shape, pattern=pattern, **kw)
        R.rflbm_load_state(box.h, img)
        R.rflbm_set_step(box.h, split)
        R.rflbm_step(box.h, 7 - split)
        got, got_img = _snapshot(R, box)
        box.close()
        assert np.array_equal(got, want) and np.array_equal(got_img, want_img), pattern


@pytest.mark.parametrize("steps", [5, 6])
def test_diagnostics_read_both_aa_layouts(R, steps):
    shape = (64, 8, 6)
    n = int(np.prod(shape))
    f0 = _state(shape, seed=61)
    pp, aa = _pair(R, shape, 0, 0, f0, tau=0.8, kT=1e-4, seed=3)
    out = []
    sites = np.array([0, 1, 63, 64, n // 2, n - 1], np.int64)
    for box in (pp, aa):
        R.rflbm_step(box.h, steps)
        rho, u, pi = box.macroscopic()
        st, _ = R.rflbm_stats(box.h)
        s1, s2 = R.rflbm_mode_sums(box.h)
        ns = R.rflbm_shell_count(box.h)
        sk, _ = R.rflbm_structure_factor(box.h, 1, ns)
        fs = np.empty((27, sites.size))
        R.rflbm_get_sites(box.h, sites, fs)
        out.append((rho, u, pi, np.array([st.mass, *st.momentum, st.max_speed]), s1, s2, sk, fs))
        box.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_aa_full_box_and_rest(R):
    L = 128
    rest = R.Box(L, L, L, tau=0.8, kT=0.0, pattern=R.RFLBM_PATTERN_AA)
    R.rflbm_init_rest(rest.h)
    R.rflbm_step(rest.h, 3)
    img = np.empty(R.rflbm_state_bytes(rest.h), np.uint8)
    R.rflbm_save_state(rest.h, img)
    rest.close()
    assert not img.any()
    imgs = []
    for pattern in (R.RFLBM_PATTERN_PINGPONG, R.RFLBM_PATTERN_AA):
        box = R.Box(L, L, L, tau=0.8, kT=1e-4, seed=1, pattern=pattern)
        assert R.rflbm_step_path(box.h) == (R.RFLBM_KERNEL_TMA, 128)
        R.rflbm_init_rest(box.h)
        R.rflbm_step(box.h, 25)
        st, _ = R.rflbm_stats(box.h)
        assert abs(st.mass / L ** 3 - 1.0) < 1e-5 and st.nonfinite == 0
        img = np.empty(R.rflbm_state_bytes(box.h), np.uint8)
        R.rflbm_save_state(box.h, img)
        imgs.append(img)
        box.close()
    assert np.array_equal(imgs[0], imgs[1])


def test_bgk_ignores_omega_g_in_both_patterns(R):
    """BGK relaxes every mode at omega_h (Eq. 12), so omega_g does not enter; AA accepts it."""
    shape = (64, 5, 4)
    f0 = _state(shape, seed=71)
    out = []
    for pattern, omega_g in ((R.RFLBM_PATTERN_PINGPONG, 1.0), (R.RFLBM_PATTERN_AA, 0.8)):
        box = R.Box(*shape, tau=0.7, kT=1e-4, seed=5, model=R.RFLBM_MODEL_BGK, omega_g=omega_g,
                    pattern=pattern)
        R.rflbm_set_populations(box.h, f0)
        R.rflbm_step(box.h, 3)
        out.append(_snapshot(R, box)[0])
        box.close()
    assert np.array_equal(out[0], out[1])


def test_structure_factor_is_reproducible(R):
    L = 64
    box = R.Box(L, L, L, tau=0.8, kT=1e-4, seed=2)
    R.rflbm_init_rest(box.h)
    R.rflbm_step(box.h, 20)
    ns = R.rflbm_shell_count(box.h)
    runs = [R.rflbm_structure_factor(box.h, k, ns) for k in (0, 0, 4, 4)]
    box.close()
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[2][0], runs[3][0])
    assert np.array_equal(runs[0][1], runs[2][1]) and runs[0][1].sum() == L ** 3


def test_aa_buffers_and_errors(R):
    torch = pytest.importorskip("torch")
    shape = (64, 4, 4)
    box = R.Box(*shape, tau=0.8, kT=1e-4, torch_buffers=True, pattern=R.RFLBM_PATTERN_AA)
    assert len(box._buffers) == 1
    R.rflbm_init_rest(box.h)
    R.rflbm_step(box.h, 3)
    st, _ = R.rflbm_stats(box.h)
    assert st.nonfinite == 0
    box.close()
    cfg = R.rflbm_config_default()
    cfg.nx, cfg.ny, cfg.nz, cfg.pattern = 64, 4, 4, R.RFLBM_PATTERN_AA
    nbytes = R.rflbm_buffer_bytes(cfg)
    bufs = [torch.empty(nbytes, dtype=torch.uint8, device="cuda") for _ in range(2)]
    cfg.buffers[0], cfg.buffers[1] = bufs[0].data_ptr(), bufs[1].data_ptr()
    with pytest.raises(R.RflbmError) as e:
        R.rflbm_create_ex(cfg)
    assert e.value.status == R.RFLBM_EINVAL
    cfg.omega_g, cfg.buffers[0], cfg.buffers[1] = 0.7, None, None
    with pytest.raises(R.RflbmError) as e:
        R.rflbm_create_ex(cfg)
    assert e.value.status == R.RFLBM_EINVAL
