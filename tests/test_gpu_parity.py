"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerance: populations within 1e-5 relative (float32 GPU vs float64 oracle after up to
100 steps), the error of f_i taken relative to max(|f_i|, w_i rho0): thermal
fluctuations carry some populations through zero (at kT = 1e-4 the corner populations
of a 32^3 box span -0.26 w_i .. 2.2 w_i), where a bare |df_i| / |f_i| has no meaning, so
the population's rest value is the floor of the scale. The Philox integer stream is
bit-exact and the float32 normals agree within 2e-5 absolute. Every test starts the oracle from the exact float32-rounded
state the GPU holds (read back through the ABI), so that only the step's arithmetic is
compared.
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


def _state(shape, seed, drho=0.02, du=0.03, amp=2e-4):
    n = int(np.prod(shape))
    rho, u = W.random_fields(*shape, seed=seed, drho=drho, du=du)
    return np.ascontiguousarray(o.equilibrium_state(rho, u) + W.population_perturbation(n, seed + 1, amp))


def _rel(got, want, rho0=1.0):
    """Largest relative population error |df_i| / max(|f_i|, w_i rho0)."""
    scale = np.maximum(np.abs(want), o.weights()[:, None] * rho0)
    return float(np.max(np.abs(got - want) / scale))


def _run_pair(R, shape, steps, tau=0.8, kT=1e-4, seed=3, t0=0, model="reg", omega_g=1.0,
              phi_rho="local", f0=None, kernel=0, rho0=1.0):
    box = R.Box(*shape, tau=tau, kT=kT, seed=seed, omega_g=omega_g, rho0=rho0,
                model=R.RFLBM_MODEL_BGK if model == "bgk" else R.RFLBM_MODEL_REG,
                phi_rho=R.RFLBM_PHI_RHO0 if phi_rho == "rho0" else R.RFLBM_PHI_LOCAL_RHO,
                kernel=kernel)
    # the state is scaled to the reference density (f^(0) is linear in rho)
    R.rflbm_set_populations(box.h, np.ascontiguousarray(rho0 * _state(shape, seed=11)) if f0 is None else f0)
    R.rflbm_set_step(box.h, t0)
    start = box.populations()
    R.rflbm_step(box.h, steps)
    got = box.populations()
    assert R.rflbm_get_step(box.h) == t0 + steps
    box.close()
    want = o.run(start, shape, tau, kT, seed, steps, t0=t0, model=model, omega_g=omega_g,
                 phi_rho=phi_rho, rho0=rho0)
    return got, want, start


# ------------------------------------------------------------------- noise source
def test_philox_integer_stream_is_bit_exact(R):
    g = np.random.default_rng(1)
    ctr = g.integers(0, 2 ** 32, (20000, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 2, 3, 4], [0x80000000, 0, 5, 0]]
    for k0, k1 in ((0, 0), (1, 0), (0xDEADBEEF, 0x12345678), (0xFFFFFFFF, 0xFFFFFFFF)):
        got = R.rflbm_philox4x32_10(ctr, k0, k1)
        want = np.stack(o.philox4x32_10(ctr.T.astype(np.uint64), (k0, k1)), axis=1)
        assert np.array_equal(got.astype(np.uint64), want)


def test_site_normals_match_oracle(R):
    sites = np.concatenate([np.arange(5000), [2 ** 31 - 1, 2 ** 30 + 7, 123456789]]).astype(np.uint32)
    for seed, step, rep in ((1, 0, 0), (0x1234567890ABCDEF, 99999, 3), (7, 2 ** 32 - 1, 0)):
        got = R.rflbm_site_normals(seed, step, rep, sites)
        want = o.normals(seed, step, sites.astype(np.uint64), rep).T
        assert np.max(np.abs(got - want)) < 2e-5


def test_normals_accurate_for_extreme_radius_draws(R):
    """Sites whose radius word x0 lies within 2^16 of 0 or 2^32 (u0 near 0 or near 1):
    the float32 radius keeps its relative accuracy where -ln u0 is tiny."""
    sites = np.arange(1 << 22, dtype=np.uint64)
    x0, _, x2, _ = o.philox4x32_10((sites, np.zeros_like(sites), np.zeros_like(sites),
                                    np.zeros_like(sites)), (5, 0))
    pick = (x0 > 2 ** 32 - 2 ** 16) | (x0 < 2 ** 16) | (x2 > 2 ** 32 - 2 ** 16) | (x2 < 2 ** 16)
    sel = sites[pick][:4000].astype(np.uint32)
    assert sel.size > 20
    got = R.rflbm_site_normals(5, 0, 0, sel)[:, :4]
    want = o.normals(5, 0, sel.astype(np.uint64), 0).T[:, :4]
    # pairs (n0, n1), (n2, n3): compare the radius relatively and the normals absolutely
    for a in (0, 2):
        rg = np.hypot(got[:, a], got[:, a + 1])
        rw = np.hypot(want[:, a], want[:, a + 1])
        assert np.max(np.abs(rg - rw) / rw) < 2e-5
    assert np.max(np.abs(got - want)) < 2e-5


# ------------------------------------------------------------------- one step, ragged boxes
# (shape, TMA row-segment width): the TMA kernels take x edges that a width divides (single-
# and multi-segment rows below), and other rows of whole 16-byte units with a ragged last
# segment where at least 77 % of the threads stay busy (100, 132, 200, 260, 300, 1000);
# other boxes run the general gather kernel (48: a 64-site segment would idle a third)
SHAPES = [((1, 1, 1), 0), ((2, 3, 4), 0), ((5, 1, 7), 0), ((17, 9, 5), 0), ((33, 31, 7), 0),
          ((32, 3, 2), 32), ((96, 4, 3), 96), ((64, 5, 3), 64), ((128, 2, 2), 128),
          ((256, 3, 1), 128), ((32, 1, 1), 32), ((128, 9, 7), 128), ((192, 3, 2), 192),
          ((288, 2, 3), 96), ((576, 2, 1), 192), ((160, 3, 2), 32), ((320, 2, 2), 64),
          ((100, 3, 2), 128), ((132, 3, 2), 32), ((200, 2, 2), 32), ((260, 2, 2), 96),
          ((300, 2, 1), 64), ((1000, 1, 2), 128), ((48, 3, 2), 0)]
KERNELS = ["gather", "tma"]


def _kernel_id(R, name):
    return {"gather": R.RFLBM_KERNEL_GATHER, "tma": R.RFLBM_KERNEL_TMA}[name]


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("shape,width", SHAPES)
def test_one_step_reg_flbm(R, shape, width, kernel):
    kid = _kernel_id(R, kernel)
    box = R.Box(*shape, tau=0.8, kernel=kid)
    tma = width > 0 and kid != R.RFLBM_KERNEL_GATHER
    assert R.rflbm_step_path(box.h) == ((kid, width) if tma else (R.RFLBM_KERNEL_GATHER, 0))
    box.close()
    got, want, _ = _run_pair(R, shape, steps=3, t0=17, kernel=kid)
    assert _rel(got, want) < POP_RTOL


def test_auto_kernel_choice(R):
    box = R.Box(128, 4, 4, tau=0.8)
    assert R.rflbm_step_path(box.h) == (R.RFLBM_KERNEL_TMA, 128)
    box.close()
    box = R.Box(48, 4, 4, tau=0.8)
    assert R.rflbm_step_path(box.h) == (R.RFLBM_KERNEL_GATHER, 0)
    box.close()


@pytest.mark.parametrize("kernel", KERNELS)
def test_kernels_agree_bitwise(R, kernel):
    """The two step kernels run the same per-site arithmetic (every operation explicitly
    rounded) on the same inputs: their populations are identical bit for bit."""
    shape = (64, 10, 6)
    f0 = _state(shape, seed=31)
    out = {}
    for name in ("gather", kernel):
        box = R.Box(*shape, tau=0.7, kT=1e-4, seed=2, kernel=_kernel_id(R, name))
        R.rflbm_set_populations(box.h, f0)
        R.rflbm_step(box.h, 4)
        out[name] = box.populations()
        box.close()
    assert np.array_equal(out[kernel], out["gather"])


VARIANTS = [
    dict(kT=0.0), dict(model="bgk"), dict(model="bgk", kT=0.0), dict(omega_g=0.7),
    dict(omega_g=1.4, kT=0.0), dict(phi_rho="rho0"), dict(tau=0.5001), dict(tau=0.51),
    dict(tau=5.0), dict(tau=100.0), dict(kT=1e-3, tau=0.6), dict(model="bgk", tau=0.505),
    dict(rho0=1.7), dict(rho0=0.6, kT=1e-3), dict(rho0=2.5, model="bgk"), dict(rho0=1.7, phi_rho="rho0"),
]


@pytest.mark.parametrize("shape,kernel", [((13, 6, 5), 0), ((64, 6, 5), 2)])
@pytest.mark.parametrize("variant", VARIANTS)
def test_one_step_variants(R, variant, shape, kernel):
    got, want, _ = _run_pair(R, shape, steps=2, t0=3, kernel=kernel, **variant)
    assert _rel(got, want, variant.get("rho0", 1.0)) < POP_RTOL, variant


# ------------------------------------------------------------------- the 32^3 x 100 run
def test_config_32cubed_100_steps_from_rest(R):
    """Periodic 32^3, tau 0.8, rho0 1, kT 1e-4, rest start, seed 1, 100 steps: populations,
    rho, u and Pi per site against the oracle; mass and momentum conservation."""
    shape, tau, kT, seed = (32, 32, 32), 0.8, 1e-4, 1
    n = 32 ** 3
    box = R.Box(*shape, tau=tau, kT=kT, seed=seed)
    R.rflbm_init_rest(box.h)
    R.rflbm_step(box.h, 100)
    got = box.populations()
    st, status = R.rflbm_stats(box.h)
    rho, u, pi = box.macroscopic()
    box.close()
    want = o.run(o.rest_state(n), shape, tau, kT, seed, 100)
    assert _rel(got, want) < POP_RTOL
    wrho, wu, wpi = o.macroscopic(want)
    # bounds implied by the population tolerance: |d rho| <= 1e-5 rho, |d j| <= 1e-5 sum f|c|
    assert np.max(np.abs(rho - wrho) / wrho) < POP_RTOL
    assert np.max(np.abs(u - wu)) < 3 * POP_RTOL
    assert np.max(np.abs(pi - wpi)) < 3 * POP_RTOL
    assert status == R.RFLBM_OK and st.nonfinite == 0 and st.step == 100
    # float32 storage: each site-step rounds its 27 stored values (~2^-24 |g_i|,
    # |g_i| ~ 3e-3); over 32^3 sites x 100 steps the sums random-walk to ~1e-6
    assert abs(st.mass - n) / n < 1e-9
    assert np.max(np.abs(np.array(st.momentum))) < 1e-5
    # the fluid did heat up: per-site density variance of order rho0 kT / cs2
    assert 0.3 < np.var(rho) / (kT * 3.0) < 1.5


def test_init_field_is_the_hermite_equilibrium(R):
    shape = (9, 8, 7)
    rho, u = W.random_fields(*shape, seed=4, drho=0.05, du=0.05)
    box = R.Box(*shape, tau=0.9)
    R.rflbm_init_field(box.h, rho, np.ascontiguousarray(u))
    got = box.populations()
    box.close()
    assert _rel(got, o.equilibrium_state(rho, u)) < 1e-6


def test_moments_of_arbitrary_state(R):
    shape = (7, 5, 6)
    f0 = _state(shape, seed=21, amp=1e-3)
    box = R.Box(*shape, tau=0.8)
    R.rflbm_set_populations(box.h, f0)
    f = box.populations()
    rho, u, pi = box.macroscopic()
    box.close()
    wr, wu, wpi = o.macroscopic(f)
    assert np.max(np.abs(rho - wr)) < 1e-12
    assert np.max(np.abs(u - wu)) < 1e-12
    assert np.max(np.abs(pi - wpi)) < 1e-12


def test_rest_without_noise_is_bitwise_stationary(R):
    box = R.Box(16, 8, 4, tau=0.7, kT=0.0, rho0=1.3)
    R.rflbm_init_rest(box.h)
    a = np.empty(R.rflbm_state_bytes(box.h), np.uint8)
    b = np.empty_like(a)
    R.rflbm_save_state(box.h, a)
    R.rflbm_step(box.h, 7)
    R.rflbm_save_state(box.h, b)
    box.close()
    assert not a.any() and np.array_equal(a, b)


def test_checkpoint_resume_is_bitwise(R):
    shape = (20, 12, 9)
    f0 = _state(shape, seed=5)
    full = R.Box(*shape, tau=0.7, kT=2e-4, seed=9)
    R.rflbm_set_populations(full.h, f0)
    R.rflbm_step(full.h, 20)
    ref = np.empty(R.rflbm_state_bytes(full.h), np.uint8)
    R.rflbm_save_state(full.h, ref)
    part = R.Box(*shape, tau=0.7, kT=2e-4, seed=9)
    R.rflbm_set_populations(part.h, f0)
    R.rflbm_step(part.h, 8)
    img = np.empty_like(ref)
    R.rflbm_save_state(part.h, img)
    resumed = R.Box(*shape, tau=0.7, kT=2e-4, seed=9)
    R.rflbm_load_state(resumed.h, img)
    R.rflbm_set_step(resumed.h, 8)
    R.rflbm_step(resumed.h, 12)
    out = np.empty_like(ref)
    R.rflbm_save_state(resumed.h, out)
    for b in (full, part, resumed):
        b.close()
    assert np.array_equal(out, ref)


def test_torch_buffers_and_stream_give_identical_results(R):
    import torch
    shape = (24, 10, 6)
    f0 = _state(shape, seed=6)
    lib_box = R.Box(*shape, tau=0.65, kT=1e-4, seed=2)
    R.rflbm_set_populations(lib_box.h, f0)
    R.rflbm_step(lib_box.h, 5)
    ref = lib_box.populations()
    lib_box.close()
    s = torch.cuda.Stream()
    tbox = R.Box(*shape, tau=0.65, kT=1e-4, seed=2, torch_buffers=True, stream=s.cuda_stream)
    fd = torch.from_numpy(f0).cuda()
    torch.cuda.synchronize()
    R.rflbm_set_populations(tbox.h, fd)
    R.rflbm_step(tbox.h, 5)
    out = torch.empty((27, int(np.prod(shape))), dtype=torch.float64, device="cuda")
    R.rflbm_get_populations(tbox.h, out)
    tbox.close()
    assert np.array_equal(out.cpu().numpy(), ref)


def test_get_sites_matches_full_readback(R):
    shape = (11, 7, 5)
    box = R.Box(*shape, tau=0.8, kT=1e-4)
    R.rflbm_set_populations(box.h, _state(shape, seed=8))
    R.rflbm_step(box.h, 3)
    full = box.populations()
    sites = np.array([0, 1, 10, 11, 76, 384, 384], dtype=np.int64)
    out = np.empty((27, sites.size))
    R.rflbm_get_sites(box.h, sites, out)
    box.close()
    assert np.array_equal(out, full[:, sites])


def test_errors_are_reported(R):
    box = R.Box(4, 4, 4, tau=0.8)
    with pytest.raises(R.RflbmError) as e:
        R.rflbm_step(box.h, 1)
    assert e.value.status == R.RFLBM_ESTATE
    R.rflbm_init_rest(box.h)
    with pytest.raises(R.RflbmError) as e:
        R.rflbm_get_sites(box.h, np.array([64]), np.empty((27, 1)))
    assert e.value.status == R.RFLBM_EINVAL
    with pytest.raises(R.RflbmError):
        R.rflbm_step(box.h, -1)
    box.close()


# ------------------------------------------------------------------- full size, sampled
def test_full_size_128cubed_sampled_sites(R):
    """The benchmark workload (128^3, tau 0.8, kT 1e-4, one launch per step): after 4
    steps from a perturbed equilibrium, the next step's post-collision populations of
    3000 sampled sites (both periodic edges included) against the oracle's per-site
    collision, read at x + c_i after streaming; mass and momentum conserved."""
    shape, tau, kT, seed = (128, 128, 128), 0.8, 1e-4, 1
    n = 128 ** 3
    c = o.velocities()
    box = R.Box(*shape, tau=tau, kT=kT, seed=seed)
    rho, u = W.random_fields(*shape, seed=12, drho=0.01, du=0.01)
    R.rflbm_init_field(box.h, rho, np.ascontiguousarray(u))
    R.rflbm_step(box.h, 4)
    st0, _ = R.rflbm_stats(box.h)
    before = box.populations()
    R.rflbm_step(box.h, 1)
    after = box.populations()
    st1, _ = R.rflbm_stats(box.h)
    box.close()
    sites = W.sample_sites(n, 3000, seed=13)
    fstar = o.collide(before[:, sites], tau, kT, seed, 4, sites.astype(np.uint64))
    x, y, z = sites % 128, (sites // 128) % 128, sites // (128 * 128)
    got = np.empty_like(fstar)
    for i in range(27):
        dst = (x + c[i, 0]) % 128 + 128 * ((y + c[i, 1]) % 128 + 128 * ((z + c[i, 2]) % 128))
        got[i] = after[i, dst]
    assert _rel(got, fstar) < POP_RTOL
    assert abs(st1.mass - st0.mass) / st0.mass < 1e-10
    # float32 rounding of the 27 stored values of each site (~2^-24 |g_i|, |g_i| < 1e-2)
    # summed with random signs over 2.1e6 sites: a drift of order 1e-6 per step
    assert np.max(np.abs(np.array(st1.momentum) - np.array(st0.momentum))) < 1e-5


@pytest.mark.parametrize("shape", [(100, 4, 3), (200, 3, 2), (260, 2, 2)])
@pytest.mark.parametrize("variant", [dict(model=1, kT=1e-4), dict(model=1, kT=0.0), dict(omega_g=1.3, kT=2e-4),
                                     dict(phi_rho=1, kT=1e-4)])
@pytest.mark.parametrize("pattern", [0, 1])
def test_ragged_segments_match_the_gather_kernel_bitwise(R, shape, variant, pattern):
    """Rows that no segment width divides run ragged last segments on the TMA kernels: BGK,
    ghost relaxation omega_g != 1 and the rho0 noise amplitude give the gather kernel's bits
    (AA: BGK only; the AA kernels carry neither omega_g != 1 nor the rho0 amplitude)."""
    if pattern == 1 and variant.get("model", 0) != 1:
        pytest.skip("AA steps run Reg-FLBM with omega_g = 1 and the local density, or BGK")
    n = int(np.prod(shape))
    rho, u = W.random_fields(*shape, seed=19, drho=0.02, du=0.03)
    f0 = np.ascontiguousarray(o.equilibrium_state(rho, u) + W.population_perturbation(n, 20, 2e-4))
    out = []
    for kernel in (R.RFLBM_KERNEL_TMA, R.RFLBM_KERNEL_GATHER):
        box = R.Box(*shape, tau=0.7, seed=5, kernel=kernel, pattern=pattern, **variant)
        if kernel == R.RFLBM_KERNEL_TMA:
            assert R.rflbm_step_path(box.h)[0] == R.RFLBM_KERNEL_TMA
        R.rflbm_set_populations(box.h, f0)
        snaps = []
        for steps in (1, 1, 3):
            R.rflbm_step(box.h, steps)
            snaps.append(box.populations())
        out.append(snaps)
        box.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b), float(np.max(np.abs(a - b)))
