"""z-slab decomposition (the paper's linear split of one box along z, Sec. IV) on one GPU.

Several handles, each the z-slab of some rows of one periodic box, step together and
exchange their faces after every step with plain device-to-device copies
(rflbm_slab_exchange). Because the noise is keyed by the global site index and the slab
kernels run the same per-site arithmetic, the slabs must reproduce the undecomposed box
bit for bit: both streaming patterns (the AA exchange alternates between filling the ghost
rows and draining them back), float32 and 16-bit storage, the TMA kernels (rows of one and
of several segments) and the general kernel, slabs of one row included. The exchange can
also be carried out by the caller (rflbm_slab_faces, rflbm_slab_faces_ready,
rflbm_slab_exchange_done), as a rank of a multi-GPU run does with its transport.
"""
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


def _state(shape, seed=11):
    n = int(np.prod(shape))
    rho, u = W.random_fields(*shape, seed=seed, drho=0.02, du=0.03)
    return np.ascontiguousarray(o.equilibrium_state(rho, u) + W.population_perturbation(n, seed + 1, 2e-4))


def _split(shape, sizes, f0, R, **kw):
    nx, ny, nz = shape
    assert sum(sizes) == nz
    slabs, z0 = [], 0
    for nzs in sizes:
        b = R.Box(nx, ny, nzs, z0=z0, nz_global=nz, **kw)
        if f0 is None:
            R.rflbm_init_thermal(b.h)
        else:
            R.rflbm_set_populations(b.h, np.ascontiguousarray(f0[:, z0 * nx * ny:(z0 + nzs) * nx * ny]))
        slabs.append(b)
        z0 += nzs
    return slabs


def _gather(slabs):
    return np.concatenate([b.populations() for b in slabs], axis=1)


CASES = [  # shape, slab sizes: TMA rows of one segment (W = nx), of several, ragged last
    # segments (ping-pong; 104 also in 16-bit storage), the general kernel
    ((64, 6, 12), (5, 6, 1)),
    ((128, 4, 7), (3, 4)),
    ((256, 3, 5), (2, 1, 2)),
    ((100, 4, 9), (4, 5)),
    ((104, 3, 6), (2, 4)),
    ((12, 10, 9), (4, 5)),
    ((12, 10, 9), (3, 3, 3)),
]


@pytest.mark.parametrize("pattern", [0, 1])
@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("shape,sizes", CASES)
def test_slabs_reproduce_the_whole_box_bitwise(R, shape, sizes, storage, pattern):
    f0 = _state(shape)
    kw = dict(tau=0.8, kT=1e-4, seed=9, storage=storage, pattern=pattern)
    whole = R.Box(*shape, **kw)
    R.rflbm_set_populations(whole.h, f0)
    slabs = _split(shape, sizes, f0, R, **kw)
    assert np.array_equal(_gather(slabs), whole.populations())
    done = 0
    for target in (1, 2, 7):
        while done < target:
            for b in slabs:
                R.rflbm_step(b.h, 1)
            R.rflbm_slab_exchange([b.h for b in slabs])
            done += 1
        R.rflbm_step(whole.h, target - R.rflbm_get_step(whole.h))
        got, want = _gather(slabs), whole.populations()
        assert np.array_equal(got, want), (target, float(np.max(np.abs(got - want))))
    whole.close()
    for b in slabs:
        b.close()


@pytest.mark.parametrize("model", [0, 1])
def test_slab_models_and_kernels(R, model):
    """BGK-FLBM and the general kernel of a box whose rows the TMA kernel also serves."""
    shape, sizes = (64, 5, 8), (3, 5)
    f0 = _state(shape, seed=5)
    for kernel in (R.RFLBM_KERNEL_GATHER, R.RFLBM_KERNEL_TMA):
        kw = dict(tau=0.7, kT=1e-3, seed=4, model=model, kernel=kernel)
        whole = R.Box(*shape, **kw)
        R.rflbm_set_populations(whole.h, f0)
        slabs = _split(shape, sizes, f0, R, **kw)
        for _ in range(4):
            for b in slabs:
                R.rflbm_step(b.h, 1)
            R.rflbm_slab_exchange([b.h for b in slabs])
        R.rflbm_step(whole.h, 4)
        assert np.array_equal(_gather(slabs), whole.populations())
        whole.close()
        for b in slabs:
            b.close()


@pytest.mark.parametrize("kernel", ["gather", "tma"])
@pytest.mark.parametrize("omega_g,phi", [(1.4, "local"), (0.7, "rho0"), (1.0, "rho0")])
def test_slab_ghost_rates_and_noise_density(R, kernel, omega_g, phi):
    """Ghost relaxation omega_g != 1 (the Eq. 22 reconstruction) and the noise amplitude at
    rho0 (Eq. 10 with rho0) on slabs, against the whole box bit for bit, on both kernels."""
    shape, sizes = (64, 5, 9), (4, 3, 2)
    f0 = _state(shape, seed=13)
    k = {"gather": R.RFLBM_KERNEL_GATHER, "tma": R.RFLBM_KERNEL_TMA}[kernel]
    p = {"local": R.RFLBM_PHI_LOCAL_RHO, "rho0": R.RFLBM_PHI_RHO0}[phi]
    kw = dict(tau=0.75, kT=2e-4, seed=17, omega_g=omega_g, phi_rho=p, kernel=k)
    whole = R.Box(*shape, **kw)
    R.rflbm_set_populations(whole.h, f0)
    slabs = _split(shape, sizes, f0, R, **kw)
    for _ in range(5):
        for b in slabs:
            R.rflbm_step(b.h, 1)
        R.rflbm_slab_exchange([b.h for b in slabs])
    R.rflbm_step(whole.h, 5)
    assert np.array_equal(_gather(slabs), whole.populations())
    whole.close()
    for b in slabs:
        b.close()


def test_one_slab_is_periodic_through_its_own_faces(R):
    shape = (32, 4, 6)
    f0 = _state(shape, seed=3)
    whole = R.Box(*shape, tau=0.9, kT=1e-4, seed=2)
    R.rflbm_set_populations(whole.h, f0)
    (slab,) = _split(shape, (6,), f0, R, tau=0.9, kT=1e-4, seed=2)
    for _ in range(3):
        R.rflbm_step(slab.h, 1)
        R.rflbm_slab_exchange([slab.h])
    R.rflbm_step(whole.h, 3)
    assert np.array_equal(slab.populations(), whole.populations())
    whole.close()
    slab.close()


@pytest.mark.parametrize("pattern", [0, 1])
def test_face_copies_one_plane_row_at_a_time(R, pattern):
    """The exchange's fallback for plane pitches beyond the copy pitch limit (one copy per
    plane row instead of one 3-D copy per face) gives the same bits."""
    shape, sizes = (64, 6, 12), (5, 6, 1)
    f0 = _state(shape, seed=8)
    kw = dict(tau=0.8, kT=1e-4, seed=3, pattern=pattern)
    whole = R.Box(*shape, **kw)
    R.rflbm_set_populations(whole.h, f0)
    slabs = _split(shape, sizes, f0, R, **kw)
    R.rflbm_testing_slab_copy_pitch_limit(1)
    try:
        for _ in range(5):
            for b in slabs:
                R.rflbm_step(b.h, 1)
            R.rflbm_slab_exchange([b.h for b in slabs])
    finally:
        R.rflbm_testing_slab_copy_pitch_limit(0)
    R.rflbm_step(whole.h, 5)
    assert np.array_equal(_gather(slabs), whole.populations())
    with pytest.raises(R.RflbmError):
        R.rflbm_testing_slab_copy_pitch_limit(-1)
    whole.close()
    for b in slabs:
        b.close()


def test_thermal_start_is_keyed_by_the_global_site(R):
    shape = (32, 6, 10)
    whole = R.Box(*shape, tau=0.8, kT=1e-4, seed=6)
    R.rflbm_init_thermal(whole.h)
    slabs = _split(shape, (4, 6), None, R, tau=0.8, kT=1e-4, seed=6)
    assert np.array_equal(_gather(slabs), whole.populations())
    for _ in range(2):
        for b in slabs:
            R.rflbm_step(b.h, 1)
        R.rflbm_slab_exchange([b.h for b in slabs])
    R.rflbm_step(whole.h, 2)
    assert np.array_equal(_gather(slabs), whole.populations())
    mass = sum(R.rflbm_stats(b.h)[0].mass for b in slabs)
    assert abs(mass - R.rflbm_stats(whole.h)[0].mass) < 1e-9 * mass
    whole.close()
    for b in slabs:
        b.close()


@pytest.mark.parametrize("pattern", [0, 1])
def test_exchange_by_the_caller(R, pattern):
    """The protocol a rank of a multi-GPU run follows: query the faces after the step, make
    its own copy stream wait for the boundary rows, move the bytes there (here with torch
    copies of the slabs' own torch-allocated buffers), and declare the exchange done."""
    import torch
    shape, sizes = (64, 4, 9), (4, 5)
    f0 = _state(shape, seed=8)
    kw = dict(tau=0.8, kT=1e-4, seed=3, pattern=pattern, torch_buffers=True)
    whole = R.Box(*shape, **{k: v for k, v in kw.items() if k != "torch_buffers"})
    R.rflbm_set_populations(whole.h, f0)
    slabs = _split(shape, sizes, f0, R, **kw)
    side = torch.cuda.Stream()

    def view(box, addr, nbytes):
        for t in box._buffers:
            off = addr - t.data_ptr()
            if 0 <= off and off + nbytes <= t.numel():
                return t[off:off + nbytes]
        raise AssertionError("face outside the slab's buffers")

    def rows(box, face):
        return [view(box, face.run[r] + p * face.plane_pitch, face.row_bytes) for r in range(3) for p in range(3)]

    for _ in range(5):
        for b in slabs:
            R.rflbm_step(b.h, 1)
        faces = [R.rflbm_slab_faces(b.h) for b in slabs]
        for b in slabs:
            R.rflbm_slab_faces_ready(b.h, side.cuda_stream)
        with torch.cuda.stream(side):
            for k, b in enumerate(slabs):
                up = slabs[(k + 1) % len(slabs)]
                fu = faces[(k + 1) % len(slabs)]
                for d, s in zip(rows(up, fu[2]), rows(b, faces[k][0])):   # send_up -> recv_below
                    d.copy_(s)
                for d, s in zip(rows(b, faces[k][3]), rows(up, fu[1])):   # send_down -> recv_above
                    d.copy_(s)
        for b in slabs:
            R.rflbm_slab_exchange_done(b.h, side.cuda_stream)
    R.rflbm_step(whole.h, 5)
    assert np.array_equal(_gather(slabs), whole.populations())
    whole.close()
    for b in slabs:
        b.close()


def test_slab_protocol_errors(R):
    shape = (32, 4, 6)
    a, b, c = _split(shape, (2, 2, 2), _state(shape), R, tau=0.8, kT=1e-4)
    with pytest.raises(R.RflbmError) as e:
        R.rflbm_step(a.h, 2)             # one step per call
    assert e.value.status == R.RFLBM_EINVAL
    with pytest.raises(R.RflbmError) as e:
        R.rflbm_slab_faces(a.h)          # nothing to exchange yet
    assert e.value.status == R.RFLBM_ESTATE
    for h in (a, b, c):
        R.rflbm_step(h.h, 1)
    assert R.rflbm_launches_per_step(a.h) == 1  # two rows: both are boundary rows
    for call in (lambda: R.rflbm_step(a.h, 1), lambda: R.rflbm_stats(a.h), a.populations):
        with pytest.raises(R.RflbmError) as e:
            call()                        # the exchange of the last step is pending
        assert e.value.status == R.RFLBM_ESTATE
    with pytest.raises(R.RflbmError) as e:
        R.rflbm_slab_exchange([a.h, c.h, b.h])  # not in z order
    assert e.value.status == R.RFLBM_EINVAL
    R.rflbm_slab_exchange([b.h, c.h, a.h])      # any rotation of the ring is the same ring
    assert R.rflbm_stats(a.h)[1] == R.RFLBM_OK
    with pytest.raises(R.RflbmError) as e:
        R.rflbm_structure_factor(a.h, "rho")
    assert e.value.status == R.RFLBM_ESTATE
    whole = R.Box(*shape, tau=0.8)
    with pytest.raises(R.RflbmError) as e:
        R.rflbm_slab_faces(whole.h)
    assert e.value.status == R.RFLBM_EINVAL
    assert R.rflbm_launches_per_step(R.Box(32, 4, 5, tau=0.8, z0=0, nz_global=5).h) == 2
    for h in (a, b, c, whole):
        h.close()


@pytest.mark.parametrize("pattern", [0, 1])
def test_rank_exchange_of_one_slab(R, pattern):
    """The rank-side exchange of the distributed path (dist.exchange_slab) with one rank:
    the slab is its own neighbour, so it must reproduce the periodic box."""
    import torch
    from paper_2507_08820_gb300 import dist
    shape = (64, 4, 6)
    f0 = _state(shape, seed=13)
    whole = R.Box(*shape, tau=0.8, kT=1e-4, seed=5, pattern=pattern)
    R.rflbm_set_populations(whole.h, f0)
    (slab,) = _split(shape, (6,), f0, R, tau=0.8, kT=1e-4, seed=5, pattern=pattern, torch_buffers=True)
    info = dist.RankInfo(0, 1, 0)
    side = torch.cuda.Stream()
    for _ in range(3):
        R.rflbm_step(slab.h, 1)
        dist.exchange_slab(R, slab, info, side)
    R.rflbm_step(whole.h, 3)
    assert np.array_equal(slab.populations(), whole.populations())
    whole.close()
    slab.close()
