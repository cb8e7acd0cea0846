"""Boxes at the limits of the index arithmetic, checked against the oracle at sampled sites.

1024 x 1024 x 2047 = 2,146,435,072 sites is just below the 2^31 site limit: site indices,
Philox counters and neighbour offsets use their full 31-bit range. 1024^3 in float32 has
4.3 GB planes, so every plane offset beyond the first needs 64 bits. Both run in the AA
pattern (one 116 GB buffer), through both of its forms, from rest; a 1024 x 1024 x 1536
float16 box (two 87 GB buffers) runs the two-site ping-pong kernel at 64-bit plane offsets.

After one step the populations are site-local functions of the noise; after two they
depend on the 27 neighbours. get_sites returns f_i(x, t) = f*_i(x - c_i, t - 1), so the
oracle collides at each neighbour x - c_i: from rest for step 1, and from the stored
populations of the neighbour (read back after step 1) for step 2.
"""
import numpy as np
import pytest

from oracle import rflbm_oracle as o
from paper_2507_08820_gb300 import workloads as W

pytestmark = pytest.mark.gpu
POP_RTOL = 1e-5
U16 = 2.0 ** -11  # float16 unit round-off


@pytest.fixture(scope="module")
def R():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_08820_gb300 import build
    build.build()
    from paper_2507_08820_gb300 import rflbm
    return rflbm


def _sites(shape, n_samples, seed):
    nx, ny, nz = shape
    n = nx * ny * nz
    corners = [x + nx * (y + ny * z) for x in (0, nx - 1) for y in (0, ny - 1) for z in (0, nz - 1)]
    edges = [nx - 1, nx, nx * ny - 1, nx * ny, n - nx, n // 2]
    return np.unique(np.concatenate([W.sample_sites(n, n_samples, seed), corners, edges])).astype(np.int64)


def _pull_neighbours(sites, shape):
    """(27, M) site indices x - c_i under periodic wrap."""
    nx, ny, nz = shape
    x, y, z = sites % nx, (sites // nx) % ny, sites // (nx * ny)
    c = o.velocities()
    xs = (x[None, :] - c[:, 0:1]) % nx
    ys = (y[None, :] - c[:, 1:2]) % ny
    zs = (z[None, :] - c[:, 2:3]) % nz
    return (xs + nx * (ys + ny * zs)).astype(np.int64)


def _streamed(fstar, nb, index_of):
    """f_i(x) = f*_i(x - c_i): population i of column nb[i, m] of fstar."""
    out = np.empty(nb.shape)
    for i in range(27):
        out[i] = fstar[i, index_of(nb[i])]
    return out


def _check(got, want, storage):
    w = o.weights()[:, None]
    if storage == 0:
        rel = np.max(np.abs(got - want) / np.maximum(np.abs(want), w))
        assert rel < POP_RTOL, rel
    else:
        bound = 1.05 * U16 * np.abs(want - w) + 1e-6 * w
        assert np.all(np.abs(got - want) <= bound), np.max(np.abs(got - want) / bound)


@pytest.mark.parametrize("shape,storage,pattern", [((1024, 1024, 2047), 1, 1), ((1024, 1024, 1024), 0, 1),
                                                   ((1024, 1024, 1536), 1, 0)])
def test_largest_boxes_two_steps_at_sampled_sites(R, shape, storage, pattern):
    n = int(np.prod(shape))
    assert n < 2 ** 31
    tau, kT, seed = 0.8, 1e-4, 5
    box = R.Box(*shape, tau=tau, kT=kT, seed=seed, storage=storage, pattern=pattern)
    try:
        R.rflbm_init_rest(box.h)
        sites = _sites(shape, 160, seed=3)
        nb = _pull_neighbours(sites, shape)
        uniq = np.unique(nb)
        index_of = lambda s: np.searchsorted(uniq, s)  # noqa: E731

        R.rflbm_step(box.h, 1)
        got1 = np.empty((27, sites.size))
        R.rflbm_get_sites(box.h, sites, got1)
        pre2 = np.empty((27, uniq.size))
        R.rflbm_get_sites(box.h, uniq, pre2)
        R.rflbm_step(box.h, 1)
        got2 = np.empty((27, sites.size))
        R.rflbm_get_sites(box.h, sites, got2)
    finally:
        box.close()

    star1 = o.collide(o.rest_state(uniq.size), tau, kT, seed, 0, uniq.astype(np.uint64))
    _check(got1, _streamed(star1, nb, index_of), storage)
    star2 = o.collide(pre2, tau, kT, seed, 1, uniq.astype(np.uint64))
    _check(got2, _streamed(star2, nb, index_of), storage)
