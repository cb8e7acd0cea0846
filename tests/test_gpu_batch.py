"""Batched ensembles: many replicas of uneven sizes, seeds, tau and kT advanced together
reproduce their single-box runs; the ensemble of the batched configuration
(64 replicas, edges in {16,24,32,48,64,96}, kT log-uniform in [1e-5, 1e-3], tau uniform in
[0.55, 1.2], rest start, 1000 steps) runs in float32 and float16 storage.

The replicas below take both kinds of tile at every tile size: rows tiles where nx divides
the tile (row blocks that fill a slab exactly, end short of it, or hold more rows than the
slab has, with one or two slabs), site tiles elsewhere; with tile 0 each replica takes its
own tile size, so one step runs launches of several sizes."""
import numpy as np
import pytest

from oracle import rflbm_oracle as o
from paper_2507_08820_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SMALL = [dict(nx=16, ny=16, nz=16, tau=0.6, kT=1e-4, seed=3),
         dict(nx=24, ny=24, nz=24, tau=0.9, kT=1e-3, seed=4),
         dict(nx=32, ny=32, nz=32, tau=1.1, kT=1e-5, seed=5),
         dict(nx=20, ny=12, nz=9, tau=0.55, kT=2e-4, seed=6),
         dict(nx=64, ny=8, nz=4, tau=0.8, kT=0.0, seed=7),
         dict(nx=1, ny=1, nz=1, tau=0.7, kT=1e-4, seed=8),
         dict(nx=32, ny=3, nz=1, tau=0.75, kT=1e-4, seed=9),
         dict(nx=16, ny=5, nz=2, tau=0.65, kT=3e-4, seed=10)]


@pytest.fixture(scope="module")
def R():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_08820_gb300 import build
    build.build()
    from paper_2507_08820_gb300 import rflbm
    return rflbm


def _single(R, rep, steps, storage):
    box = R.Box(rep["nx"], rep["ny"], rep["nz"], tau=rep["tau"], kT=rep["kT"], seed=rep["seed"],
                storage=storage, kernel=R.RFLBM_KERNEL_GATHER)
    R.rflbm_init_rest(box.h)
    R.rflbm_step(box.h, steps)
    f = box.populations()
    box.close()
    return f


def _batch_pops(R, b, reps, r):
    n = reps[r]["nx"] * reps[r]["ny"] * reps[r]["nz"]
    f = np.empty((27, n))
    R.rflbm_batch_get_populations(b, r, f)
    return f


def _launch_kinds(reps, storage, tile):
    """Launch kinds of one step at an explicit tile size: full rows tiles (the row length
    divides the tile), partial rows tiles (whole rows keeping at least 85 % of the threads
    busy) and site tiles (rows that are no whole 16-byte units, longer than the tile, or
    leaving too many threads idle)."""
    elem = 4 if storage == 0 else 2
    kinds = set()
    for rep in reps:
        nx = rep["nx"]
        if (nx * elem) % 16 == 0 and nx <= 256 and nx <= tile and (
                tile % nx == 0 or (tile // nx * nx) >= 0.85 * tile):
            kinds.add("full" if tile % nx == 0 else "partial")
        else:
            kinds.add("sites")
    return len(kinds)


@pytest.mark.parametrize("storage", [0, 1, 2])
@pytest.mark.parametrize("tile", [96, 128, 192, 256, 512])
def test_replicas_reproduce_their_single_box_runs(R, storage, tile):
    b = R.rflbm_batch_create(SMALL, storage=storage, tile=tile)
    assert R.rflbm_batch_tuning(b)[0] == tile
    assert R.rflbm_batch_launches_per_step(b) == _launch_kinds(SMALL, storage, tile)
    R.rflbm_batch_init_rest(b)
    for n in (3, 4, 3):  # several calls: odd/even buffer parity and the step index
        R.rflbm_batch_run(b, n)
    R.rflbm_batch_synchronize(b)
    for r, rep in enumerate(SMALL):
        got = _batch_pops(R, b, SMALL, r)
        want = _single(R, rep, 10, storage)
        assert np.array_equal(got, want), r
    R.rflbm_batch_destroy(b)


# per-replica tile sizes of SMALL (tile size, rows per tile) in float32 and in 16-bit storage
PER_REPLICA = {0: [(128, 8), (96, 4), (128, 4), (128, 6), (128, 2), (128, 0), (128, 4), (128, 8)],
               1: [(128, 8), (192, 8), (128, 4), (128, 0), (128, 2), (128, 0), (128, 4), (128, 8)]}


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_per_replica_tiles_reproduce_single_box_runs(R, storage):
    """tile -1: every replica at the tile size its row length and storage select in the order
    of preference; the step runs one launch per size and kind (rows at 128 and at 96 or 192,
    in float32 also partial rows tiles at 128 for nx = 20: 6 rows of 20 sites; sites at 128)."""
    b = R.rflbm_batch_create(SMALL, storage=storage, tile=-1)
    assert R.rflbm_batch_tuning(b)[0] == -1
    assert [R.rflbm_batch_replica_tiling(b, r) for r in range(len(SMALL))] == PER_REPLICA[min(storage, 1)]
    assert R.rflbm_batch_launches_per_step(b) == (4 if storage == 0 else 3)
    R.rflbm_batch_init_rest(b)
    for n in (3, 4, 3):
        R.rflbm_batch_run(b, n)
    R.rflbm_batch_synchronize(b)
    for r, rep in enumerate(SMALL):
        assert np.array_equal(_batch_pops(R, b, SMALL, r), _single(R, rep, 10, storage)), r
    R.rflbm_batch_destroy(b)


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_autotuned_tiles_are_valid_and_reproduce_single_box_runs(R, storage):
    """tile 0: the autotuner gives every replica of one row length the same size, one that
    its rows divide where they take row tiles (site tiles of 128 elsewhere), and the run
    reproduces the single-box runs bit for bit."""
    b = R.rflbm_batch_create(SMALL, storage=storage, tile=0)
    assert R.rflbm_batch_tuning(b)[0] == 0
    by_length = {}
    for r, rep in enumerate(SMALL):
        tile, rows = R.rflbm_batch_replica_tiling(b, r)
        assert tile in (96, 128, 192, 256, 512)
        if rows:
            assert rows == tile // rep["nx"] and rows * rep["nx"] >= 0.85 * tile
            assert by_length.setdefault(rep["nx"], tile) == tile
        else:
            assert tile == 128 and PER_REPLICA[min(storage, 1)][r][1] == 0
    R.rflbm_batch_init_rest(b)
    for n in (3, 4):
        R.rflbm_batch_run(b, n)
    R.rflbm_batch_synchronize(b)
    for r, rep in enumerate(SMALL):
        assert np.array_equal(_batch_pops(R, b, SMALL, r), _single(R, rep, 7, storage)), r
    R.rflbm_batch_destroy(b)


@pytest.mark.parametrize("storage", [0, 1])
@pytest.mark.parametrize("tile", [-1, 0])
def test_partial_row_tiles_reproduce_single_box_runs(R, storage, tile):
    """Row lengths that divide no tile size take tiles of whole rows with idle threads where
    at least 85 % of the threads stay busy (40 and 120 at 128), else site tiles (100: one row
    of a 128-site tile would idle 22 %; 72), bit for bit as single boxes."""
    reps = [dict(nx=40, ny=9, nz=5, tau=0.6, kT=1e-4, seed=31), dict(nx=100, ny=5, nz=4, tau=0.9, kT=2e-4, seed=32),
            dict(nx=120, ny=3, nz=3, tau=0.7, kT=0.0, seed=33), dict(nx=72, ny=7, nz=3, tau=1.1, kT=1e-3, seed=34)]
    b = R.rflbm_batch_create(reps, storage=storage, tile=tile)
    tiling = [R.rflbm_batch_replica_tiling(b, r) for r in range(len(reps))]
    if tile == -1:
        assert tiling == [(128, 3), (128, 0), (128, 1), (128, 0)]
    R.rflbm_batch_init_rest(b)
    R.rflbm_batch_run(b, 3)
    R.rflbm_batch_run(b, 2)
    R.rflbm_batch_synchronize(b)
    for r, rep in enumerate(reps):
        assert np.array_equal(_batch_pops(R, b, reps, r), _single(R, rep, 5, storage)), (r, tiling[r])
    R.rflbm_batch_destroy(b)


def test_prepare_builds_the_run_without_running_it(R):
    """rflbm_batch_prepare(n) launches nothing (the state and step stay), and the run of n
    steps that follows replays its graph with the same result as an unprepared run."""
    reps = SMALL[:5]
    b = R.rflbm_batch_create(reps, storage=0, tile=0)
    R.rflbm_batch_init_rest(b)
    R.rflbm_batch_run(b, 2)
    R.rflbm_batch_synchronize(b)
    before = [_batch_pops(R, b, reps, r) for r in range(len(reps))]
    R.rflbm_batch_prepare(b, 5)
    R.rflbm_batch_synchronize(b)
    for r in range(len(reps)):
        assert np.array_equal(_batch_pops(R, b, reps, r), before[r]), r
    assert R.rflbm_batch_stats(b, 0)[0].step == 2
    R.rflbm_batch_run(b, 5)
    R.rflbm_batch_synchronize(b)
    for r, rep in enumerate(reps):
        assert np.array_equal(_batch_pops(R, b, reps, r), _single(R, rep, 7, 0)), r
    with pytest.raises(R.RflbmError) as e:
        R.rflbm_batch_prepare(b, 0)
    assert e.value.status == R.RFLBM_EINVAL
    R.rflbm_batch_destroy(b)


@pytest.mark.parametrize("storage", [0, 1])
def test_three_launch_groups_and_more_launches_than_chains(R, storage):
    """140 replicas: three groups of up to 64, each with row tiles at two sizes and site
    tiles (9 launches per step, more than the 8 launch-chain streams, so that some chains
    carry two launches). Sampled replicas, the last one included, reproduce their
    single-box runs bit for bit."""
    edges = [8, 12, 16, 20, 24]
    reps = [dict(nx=e, ny=e + (r % 3), nz=4 + r % 5, tau=0.55 + 0.01 * (r % 50), kT=1e-4 * (1 + r % 4),
                 seed=100 + r) for r, e in enumerate(edges[r % 5] for r in range(140))]
    b = R.rflbm_batch_create(reps, storage=storage, tile=-1)
    # per group: rows at 128 (edges 8, 16; float32 also 20 as partial tiles of 6 rows) and at
    # 96 (float32: 12, 24) or 192 (16-bit: 24); 16-bit: sites at 128 for 12 and 20, whose rows
    # are no whole 16-byte units
    assert R.rflbm_batch_launches_per_step(b) == 9
    R.rflbm_batch_init_rest(b)
    R.rflbm_batch_run(b, 4)
    R.rflbm_batch_run(b, 3)
    R.rflbm_batch_synchronize(b)
    for r in list(range(0, 140, 9)) + [63, 64, 127, 128, 139]:
        assert np.array_equal(_batch_pops(R, b, reps, r), _single(R, reps[r], 7, storage)), r
    R.rflbm_batch_destroy(b)


def test_tuning_and_errors(R):
    b = R.rflbm_batch_create(SMALL[:3], tile=0)
    tile, per_sm, tiles = R.rflbm_batch_tuning(b)
    assert tile == 0 and per_sm >= 1 and tiles > 0
    assert 1 <= R.rflbm_batch_launches_per_step(b) <= 3  # row tiles at up to three sizes
    with pytest.raises(R.RflbmError) as e:
        R.rflbm_batch_replica_tiling(b, 3)
    assert e.value.status == R.RFLBM_EINVAL
    with pytest.raises(R.RflbmError) as e:
        R.rflbm_batch_run(b, 1)  # not initialised
    assert e.value.status == R.RFLBM_ESTATE
    R.rflbm_batch_destroy(b)
    with pytest.raises(R.RflbmError):
        R.rflbm_batch_create([dict(nx=8, ny=8, nz=8, tau=0.4, kT=0.0, seed=1)])
    for bad in (-2, 64, 100):
        with pytest.raises(R.RflbmError):
            R.rflbm_batch_create(SMALL[:1], tile=bad)


@pytest.mark.parametrize("storage", [0, 1])
def test_ensemble_of_64_replicas_1000_steps(R, storage):
    reps = W.replica_ensemble(64, seed=0)
    b = R.rflbm_batch_create(reps, storage=storage, tile=0)
    R.rflbm_batch_init_rest(b)
    R.rflbm_batch_run(b, 1000)
    R.rflbm_batch_synchronize(b)
    for r, rep in enumerate(reps):
        st, status = R.rflbm_batch_stats(b, r)
        n = rep["nx"] * rep["ny"] * rep["nz"]
        assert status == R.RFLBM_OK and st.step == 1000
        assert abs(st.mass - n) / n < (1e-7 if storage == 0 else 1e-4)
    # the smallest and the largest replica against their single-box runs
    sizes = [rep["nx"] for rep in reps]
    for r in (int(np.argmin(sizes)), int(np.argmax(sizes))):
        assert np.array_equal(_batch_pops(R, b, reps, r), _single(R, reps[r], 1000, storage)), r
    R.rflbm_batch_destroy(b)


def test_replica_against_the_oracle(R):
    """One replica of an ensemble against the FP64 oracle directly (not only through its
    single-box run): a 16^3 box with noise, 5 steps from rest, populations within 1e-5
    relative to max(|f_i|, w_i rho0)."""
    reps = [dict(nx=16, ny=16, nz=16, tau=0.7, kT=1e-4, seed=12),
            dict(nx=24, ny=8, nz=8, tau=0.9, kT=1e-3, seed=13)]
    b = R.rflbm_batch_create(reps, storage=0, tile=192)
    R.rflbm_batch_init_rest(b)
    R.rflbm_batch_run(b, 5)
    R.rflbm_batch_synchronize(b)
    for r, rep in enumerate(reps):
        shape = (rep["nx"], rep["ny"], rep["nz"])
        n = int(np.prod(shape))
        got = _batch_pops(R, b, reps, r)
        want = o.run(o.rest_state(n), shape, rep["tau"], rep["kT"], rep["seed"], 5)
        scale = np.maximum(np.abs(want), o.weights()[:, None])
        assert float(np.max(np.abs(got - want) / scale)) < 1e-5, r
    R.rflbm_batch_destroy(b)


@pytest.mark.parametrize("storage", [0, 1])
def test_random_ensemble_autotuned(R, storage):
    """A seeded random ensemble: 24 replicas with row lengths in 8..132 (multiples of 4, so
    exact, partial and site tiles mix), random tau and kT, autotuned tiles; five sampled
    replicas reproduce their single-box runs bit for bit after 3 steps."""
    g = np.random.default_rng(2024 + storage)
    reps = [dict(nx=int(4 * g.integers(2, 34)), ny=int(g.integers(2, 9)), nz=int(g.integers(1, 6)),
                 tau=float(g.uniform(0.55, 1.3)), kT=float(10 ** g.uniform(-5, -3)), seed=int(500 + r))
            for r in range(24)]
    b = R.rflbm_batch_create(reps, storage=storage, tile=0)
    R.rflbm_batch_init_rest(b)
    R.rflbm_batch_run(b, 3)
    R.rflbm_batch_synchronize(b)
    for r in g.choice(len(reps), 5, replace=False):
        r = int(r)
        assert np.array_equal(_batch_pops(R, b, reps, r), _single(R, reps[r], 3, storage)), (r, reps[r]["nx"])
    R.rflbm_batch_destroy(b)
