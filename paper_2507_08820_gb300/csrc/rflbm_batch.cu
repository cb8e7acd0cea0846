// Batched ensembles: many independent periodic boxes (replicas) of uneven sizes, seeds,
// relaxation times and thermal energies, advanced together.
//
// One launch per step covers the tiles of every replica (a tile table maps CTA j to its
// replica); a run of n steps is one CUDA graph of n launches, chained by programmatic
// dependent launch like the single-box step: a CTA draws its noise while the previous
// step drains and touches the populations only after griddepcontrol.wait. Two kinds of
// tile, per replica:
//  - rows: when a row of the replica is a whole number of 16-byte units and divides the
//    CTA size (kTile = R nx), a tile is R consecutive rows (y0 .. y0 + R - 1) of one slab
//    z. Lanes 0..8 load, for group g = 3 (c_y + 1) + (c_z + 1), the three planes of the R
//    source rows (y0 - c_y .., z - c_z) with one TMA copy each; the rows that wrap around
//    the y edge are copied in afterwards and x wraps by index. The 27 outputs go through
//    shared memory and leave as one TMA store of the (nx, R, 27) box.
//  - sites: otherwise, kTile consecutive sites, each gathering its 27 populations.
// Rows tiles of 16-bit ensembles run two sites per thread (k_batch_rows_pair).
// Each replica's arithmetic is the single-box kernels' (same tile order, same Philox key =
// the replica's seed, replica word 0), so a replica reproduces its single-box run bit for
// bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/rflbm.h"
#include "rflbm_aux.h"
#include "tma.cuh"

namespace rflbm_dev {

// One replica as the step kernels see it. The kernels take the descriptors of up to
// kGroupReps replicas in their launch parameters (the constant bank): a CTA reads its
// replica's fields there, with no per-CTA copy, and the compiler may reload any of them
// instead of holding it in a register.
struct ReplicaDev {
  Geometry geo;
  CollideParams cp;
  StoreScale ss;
  void* buf[2];
  const CUtensorMap* maps;  // rows tiles, per buffer b: [2 b] loads (nx, rows, 1, 3), [2 b + 1] stores (nx, rows, 1, 27)
  int64_t tile_begin;  // first global tile index of this replica
  int64_t ntiles;      // tiles per step
  uint32_t key0, key1;
  PhiloxRoundKeys rk;  // round keys of (key0, key1) (float32 rows tiles: 88.7 % against 88.0 % computed in the rounds)
  uint32_t rows;       // rows per tile (rows tiles), 0: sites tiles
  uint32_t yblocks;    // row blocks per slab: ceil(ny / rows)
  int noise;           // kT > 0
};

constexpr int kGroupReps = 64;  // replicas whose descriptors one launch carries
struct ReplicaTable {
  ReplicaDev r[kGroupReps];
};
static_assert(sizeof(ReplicaTable) <= 30 * 1024, "the replica table stays inside the launch parameters (32 KB)");

// Dynamic shared memory of a rows tile: 9 groups of 3 planes x kTile sites (each group
// rounded to 128 bytes), which then holds the 27-plane output tile.
__host__ __device__ constexpr size_t batch_group_bytes(int tile, size_t elem) {
  return (3 * (size_t)tile * elem + 127) / 128 * 128;
}
__host__ __device__ constexpr size_t batch_smem_bytes(int tile, size_t elem) {
  return 9 * batch_group_bytes(tile, elem) + 128;
}

constexpr uint32_t kBatchTmaPolls = 1u << 22;
constexpr int kBatchPreWaitCalls = 2;  // Philox calls a row tile draws before the dependency wait
// Philox calls (raw words) the two-site row tiles draw before the dependency wait (float16
// ensemble: 3 measured 46.0 % against 45.3 % for 2; the single-box two-site kernels keep 2)
constexpr int kBatchPairPreDrawn = 3;
constexpr int kBatchGroups = 9;  // source rows (c_y, c_z) of a site

// One step of the tiles [tile0, tile0 + gridDim.x) of the tile table, all of one kind
// (rows tiles when kRows, else sites tiles).
// Rows tiles are held to 56 registers (65536 / (kTile 56) resident CTAs per SM), which they
// fit without spilling: the replica's parameters are read from the launch parameters and
// the noise is held as 24 normals.
template <int kStore, int kTile, bool kRows, bool kFull = true>
__global__ void __launch_bounds__(kTile, kRows ? 65536 / (kTile * 56) : 0)
    k_batch_step(const __grid_constant__ ReplicaTable tab, const int* __restrict__ tile_rep, int64_t tile0,
                 const unsigned long long* run, uint32_t k, int* err) {
  using S = Storage<kStore>;
  using T = typename S::T;
  constexpr int kGroup = (int)(batch_group_bytes(kTile, sizeof(T)) / sizeof(T));  // elements
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  T* const sm = reinterpret_cast<T*>(smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u));
  const int tid = threadIdx.x;
  const int64_t j = tile0 + blockIdx.x;
  const ReplicaDev& rep = tab.r[__ldg(tile_rep + j)];  // this tile's replica
  if (kRows && tid == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  if (kRows) __syncthreads();
  grid_launch_dependents();
  // run[0]: the first step of this run, run[1]: the buffer holding its state
  const uint32_t step = (uint32_t)__ldg(run) + k;
  const int parity = (int)((__ldg(run + 1) + k) & 1u);
  const T* src = static_cast<const T*>(rep.buf[parity]);
  T* dst = static_cast<T*>(rep.buf[parity ^ 1]);
  const uint32_t li = (uint32_t)(j - rep.tile_begin);  // tile index within the replica

  if (!kRows) {
    // ---- sites tile: kTile consecutive sites, gathered
    const int64_t s64 = (int64_t)li * kTile + tid;
    if (s64 >= (int64_t)rep.geo.n) return;
    const uint32_t s = (uint32_t)s64;
    SiteNoise noise;
    if (rep.noise) site_noise(s, step, 0u, rep.key0, rep.key1, noise);
    const PullDeltas d = pull_deltas(s, rep.geo);
    grid_dependency_wait();
    float G[3][3][3];
#pragma unroll
    for (int i = 0; i < kQ; ++i)
      G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1] =
          S::load(__ldg(src + s + pull_delta(d, i) + plane_of(i) * rep.geo.ps), class_of(i), rep.ss);
    if (rep.noise)
      collide_site<kModelReg, true, false, false>(G, rep.cp, noise);
    else
      collide_site<kModelReg, false, false, false>(G, rep.cp, noise);
#pragma unroll
    for (int i = 0; i < kQ; ++i)
      dst[s + plane_of(i) * rep.geo.ps] = S::store(G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1], class_of(i), rep.ss);
    return;
  }

  // ---- rows tile: R rows of slab z from y0
  const uint32_t R = rep.rows;
  // sites of the tile (R nx): kTile for full tiles, fewer where nx does not divide kTile (the
  // threads from R nx on stay idle)
  const int rn = kFull ? kTile : (int)(R * rep.geo.nx);
  const uint32_t nx = rep.geo.nx, ny = rep.geo.ny, nz = rep.geo.nz;
  const uint32_t z = li / rep.yblocks;
  const uint32_t y0 = (li - z * rep.yblocks) * R;
  const uint32_t nrows = min(R, ny - y0);
  const uint32_t row = fastdiv((uint32_t)tid, rep.geo.div_nx);
  const uint32_t x = (uint32_t)tid - row * nx;
  const bool active = row < nrows;
  // the normals of calls 0 and 1 while the previous step drains, of calls 2 to 5 while the
  // copies are in flight
  const uint32_t site = x + nx * ((y0 + row) + ny * z);
  SiteNoise noise;
  if (rep.noise && active) site_noise_part<0, kBatchPreWaitCalls>(site, step, 0u, rep.rk, noise);

  grid_dependency_wait();  // the previous step's writes (our source) are complete
  if (tid < kBatchGroups) {
    if (tid == 0) mbar_arrive_expect_tx(&bar, (uint32_t)(kBatchGroups * 3 * rn * sizeof(T)));
    const int cy = tid / 3 - 1, cz = tid % 3 - 1;
    int zs = (int)z - cz;
    zs += zs < 0 ? (int)nz : 0;
    zs -= zs >= (int)nz ? (int)nz : 0;
    tma_load_4d(sm + tid * kGroup, rep.maps + 2 * parity, 0, (int)y0 - cy, zs, 3 * tid, &bar);
  }
  if (rep.noise && active) site_noise_part<kBatchPreWaitCalls, 6>(site, step, 0u, rep.rk, noise);
  const bool ok = mbar_wait_bounded(&bar, 0, kBatchTmaPolls);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) atomicOr(err, 1);
    mbar_wait_bounded(&bar, 0, kBatchTmaPolls);  // copies in flight land first
    return;
  }
  // Rows that wrap around the y edge. The box of c_y = +1 (groups 6..8) starts at row
  // y0 - 1: for y0 = 0 its first row must be row ny - 1. The box of c_y = -1 (groups 0..2)
  // reads row y + 1 for row y: for the tile holding row ny - 1 that is row 0 (a slab of
  // one row block takes both).
  if (tid < (int)nx && (y0 == 0 || y0 + nrows == ny)) {
    // one x of each patched row: 3 groups x 3 planes per patched row position
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
      if (side == 0 ? y0 != 0 : y0 + nrows != ny) continue;
      const int64_t ys = side == 0 ? (int64_t)ny - 1 : 0;
      const int brow = side == 0 ? 0 : (int)nrows - 1;
#pragma unroll
      for (int gi = 0; gi < 3; ++gi) {
        const int g = side == 0 ? 6 + gi : gi;  // c_y = +1: groups 6..8, c_y = -1: groups 0..2
        int zs = (int)z - (gi - 1);              // c_z = gi - 1
        zs += zs < 0 ? (int)nz : 0;
        zs -= zs >= (int)nz ? (int)nz : 0;
        const T* from = src + (int64_t)3 * g * rep.geo.ps + (int64_t)nx * (ys + (int64_t)ny * zs) + tid;
#pragma unroll
        for (int a = 0; a < 3; ++a) sm[g * kGroup + a * rn + brow * (int)nx + tid] = from[(int64_t)a * rep.geo.ps];
      }
    }
  }
  __syncthreads();
  float G[3][3][3];
  if (active) {
    const int xm = x == 0 ? (int)nx - 1 : (int)x - 1, xp = x + 1 == nx ? 0 : (int)x + 1;
    // plane a of every group: the value at x - c_x = x + 1, x, x - 1 (periodic in x)
    const T* const pa[3] = {sm + row * nx + xp, sm + rn + row * nx + x, sm + 2 * rn + row * nx + xm};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          G[a][b][c] = S::load(pa[a][(3 * b + c) * kGroup], class_at(a, b, c), rep.ss);
    if (rep.noise)
      collide_site<kModelReg, true, false, false>(G, rep.cp, noise);
    else
      collide_site<kModelReg, false, false, false>(G, rep.cp, noise);
  }
  __syncthreads();  // every input is read: the tile takes the outputs
  if (active) {
    T* out = sm + row * nx + x;
#pragma unroll
    for (int i = 0; i < kQ; ++i)
      out[plane_of(i) * rn] = S::store(G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1], class_of(i), rep.ss);
  }
  fence_proxy_async_smem();
  __syncthreads();
  if (tid == 0) {
    tma_store_4d(rep.maps + 2 * (parity ^ 1) + 1, sm, 0, (int)y0, (int)z, 0);
    bulk_commit();
    bulk_wait_read();
  }
}

// Rows tiles with two sites per thread (16-bit storage): kTile sites, kTile / 2 threads,
// thread t updating sites 2t and 2t + 1 of the tile (one row: nx is even) with the packed
// collision of the single-box two-site kernels, the storage scale folded into the weights.
template <int kStore, int kTile, bool kFull = true>
__global__ void __launch_bounds__(kTile / 2)
    k_batch_rows_pair(const __grid_constant__ ReplicaTable tab, const int* __restrict__ tile_rep, int64_t tile0,
                      const unsigned long long* run, uint32_t k, int* err) {
  using S = Storage<kStore>;
  using T = typename S::T;
  constexpr int kGroup = (int)(batch_group_bytes(kTile, sizeof(T)) / sizeof(T));
  constexpr int kThreads = kTile / 2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  T* const sm = reinterpret_cast<T*>(smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u));
  const int tid = threadIdx.x;
  const int64_t j = tile0 + blockIdx.x;
  const ReplicaDev& rep = tab.r[__ldg(tile_rep + j)];
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  grid_launch_dependents();
  const uint32_t step = (uint32_t)__ldg(run) + k;
  const int parity = (int)((__ldg(run + 1) + k) & 1u);
  const T* src = static_cast<const T*>(rep.buf[parity]);
  const uint32_t li = (uint32_t)(j - rep.tile_begin);

  const uint32_t R = rep.rows;
  const int rn = kFull ? kTile : (int)(R * rep.geo.nx);  // sites of the tile, as in k_batch_step
  const uint32_t nx = rep.geo.nx, ny = rep.geo.ny, nz = rep.geo.nz;
  const uint32_t z = li / rep.yblocks;
  const uint32_t y0 = (li - z * rep.yblocks) * R;
  const uint32_t nrows = min(R, ny - y0);
  const uint32_t q = 2u * (uint32_t)tid;  // first site of the pair in the tile
  const uint32_t row = fastdiv(q, rep.geo.div_nx);
  const uint32_t x = q - row * nx;  // even
  const bool active = row < nrows;
  // (round keys computed in the rounds: from the replica table they measured 0.9 % slower here)
  const PhiloxKey key{rep.key0, rep.key1};
  PairNoise<kBatchPairPreDrawn, PhiloxKey> noise{x + nx * ((y0 + row) + ny * z), step, 0u, key};
  if (rep.noise && active) noise.draw();

  grid_dependency_wait();
  if (tid < kBatchGroups) {
    if (tid == 0) mbar_arrive_expect_tx(&bar, (uint32_t)(kBatchGroups * 3 * rn * sizeof(T)));
    const int cy = tid / 3 - 1, cz = tid % 3 - 1;
    int zs = (int)z - cz;
    zs += zs < 0 ? (int)nz : 0;
    zs -= zs >= (int)nz ? (int)nz : 0;
    tma_load_4d(sm + tid * kGroup, rep.maps + 2 * parity, 0, (int)y0 - cy, zs, 3 * tid, &bar);
  }
  const bool ok = mbar_wait_bounded(&bar, 0, kBatchTmaPolls);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) atomicOr(err, 1);
    mbar_wait_bounded(&bar, 0, kBatchTmaPolls);
    return;
  }
  // rows that wrap around the y edge, as in k_batch_step (x strided over the threads)
  if (y0 == 0 || y0 + nrows == ny) {
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
      if (side == 0 ? y0 != 0 : y0 + nrows != ny) continue;
      const int64_t ys = side == 0 ? (int64_t)ny - 1 : 0;
      const int brow = side == 0 ? 0 : (int)nrows - 1;
#pragma unroll 1
      for (int xx = tid; xx < (int)nx; xx += kThreads) {
#pragma unroll
        for (int gi = 0; gi < 3; ++gi) {
          const int g = side == 0 ? 6 + gi : gi;
          int zs = (int)z - (gi - 1);
          zs += zs < 0 ? (int)nz : 0;
          zs -= zs >= (int)nz ? (int)nz : 0;
          const T* from = src + (int64_t)3 * g * rep.geo.ps + (int64_t)nx * (ys + (int64_t)ny * zs) + xx;
#pragma unroll
          for (int a = 0; a < 3; ++a) sm[g * kGroup + a * rn + brow * (int)nx + xx] = from[(int64_t)a * rep.geo.ps];
        }
      }
    }
  }
  __syncthreads();
  float2 G[3][3][3];
  if (active) {
    // plane a of a group holds the value at x - c_x: x + 1, x, x - 1 (periodic in x); for
    // the pair (x, x + 1): (x + 1, x + 2), (x, x + 1), (x - 1, x)
    const int xm = x == 0 ? (int)nx - 1 : (int)x - 1, xp2 = x + 2 == nx ? 0 : (int)x + 2;
    const T* const base = sm + row * nx;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const T* pl = base + (3 * b + c) * kGroup + a * rn;
          float2 v = a == 1 ? S::load2(pl + x)
                            : (a == 0 ? make_float2(S::to_float(pl[x + 1]), S::to_float(pl[xp2]))
                                      : make_float2(S::to_float(pl[xm]), S::to_float(pl[x])));
          if (S::kScaled) v = kmul(rep.ss.inv_scale[class_at(a, b, c)], v);
          G[a][b][c] = v;
        }
    if (rep.noise)
      collide_tile<kModelReg, true, false, false>(G, rep.cp, noise, ScaledWeight<kStore>{rep.ss});
    else
      collide_tile<kModelReg, false, false, false>(G, rep.cp, noise, ScaledWeight<kStore>{rep.ss});
  }
  __syncthreads();
  if (active) {
    T* out = sm + row * nx + x;
#pragma unroll
    for (int i = 0; i < kQ; ++i) S::store2(out + plane_of(i) * rn, G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1]);
  }
  fence_proxy_async_smem();
  __syncthreads();
  if (tid == 0) {
    tma_store_4d(rep.maps + 2 * (parity ^ 1) + 1, sm, 0, (int)y0, (int)z, 0);
    bulk_commit();
    bulk_wait_read();
  }
}

// Rows tiles of 16-bit ensembles run two sites per thread (issue-bound, like the single-box
// 16-bit steps); float32 ensembles one.
// (float32 row tiles in the two-site form measured 78.3 % against 79.2 % at tile 192)
template <int kStore>
constexpr bool batch_rows_pairs() { return kStore != kStoreF32; }

// One launch of a step: the rows tiles (or the sites tiles) of one tile size within one
// group of kGroupReps replicas, global tiles [begin, end).
struct BatchLaunch {
  int group;
  int tile;
  bool rows;
  bool full;  // rows tiles: R nx = tile (else fewer sites, the rest of the threads idle)
  int64_t begin, end;
};

template <int kStore, int kTile>
static cudaError_t prepare_t() {
  const size_t smem = batch_smem_bytes(kTile, storage_bytes(kStore));
  if (smem <= 48 * 1024) return cudaSuccess;
  if constexpr (batch_rows_pairs<kStore>()) {
    if (cudaError_t e = cudaFuncSetAttribute(k_batch_rows_pair<kStore, kTile, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))
      return e;
    return cudaFuncSetAttribute(k_batch_rows_pair<kStore, kTile, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
  }
  if (cudaError_t e = cudaFuncSetAttribute(k_batch_step<kStore, kTile, true, true>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))
    return e;
  return cudaFuncSetAttribute(k_batch_step<kStore, kTile, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

// Step k of a run for the tiles of launch L, chained to the previous launch on the stream
// by programmatic dependent launch.
template <int kStore, int kTile>
static cudaError_t launch_one_t(const ReplicaTable& tab, const BatchLaunch& L, const int* tile_rep, uint32_t k,
                                const unsigned long long* run, int* err, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(L.end - L.begin));
  cfg.blockDim = dim3(kTile);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (!L.rows) return cudaLaunchKernelEx(&cfg, k_batch_step<kStore, kTile, false>, tab, tile_rep, L.begin, run, k, err);
  cfg.dynamicSmemBytes = batch_smem_bytes(kTile, storage_bytes(kStore));
  if constexpr (batch_rows_pairs<kStore>()) {
    cfg.blockDim = dim3(kTile / 2);
    if (L.full) return cudaLaunchKernelEx(&cfg, k_batch_rows_pair<kStore, kTile, true>, tab, tile_rep, L.begin, run, k, err);
    return cudaLaunchKernelEx(&cfg, k_batch_rows_pair<kStore, kTile, false>, tab, tile_rep, L.begin, run, k, err);
  } else {
    if (L.full) return cudaLaunchKernelEx(&cfg, k_batch_step<kStore, kTile, true, true>, tab, tile_rep, L.begin, run, k, err);
    return cudaLaunchKernelEx(&cfg, k_batch_step<kStore, kTile, true, false>, tab, tile_rep, L.begin, run, k, err);
  }
}

// Resident CTAs per SM of the rows-tile kernel (rows) or the sites-tile kernel.
template <int kStore, int kTile>
static int occupancy_t(bool rows) {
  int n = 0;
  cudaError_t e;
  if (!rows) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_step<kStore, kTile, false>, kTile, 0);
  } else {
    if (prepare_t<kStore, kTile>() != cudaSuccess) return 1;
    const size_t smem = batch_smem_bytes(kTile, storage_bytes(kStore));
    if constexpr (batch_rows_pairs<kStore>())
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_rows_pair<kStore, kTile, true>, kTile / 2, smem);
    else
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_step<kStore, kTile, true, true>, kTile, smem);
  }
  if (e != cudaSuccess) return 1;
  return std::max(n, 1);
}

// Tile sizes: CTA threads of a tile (half as many threads for two-site rows tiles), and
// sites per tile.
constexpr int kNumTiles = 5;
constexpr int kBatchTiles[kNumTiles] = {96, 128, 192, 256, 512};

// Per-replica tile choice: the first size of the storage format's order of preference
// that the row length divides. Uniform 2000-step ensembles, fraction of the copy bandwidth:
// float32 rows of 96 at tile 96 92.3 % (192: 89.7 %), of 64 at 128 92.8 % (192: 88.2 %,
// 256: 85.1 %, 64: 86.5 %), of 48 at 96 90.2 % (192: 87.2 %), of 32 at 128 84.2 % (96:
// 83.3 %, 192: 77.5 %); two-site 16-bit rows of 64 at 128 49.6 % (192: 45.7 %), of 96 at
// 192 47.1 % (96: 38.0 %). Smaller CTAs at the same resident threads interleave more
// independent copy-collide-store phases per SM, down to 96-128 threads.
constexpr int kPrefF32[kNumTiles] = {128, 96, 192, 256, 512};
constexpr int kPref16[kNumTiles] = {128, 192, 256, 512, 96};
constexpr int kAutoSitesTile = 128;  // sites tiles in per-replica mode

static int tile_index(int tile) {
  for (int k = 0; k < kNumTiles; ++k)
    if (kBatchTiles[k] == tile) return k;
  return -1;
}

#define RFLBM_BATCH_DISPATCH(storage, tile, CALL)               \
  switch (tile_index(tile) < 0 ? -1 : (storage) * kNumTiles + tile_index(tile)) { \
    case 0: { constexpr int S = kStoreF32, T = 96; CALL; }      \
    case 1: { constexpr int S = kStoreF32, T = 128; CALL; }     \
    case 2: { constexpr int S = kStoreF32, T = 192; CALL; }     \
    case 3: { constexpr int S = kStoreF32, T = 256; CALL; }     \
    case 4: { constexpr int S = kStoreF32, T = 512; CALL; }     \
    case 5: { constexpr int S = kStoreF16, T = 96; CALL; }      \
    case 6: { constexpr int S = kStoreF16, T = 128; CALL; }     \
    case 7: { constexpr int S = kStoreF16, T = 192; CALL; }     \
    case 8: { constexpr int S = kStoreF16, T = 256; CALL; }     \
    case 9: { constexpr int S = kStoreF16, T = 512; CALL; }     \
    case 10: { constexpr int S = kStoreBF16, T = 96; CALL; }    \
    case 11: { constexpr int S = kStoreBF16, T = 128; CALL; }   \
    case 12: { constexpr int S = kStoreBF16, T = 192; CALL; }   \
    case 13: { constexpr int S = kStoreBF16, T = 256; CALL; }   \
    case 14: { constexpr int S = kStoreBF16, T = 512; CALL; }   \
    default: break;                                             \
  }

static cudaError_t batch_prepare(int storage, int tile) {
  RFLBM_BATCH_DISPATCH(storage, tile, return (prepare_t<S, T>()));
  return cudaErrorInvalidValue;
}

static int batch_occupancy(int storage, int tile, bool rows) {
  RFLBM_BATCH_DISPATCH(storage, tile, return (occupancy_t<S, T>(rows)));
  return 1;
}

// nsteps steps of every launch; launch l runs on stream l % nstreams. The launches of a
// step update disjoint replicas, so each stream is an independent chain of steps: a launch
// waits only for the previous step of the launches on its own stream.
static cudaError_t launch_batch(int storage, const ReplicaTable* tabs, const BatchLaunch* launches, int nlaunches,
                                const int* tile_rep, int64_t nsteps, const unsigned long long* run, int* err,
                                const cudaStream_t* streams, int nstreams) {
  for (int64_t k = 0; k < nsteps; ++k) {
    for (int l = 0; l < nlaunches; ++l) {
      const BatchLaunch& L = launches[l];
      cudaError_t e = cudaErrorInvalidValue;
      RFLBM_BATCH_DISPATCH(storage, L.tile,
                           e = (launch_one_t<S, T>(tabs[L.group], L, tile_rep, (uint32_t)k, run, err,
                                                   streams[l % nstreams]));
                           break);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace rflbm_dev

using namespace rflbm_dev;

struct rflbm_batch {
  int n = 0;
  int device = 0;
  int num_sms = 1;
  int storage = kStoreF32;
  double rho0 = 1.0;
  cudaStream_t stream = nullptr;
  std::vector<rflbm_replica_t> cfg;
  std::vector<ReplicaDev> host;
  std::vector<int> rep_tile;           // per replica: its tile size
  std::vector<ReplicaTable> tables;    // per group of kGroupReps replicas: their descriptors
  std::vector<BatchLaunch> launches;   // the launches of one step, in order
  std::vector<cudaStream_t> chains;    // streams of the independent launch chains of a run
  std::vector<cudaEvent_t> chain_ev;   // [0]: fork, [1 + c]: join of chain c
  int cur = 0;                         // buffer holding every replica's current state
  int* tile_rep = nullptr;             // per global tile: its replica's index within its group
  CUtensorMap* maps = nullptr;  // 4 per replica (rows tiles), device memory
  int64_t tiles = 0;
  int tile = 0;  // requested tile size (0: autotuned per row length, -1: by the order of preference)
  int ctas_per_sm = 1;
  unsigned long long* run = nullptr;  // device: first step of the current run, its buffer
  int* err = nullptr;
  double* partials = nullptr;
  int stat_blocks = 0;
  int64_t step = 0;
  bool initialised = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t graph_steps = -1;
};

namespace {

int bfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  return record_error(code, buf, nullptr);
}

int bcuda(cudaError_t e, const char* what) {
  return record_error(e == cudaErrorMemoryAllocation ? RFLBM_ENOMEM : RFLBM_ECUDA, what,
                      cudaGetErrorString(e));
}

#define BCUDA(call, what)                       \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return bcuda(e_, what); \
  } while (0)

int64_t pstride(int64_t n) { return (n + 63) / 64 * 64; }


constexpr int kBatchChains = 8;  // streams of the independent launch chains of a run

// Streams and events for the launch chains of a run (created outside any stream capture).
int ensure_chains(rflbm_batch* b) {
  const int nc = std::min((int)b->launches.size(), kBatchChains);
  while ((int)b->chains.size() < nc) {
    cudaStream_t c;
    BCUDA(cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking), "creating a launch-chain stream");
    b->chains.push_back(c);
  }
  while ((int)b->chain_ev.size() < nc + 1) {
    cudaEvent_t e;
    BCUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "creating a launch-chain event");
    b->chain_ev.push_back(e);
  }
  return RFLBM_OK;
}

// A replica whose rows can move as TMA row tiles: a row of whole 16-byte units, at most
// 256 sites (the TMA box limit).
bool rows_eligible(const rflbm_batch* b, const Geometry& g) {
  return (g.nx * storage_bytes(b->storage)) % 16 == 0 && g.nx <= 256;
}

// Share of a tile's threads that a replica's rows tiles keep busy (whole rows, floor(t / nx)
// of them; 0 when a row is longer than the tile).
double row_tile_use(const Geometry& g, int t) { return (double)((uint32_t)t / g.nx * g.nx) / t; }
// partial rows tiles below this take site tiles (uniform float32 ensembles, 2000 steps: rows of
// 40 sites 3 to a 128-site tile, 94 % busy, 71.7 % against 64.0 % in site tiles; rows of 100
// one to a tile, 78 % busy, 63.1 % against 65.5 %)
constexpr double kMinRowTileUse = 0.85;

// Whether a replica at tile size t takes rows tiles: eligible rows that t divides, or whose
// whole rows keep at least kMinRowTileUse of t's threads busy.
bool takes_rows(const rflbm_batch* b, const Geometry& g, int t) {
  return rows_eligible(b, g) && (uint32_t)t >= g.nx &&
         ((uint32_t)t % g.nx == 0 || row_tile_use(g, t) >= kMinRowTileUse);
}

// Tile size of a replica: `tile` when positive, else the first size of the storage format's
// order of preference that its row length divides, else the first of at most 256 sites whose
// whole-row tiles keep at least kMinRowTileUse of the threads busy, else sites tiles of
// kAutoSitesTile.
int replica_tile(const rflbm_batch* b, const Geometry& g, int tile) {
  if (tile > 0) return tile;
  const int* pref = b->storage == kStoreF32 ? kPrefF32 : kPref16;
  if (!rows_eligible(b, g)) return kAutoSitesTile;
  for (int k = 0; k < kNumTiles; ++k)
    if (pref[k] % (int)g.nx == 0) return pref[k];
  for (int k = 0; k < kNumTiles; ++k)
    if (pref[k] <= 256 && takes_rows(b, g, pref[k])) return pref[k];
  return kAutoSitesTile;
}

// Builds the per-replica descriptors, their tensor maps, the launches of a step and the
// tile map, replica r at tile size tile_of[r]. A replica takes rows tiles when its rows are
// eligible (rows_eligible), divide its tile, and its maps encode; else sites tiles.
int layout_replicas(rflbm_batch* b, const std::vector<int>& tile_of) {
  std::vector<CUtensorMap> maps((size_t)b->n * 4);
  if (!b->maps) BCUDA(cudaMalloc((void**)&b->maps, sizeof(CUtensorMap) * maps.size()), "allocating tensor maps");
  b->rep_tile = tile_of;
  for (int r = 0; r < b->n; ++r) {
    ReplicaDev& d = b->host[r];
    const Geometry& g = d.geo;
    const int t = tile_of[(size_t)r];
    d.rows = 0;
    d.yblocks = 0;
    d.maps = nullptr;
    if (takes_rows(b, g, t)) {
      const uint32_t R = (uint32_t)t / g.nx;
      bool ok = true;
      for (int k = 0; k < 2 && ok; ++k)
        ok = encode_population_map(&maps[4 * r + 2 * k], d.buf[k], g, g.nx, R, 3, b->storage) &&
             encode_population_map(&maps[4 * r + 2 * k + 1], d.buf[k], g, g.nx, R, kQ, b->storage);
      if (ok) {
        d.rows = R;
        d.yblocks = (g.ny + R - 1) / R;
        d.maps = b->maps + 4 * r;
      }
    }
    d.ntiles = d.rows ? (int64_t)g.nz * d.yblocks : ((int64_t)g.n + t - 1) / t;
  }
  // per group of kGroupReps replicas: one launch per tile size of its rows tiles, then one
  // per tile size of its sites tiles
  const int ngroups = (b->n + kGroupReps - 1) / kGroupReps;
  b->tables.assign((size_t)ngroups, ReplicaTable{});
  b->launches.clear();
  int64_t tiles = 0;
  std::vector<int64_t> sites_at(kNumTiles * 2, 0);  // [kind][tile]: sites updated by such tiles
  for (int g = 0; g < ngroups; ++g) {
    const int r0 = g * kGroupReps, r1 = std::min(b->n, r0 + kGroupReps);
    // passes: full rows tiles, partial rows tiles, sites tiles
    for (int pass = 0; pass < 3; ++pass) {
      for (int ti = 0; ti < kNumTiles; ++ti) {
        BatchLaunch L{g, kBatchTiles[ti], pass < 2, pass == 0, tiles, tiles};
        for (int r = r0; r < r1; ++r) {
          ReplicaDev& d = b->host[r];
          const bool full = d.rows * d.geo.nx == (uint32_t)L.tile;
          if ((d.rows != 0) != L.rows || b->rep_tile[(size_t)r] != L.tile || (L.rows && full != L.full)) continue;
          d.tile_begin = tiles;
          tiles += d.ntiles;
          sites_at[(size_t)((pass == 2 ? 1 : 0) * kNumTiles + ti)] += d.geo.n;
        }
        L.end = tiles;
        if (L.end > L.begin) b->launches.push_back(L);
      }
    }
  }
  BCUDA(cudaMemcpy(b->maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice),
        "uploading tensor maps");
  std::vector<int> map((size_t)tiles);
  for (int r = 0; r < b->n; ++r)
    for (int64_t j = 0; j < b->host[r].ntiles; ++j) map[(size_t)(b->host[r].tile_begin + j)] = r % kGroupReps;
  for (int r = 0; r < b->n; ++r) b->tables[(size_t)(r / kGroupReps)].r[r % kGroupReps] = b->host[r];
  cudaFree(b->tile_rep);
  b->tile_rep = nullptr;
  BCUDA(cudaMalloc(&b->tile_rep, sizeof(int) * (size_t)std::max<int64_t>(tiles, 1)), "allocating the tile map");
  if (tiles > 0)
    BCUDA(cudaMemcpy(b->tile_rep, map.data(), sizeof(int) * (size_t)tiles, cudaMemcpyHostToDevice),
          "uploading the tile map");
  for (const BatchLaunch& L : b->launches)
    if (L.rows) BCUDA(batch_prepare(b->storage, L.tile), "setting the shared-memory size of the batched step kernel");
  if (int e = ensure_chains(b)) return e;
  b->tiles = tiles;
  // occupancy of the kernel that updates the most sites
  size_t top = 0;
  for (size_t k = 1; k < sites_at.size(); ++k)
    if (sites_at[k] > sites_at[top]) top = k;
  b->ctas_per_sm = batch_occupancy(b->storage, kBatchTiles[top % kNumTiles], top < (size_t)kNumTiles);
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (b->graph) {
    cudaGraphDestroy(b->graph);
    b->graph = nullptr;
  }
  b->graph_steps = -1;
  return RFLBM_OK;
}

int enqueue_run(rflbm_batch* b, int64_t nsteps, cudaStream_t st);
int bsync(rflbm_batch* b, const char* what);

// Autotuner of tile 0. Every replica starts at its size from the order of preference; then,
// per row length (largest share of the sites first), the step of the whole ensemble is timed
// with the replicas of that row length at every tile size their rows divide, the other
// replicas at their current sizes, from a rest state: after one warm-up step, the shorter of
// two timings of enough steps for about kTuneSites site updates (at least 3, at most 64).
// Candidates come in the storage format's order of preference, and a later one replaces the
// best so far only when the whole step is more than 2 % faster. (Timed alone, a small class
// of replicas is launch-bound and prefers large tiles; in the ensemble the extra tile size
// is one more launch per step and costs more than it saves.) The populations it leaves are
// undefined until the initialisation call that must follow.
constexpr double kTuneSites = 2e7;
int autotune_tiles(rflbm_batch* b, std::vector<int>& tile_of) {
  for (int r = 0; r < b->n; ++r) tile_of[(size_t)r] = replica_tile(b, b->host[r].geo, -1);
  std::vector<std::pair<double, uint32_t>> classes;  // (sites, row length)
  double total = 0.0;
  for (int r = 0; r < b->n; ++r) {
    const Geometry& g = b->host[r].geo;
    total += g.n;
    if (!rows_eligible(b, g)) continue;
    auto it = std::find_if(classes.begin(), classes.end(), [&](const auto& c) { return c.second == g.nx; });
    if (it == classes.end()) classes.push_back({(double)g.n, g.nx});
    else it->first += g.n;
  }
  std::sort(classes.begin(), classes.end(), [](const auto& a, const auto& c) { return a.first > c.first; });
  const int64_t steps = std::min<int64_t>(64, std::max<int64_t>(3, (int64_t)(kTuneSites / total)));
  for (auto& d : b->host)
    for (int k = 0; k < 2; ++k)
      BCUDA(cudaMemsetAsync(d.buf[k], 0, (size_t)d.geo.ps * kQ * storage_bytes(b->storage), b->stream),
            "clearing replica populations");
  const unsigned long long r0[2] = {0ull, 0ull};
  BCUDA(cudaMemcpyAsync(b->run, r0, sizeof(r0), cudaMemcpyHostToDevice, b->stream), "setting the step index");
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  BCUDA(cudaEventCreate(&t0), "creating the autotuner's events");
  cudaError_t ce = cudaEventCreate(&t1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(t0);
    return bcuda(ce, "creating the autotuner's events");
  }
  const int* pref = b->storage == kStoreF32 ? kPrefF32 : kPref16;
  int rc = RFLBM_OK;
  for (const auto& cls : classes) {
    const uint32_t nx = cls.second;
    std::vector<char> in_class((size_t)b->n, 0);
    for (int r = 0; r < b->n; ++r) in_class[(size_t)r] = b->host[r].geo.nx == nx && rows_eligible(b, b->host[r].geo);
    float best = 0.0f;
    int best_t = 0;
    // the class's size from the order of preference first (a size the row divides where there
    // is one), then the other sizes that take its rows, and kAutoSitesTile (site tiles where
    // it does not take them)
    int cand[kNumTiles + 1];
    int ncand = 0;
    int first_in_class = 0;
    for (int r = 0; r < b->n; ++r)
      if (in_class[(size_t)r]) {
        cand[ncand++] = tile_of[(size_t)r];
        first_in_class = r;
        break;
      }
    const Geometry& gc = b->host[first_in_class].geo;
    for (int k = 0; k < kNumTiles; ++k)
      if (pref[k] != cand[0] && (takes_rows(b, gc, pref[k]) || pref[k] == kAutoSitesTile)) cand[ncand++] = pref[k];
    for (int c = 0; c < ncand && rc == RFLBM_OK; ++c) {
      const int t = cand[c];
      for (int r = 0; r < b->n; ++r)
        if (in_class[(size_t)r]) tile_of[(size_t)r] = t;
      rc = layout_replicas(b, tile_of);
      if (rc == RFLBM_OK) rc = enqueue_run(b, 1, b->stream);  // warm-up
      float ms = 0.0f;
      for (int rep = 0; rep < 2 && rc == RFLBM_OK; ++rep) {
        ce = cudaEventRecord(t0, b->stream);
        if (ce == cudaSuccess) rc = enqueue_run(b, steps, b->stream);
        if (rc == RFLBM_OK && ce == cudaSuccess) ce = cudaEventRecord(t1, b->stream);
        if (rc == RFLBM_OK && ce == cudaSuccess) ce = cudaEventSynchronize(t1);
        float m = 0.0f;
        if (rc == RFLBM_OK && ce == cudaSuccess) ce = cudaEventElapsedTime(&m, t0, t1);
        if (rc == RFLBM_OK && ce != cudaSuccess) rc = bcuda(ce, "timing a tile size");
        if (rep == 0 || m < ms) ms = m;
      }
      if (rc == RFLBM_OK && (best_t == 0 || ms < 0.98f * best)) {
        best = ms;
        best_t = t;
      }
    }
    if (rc != RFLBM_OK) break;
    for (int r = 0; r < b->n; ++r)  // (no size divides the row: the replicas keep site tiles)
      if (in_class[(size_t)r]) tile_of[(size_t)r] = best_t ? best_t : replica_tile(b, b->host[r].geo, -1);
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  return rc;
}

// The layout of tile request `tile`: every replica at `tile` (> 0), at its size from the
// order of preference (-1), or autotuned (0).
int layout_tiles(rflbm_batch* b, int tile) {
  std::vector<int> tile_of((size_t)b->n);
  if (tile == 0) {
    if (int e = autotune_tiles(b, tile_of)) return e;
  } else {
    for (int r = 0; r < b->n; ++r) tile_of[(size_t)r] = replica_tile(b, b->host[r].geo, tile);
  }
  if (int e = layout_replicas(b, tile_of)) return e;
  b->tile = tile;
  return tile == 0 ? bsync(b, "autotuning the batch") : RFLBM_OK;
}

// The launch sequence of one run on stream st: a single launch per step chains on st
// itself; several fork into one chain each (up to kBatchChains streams, launches beyond
// that share them round-robin) and join back into st at the end.
int enqueue_run(rflbm_batch* b, int64_t nsteps, cudaStream_t st) {
  const int nl = (int)b->launches.size();
  const int nc = std::min(nl, kBatchChains);
  if (nc <= 1) {
    BCUDA(launch_batch(b->storage, b->tables.data(), b->launches.data(), nl, b->tile_rep, nsteps, b->run, b->err, &st,
                       1),
          "launching the batched step kernel");
    return RFLBM_OK;
  }
  if ((int)b->chains.size() < nc || (int)b->chain_ev.size() < nc + 1)
    return bfail(RFLBM_ESTATE, "batch launch chains not set up");
  BCUDA(cudaEventRecord(b->chain_ev[0], st), "forking the launch chains");
  for (int c = 0; c < nc; ++c) BCUDA(cudaStreamWaitEvent(b->chains[c], b->chain_ev[0], 0), "forking the launch chains");
  BCUDA(launch_batch(b->storage, b->tables.data(), b->launches.data(), nl, b->tile_rep, nsteps, b->run, b->err,
                     b->chains.data(), nc),
        "launching the batched step kernel");
  for (int c = 0; c < nc; ++c) {
    BCUDA(cudaEventRecord(b->chain_ev[1 + c], b->chains[c]), "joining the launch chains");
    BCUDA(cudaStreamWaitEvent(st, b->chain_ev[1 + c], 0), "joining the launch chains");
  }
  return RFLBM_OK;
}

int bsync(rflbm_batch* b, const char* what) {
  BCUDA(cudaStreamSynchronize(b->stream), what);
  int flag = 0;
  BCUDA(cudaMemcpy(&flag, b->err, sizeof(int), cudaMemcpyDeviceToHost), "reading the error flag");
  if (flag) {
    cudaMemset(b->err, 0, sizeof(int));
    return bfail(RFLBM_ETIMEOUT, "%s: a CTA gave up waiting for its bulk copies (bounded wait expired)", what);
  }
  return RFLBM_OK;
}

// Runs n steps through a CUDA graph of the launch sequence (captured once per n; the
// starting step is read by the kernel from device memory, written before each launch).
int build_graph(rflbm_batch* b, int64_t n) {
  if (!b->exec || b->graph_steps != n) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    cudaStream_t cap;
    BCUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "creating the capture stream");
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    int rc = RFLBM_OK;
    if (e == cudaSuccess) rc = enqueue_run(b, n, cap);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) return bcuda(e, "capturing the batched run");
    if (rc != RFLBM_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e2 != cudaSuccess) return bcuda(e2, "capturing the batched run");
    BCUDA(cudaGraphInstantiate(&b->exec, g, 0), "instantiating the batched run graph");
    b->graph = g;
    b->graph_steps = n;
  }
  return RFLBM_OK;
}

int run_graph(rflbm_batch* b, int64_t n) {
  const unsigned long long r0[2] = {(unsigned long long)b->step, (unsigned long long)b->cur};
  BCUDA(cudaMemcpyAsync(b->run, r0, sizeof(r0), cudaMemcpyHostToDevice, b->stream), "setting the step index");
  if (int e = build_graph(b, n)) return e;
  BCUDA(cudaGraphLaunch(b->exec, b->stream), "launching the batched run graph");
  return RFLBM_OK;
}

}  // namespace

extern "C" {

rflbm_batch_t* rflbm_batch_create(const rflbm_replica_t* reps, int n, double rho0, int storage,
                                  int tile) {
  if (!reps || n < 1) {
    bfail(RFLBM_EINVAL, "rflbm_batch_create: no replicas");
    return nullptr;
  }
  if (!(rho0 > 0.0) || (storage != RFLBM_STORE_F32 && storage != RFLBM_STORE_F16 && storage != RFLBM_STORE_BF16) ||
      (tile != 0 && tile != -1 && tile_index(tile) < 0)) {
    bfail(RFLBM_EINVAL, "rflbm_batch_create: invalid rho0, storage or tile");
    return nullptr;
  }
  for (int r = 0; r < n; ++r) {
    rflbm_config_t c;
    rflbm_config_default(&c);
    c.nx = reps[r].nx; c.ny = reps[r].ny; c.nz = reps[r].nz;
    c.tau = reps[r].tau; c.kT = reps[r].kT; c.rho0 = rho0; c.storage = storage;
    if (rflbm_buffer_bytes(&c) < 0) return nullptr;  // validation message already recorded
  }
  rflbm_batch* b = new (std::nothrow) rflbm_batch();
  if (!b) {
    bfail(RFLBM_ENOMEM, "allocating the batch handle");
    return nullptr;
  }
  b->n = n;
  b->rho0 = rho0;
  b->storage = storage == RFLBM_STORE_F16 ? kStoreF16 : (storage == RFLBM_STORE_BF16 ? kStoreBF16 : kStoreF32);
  b->cfg.assign(reps, reps + n);
  b->host.resize(n);
  cudaGetDevice(&b->device);
  cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
  const size_t elem = storage_bytes(b->storage);
  int rc = RFLBM_OK;
  for (int r = 0; r < n && rc == RFLBM_OK; ++r) {
    ReplicaDev& d = b->host[r];
    std::memset(&d, 0, sizeof(d));
    const rflbm_replica_t& c = reps[r];
    Geometry& g = d.geo;
    g.nx = c.nx; g.ny = c.ny; g.nz = c.nz;
    g.view = kViewPull;
    g.nxy = (uint32_t)c.nx * (uint32_t)c.ny;
    g.n = (uint32_t)((int64_t)c.nx * c.ny * c.nz);
    g.ps = pstride(g.n);
    g.div_nx = make_fastdiv(g.nx);
    g.div_nxy = make_fastdiv(g.nxy);
    // collision and noise parameters: the single-box handle's (Reg-FLBM, omega_g = 1)
    const double om = 1.0 / c.tau;
    d.cp.rho0 = (float)rho0;
    d.cp.omega = (float)om;
    d.cp.neq_diag = (float)((1.0 - om) / bnorm(2, 0, 0));
    d.cp.neq_off = (float)((1.0 - om) / bnorm(1, 1, 0));
    d.cp.ghost_keep = 0.0f;
    d.cp.sqrt_rho0 = (float)std::sqrt(rho0);
    d.cp.amp_h = (float)std::sqrt(c.kT * om * (2.0 - om));  // Eq. 10 rate parts (omega_g = 1)
    d.cp.amp_g = (float)std::sqrt(c.kT);
    const double wc[4] = {8.0 / 27.0, 2.0 / 27.0, 1.0 / 54.0, 1.0 / 216.0};
    for (int k = 0; k < 4; ++k) {
      if (b->storage == kStoreF32) {
        d.ss.scale[k] = d.ss.inv_scale[k] = 1.0f;
      } else {
        const int e = (int)std::lround(-std::log2(std::sqrt(3.0 * wc[k] * rho0 * std::max(c.kT, 1e-6))));
        d.ss.scale[k] = std::ldexp(1.0f, e);
        d.ss.inv_scale[k] = std::ldexp(1.0f, -e);
      }
    }
    d.key0 = (uint32_t)(c.seed & 0xffffffffu);
    d.key1 = (uint32_t)(c.seed >> 32);
    d.rk = philox_round_keys(d.key0, d.key1);
    d.noise = c.kT > 0.0;
    for (int k = 0; k < 2 && rc == RFLBM_OK; ++k) {
      cudaError_t e = cudaMalloc(&d.buf[k], (size_t)g.ps * kQ * elem);
      if (e == cudaSuccess) e = cudaMemset(d.buf[k], 0, (size_t)g.ps * kQ * elem);
      if (e != cudaSuccess) rc = bcuda(e, "allocating replica populations");
    }
  }
  if (rc == RFLBM_OK) {
    cudaError_t e = cudaMalloc((void**)&b->run, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(b->run, 0, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->err, 0, sizeof(int));
    if (e != cudaSuccess) rc = bcuda(e, "allocating batch descriptors");
  }
  if (rc == RFLBM_OK) {
    int64_t nmax = 0;
    for (int r = 0; r < n; ++r) nmax = std::max<int64_t>(nmax, b->host[r].geo.n);
    b->stat_blocks = std::max(1, (int)std::min<int64_t>(4 * (int64_t)b->num_sms, (nmax + 255) / 256));
    cudaError_t e = cudaMalloc((void**)&b->partials, sizeof(double) * ((size_t)b->stat_blocks * kStatOutFields + 8));
    if (e != cudaSuccess) rc = bcuda(e, "allocating the reduction scratch");
  }
  if (rc == RFLBM_OK) rc = layout_tiles(b, tile);
  if (rc != RFLBM_OK) {
    rflbm_batch_destroy(b);
    return nullptr;
  }
  return b;
}

void rflbm_batch_destroy(rflbm_batch_t* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  for (auto& d : b->host) {
    cudaFree(d.buf[0]);
    cudaFree(d.buf[1]);
  }
  cudaFree(b->tile_rep);
  cudaFree(b->maps);
  cudaFree(b->run);
  cudaFree(b->err);
  cudaFree(b->partials);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaStream_t c : b->chains) cudaStreamDestroy(c);
  for (cudaEvent_t e : b->chain_ev) cudaEventDestroy(e);
  delete b;
}

int rflbm_batch_launches_per_step(const rflbm_batch_t* b) {
  if (!b) return bfail(RFLBM_EINVAL, "batch handle is NULL");
  return (int)b->launches.size();
}

int rflbm_batch_tuning(const rflbm_batch_t* b, int* tile, int* ctas_per_sm, int64_t* tiles_per_step) {
  if (!b) return bfail(RFLBM_EINVAL, "batch handle is NULL");
  if (tile) *tile = b->tile;
  if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
  if (tiles_per_step) *tiles_per_step = b->tiles;
  return RFLBM_OK;
}

int rflbm_batch_replica_tiling(const rflbm_batch_t* b, int r, int* tile, int* rows) {
  if (!b || r < 0 || r >= b->n) return bfail(RFLBM_EINVAL, "invalid batch or replica");
  if (tile) *tile = b->rep_tile[(size_t)r];
  if (rows) *rows = (int)b->host[r].rows;
  return RFLBM_OK;
}

int rflbm_batch_replica_dims(const rflbm_batch_t* b, int r, int* nx, int* ny, int* nz) {
  if (!b || r < 0 || r >= b->n) return bfail(RFLBM_EINVAL, "invalid batch or replica");
  const Geometry& g = b->host[r].geo;
  if (nx) *nx = (int)g.nx;
  if (ny) *ny = (int)g.ny;
  if (nz) *nz = (int)g.nz;
  return RFLBM_OK;
}

int rflbm_batch_init_rest(rflbm_batch_t* b) {
  if (!b) return bfail(RFLBM_EINVAL, "batch handle is NULL");
  for (auto& d : b->host)
    BCUDA(cudaMemsetAsync(d.buf[0], 0, (size_t)d.geo.ps * kQ * storage_bytes(b->storage), b->stream),
          "clearing replica populations");
  b->cur = 0;
  b->step = 0;
  b->initialised = true;
  return bsync(b, "rflbm_batch_init_rest");
}

int rflbm_batch_run(rflbm_batch_t* b, int64_t n) {
  if (!b) return bfail(RFLBM_EINVAL, "batch handle is NULL");
  if (!b->initialised) return bfail(RFLBM_ESTATE, "batch state not initialised (call rflbm_batch_init_rest)");
  if (n < 0) return bfail(RFLBM_EINVAL, "negative step count");
  if (n == 0) return RFLBM_OK;
  if (int e = run_graph(b, n)) return e;
  b->step += n;
  if (n & 1) b->cur ^= 1;
  return RFLBM_OK;
}

int rflbm_batch_prepare(rflbm_batch_t* b, int64_t n) {
  if (!b) return bfail(RFLBM_EINVAL, "batch handle is NULL");
  if (n < 1) return bfail(RFLBM_EINVAL, "rflbm_batch_prepare: n must be positive");
  return build_graph(b, n);
}

int rflbm_batch_synchronize(rflbm_batch_t* b) {
  if (!b) return bfail(RFLBM_EINVAL, "batch handle is NULL");
  return bsync(b, "rflbm_batch_synchronize");
}

int rflbm_batch_get_populations(rflbm_batch_t* b, int r, double* f) {
  if (!b || r < 0 || r >= b->n || !f) return bfail(RFLBM_EINVAL, "invalid batch, replica or output");
  if (!b->initialised) return bfail(RFLBM_ESTATE, "batch state not initialised");
  const ReplicaDev& d = b->host[r];
  double* dev = nullptr;
  const size_t bytes = sizeof(double) * kQ * (size_t)d.geo.n;
  BCUDA(cudaMalloc((void**)&dev, bytes), "allocating the export buffer");
  cudaError_t e = launch_get_populations_f64(d.geo, d.cp.rho0, d.ss, b->storage, d.buf[b->cur], dev, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f, dev, bytes, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  cudaFree(dev);
  if (e != cudaSuccess) return bcuda(e, "exporting replica populations");
  return bsync(b, "rflbm_batch_get_populations");
}

int rflbm_batch_stats(rflbm_batch_t* b, int r, rflbm_stats_t* out) {
  if (!b || r < 0 || r >= b->n || !out) return bfail(RFLBM_EINVAL, "invalid batch, replica or output");
  if (!b->initialised) return bfail(RFLBM_ESTATE, "batch state not initialised");
  const ReplicaDev& d = b->host[r];
  const int blocks = std::max(1, (int)std::min<int64_t>(b->stat_blocks, ((int64_t)d.geo.n + 255) / 256));
  double* res = b->partials + (size_t)b->stat_blocks * kStatOutFields;
  BCUDA(launch_stats(d.geo, d.cp.rho0, d.ss, b->storage, d.buf[b->cur], b->partials, blocks, res, b->stream),
        "launching replica stats");
  double host[kStatOutFields];
  BCUDA(cudaMemcpyAsync(host, res, sizeof(host), cudaMemcpyDeviceToHost, b->stream), "copying replica stats");
  if (int e = bsync(b, "rflbm_batch_stats")) return e;
  out->step = b->step;
  out->mass = (double)d.geo.n * b->rho0 + host[0];
  out->momentum[0] = host[1];
  out->momentum[1] = host[2];
  out->momentum[2] = host[3];
  out->max_speed = host[4];
  out->nonfinite = (int64_t)host[5];
  if (out->nonfinite > 0) return bfail(RFLBM_EUNSTABLE, "replica %d holds unstable sites (non-finite values or non-positive densities)", r);
  return RFLBM_OK;
}

}  // extern "C"
