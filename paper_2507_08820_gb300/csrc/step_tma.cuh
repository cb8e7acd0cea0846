// The fused stream-and-collide step with TMA staging, for boxes whose rows are whole
// 16-byte units, in row segments of width kW in {32, 64, 96, 128, 192}; templated on the
// storage format. Where kW does not divide the x edge, the last segment of each row ends
// past it: the copies fill its missing sites with zeros, its excess threads compute on
// them, and the store of the segment is clipped at the row's end.
//
// One CTA of kW threads updates one row segment [x0, x0 + kW) of one lattice row (y, z).
// The 27 populations of a site are pulled from 9 source rows (y - c_y, z - c_z), shifted
// by -c_x along x. The three populations of a source row (c_x = -1, 0, +1) occupy three
// adjacent planes of the buffer, so lane g of warp 0 (g = 0..8) fetches group g with one
// tiled TMA load of three planes x [x0 - H, x0 + kW + H) (H = 4 float32 or 8 16-bit
// elements: 16-byte aligned coordinates); the 9 loads complete on one mbarrier. Where the
// segment touches the periodic x edge the wrapped neighbour is fetched with a plain load.
// The first 8 of the 24 normals (Philox calls 0 and 1) are drawn before the kernel waits for
// the previous step (programmatic dependent launch lets this grid start while the previous
// one drains), the other 16 while the copies are in flight, with the Philox round keys
// precomputed in the launch parameters. Each thread then reads its 27 values from
// shared memory at fixed offsets (x - c_x within its group row), collides in registers in
// float32 and writes its 27 results into a dense [plane][kW] tile, which lane 0 stores
// with one TMA copy of all 27 planes.
//
// Every wait on the mbarrier is bounded; a CTA that gives up sets the handle's error flag,
// waits (again bounded) for its copies in flight and exits without storing.
#pragma once

#include "rflbm_internal.h"
#include "tma.cuh"

namespace rflbm_dev {

constexpr uint32_t kMaxPolls = 1u << 22;  // bounded mbarrier waits
// Philox calls (of 6) a one-site CTA draws before it waits for the previous step; the rest
// while its copies are in flight (128^3 float32: 1 call 95.1 %, 2 calls 96.6 %, 3 calls
// 95.3 %, 4 calls 94.3 %, all 6 91.7 % of the copy bandwidth).
constexpr int kPreWaitCalls = 2;
constexpr int kGroups = 9;                 // source rows (c_y, c_z)

// Shared-memory geometry of one CTA.
template <int kStore, int kW>
struct TmaLayout {
  using T = typename Storage<kStore>::T;
  static constexpr int kH = Storage<kStore>::kHalo;
  static constexpr int kSeg = kW + 2 * kH;  // elements per plane row of a group
  static constexpr int kGroupBytes = (3 * kSeg * (int)sizeof(T) + 127) / 128 * 128;
  static constexpr int kGroup = kGroupBytes / (int)sizeof(T);  // group stride in elements
  static constexpr size_t kBytes = (size_t)kGroups * kGroupBytes + 128;  // + alignment slack
  static_assert((size_t)kQ * kW * sizeof(T) <= (size_t)kGroups * kGroupBytes,
                "the output tile must fit in the input tile");
};

template <int kStore, int kW, int kModel, bool kNoise, bool kGhostNeq, bool kPhiRho0>
__global__ void __launch_bounds__(kW, kModel == kModelBgk ? 1024 / kW : 0) step_tma(const __grid_constant__ CUtensorMap load_map,
                                               const __grid_constant__ CUtensorMap store_map,
                                               const StepParams p) {
  using S = Storage<kStore>;
  using L = TmaLayout<kStore, kW>;
  using T = typename L::T;
  constexpr int kH = L::kH;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  // groups start on 128-byte boundaries of the shared window (the launch adds 128 bytes)
  T* const sm = reinterpret_cast<T*>(smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u));

  const int t = threadIdx.x;
  const uint32_t nseg = (p.geo.nx + kW - 1) / kW;  // the last segment of a row may end past x = nx - 1
  const uint32_t rb = blockIdx.x / nseg;
  const uint32_t row = p.row0 + rb + (rb >= p.row_split ? p.row_gap : 0u);  // y + ny * z
  const uint32_t x0 = (blockIdx.x - rb * nseg) * kW;
  const uint32_t z = row / p.geo.ny, y = row - z * p.geo.ny;

  // the next step may start launching now: its CTAs draw their noise while this grid's
  // last CTAs finish; they touch global memory only after their grid_dependency_wait
  grid_launch_dependents();
  const uint32_t s = x0 + t + p.geo.nx * row + p.geo.site0;  // global site (Philox counter)
  // the normals of calls 0 and 1 before the dependency wait, of calls 2 to 5 while the
  // copies are in flight
  SiteNoise noise;
  if (kNoise) site_noise_part<0, kPreWaitCalls>(s, p.step, p.replica, p.rk, noise);

  if (t == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  grid_dependency_wait();  // the previous step's writes (our source) are complete

  // lane g of warp 0 loads the source row of group g = 3 (c_y + 1) + (c_z + 1)
  T patch_l = T(), patch_r = T();
  int at_l = -1, at_r = -1;
  if (t < kGroups) {
    if (t == 0) mbar_arrive_expect_tx(&bar, (uint32_t)(kGroups * 3 * L::kSeg * sizeof(T)) + p.test_extra_tx);
    const int cy = t / 3 - 1, cz = t % 3 - 1;
    int ys = (int)y - cy;
    ys += ys < 0 ? (int)p.geo.ny : 0;
    ys -= ys >= (int)p.geo.ny ? (int)p.geo.ny : 0;
    const int zs = zrow(p.geo, (int)z, -cz);  // buffer row (a z-slab's ghost rows at its faces)
    tma_load_4d(sm + t * L::kGroup, &load_map, (int)x0 - kH, ys, zs, 3 * t, &bar);
    // periodic x edge: plane c_x = +1 needs x = nx - 1 left of x = 0, plane c_x = -1
    // needs x = 0 right of x = nx - 1
    const T* src = static_cast<const T*>(p.src);
    const int64_t rowoff = (int64_t)p.geo.nx * ((int64_t)ys + (int64_t)p.geo.ny * zs);
    if (x0 == 0) {
      patch_l = src[(int64_t)(3 * t + 2) * p.geo.ps + rowoff + (p.geo.nx - 1)];
      at_l = t * L::kGroup + 2 * L::kSeg + kH - 1;
    }
    if (x0 + kW >= p.geo.nx) {  // right of the row's last site, at x0 + kW or inside the segment
      patch_r = src[(int64_t)(3 * t) * p.geo.ps + rowoff];
      at_r = t * L::kGroup + kH + (int)(p.geo.nx - x0);
    }
  }

  if (kNoise) site_noise_part<kPreWaitCalls, 6>(s, p.step, p.replica, p.rk, noise);

  const bool ok = mbar_wait_bounded(&bar, 0, kMaxPolls);
  if (__syncthreads_or(!ok)) {
    if (t == 0) atomicOr(p.err, 1);
    mbar_wait_bounded(&bar, 0, kMaxPolls);  // let copies in flight land before exiting
    return;
  }
  if (at_l >= 0) sm[at_l] = patch_l;
  if (at_r >= 0) sm[at_r] = patch_r;
  __syncthreads();

  float G[3][3][3];
  const T* mine = sm + kH + t;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const int gi = 3 * (cy_of(i) + 1) + (cz_of(i) + 1);
    G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1] =
        S::load(mine[gi * L::kGroup + (cx_of(i) + 1) * L::kSeg - cx_of(i)], class_of(i), p.ss);
  }

  if (kModel == kModelBgk) {
    // BGK re-reads its inputs from the tile at the end instead of keeping them in registers
    const auto reload = [&](int a, int b, int c, float) {
      return S::load(mine[(3 * b + c) * L::kGroup + a * L::kSeg - (a - 1)], class_at(a, b, c), p.ss);
    };
    collide_site<kModel, kNoise, kGhostNeq, kPhiRho0>(G, p.cp, noise, reload);
  } else {
    collide_site<kModel, kNoise, kGhostNeq, kPhiRho0>(G, p.cp, noise);
  }

  __syncthreads();  // every thread has read its inputs: the tile can hold the outputs
  T* out = sm + t;  // dense [plane][kW] output tile at the (128-byte aligned) start
#pragma unroll
  for (int i = 0; i < kQ; ++i)
    out[plane_of(i) * kW] = S::store(G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1], class_of(i), p.ss);
  fence_proxy_async_smem();
  __syncthreads();
  if (t == 0) {
    tma_store_4d(&store_map, sm, (int)x0, (int)y, (int)(z + p.geo.zlo), 0);
    bulk_commit();
    bulk_wait_read();
  }
}

// The same step with two adjacent sites per thread: kW / 2 threads per segment, thread t
// updates x0 + 2t and x0 + 2t + 1 with the collision in packed f32x2 arithmetic (Reg-FLBM,
// omega_g = 1, local rho in Eq. 10). Plane c_x = 0 of a site pair is read from shared memory
// as one aligned pair, the shifted planes c_x = -1, +1 as two elements; the 27 results go
// out as pairs (16-bit storage: one packed conversion per pair) with the storage scale
// folded into the lattice weights. Philox calls 0 and 1 of both sites are drawn before the
// kernel waits for the previous step, the other four inside the collision.
template <int kStore, int kW, bool kNoise>
__global__ void __launch_bounds__(kW / 2) step_tma_pair(const __grid_constant__ CUtensorMap load_map,
                                                         const __grid_constant__ CUtensorMap store_map,
                                                         const StepParams p) {
  using S = Storage<kStore>;
  using L = TmaLayout<kStore, kW>;
  using T = typename L::T;
  constexpr int kH = L::kH;
  static_assert(kW / 2 >= kGroups, "one lane per source row");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  T* const sm = reinterpret_cast<T*>(smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u));

  const int t = threadIdx.x;
  const uint32_t nseg = (p.geo.nx + kW - 1) / kW;  // the last segment of a row may end past x = nx - 1
  const uint32_t rb = blockIdx.x / nseg;
  const uint32_t row = p.row0 + rb + (rb >= p.row_split ? p.row_gap : 0u);  // y + ny * z
  const uint32_t x0 = (blockIdx.x - rb * nseg) * kW;
  const uint32_t z = row / p.geo.ny, y = row - z * p.geo.ny;

  grid_launch_dependents();
  // (round keys computed in the rounds: from the parameter bank they measured 5 % slower here)
  const PhiloxKey key{p.key0, p.key1};
  PairNoise<kPairPreDrawn, PhiloxKey> noise{x0 + 2u * t + p.geo.nx * row + p.geo.site0, p.step, p.replica, key};
  if (kNoise) noise.draw();
  if (t == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  grid_dependency_wait();

  T patch_l = T(), patch_r = T();
  int at_l = -1, at_r = -1;
  if (t < kGroups) {
    if (t == 0) mbar_arrive_expect_tx(&bar, (uint32_t)(kGroups * 3 * L::kSeg * sizeof(T)) + p.test_extra_tx);
    const int cy = t / 3 - 1, cz = t % 3 - 1;
    int ys = (int)y - cy;
    ys += ys < 0 ? (int)p.geo.ny : 0;
    ys -= ys >= (int)p.geo.ny ? (int)p.geo.ny : 0;
    const int zs = zrow(p.geo, (int)z, -cz);  // buffer row (a z-slab's ghost rows at its faces)
    tma_load_4d(sm + t * L::kGroup, &load_map, (int)x0 - kH, ys, zs, 3 * t, &bar);
    const T* src = static_cast<const T*>(p.src);
    const int64_t rowoff = (int64_t)p.geo.nx * ((int64_t)ys + (int64_t)p.geo.ny * zs);
    if (x0 == 0) {
      patch_l = src[(int64_t)(3 * t + 2) * p.geo.ps + rowoff + (p.geo.nx - 1)];
      at_l = t * L::kGroup + 2 * L::kSeg + kH - 1;
    }
    if (x0 + kW >= p.geo.nx) {  // right of the row's last site, at x0 + kW or inside the segment
      patch_r = src[(int64_t)(3 * t) * p.geo.ps + rowoff];
      at_r = t * L::kGroup + kH + (int)(p.geo.nx - x0);
    }
  }

  const bool ok = mbar_wait_bounded(&bar, 0, kMaxPolls);
  if (__syncthreads_or(!ok)) {
    if (t == 0) atomicOr(p.err, 1);
    mbar_wait_bounded(&bar, 0, kMaxPolls);
    return;
  }
  if (at_l >= 0) sm[at_l] = patch_l;
  if (at_r >= 0) sm[at_r] = patch_r;
  __syncthreads();

  // sites x0 + 2t and x0 + 2t + 1: plane c_x = 0 is read as one aligned pair, the shifted
  // planes c_x = -+1 as two elements
  float2 G[3][3][3];
  const T* mine = sm + kH + 2 * t;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const int gi = 3 * (cy_of(i) + 1) + (cz_of(i) + 1);
    const T* at = mine + gi * L::kGroup + (cx_of(i) + 1) * L::kSeg - cx_of(i);
    float2 v = cx_of(i) == 0 ? S::load2(at) : S::load1x2(at);
    if (S::kScaled) v = kmul(p.ss.inv_scale[class_of(i)], v);
    G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1] = v;
  }

  collide_tile<kModelReg, kNoise, false, false>(G, p.cp, noise,
                                                    ScaledWeight<kStore>{p.ss});

  __syncthreads();
  T* out = sm + 2 * t;
#pragma unroll
  for (int i = 0; i < kQ; ++i) S::store2(out + plane_of(i) * kW, G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1]);
  fence_proxy_async_smem();
  __syncthreads();
  if (t == 0) {
    tma_store_4d(&store_map, sm, (int)x0, (int)y, (int)(z + p.geo.zlo), 0);
    bulk_commit();
    bulk_wait_read();
  }
}

template <int kStore, int kW, bool kNoise>
cudaError_t launch_tma_pair(const TmaMaps& m, const StepParams& p, cudaStream_t st) {
  const uint64_t blocks = (uint64_t)((p.geo.nx + kW - 1) / kW) * p.nrows;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(kW / 2);
  cfg.dynamicSmemBytes = TmaLayout<kStore, kW>::kBytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, step_tma_pair<kStore, kW, kNoise>, *m.load,
                            *m.store, p);
}

template <int kStore, int kW, int kModel, bool kNoise, bool kGhostNeq, bool kPhiRho0>
cudaError_t launch_tma_segment(const TmaMaps& m, const StepParams& p, cudaStream_t st) {
  const uint64_t blocks = (uint64_t)((p.geo.nx + kW - 1) / kW) * p.nrows;
  // programmatic stream serialisation: this launch may begin while the previous kernel
  // of the stream drains (the kernel waits for it before touching global memory)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(kW);
  cfg.dynamicSmemBytes = TmaLayout<kStore, kW>::kBytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, step_tma<kStore, kW, kModel, kNoise, kGhostNeq, kPhiRho0>, *m.load,
                            *m.store, p);
}

}  // namespace rflbm_dev
