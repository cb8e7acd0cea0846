// The fused stream-and-collide step with TMA staging, for boxes whose x edge is a
// multiple of the row-segment width kW in {32, 64, 128}; templated on the storage format.
//
// One CTA of kW threads updates one row segment [x0, x0 + kW) of one lattice row (y, z).
// The 27 populations of a site are pulled from 9 source rows (y - c_y, z - c_z), shifted
// by -c_x along x. One thread per population (spread over the warps) issues one tiled TMA
// load of the source row segment [x0 - H, x0 + kW + H) of plane i into shared memory
// (H = 4 float32 or 8 16-bit elements: 16-byte aligned coordinates; 27 loads complete on
// one mbarrier); where the segment touches the periodic x edge the wrapped neighbour is
// fetched with a plain load. The first half of the 24 normals is drawn before the kernel
// waits for the previous step (programmatic dependent launch lets this grid start while
// the previous one drains), the second half while the copies are in flight. Each thread
// then reads its 27 values from shared memory at fixed offsets (x - c_x within the row),
// collides in registers in float32, writes its 27 results back to shared memory, and the
// same threads issue 27 tiled TMA stores of the row segment into the destination planes.
//
// Every wait on the mbarrier is bounded; a CTA that gives up sets the handle's error flag,
// waits (again bounded) for its copies in flight and exits without storing.
#pragma once

#include "rflbm_internal.h"
#include "tma.cuh"

namespace rflbm_dev {

// Velocity component of population i for a run-time i (2 bits per population).
__host__ __device__ constexpr uint64_t pack_component(int axis) {
  uint64_t v = 0;
  for (int i = 0; i < kQ; ++i) {
    const int c = axis == 0 ? cx_of(i) : (axis == 1 ? cy_of(i) : cz_of(i));
    v |= (uint64_t)(c + 1) << (2 * i);
  }
  return v;
}
constexpr uint64_t kPackCx = pack_component(0), kPackCy = pack_component(1),
                   kPackCz = pack_component(2);
__device__ __forceinline__ int comp(uint64_t pack, int i) { return (int)((pack >> (2 * i)) & 3u) - 1; }

constexpr uint32_t kMaxPolls = 1u << 22;  // bounded mbarrier waits

template <int kStore, int kW, int kModel, bool kNoise, bool kGhostNeq, bool kPhiRho0>
__global__ void __launch_bounds__(kW) step_tma(const __grid_constant__ CUtensorMap load_map,
                                               const __grid_constant__ CUtensorMap store_map,
                                               const StepParams p) {
  using S = Storage<kStore>;
  using T = typename S::T;
  constexpr int kH = S::kHalo;
  constexpr int kSeg = kW + 2 * kH;                                       // loaded elements
  constexpr int kRow = ((kSeg * (int)sizeof(T) + 127) / 128 * 128) / (int)sizeof(T);  // row stride
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  // rows start on 128-byte boundaries of the shared window (the launch adds 128 bytes)
  T* const sm = reinterpret_cast<T*>(smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u));

  const int t = threadIdx.x;
  const uint32_t nseg = p.geo.nx / kW;
  const uint32_t row = blockIdx.x / nseg;            // y + ny * z
  const uint32_t x0 = (blockIdx.x - row * nseg) * kW;
  const uint32_t z = row / p.geo.ny, y = row - z * p.geo.ny;

  // the next step may start launching now: its CTAs draw their noise while this grid's
  // last CTAs finish; they touch global memory only after their grid_dependency_wait
  grid_launch_dependents();
  const uint32_t s = x0 + t + p.geo.nx * row;
  SiteNoise noise;
  if (kNoise) site_noise_part<0, 3>(s, p.step, p.replica, p.key0, p.key1, noise);

  if (t == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  grid_dependency_wait();  // the previous step's writes (our source) are complete

  // population i is fetched by lane i / nw of warp i % nw (spread over the nw warps)
  constexpr int kWarps = kW / 32;
  const int my_pop = (t & 31) * kWarps + (t >> 5);
  T patch = T();
  int patch_at = -1;
  if (t == 0) mbar_arrive_expect_tx(&bar, (uint32_t)(kQ * kSeg * sizeof(T)));
  if (my_pop < kQ) {
    const int i = my_pop;
    const int cx = comp(kPackCx, i), cy = comp(kPackCy, i), cz = comp(kPackCz, i);
    int ys = (int)y - cy, zs = (int)z - cz;
    ys += ys < 0 ? (int)p.geo.ny : 0;
    ys -= ys >= (int)p.geo.ny ? (int)p.geo.ny : 0;
    zs += zs < 0 ? (int)p.geo.nz : 0;
    zs -= zs >= (int)p.geo.nz ? (int)p.geo.nz : 0;
    tma_load_4d(sm + i * kRow, &load_map, (int)x0 - kH, ys, zs, i, &bar);
    // periodic x edge: the element left of x = 0 is x = nx - 1, right of nx - 1 is 0
    const T* src = static_cast<const T*>(p.src);
    const int64_t rowoff = (int64_t)i * p.geo.ps + (int64_t)p.geo.nx * ((int64_t)ys + (int64_t)p.geo.ny * zs);
    if (cx == 1 && x0 == 0) {
      patch = src[rowoff + (p.geo.nx - 1)];
      patch_at = i * kRow + kH - 1;
    } else if (cx == -1 && x0 + kW == p.geo.nx) {
      patch = src[rowoff];
      patch_at = i * kRow + kH + kW;
    }
  }

  if (kNoise) site_noise_part<3, 6>(s, p.step, p.replica, p.key0, p.key1, noise);

  const bool ok = mbar_wait_bounded(&bar, 0, kMaxPolls);
  if (__syncthreads_or(!ok)) {
    if (t == 0) atomicOr(p.err, 1);
    mbar_wait_bounded(&bar, 0, kMaxPolls);  // let copies in flight land before exiting
    return;
  }
  if (patch_at >= 0) sm[patch_at] = patch;
  __syncthreads();

  float G[3][3][3];
  const T* mine = sm + kH + t;
#pragma unroll
  for (int i = 0; i < kQ; ++i)
    G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1] = S::load(mine[i * kRow - cx_of(i)], class_of(i), p.ss);

  collide_site<kModel, kNoise, kGhostNeq, kPhiRho0>(G, p.cp, noise);

  __syncthreads();  // every thread has read its inputs: the rows can hold the outputs
  T* out = sm + t;  // output row i at the (128-byte aligned) start of shared row i
#pragma unroll
  for (int i = 0; i < kQ; ++i) out[i * kRow] = S::store(G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1], class_of(i), p.ss);
  fence_proxy_async_smem();
  __syncthreads();
  if (my_pop < kQ) {
    tma_store_4d(&store_map, sm + my_pop * kRow, (int)x0, (int)y, (int)z, my_pop);
    bulk_commit();
    bulk_wait_read();
  }
}

// Dynamic shared memory of one CTA (27 rows + 128 bytes of alignment slack).
template <int kStore, int kW>
constexpr size_t tma_smem_bytes() {
  using T = typename Storage<kStore>::T;
  constexpr int kSeg = kW + 2 * Storage<kStore>::kHalo;
  return (size_t)kQ * ((kSeg * sizeof(T) + 127) / 128 * 128) + 128;
}

template <int kStore, int kW, int kModel, bool kNoise, bool kGhostNeq, bool kPhiRho0>
cudaError_t launch_tma_segment(const TmaMaps& m, const StepParams& p, cudaStream_t st) {
  const uint64_t blocks = (uint64_t)(p.geo.nx / kW) * p.geo.ny * p.geo.nz;
  // programmatic stream serialisation: this launch may begin while the previous kernel
  // of the stream drains (the kernel waits for it before touching global memory)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(kW);
  cfg.dynamicSmemBytes = tma_smem_bytes<kStore, kW>();
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
