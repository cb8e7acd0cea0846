// The fused stream-and-collide step with TMA staging (boxes whose x edge is a multiple of
// the row-segment width kW in {32, 64, 128}).
//
// One CTA of kW threads updates one row segment [x0, x0 + kW) of one lattice row (y, z).
// The 27 populations of a site are pulled from 9 source rows (y - c_y, z - c_z), shifted
// by -c_x along x. One thread per population (spread over the warps) issues one tiled TMA load of the
// source row segment [x0 - 4, x0 + kW + 4) of plane i into shared memory (27 loads of
// (kW + 8) floats, completion counted on one mbarrier); lanes whose segment touches the
// periodic x edge also fetch the wrapped neighbour with a plain load. While the copies are
// in flight every thread draws the second half of its 24 normals (the first half is drawn
// before the kernel waits for the previous step: programmatic dependent launch lets this
// grid start while the previous one drains). Each thread then reads its 27 values from
// shared memory at fixed offsets (x - c_x within the row), collides in registers, writes
// its 27 results back to shared memory, and the same threads issue 27 tiled TMA stores of the
// row segment into the destination planes.
//
// Every wait on the mbarrier is bounded; a CTA that gives up sets the handle's error flag,
// waits (again bounded) for its copies in flight and exits without storing.
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

template <int kW, int kModel, bool kNoise, bool kGhostNeq, bool kPhiRho0>
__global__ void __launch_bounds__(kW) step_tma_f32(const __grid_constant__ CUtensorMap load_map,
                                                   const __grid_constant__ CUtensorMap store_map,
                                                   const StepParams p) {
  constexpr int kSeg = kW + 8;                 // loaded segment: x0 - 4 .. x0 + kW + 3
  constexpr int kRow = (kSeg + 31) / 32 * 32;  // shared row stride (128-byte multiple)
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  // rows start on 128-byte boundaries of the shared window (the launch adds 128 bytes)
  float* const sm = reinterpret_cast<float*>(smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u));

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
  float patch = 0.0f;
  int patch_at = -1;
  if (t == 0) mbar_arrive_expect_tx(&bar, (uint32_t)(kQ * kSeg * sizeof(float)));
  {
    if (my_pop < kQ) {
      const int i = my_pop;
      const int cx = comp(kPackCx, i), cy = comp(kPackCy, i), cz = comp(kPackCz, i);
      int ys = (int)y - cy, zs = (int)z - cz;
      ys += ys < 0 ? (int)p.geo.ny : 0;
      ys -= ys >= (int)p.geo.ny ? (int)p.geo.ny : 0;
      zs += zs < 0 ? (int)p.geo.nz : 0;
      zs -= zs >= (int)p.geo.nz ? (int)p.geo.nz : 0;
      tma_load_4d(sm + i * kRow, &load_map, (int)x0 - 4, ys, zs, i, &bar);
      // periodic x edge: the element left of x = 0 is x = nx - 1, right of nx - 1 is 0
      const int64_t rowoff = (int64_t)i * p.geo.ps + (int64_t)p.geo.nx * ((int64_t)ys + (int64_t)p.geo.ny * zs);
      if (cx == 1 && x0 == 0) {
        patch = __ldg(p.src + rowoff + (p.geo.nx - 1));
        patch_at = i * kRow + 3;
      } else if (cx == -1 && x0 + kW == p.geo.nx) {
        patch = __ldg(p.src + rowoff);
        patch_at = i * kRow + 4 + kW;
      }
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
  const float* mine = sm + 4 + t;
#pragma unroll
  for (int i = 0; i < kQ; ++i) G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1] = mine[i * kRow - cx_of(i)];

  collide_site<kModel, kNoise, kGhostNeq, kPhiRho0>(G, p.cp, noise);

  __syncthreads();  // every thread has read its inputs: the rows can hold the outputs
  float* out = sm + t;  // output row i at the (128-byte aligned) start of shared row i
#pragma unroll
  for (int i = 0; i < kQ; ++i) out[i * kRow] = G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1];
  fence_proxy_async_smem();
  __syncthreads();
  if (my_pop < kQ) {
    tma_store_4d(&store_map, sm + my_pop * kRow, (int)x0, (int)y, (int)z, my_pop);
    bulk_commit();
    bulk_wait_read();
  }
}

// Persistent, double-buffered variant: a grid of a few CTAs per SM walks the row
// segments (segment T = blockIdx.x + k gridDim.x); while segment k is collided, the 27 TMA
// loads of segment k + 1 are already in flight into the other shared-memory stage.
// Stage reuse: before a stage is reloaded, the lanes that stored from it wait until their
// bulk stores have read it. Barrier phases: stage s is armed once per use, so its k-th
// use (k counted per stage) completes phase parity k & 1.
template <int kW>
struct TmaSegment {
  static __device__ __forceinline__ void issue(const CUtensorMap* load_map, const StepParams& p,
                                               float* stage, uint64_t* bar, uint32_t tile,
                                               uint32_t nseg, float& patch, int& patch_at) {
    constexpr int kSeg = kW + 8;
    constexpr int kRow = (kSeg + 31) / 32 * 32;
    const int t = threadIdx.x;  // warp 0 only
    const uint32_t row = tile / nseg;
    const uint32_t x0 = (tile - row * nseg) * kW;
    const uint32_t z = row / p.geo.ny, y = row - z * p.geo.ny;
    if (t == 0) mbar_arrive_expect_tx(bar, (uint32_t)(kQ * kSeg * sizeof(float)));
    __syncwarp();
    patch_at = -1;
    if (t < kQ) {
      const int i = t;
      const int cx = comp(kPackCx, i), cy = comp(kPackCy, i), cz = comp(kPackCz, i);
      int ys = (int)y - cy, zs = (int)z - cz;
      ys += ys < 0 ? (int)p.geo.ny : 0;
      ys -= ys >= (int)p.geo.ny ? (int)p.geo.ny : 0;
      zs += zs < 0 ? (int)p.geo.nz : 0;
      zs -= zs >= (int)p.geo.nz ? (int)p.geo.nz : 0;
      tma_load_4d(stage + i * kRow, load_map, (int)x0 - 4, ys, zs, i, bar);
      const int64_t rowoff = (int64_t)i * p.geo.ps + (int64_t)p.geo.nx * ((int64_t)ys + (int64_t)p.geo.ny * zs);
      if (cx == 1 && x0 == 0) {
        patch = __ldg(p.src + rowoff + (p.geo.nx - 1));
        patch_at = i * kRow + 3;
      } else if (cx == -1 && x0 + kW == p.geo.nx) {
        patch = __ldg(p.src + rowoff);
        patch_at = i * kRow + 4 + kW;
      }
    }
  }
};

template <int kW, int kModel, bool kNoise, bool kGhostNeq, bool kPhiRho0>
__global__ void __launch_bounds__(kW) step_tma_persistent_f32(
    const __grid_constant__ CUtensorMap load_map, const __grid_constant__ CUtensorMap store_map,
    const StepParams p) {
  constexpr int kSeg = kW + 8;
  constexpr int kRow = (kSeg + 31) / 32 * 32;
  constexpr int kStage = kQ * kRow;  // floats per stage
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[2];
  float* const sm = reinterpret_cast<float*>(smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u));

  const int t = threadIdx.x;
  const uint32_t nseg = p.geo.nx / kW;
  const uint32_t ntiles = nseg * p.geo.ny * p.geo.nz;
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
  }
  __syncthreads();

  float patch_next = 0.0f, patch = 0.0f;
  int patch_next_at = -1, patch_at = -1;
  uint32_t tile = blockIdx.x;
  if (t < 32 && tile < ntiles)
    TmaSegment<kW>::issue(&load_map, p, sm, &bar[0], tile, nseg, patch_next, patch_next_at);

  for (uint32_t k = 0; tile < ntiles; ++k, tile += gridDim.x) {
    const int st = k & 1;
    float* const cur = sm + st * kStage;
    patch = patch_next;
    patch_at = patch_next_at;
    const uint32_t next = tile + gridDim.x;
    if (t < 32 && next < ntiles) {
      if (t < kQ) bulk_wait_read();  // stores that read the other stage are done with it
      __syncwarp();
      TmaSegment<kW>::issue(&load_map, p, sm + (st ^ 1) * kStage, &bar[st ^ 1], next, nseg,
                            patch_next, patch_next_at);
    }
    const uint32_t row = tile / nseg;
    const uint32_t x0 = (tile - row * nseg) * kW;
    const uint32_t z = row / p.geo.ny, y = row - z * p.geo.ny;
    const uint32_t s = x0 + t + p.geo.nx * row;
    SiteNoise noise;
    if (kNoise) site_noise(s, p.step, p.replica, p.key0, p.key1, noise);

    const bool ok = mbar_wait_bounded(&bar[st], (k >> 1) & 1u, kMaxPolls);
    if (__syncthreads_or(!ok)) {
      if (t == 0) atomicOr(p.err, 1);
      mbar_wait_bounded(&bar[st], (k >> 1) & 1u, kMaxPolls);
      mbar_wait_bounded(&bar[st ^ 1], ((k + 1) >> 1) & 1u, kMaxPolls);
      if (t < kQ) bulk_wait_read();
      return;
    }
    if (patch_at >= 0) cur[patch_at] = patch;
    __syncthreads();

    float G[3][3][3];
    const float* mine = cur + 4 + t;
#pragma unroll
    for (int i = 0; i < kQ; ++i) G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1] = mine[i * kRow - cx_of(i)];

    collide_site<kModel, kNoise, kGhostNeq, kPhiRho0>(G, p.cp, noise);

    __syncthreads();
    float* out = cur + t;
#pragma unroll
    for (int i = 0; i < kQ; ++i) out[i * kRow] = G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1];
    fence_proxy_async_smem();
    __syncthreads();
    if (t < kQ) {
      tma_store_4d(&store_map, cur + t * kRow, (int)x0, (int)y, (int)z, t);
      bulk_commit();
    }
  }
  if (t < kQ) bulk_wait_read();
}

template <int kW, int kModel, bool kNoise, bool kGhostNeq, bool kPhiRho0>
static cudaError_t launch_w(const TmaMaps& m, const StepParams& p, cudaStream_t st) {
  const uint64_t blocks = (uint64_t)(p.geo.nx / kW) * p.geo.ny * p.geo.nz;
  const size_t stage = (size_t)kQ * ((kW + 8 + 31) / 32 * 32) * sizeof(float);
  if (m.persistent_sms > 0) {
    auto kern = step_tma_persistent_f32<kW, kModel, kNoise, kGhostNeq, kPhiRho0>;
    const size_t smem = 2 * stage + 128;  // below the 48 KB default for kW <= 128
    static int per_sm = 0;                // resident CTAs per SM, queried once
    if (per_sm <= 0) {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kW, smem) != cudaSuccess ||
          per_sm <= 0)
        per_sm = 1;
    }
    const uint64_t full = (uint64_t)per_sm * (uint64_t)m.persistent_sms;
    const uint64_t grid = blocks < full ? blocks : full;
    kern<<<(unsigned)grid, kW, smem, st>>>(*m.load, *m.store, p);
    return cudaGetLastError();
  }
  // programmatic stream serialisation: this launch may begin while the previous kernel
  // of the stream drains (the kernel waits for it before touching global memory)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(kW);
  cfg.dynamicSmemBytes = stage + 128;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, step_tma_f32<kW, kModel, kNoise, kGhostNeq, kPhiRho0>, *m.load,
                            *m.store, p);
}

template <int kW>
static cudaError_t launch_variant(const TmaMaps& m, const StepParams& p, const StepVariant& v,
                                  cudaStream_t st) {
  if (v.model == kModelBgk) {
    if (!v.noise) return launch_w<kW, kModelBgk, false, false, false>(m, p, st);
    return v.phi_rho0 ? launch_w<kW, kModelBgk, true, false, true>(m, p, st)
                      : launch_w<kW, kModelBgk, true, false, false>(m, p, st);
  }
  if (!v.noise) {
    return v.ghost_neq ? launch_w<kW, kModelReg, false, true, false>(m, p, st)
                       : launch_w<kW, kModelReg, false, false, false>(m, p, st);
  }
  if (v.ghost_neq) {
    return v.phi_rho0 ? launch_w<kW, kModelReg, true, true, true>(m, p, st)
                      : launch_w<kW, kModelReg, true, true, false>(m, p, st);
  }
  return v.phi_rho0 ? launch_w<kW, kModelReg, true, false, true>(m, p, st)
                    : launch_w<kW, kModelReg, true, false, false>(m, p, st);
}

int tma_segment_width(uint32_t nx) {
  if (nx % 128 == 0) return 128;
  if (nx % 64 == 0) return 64;
  if (nx % 32 == 0) return 32;
  return 0;
}

cudaError_t launch_step_tma_f32(const TmaMaps& m, const StepParams& p, const StepVariant& v,
                                cudaStream_t stream) {
  switch (m.width) {
    case 128: return launch_variant<128>(m, p, v, stream);
    case 64: return launch_variant<64>(m, p, v, stream);
    case 32: return launch_variant<32>(m, p, v, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace rflbm_dev
