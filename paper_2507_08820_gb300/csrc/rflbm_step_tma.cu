// Step kernels with TMA staging for float32 storage: the per-segment kernel
// (step_tma.cuh) and a persistent, double-buffered variant; dispatch for all formats.
#include "step_tma.cuh"

namespace rflbm_dev {

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
        patch = __ldg(static_cast<const float*>(p.src) + rowoff + (p.geo.nx - 1));
        patch_at = i * kRow + 3;
      } else if (cx == -1 && x0 + kW == p.geo.nx) {
        patch = __ldg(static_cast<const float*>(p.src) + rowoff);
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
  if (m.persistent_sms > 0) {
    const uint64_t blocks = (uint64_t)(p.geo.nx / kW) * p.geo.ny * p.geo.nz;
    auto kern = step_tma_persistent_f32<kW, kModel, kNoise, kGhostNeq, kPhiRho0>;
    const size_t smem = 2 * (tma_smem_bytes<kStoreF32, kW>() - 128) + 128;  // below 48 KB
    static int per_sm = 0;  // resident CTAs per SM, queried once
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
  return launch_tma_segment<kStoreF32, kW, kModel, kNoise, kGhostNeq, kPhiRho0>(m, p, st);
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

cudaError_t launch_step_tma(const TmaMaps& m, const StepParams& p, const StepVariant& v,
                            cudaStream_t stream) {
  if (v.storage != kStoreF32) {
    if (m.persistent_sms > 0) return cudaErrorInvalidValue;
    return launch_step_tma_16(m, p, v, stream);
  }
  switch (m.width) {
    case 128: return launch_variant<128>(m, p, v, stream);
    case 64: return launch_variant<64>(m, p, v, stream);
    case 32: return launch_variant<32>(m, p, v, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace rflbm_dev
