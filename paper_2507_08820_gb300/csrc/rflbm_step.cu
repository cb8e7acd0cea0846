// The fused stream-and-collide step (Eq. 25 / Eq. 12 followed by Eq. 8) in the pull
// layout, for any box: the general kernel.
//
// One thread per site. The thread gathers the 27 pre-collision populations of its site
// from the 27 neighbours x - c_i (periodic wrap; consecutive threads read consecutive
// addresses of every plane, so each warp-wide load is one coalesced row segment), draws
// its 24 normals (Philox4x32-10 + Box-Muller, independent of the loads so that the
// arithmetic overlaps the memory latency), collides in registers and writes the 27
// post-collision values to its own site of the other buffer (27 coalesced stores).
// Algorithmic traffic per site update: 27 populations read + 27 written (216 bytes in
// float32, 108 bytes in 16-bit storage).
#include "rflbm_internal.h"

namespace rflbm_dev {

template <int kStore, int kModel, bool kNoise, bool kGhostNeq, bool kPhiRho0>
__global__ void __launch_bounds__(kStepBlock) step_pull(const StepParams p) {
  using S = Storage<kStore>;
  using T = typename S::T;
  // local site s of the launched rows (see StepParams); a z-slab's buffer holds it zlo rows up
  const uint32_t q = blockIdx.x * kStepBlock + threadIdx.x;
  if (q >= p.nrows * p.geo.nx) return;
  const uint32_t s = p.row0 * p.geo.nx + q + (q >= p.row_split * p.geo.nx ? p.row_gap * p.geo.nx : 0u);
  const PullDeltas d = pull_deltas(s, p.geo);
  const int64_t sb = s + (int64_t)p.geo.zlo * p.geo.nxy;
  const T* __restrict__ src = static_cast<const T*>(p.src) + sb;

  float G[3][3][3];
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    // per-thread neighbour pointer plus the plane offset i * ps (uniform across the grid)
    G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1] =
        S::load(__ldg((src + pull_delta(d, i)) + plane_of(i) * p.geo.ps), class_of(i), p.ss);
  }

  SiteNoise noise;
  if (kNoise) site_noise(s + p.geo.site0, p.step, p.replica, p.key0, p.key1, noise);

  collide_site<kModel, kNoise, kGhostNeq, kPhiRho0>(G, p.cp, noise);

  T* __restrict__ dst = static_cast<T*>(p.dst) + sb;
#pragma unroll
  for (int i = 0; i < kQ; ++i)
    dst[plane_of(i) * p.geo.ps] = S::store(G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1], class_of(i), p.ss);
}

// One in-place step of the AA pattern (even or odd form, see step_aa.cuh) for any box.
// Plain loads: the buffer is written during the kernel (each slot by the one thread that
// read it), so the read-only path does not apply.
template <int kStore, bool kOdd, int kModel, bool kNoise>
__global__ void __launch_bounds__(kStepBlock) step_aa_gather(const StepParams p) {
  using S = Storage<kStore>;
  using T = typename S::T;
  const uint32_t q = blockIdx.x * kStepBlock + threadIdx.x;
  if (q >= p.nrows * p.geo.nx) return;
  const uint32_t s = p.row0 * p.geo.nx + q + (q >= p.row_split * p.geo.nx ? p.row_gap * p.geo.nx : 0u);
  T* const buf = static_cast<T*>(p.dst) + s + (int64_t)p.geo.zlo * p.geo.nxy;
  PullDeltas d{};
  if (kOdd) d = pull_deltas(s, p.geo);

  float G[3][3][3];
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    // even: own slot of plane P(i); odd: plane 26 - P(i) at x - c_i
    const int64_t at = kOdd ? (int64_t)(kQ - 1 - plane_of(i)) * p.geo.ps + pull_delta(d, i)
                            : (int64_t)plane_of(i) * p.geo.ps;
    G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1] = S::load(buf[at], class_of(i), p.ss);
  }

  SiteNoise noise;
  if (kNoise) site_noise(s + p.geo.site0, p.step, p.replica, p.key0, p.key1, noise);

  collide_site<kModel, kNoise, false, false>(G, p.cp, noise);

#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    // even: own slot of plane 26 - P(i); odd: plane P(i) at x + c_i
    const int64_t at = kOdd ? (int64_t)plane_of(i) * p.geo.ps + push_delta(d, i)
                            : (int64_t)(kQ - 1 - plane_of(i)) * p.geo.ps;
    buf[at] = S::store(G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1], class_of(i), p.ss);
  }
}

template <int kStore, bool kOdd, int kModel, bool kNoise>
static cudaError_t launch_aa(const StepParams& p, cudaStream_t stream) {
  const uint32_t blocks = (p.nrows * p.geo.nx + kStepBlock - 1) / kStepBlock;
  step_aa_gather<kStore, kOdd, kModel, kNoise><<<blocks, kStepBlock, 0, stream>>>(p);
  return cudaGetLastError();
}

template <int kStore, bool kOdd>
static cudaError_t launch_aa_model(const StepParams& p, const StepVariant& v, cudaStream_t stream) {
  if (v.model == kModelBgk)
    return v.noise ? launch_aa<kStore, kOdd, kModelBgk, true>(p, stream)
                   : launch_aa<kStore, kOdd, kModelBgk, false>(p, stream);
  return v.noise ? launch_aa<kStore, kOdd, kModelReg, true>(p, stream)
                 : launch_aa<kStore, kOdd, kModelReg, false>(p, stream);
}

template <int kStore>
static cudaError_t launch_aa_gather_storage(const StepParams& p, const StepVariant& v, bool odd, cudaStream_t stream) {
  return odd ? launch_aa_model<kStore, true>(p, v, stream) : launch_aa_model<kStore, false>(p, v, stream);
}

cudaError_t launch_step_aa_gather(const StepParams& p, const StepVariant& v, bool odd, cudaStream_t stream) {
  if (v.ghost_neq || v.phi_rho0) return cudaErrorInvalidValue;
  switch (v.storage) {
    case kStoreF32: return launch_aa_gather_storage<kStoreF32>(p, v, odd, stream);
    case kStoreF16: return launch_aa_gather_storage<kStoreF16>(p, v, odd, stream);
    case kStoreBF16: return launch_aa_gather_storage<kStoreBF16>(p, v, odd, stream);
    default: return cudaErrorInvalidValue;
  }
}

template <int kStore, int kModel, bool kNoise, bool kGhostNeq, bool kPhiRho0>
static cudaError_t launch(const StepParams& p, cudaStream_t stream) {
  const uint32_t blocks = (p.nrows * p.geo.nx + kStepBlock - 1) / kStepBlock;
  step_pull<kStore, kModel, kNoise, kGhostNeq, kPhiRho0><<<blocks, kStepBlock, 0, stream>>>(p);
  return cudaGetLastError();
}

// 16-bit storage supports the paper's configuration (omega_g = 1, local rho in Eq. 10).
template <int kStore>
static cudaError_t launch_16(const StepParams& p, const StepVariant& v, cudaStream_t stream) {
  if (v.ghost_neq || v.phi_rho0) return cudaErrorInvalidValue;
  if (v.model == kModelBgk)
    return v.noise ? launch<kStore, kModelBgk, true, false, false>(p, stream)
                   : launch<kStore, kModelBgk, false, false, false>(p, stream);
  return v.noise ? launch<kStore, kModelReg, true, false, false>(p, stream)
                 : launch<kStore, kModelReg, false, false, false>(p, stream);
}

cudaError_t launch_step_gather(const StepParams& p, const StepVariant& v, cudaStream_t stream) {
  if (v.storage == kStoreF16) return launch_16<kStoreF16>(p, v, stream);
  if (v.storage == kStoreBF16) return launch_16<kStoreBF16>(p, v, stream);
  constexpr int F = kStoreF32;
  if (v.model == kModelBgk) {
    if (!v.noise) return launch<F, kModelBgk, false, false, false>(p, stream);
    return v.phi_rho0 ? launch<F, kModelBgk, true, false, true>(p, stream)
                      : launch<F, kModelBgk, true, false, false>(p, stream);
  }
  if (!v.noise) {
    return v.ghost_neq ? launch<F, kModelReg, false, true, false>(p, stream)
                       : launch<F, kModelReg, false, false, false>(p, stream);
  }
  if (v.ghost_neq) {
    return v.phi_rho0 ? launch<F, kModelReg, true, true, true>(p, stream)
                      : launch<F, kModelReg, true, true, false>(p, stream);
  }
  return v.phi_rho0 ? launch<F, kModelReg, true, false, true>(p, stream)
                    : launch<F, kModelReg, true, false, false>(p, stream);
}

}  // namespace rflbm_dev
