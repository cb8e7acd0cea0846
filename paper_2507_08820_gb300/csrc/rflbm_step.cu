// The fused stream-and-collide step (Eq. 25 / Eq. 12 followed by Eq. 8) for float32
// populations in the pull layout.
//
// One thread per site. The thread gathers the 27 pre-collision populations of its site
// from the 27 neighbours x - c_i (periodic wrap; consecutive threads read consecutive
// addresses of every plane, so each warp-wide load is one coalesced 128-byte row segment),
// draws its 24 normals (Philox4x32-10 + Box-Muller, independent of the loads so that
// the arithmetic overlaps the memory latency), collides in registers and writes the 27
// post-collision values to its own site of the other buffer (27 coalesced stores).
// Algorithmic traffic: 108 bytes read + 108 bytes written per site update.
#include "rflbm_internal.h"

namespace rflbm_dev {

template <int kModel, bool kNoise, bool kGhostNeq, bool kPhiRho0>
__global__ void __launch_bounds__(kStepBlock) step_pull_f32(const StepParams p) {
  const uint32_t s = blockIdx.x * kStepBlock + threadIdx.x;
  if (s >= p.geo.n) return;
  const PullDeltas d = pull_deltas(s, p.geo);
  const float* __restrict__ src = p.src + s;

  float G[3][3][3];
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    // per-thread neighbour pointer plus the plane offset i * ps (uniform across the grid)
    G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1] = __ldg((src + pull_delta(d, i)) + i * p.geo.ps);
  }

  SiteNoise noise;
  if (kNoise) site_noise(s, p.step, p.replica, p.key0, p.key1, noise);

  collide_site<kModel, kNoise, kGhostNeq, kPhiRho0>(G, p.cp, noise);

  float* __restrict__ dst = p.dst + s;
#pragma unroll
  for (int i = 0; i < kQ; ++i) dst[i * p.geo.ps] = G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1];
}

template <int kModel, bool kNoise, bool kGhostNeq, bool kPhiRho0>
static cudaError_t launch(const StepParams& p, cudaStream_t stream) {
  const uint32_t blocks = (p.geo.n + kStepBlock - 1) / kStepBlock;
  step_pull_f32<kModel, kNoise, kGhostNeq, kPhiRho0><<<blocks, kStepBlock, 0, stream>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_step_f32(const StepParams& p, const StepVariant& v, cudaStream_t stream) {
  if (v.model == kModelBgk) {
    if (!v.noise) return launch<kModelBgk, false, false, false>(p, stream);
    return v.phi_rho0 ? launch<kModelBgk, true, false, true>(p, stream)
                      : launch<kModelBgk, true, false, false>(p, stream);
  }
  if (!v.noise) {
    return v.ghost_neq ? launch<kModelReg, false, true, false>(p, stream)
                       : launch<kModelReg, false, false, false>(p, stream);
  }
  if (v.ghost_neq) {
    return v.phi_rho0 ? launch<kModelReg, true, true, true>(p, stream)
                      : launch<kModelReg, true, true, false>(p, stream);
  }
  return v.phi_rho0 ? launch<kModelReg, true, false, true>(p, stream)
                    : launch<kModelReg, true, false, false>(p, stream);
}

}  // namespace rflbm_dev
