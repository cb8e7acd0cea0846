// Step kernels with TMA staging for 16-bit storage (float16, bfloat16), the paper's
// configuration only (omega_g = 1, local rho in Eq. 10); the Reg-FLBM steps run two sites
// per thread (step_tma_pair).
#include "step_tma.cuh"

namespace rflbm_dev {

template <int kStore, int kW>
static cudaError_t launch_16_w(const TmaMaps& m, const StepParams& p, const StepVariant& v,
                               cudaStream_t st) {
  if (v.ghost_neq || v.phi_rho0) return cudaErrorInvalidValue;
  if (v.model == kModelBgk)
    return v.noise ? launch_tma_segment<kStore, kW, kModelBgk, true, false, false>(m, p, st)
                   : launch_tma_segment<kStore, kW, kModelBgk, false, false, false>(m, p, st);
  if (tma_uses_pairs(v))
    return v.noise ? launch_tma_pair<kStore, kW, true>(m, p, st) : launch_tma_pair<kStore, kW, false>(m, p, st);
  return v.noise ? launch_tma_segment<kStore, kW, kModelReg, true, false, false>(m, p, st)
                 : launch_tma_segment<kStore, kW, kModelReg, false, false, false>(m, p, st);
}

template <int kStore>
static cudaError_t launch_16_store(const TmaMaps& m, const StepParams& p, const StepVariant& v,
                                   cudaStream_t st) {
  switch (m.width) {
    case 128: return launch_16_w<kStore, 128>(m, p, v, st);
    case 192: return launch_16_w<kStore, 192>(m, p, v, st);
    case 96: return launch_16_w<kStore, 96>(m, p, v, st);
    case 64: return launch_16_w<kStore, 64>(m, p, v, st);
    case 32: return launch_16_w<kStore, 32>(m, p, v, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_step_tma_16(const TmaMaps& m, const StepParams& p, const StepVariant& v,
                               cudaStream_t stream) {
  if (v.storage == kStoreF16) return launch_16_store<kStoreF16>(m, p, v, stream);
  if (v.storage == kStoreBF16) return launch_16_store<kStoreBF16>(m, p, v, stream);
  return cudaErrorInvalidValue;
}

}  // namespace rflbm_dev
