// Step kernels with TMA staging for float32 storage (step_tma.cuh), and the dispatch for
// all storage formats.
#include "step_tma.cuh"

namespace rflbm_dev {

template <int kW>
static cudaError_t launch_variant(const TmaMaps& m, const StepParams& p, const StepVariant& v,
                                  cudaStream_t st) {
  constexpr int F = kStoreF32;
  if (tma_uses_pairs(v)) return launch_tma_pair<F, kW, false>(m, p, st);  // kT = 0
  if (v.model == kModelBgk) {
    if (!v.noise) return launch_tma_segment<F, kW, kModelBgk, false, false, false>(m, p, st);
    return v.phi_rho0 ? launch_tma_segment<F, kW, kModelBgk, true, false, true>(m, p, st)
                      : launch_tma_segment<F, kW, kModelBgk, true, false, false>(m, p, st);
  }
  if (!v.noise) {
    return v.ghost_neq ? launch_tma_segment<F, kW, kModelReg, false, true, false>(m, p, st)
                       : launch_tma_segment<F, kW, kModelReg, false, false, false>(m, p, st);
  }
  if (v.ghost_neq) {
    return v.phi_rho0 ? launch_tma_segment<F, kW, kModelReg, true, true, true>(m, p, st)
                      : launch_tma_segment<F, kW, kModelReg, true, true, false>(m, p, st);
  }
  return v.phi_rho0 ? launch_tma_segment<F, kW, kModelReg, true, false, true>(m, p, st)
                    : launch_tma_segment<F, kW, kModelReg, true, false, false>(m, p, st);
}

bool tma_uses_pairs(const StepVariant& v) {
  // two sites per thread where it measured faster: every 16-bit Reg step (issue-bound; the
  // packed arithmetic saves a fifth of the instructions) and the float32 step without noise.
  // The float32 fluctuating step stays at one site per thread, where the halved occupancy
  // of the two-site form costs more than the instructions it saves.
  if (v.model != kModelReg || v.ghost_neq || (v.noise && v.phi_rho0)) return false;
  return v.storage != kStoreF32 || !v.noise;
}

bool aa_uses_pairs(const StepVariant& v, bool odd, bool full_row) {
  if (tma_uses_pairs(v)) return true;
  // float32 fluctuating odd steps whose stores go straight to the neighbours (rows of
  // several segments): the two sites of a thread share the address arithmetic of the 27
  // stores, which outweighs the lower occupancy (256^3: 94.9 % against 87.9 %). Where the
  // odd step stores rotated whole rows the one-site form stays faster (128^3: 94.3 % against
  // 90.0 % for the pair).
  return odd && !full_row && v.model == kModelReg && !v.ghost_neq && !v.phi_rho0 && v.noise;
}

int tma_segment_width(uint32_t nx) {
  // the widest segment that tiles the row: wider CTAs amortise their fixed costs (128 sites
  // measured 94 %, 64 sites 87 %, 32 sites 85 % of the copy bandwidth at 128^3)
  if (nx % 128 == 0) return 128;
  if (nx % 192 == 0) return 192;
  if (nx % 96 == 0) return 96;
  if (nx % 64 == 0) return 64;
  if (nx % 32 == 0) return 32;
  return 0;
}

cudaError_t launch_step_tma(const TmaMaps& m, const StepParams& p, const StepVariant& v,
                            cudaStream_t stream) {
  if (v.storage != kStoreF32) return launch_step_tma_16(m, p, v, stream);
  switch (m.width) {
    case 128: return launch_variant<128>(m, p, v, stream);
    case 192: return launch_variant<192>(m, p, v, stream);
    case 96: return launch_variant<96>(m, p, v, stream);
    case 64: return launch_variant<64>(m, p, v, stream);
    case 32: return launch_variant<32>(m, p, v, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace rflbm_dev
