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

int tma_ragged_width(uint32_t nx, size_t elem) {
  // rows that no width divides but that are whole 16-byte units (the tensor maps' row
  // pitch): the last segment of each row ends past the row. Of the widths whose padded row
  // keeps at least 77 % of the threads busy, the one with the fewest padded threads per
  // measured efficiency of its width (one-site float32 at 128^3: 128 and 192 sites 94-96 %,
  // 96 sites about 91 %, 64 sites 87 %, 32 sites 85 %); 0 when none qualifies.
  if (nx == 0 || (nx * elem) % 16 != 0) return 0;
  const int widths[5] = {128, 192, 96, 64, 32};
  const double eff[5] = {1.0, 1.0, 0.97, 0.92, 0.90};
  int best = 0;
  double best_cost = 0.0;
  for (int k = 0; k < 5; ++k) {
    const uint32_t padded = (nx + widths[k] - 1) / widths[k] * widths[k];
    if (padded > 1.3 * nx) continue;
    const double cost = padded / eff[k];
    if (best == 0 || cost < best_cost) {
      best = widths[k];
      best_cost = cost;
    }
  }
  return best;
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
