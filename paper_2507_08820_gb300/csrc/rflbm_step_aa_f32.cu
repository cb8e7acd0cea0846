// In-place AA step kernels (step_aa.cuh) for float32 storage, and the dispatch over the
// storage formats.
#include "step_aa.cuh"

namespace rflbm_dev {

cudaError_t launch_step_aa_tma_f32(const TmaMaps& m, const StepParams& p, const StepVariant& v, bool odd,
                                   cudaStream_t st) {
  return launch_aa_storage<kStoreF32>(m, p, v, odd, st);
}

cudaError_t launch_step_aa_tma(const TmaMaps& m, const StepParams& p, const StepVariant& v, bool odd,
                               cudaStream_t stream) {
  switch (v.storage) {
    case kStoreF32: return launch_step_aa_tma_f32(m, p, v, odd, stream);
    case kStoreF16: return launch_step_aa_tma_f16(m, p, v, odd, stream);
    case kStoreBF16: return launch_step_aa_tma_bf16(m, p, v, odd, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace rflbm_dev
