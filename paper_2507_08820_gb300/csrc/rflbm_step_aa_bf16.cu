// In-place AA step kernels (step_aa.cuh) for bfloat16 storage.
#include "step_aa.cuh"

namespace rflbm_dev {

cudaError_t launch_step_aa_tma_bf16(const TmaMaps& m, const StepParams& p, const StepVariant& v, bool odd,
                                   cudaStream_t st) {
  return launch_aa_storage<kStoreBF16>(m, p, v, odd, st);
}

}  // namespace rflbm_dev
