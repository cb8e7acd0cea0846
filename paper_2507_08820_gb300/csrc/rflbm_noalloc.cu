// Global diagnostics of caller-owned populations without any run-time allocation.
//
// Some callers cannot allocate device memory when they need these numbers: an application
// whose framework has reserved the device memory for its own pool up front (so that a
// cudaMalloc would fail or, being device-synchronising, would stall a pipeline that must
// not stall), or a monitoring hook that runs between the steps of someone else's solver.
// This entry point reduces their populations with a fixed scratch area that lives in the
// library's static device memory instead: every GPU that loads the library holds
// kNoAllocScratchBytes (about 512 KB) until the process exits.
//
// The reduction is the same as rflbm_stats (FP64 sums of density and momentum, maximum
// speed, unstable sites), applied to populations in the public layout (27 planes of
// n_sites float32 values) rather than to a handle's internal storage. Like rflbm_stats it
// sums the populations shifted by the rest state of unit density, f_i - w_i (the shift
// cancels in the momentum, and sum_i w_i = 1 restores the density), so the per-site
// float32 sums keep the relative precision of the fluctuations. Each block of 256 threads
// reduces a fixed chunk of kNoAllocChunk sites into one partial (deterministic for a given
// n_sites); the last block to finish sums the partials in a fixed order.
//
// The scratch is shared by all calls in the process: calls that overlap on the GPU (two
// streams, or two host threads at once) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/rflbm.h"
#include "rflbm_internal.h"

namespace {

constexpr int kNaThreads = 256;
constexpr int64_t kNoAllocChunk = 16384;     // sites per block (64 per thread)
constexpr int kNoAllocMaxBlocks = 8192;      // partial slots in the scratch
static_assert((int64_t)kNoAllocMaxBlocks * kNoAllocChunk == RFLBM_STATS_NOALLOC_MAX_SITES,
              "capacity must match the public constant");
constexpr int kNaFields = 6;                 // mass, momentum x/y/z, max speed, non-finite
constexpr int kSlot = 8;                     // doubles per partial slot
// words: partial slots, then the result slot, then the completion counter
constexpr int64_t kScratchWords = (int64_t)kNoAllocMaxBlocks * kSlot + kSlot + kSlot;
constexpr int64_t kNoAllocScratchBytes = kScratchWords * (int64_t)sizeof(double);

static_assert(kNoAllocScratchBytes < 600 * 1024, "the static scratch stays modest");
static __device__ __align__(256) double g_noalloc_scratch[kScratchWords];

__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double na_warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__global__ void __launch_bounds__(kNaThreads) k_stats_noalloc(const float* __restrict__ f,
                                                              int64_t n, double* scratch) {
  double acc[kNaFields] = {0, 0, 0, 0, 0, 0};
  const int64_t begin = (int64_t)blockIdx.x * kNoAllocChunk;
  const int64_t end = begin + kNoAllocChunk < n ? begin + kNoAllocChunk : n;
  for (int64_t s = begin + threadIdx.x; s < end; s += kNaThreads) {
    float drho = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
    for (int i = 0; i < rflbm_dev::kQ; ++i) {
      const float v = __ldg(f + i * n + s) - (float)rflbm_dev::weight_of(i);
      drho += v;
      if (rflbm_dev::cx_of(i)) jx += rflbm_dev::cx_of(i) * v;
      if (rflbm_dev::cy_of(i)) jy += rflbm_dev::cy_of(i) * v;
      if (rflbm_dev::cz_of(i)) jz += rflbm_dev::cz_of(i) * v;
    }
    const float rho = 1.0f + drho;
    // a non-finite site, or one whose density is not positive, counts as unstable
    if (isfinite(drho) && isfinite(jx) && isfinite(jy) && isfinite(jz) && rho > 0.0f) {
      acc[0] += drho;
      acc[1] += jx;
      acc[2] += jy;
      acc[3] += jz;
      acc[4] = fmax(acc[4], (double)(sqrtf(jx * jx + jy * jy + jz * jz) / rho));
    } else {
      acc[5] += 1.0;
    }
  }
  __shared__ double sh[kNaThreads / 32][kNaFields];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kNaFields; ++q) {
    const double v = (q == 4) ? na_warp_max(acc[q]) : na_warp_sum(acc[q]);
    if (lane == 0) sh[wid][q] = v;
  }
  __syncthreads();
  double* partial = scratch + (int64_t)blockIdx.x * kSlot;
  if (threadIdx.x < kNaFields) {
    const int q = threadIdx.x;
    double v = sh[0][q];
    for (int w = 1; w < kNaThreads / 32; ++w) v = (q == 4) ? fmax(v, sh[w][q]) : v + sh[w][q];
    partial[q] = v;
  }
  // the last block to finish sums every partial in a fixed order
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + (int64_t)kNoAllocMaxBlocks * kSlot + kSlot);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  double* result = scratch + (int64_t)kNoAllocMaxBlocks * kSlot;
  if (wid < kNaFields) {  // warp q reduces field q: lane l takes blocks l, l + 32, ...
    const int q = wid;
    double v = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) {
      const double p = __ldcg(scratch + (int64_t)b * kSlot + q);
      v = (q == 4) ? fmax(v, p) : v + p;
    }
    v = (q == 4) ? na_warp_max(v) : na_warp_sum(v);
    if (lane == 0) result[q] = v;
  }
  if (threadIdx.x == 0) *counter = 0u;  // ready for the next call
}

int na_fail(int code, const char* msg, cudaError_t e = cudaSuccess) {
  return rflbm_dev::record_error(code, msg, e == cudaSuccess ? nullptr : cudaGetErrorString(e));
}

}  // namespace

extern "C" int rflbm_stats_f32_noalloc(const float* f, int64_t n_sites, void* stream,
                                       rflbm_stats_t* out) {
  if (!f || !out || n_sites < 1) return na_fail(RFLBM_EINVAL, "rflbm_stats_f32_noalloc: invalid arguments");
  if (n_sites > RFLBM_STATS_NOALLOC_MAX_SITES)
    return na_fail(RFLBM_EINVAL,
                   "rflbm_stats_f32_noalloc: n_sites exceeds the fixed scratch capacity of "
                   "134217728 sites (8192 partial sums of 16384 sites)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(RFLBM_ECUDA, "rflbm_stats_f32_noalloc: no current device", e);
  // the device address of the static scratch array on the current device (the host-side
  // symbol is not a device address). Looked up on every call: it allocates nothing, and a
  // cached address would go stale if the caller reset the device (cudaDeviceReset recreates
  // the module's static memory).
  void* sym = nullptr;
  e = cudaGetSymbolAddress(&sym, g_noalloc_scratch);
  if (e != cudaSuccess) return na_fail(RFLBM_ECUDA, "rflbm_stats_f32_noalloc: cudaGetSymbolAddress failed", e);
  double* const scratch = static_cast<double*>(sym);
  cudaStream_t st = (cudaStream_t)stream;
  double* counter = scratch + (int64_t)(kNoAllocMaxBlocks + 1) * kSlot;
  double* result = scratch + (int64_t)kNoAllocMaxBlocks * kSlot;
  // the completion counter must start at zero (an earlier call may have been interrupted)
  e = cudaMemsetAsync(counter, 0, sizeof(double), st);
  if (e != cudaSuccess) return na_fail(RFLBM_ECUDA, "rflbm_stats_f32_noalloc: clearing the counter failed", e);
  const unsigned blocks = (unsigned)((n_sites + kNoAllocChunk - 1) / kNoAllocChunk);
  k_stats_noalloc<<<blocks, kNaThreads, 0, st>>>(f, n_sites, scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(RFLBM_ECUDA, "rflbm_stats_f32_noalloc: launch failed", e);
  double host[kNaFields];
  e = cudaMemcpyAsync(host, result, sizeof(host), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return na_fail(RFLBM_ECUDA, "rflbm_stats_f32_noalloc: reduction failed", e);
  out->step = 0;
  out->mass = (double)n_sites + host[0];  // sum_s rho = N + sum_s sum_i (f_i - w_i)
  out->momentum[0] = host[1];
  out->momentum[1] = host[2];
  out->momentum[2] = host[3];
  out->max_speed = host[4];
  out->nonfinite = (int64_t)host[5];
  if (out->nonfinite > 0) return na_fail(RFLBM_EUNSTABLE, "rflbm_stats_f32_noalloc: non-finite or non-positive densities");
  return RFLBM_OK;
}
