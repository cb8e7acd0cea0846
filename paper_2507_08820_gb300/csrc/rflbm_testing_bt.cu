// Measurements of design choices (not production paths). The noise draw of a step on its own
// (rflbm_testing_noise_time). The back transform of Eq. 11 on its own, f_i = w_i sum_k e_ki m_k / b_k
// over tiles of 128 sites, in two forms: the step kernels' sum-factorised float32 FMAs (back_transform of
// collide.cuh), and fifth-generation tensor-core MMA. A measurement of that design choice;
// the step kernels use the FMA form.
//
// MMA form: D[site][i] = sum_k A[site][k] B[i][k] on one tcgen05 kind::f16 MMA tile of
// M = 128 sites x N = 32 populations (27 used), K = 32 modes (27 used), with the float32
// accumulator in tensor memory. B[i][k] = e'_ki = h'_p(c_x) h'_q(c_y) h'_r(c_z) with
// h' = (1, c, 3c^2 - 1): small integers, exact in bfloat16. A[site][k] = M_k / 3^(n_k), n_k the
// number of second-order factors of mode k, so that A B = sum_k e_ki M_k; each thread writes
// its site's row of A split into a bfloat16 high part and a bfloat16 remainder (two MMAs per
// K chunk accumulate both), which keeps about 16 significant bits of M. The threads then read
// their rows back from tensor memory and apply the weights w_i.
//
// The forward projection (Eq. 5) of the moments the step needs, order <= 2, on its own, in the
// same two forms, with the operands the 16-bit storage formats give exactly: the ten raw
// moments m_pqr = sum_i f_i c_x^p c_y^q c_z^r (p + q + r <= 2) of float16 populations. FMA
// form: the step kernels' sum-factorised sweeps (moments_order2 of collide.cuh), in float32.
// MMA form: D[site][k] = sum_i A[site][i] B[k][i] on one tcgen05 kind::f16 tile of M = 128
// sites x N = 16 moments (10 used), K = 32 populations (27 used), float16 operands: A holds the
// populations (exact: they are float16 values), B the products c_x^p c_y^q c_z^r in {-1, 0, 1};
// the float32 accumulator in tensor memory, no split needed.
//
// Both operands sit in shared memory in the canonical K-major layout without swizzling:
// element (row, k) at byte (row % 8) 16 + (row / 8) 512 + (k % 8) 2 + (k / 8) 128, i.e. core
// matrices of 8 rows x 16 bytes, 128 bytes apart along K and 512 bytes apart along the rows.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/rflbm_testing.h"
#include "rflbm_internal.h"
#include "tcgen05.cuh"

namespace rflbm_dev {
namespace {

constexpr int kBtTile = 128;  // sites per CTA: the MMA's M
constexpr int kBtK = 32;      // modes, padded: the MMA's K (two K = 16 instructions)
constexpr int kBtN = 32;      // populations, padded: the MMA's N
constexpr uint32_t kBtPolls = 1u << 22;

// element offset of (row, k) in a canonical K-major operand of 32 columns
__host__ __device__ constexpr int canon(int row, int k) { return (row % 8) * 8 + (row / 8) * 256 + (k % 8) + (k / 8) * 64; }
// scaled 1-D Hermite value h'_p(c) = 1, c, 3c^2 - 1
__host__ __device__ constexpr int hs(int p, int c) { return p == 0 ? 1 : (p == 1 ? c : 3 * c * c - 1); }
// second-order factors of mode k = 9p + 3q + r
__host__ __device__ constexpr int n2_of(int k) { return (k / 9 == 2) + ((k / 3) % 3 == 2) + (k % 3 == 2); }

// The moments of a site: loaded (27 planes of n values), or synthetic values for timing.
template <bool kSynth>
__device__ __forceinline__ void site_moments_in(const float* m, int64_t n, int64_t site, float (&M)[27]) {
#pragma unroll
  for (int k = 0; k < 27; ++k)
    M[k] = kSynth ? 1e-3f * (float)(((uint32_t)site * 2654435761u + 40503u * (uint32_t)k) >> 20) - 2.0f
                  : m[(int64_t)k * n + site];
}

// ---- FMA form: the step kernels' back transform, per thread and site
template <bool kSynth>
__global__ void __launch_bounds__(kBtTile) k_bt_fma(const float* __restrict__ m, int64_t n, int reps,
                                                    float* __restrict__ out) {
  const int64_t site = (int64_t)blockIdx.x * kBtTile + threadIdx.x;
  float Mv[27];
  site_moments_in<kSynth>(m, n, site, Mv);
  float acc[27];
#pragma unroll
  for (int i = 0; i < 27; ++i) acc[i] = 0.0f;
  for (int rep = 0; rep < reps; ++rep) {
    float M[3][3][3], G[3][3][3];
#pragma unroll
    for (int k = 0; k < 27; ++k) M[k / 9][(k / 3) % 3][k % 3] = kSynth ? Mv[k] + 1e-4f * (float)rep : Mv[k];
    back_transform(M, G, LatticeWeight());
#pragma unroll
    for (int i = 0; i < 27; ++i) acc[i] += G[i / 9][(i / 3) % 3][i % 3];
  }
#pragma unroll
  for (int i = 0; i < 27; ++i) out[(int64_t)i * n + site] = acc[i];
}

// ---- MMA form
template <bool kSynth>
__global__ void __launch_bounds__(kBtTile) k_bt_mma(const float* __restrict__ m, int64_t n, int reps,
                                                    float* __restrict__ out, int* err) {
  __shared__ __align__(1024) __nv_bfloat16 sA[2][kBtTile * kBtK];  // high parts, remainders
  __shared__ __align__(1024) __nv_bfloat16 sB[kBtN * kBtK];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_base;
  const int t = threadIdx.x, warp = t >> 5;
  const int64_t site = (int64_t)blockIdx.x * kBtTile + t;

  for (int e = t; e < kBtN * kBtK; e += kBtTile) {
    const int i = e / kBtK, k = e % kBtK;
    const int v = (i < 27 && k < 27) ? hs(k / 9, i / 9 - 1) * hs((k / 3) % 3, (i / 3) % 3 - 1) * hs(k % 3, i % 3 - 1) : 0;
    sB[canon(i, k)] = __float2bfloat16((float)v);
  }
  if (t == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  if (warp == 0) tmem_alloc(&tmem_base, 32);
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tmem = tmem_base;

  float Mv[27];
  site_moments_in<kSynth>(m, n, site, Mv);
  float acc[27];
#pragma unroll
  for (int i = 0; i < 27; ++i) acc[i] = 0.0f;
  uint32_t phase = 0;
  bool ok = true;
  for (int rep = 0; rep < reps && ok; ++rep) {
    // this site's row of A: M_k / 3^n_k as a bfloat16 high part and remainder, 8 modes per
    // 16-byte store
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      __align__(16) __nv_bfloat162 hi[4], lo[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        float v[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int k = 8 * j + 2 * h + e;
          const float scale = n2_of(k) == 0 ? 1.0f : (n2_of(k) == 1 ? 1.0f / 3.0f : (n2_of(k) == 2 ? 1.0f / 9.0f : 1.0f / 27.0f));
          v[e] = k < 27 ? (kSynth ? Mv[k] + 1e-4f * (float)rep : Mv[k]) * scale : 0.0f;
        }
        hi[h] = __floats2bfloat162_rn(v[0], v[1]);
        const float2 back = __bfloat1622float2(hi[h]);
        lo[h] = __floats2bfloat162_rn(v[0] - back.x, v[1] - back.y);
      }
      *reinterpret_cast<uint4*>(&sA[0][canon(t, 8 * j)]) = *reinterpret_cast<const uint4*>(hi);
      *reinterpret_cast<uint4*>(&sA[1][canon(t, 8 * j)]) = *reinterpret_cast<const uint4*>(lo);
    }
    fence_proxy_async_smem();  // the rows become visible to the tensor core's reads
    __syncthreads();
    if (t == 0) {
      tc_fence_after_sync();
      constexpr uint32_t idesc = idesc_bf16_f32(kBtTile, kBtN);
#pragma unroll
      for (int part = 0; part < 2; ++part)
#pragma unroll
        for (int s = 0; s < 2; ++s)  // K = 16 per instruction: two core matrices along K
          tc_mma_bf16(tmem, smem_desc_noswizzle(smem_addr(&sA[part][0]) + 256u * s, 128u, 512u),
                      smem_desc_noswizzle(smem_addr(&sB[0]) + 256u * s, 128u, 512u), idesc, (part | s) != 0);
      tc_commit(&bar);
    }
    ok = mbar_wait_bounded(&bar, phase, kBtPolls);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (t == 0) atomicOr(err, 1);
      mbar_wait_bounded(&bar, phase ^ 1u, kBtPolls);  // the MMA in flight completes first
      ok = false;
      break;
    }
    tc_fence_after_sync();
    float D[32];
    tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16), D);
#pragma unroll
    for (int i = 0; i < 27; ++i) acc[i] = fmaf((float)(w1d(i / 9) * w1d((i / 3) % 3) * w1d(i % 3)), D[i], acc[i]);
    tc_fence_before_sync();
    __syncthreads();  // every row is read before the next MMA overwrites the accumulator
  }
  if (ok) {
#pragma unroll
    for (int i = 0; i < 27; ++i) out[(int64_t)i * n + site] = acc[i];
  }
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 32);
}

// ---- the noise draw alone: the 24 normals of every site at one step (6 Philox4x32-10 calls
// and 12 Box-Muller pairs, site_noise), two sites per thread as in the 16-bit step kernels,
// folded into one sum per thread so that nothing but the draw costs time
__global__ void __launch_bounds__(128) k_noise_only(uint32_t nsites, uint32_t step, float* __restrict__ out) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  float acc = 0.0f;
  for (uint32_t s = 2 * tid; s + 1 < nsites; s += 2 * gridDim.x * blockDim.x) {
    SiteNoise a, b;
    site_noise(s, step, 0u, 1u, 0u, a);
    site_noise(s + 1, step, 0u, 1u, 0u, b);
#pragma unroll
    for (int m = 0; m < 23; ++m) acc = fmaf(a.n[m], b.n[m], acc);
  }
  out[tid] = acc;
}

// ---- forward projection: the ten raw moments of order <= 2, in the order of fw_exps
constexpr int kFwN = 16;  // moments, padded: the MMA's N
__host__ __device__ constexpr int fw_exp(int k, int axis) {
  // (p, q, r) of moment k: 1, c_x, c_y, c_z, c_x^2, c_y^2, c_z^2, c_x c_y, c_x c_z, c_y c_z
  return k == 0 ? 0
       : k <= 3 ? (axis == k - 1)
       : k <= 6 ? 2 * (axis == k - 4)
       : k == 7 ? (axis == 0 || axis == 1)
       : k == 8 ? (axis == 0 || axis == 2)
                : (axis == 1 || axis == 2);
}
__host__ __device__ constexpr int ipow(int c, int p) { return p == 0 ? 1 : (p == 1 ? c : c * c); }

// The populations of a site as float16 values: loaded, or synthetic values for timing.
template <bool kSynth>
__device__ __forceinline__ void site_pops_in(const float* f, int64_t n, int64_t site, float (&g)[27]) {
#pragma unroll
  for (int i = 0; i < 27; ++i)
    g[i] = kSynth ? __half2float(__float2half_rn(
                        1e-3f * (float)(((uint32_t)site * 2654435761u + 40503u * (uint32_t)i) >> 20) - 2.0f))
                  : f[(int64_t)i * n + site];
}

template <bool kSynth>
__global__ void __launch_bounds__(kBtTile) k_fw_fma(const float* __restrict__ f, int64_t n, int reps,
                                                    float* __restrict__ out) {
  const int64_t site = (int64_t)blockIdx.x * kBtTile + threadIdx.x;
  float gv[27];
  site_pops_in<kSynth>(f, n, site, gv);
  float acc[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) acc[k] = 0.0f;
  for (int rep = 0; rep < reps; ++rep) {
    float G[3][3][3];
#pragma unroll
    for (int i = 0; i < 27; ++i) G[i / 9][(i / 3) % 3][i % 3] = kSynth ? gv[i] + 1e-4f * (float)rep : gv[i];
    float drho, jx, jy, jz, sxy, sxz, syz, axx, ayy, azz;
    moments_order2(G, drho, jx, jy, jz, sxy, sxz, syz, axx, ayy, azz);
    const float third = drho * (1.0f / 3.0f);  // raw diagonal moments from the Hermite ones
    const float m[10] = {drho, jx, jy, jz, axx + third, ayy + third, azz + third, sxy, sxz, syz};
#pragma unroll
    for (int k = 0; k < 10; ++k) acc[k] += m[k];
  }
#pragma unroll
  for (int k = 0; k < 10; ++k) out[(int64_t)k * n + site] = acc[k];
}

// D = A B with float16 operands (kind::f16, A and B of one type), float32 accumulator
__host__ __device__ constexpr uint32_t idesc_f16_f32(int m, int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

template <bool kSynth>
__global__ void __launch_bounds__(kBtTile) k_fw_mma(const float* __restrict__ f, int64_t n, int reps,
                                                    float* __restrict__ out, int* err) {
  __shared__ __align__(1024) __half sA[kBtTile * kBtK];
  __shared__ __align__(1024) __half sB[kFwN * kBtK];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_base;
  const int t = threadIdx.x, warp = t >> 5;
  const int64_t site = (int64_t)blockIdx.x * kBtTile + t;

  for (int e = t; e < kFwN * kBtK; e += kBtTile) {
    const int k = e / kBtK, i = e % kBtK;
    const int cx = i / 9 - 1, cy = (i / 3) % 3 - 1, cz = i % 3 - 1;
    const int v = (k < 10 && i < 27) ? ipow(cx, fw_exp(k, 0)) * ipow(cy, fw_exp(k, 1)) * ipow(cz, fw_exp(k, 2)) : 0;
    sB[canon(k, i)] = __float2half_rn((float)v);
  }
  if (t == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  if (warp == 0) tmem_alloc(&tmem_base, 32);
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tmem = tmem_base;

  float gv[27];
  site_pops_in<kSynth>(f, n, site, gv);
  float acc[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) acc[k] = 0.0f;
  uint32_t phase = 0;
  bool ok = true;
  for (int rep = 0; rep < reps && ok; ++rep) {
    // this site's row of A: its 27 populations as float16, 8 per 16-byte store
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      __align__(16) __half2 h[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i0 = 8 * j + 2 * q;
        const float a = i0 < 27 ? (kSynth ? gv[i0] + 1e-4f * (float)rep : gv[i0]) : 0.0f;
        const float b = i0 + 1 < 27 ? (kSynth ? gv[i0 + 1] + 1e-4f * (float)rep : gv[i0 + 1]) : 0.0f;
        h[q] = __floats2half2_rn(a, b);
      }
      *reinterpret_cast<uint4*>(&sA[canon(t, 8 * j)]) = *reinterpret_cast<const uint4*>(h);
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (t == 0) {
      tc_fence_after_sync();
      constexpr uint32_t idesc = idesc_f16_f32(kBtTile, kFwN);
#pragma unroll
      for (int s = 0; s < 2; ++s)
        tc_mma_bf16(tmem, smem_desc_noswizzle(smem_addr(&sA[0]) + 256u * s, 128u, 512u),
                    smem_desc_noswizzle(smem_addr(&sB[0]) + 256u * s, 128u, 512u), idesc, s != 0);
      tc_commit(&bar);
    }
    ok = mbar_wait_bounded(&bar, phase, kBtPolls);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (t == 0) atomicOr(err, 1);
      mbar_wait_bounded(&bar, phase ^ 1u, kBtPolls);
      ok = false;
      break;
    }
    tc_fence_after_sync();
    float D[32];
    tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16), D);
#pragma unroll
    for (int k = 0; k < 10; ++k) acc[k] += D[k];
    tc_fence_before_sync();
    __syncthreads();
  }
  if (ok) {
#pragma unroll
    for (int k = 0; k < 10; ++k) out[(int64_t)k * n + site] = acc[k];
  }
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 32);
}

int bt_fail(int code, const char* msg, cudaError_t e = cudaSuccess) {
  return record_error(code, msg, e == cudaSuccess ? nullptr : cudaGetErrorString(e));
}

}  // namespace
}  // namespace rflbm_dev

using namespace rflbm_dev;

extern "C" int rflbm_testing_backtransform(int method, const float* m, int64_t n, float* f) {
  if ((method != 0 && method != 1) || !m || !f || n < kBtTile || n % kBtTile)
    return bt_fail(RFLBM_EINVAL, "rflbm_testing_backtransform: method 0 or 1, n a positive multiple of 128");
  float *dm = nullptr, *df = nullptr;
  int* derr = nullptr;
  const size_t bytes = sizeof(float) * 27 * (size_t)n;
  cudaError_t e = cudaMalloc(&dm, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&df, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&derr, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(derr, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(dm, m, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    const unsigned blocks = (unsigned)(n / kBtTile);
    if (method == 0) k_bt_fma<false><<<blocks, kBtTile>>>(dm, n, 1, df);
    else k_bt_mma<false><<<blocks, kBtTile>>>(dm, n, 1, df, derr);
    e = cudaGetLastError();
  }
  int err = 0;
  if (e == cudaSuccess) e = cudaMemcpy(f, df, bytes, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&err, derr, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(dm);
  cudaFree(df);
  cudaFree(derr);
  if (e != cudaSuccess) return bt_fail(RFLBM_ECUDA, "rflbm_testing_backtransform", e);
  if (err) return bt_fail(RFLBM_ETIMEOUT, "rflbm_testing_backtransform: a bounded wait for the MMA expired");
  return RFLBM_OK;
}

extern "C" int rflbm_testing_backtransform_time(int method, int64_t tiles, int reps, float* ms) {
  if ((method != 0 && method != 1) || tiles < 1 || reps < 1 || !ms)
    return bt_fail(RFLBM_EINVAL, "rflbm_testing_backtransform_time: invalid arguments");
  const int64_t n = tiles * kBtTile;
  float* dout = nullptr;
  int* derr = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&dout, sizeof(float) * 27 * (size_t)n);
  if (e == cudaSuccess) e = cudaMalloc(&derr, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(derr, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {  // warm-up, then timed
    if (pass == 1) e = cudaEventRecord(e0);
    if (method == 0) k_bt_fma<true><<<(unsigned)tiles, kBtTile>>>(nullptr, n, reps, dout);
    else k_bt_mma<true><<<(unsigned)tiles, kBtTile>>>(nullptr, n, reps, dout, derr);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (pass == 1 && e == cudaSuccess) e = cudaEventRecord(e1);
  }
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  int err = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&err, derr, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(dout);
  cudaFree(derr);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return bt_fail(RFLBM_ECUDA, "rflbm_testing_backtransform_time", e);
  if (err) return bt_fail(RFLBM_ETIMEOUT, "rflbm_testing_backtransform_time: a bounded wait for the MMA expired");
  return RFLBM_OK;
}

extern "C" int rflbm_testing_forward(int method, const float* f, int64_t n, float* m) {
  if ((method != 0 && method != 1) || !f || !m || n < kBtTile || n % kBtTile)
    return bt_fail(RFLBM_EINVAL, "rflbm_testing_forward: method 0 or 1, n a positive multiple of 128");
  float *df = nullptr, *dm = nullptr;
  int* derr = nullptr;
  cudaError_t e = cudaMalloc(&df, sizeof(float) * 27 * (size_t)n);
  if (e == cudaSuccess) e = cudaMalloc(&dm, sizeof(float) * 10 * (size_t)n);
  if (e == cudaSuccess) e = cudaMalloc(&derr, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(derr, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(df, f, sizeof(float) * 27 * (size_t)n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    const unsigned blocks = (unsigned)(n / kBtTile);
    if (method == 0) k_fw_fma<false><<<blocks, kBtTile>>>(df, n, 1, dm);
    else k_fw_mma<false><<<blocks, kBtTile>>>(df, n, 1, dm, derr);
    e = cudaGetLastError();
  }
  int err = 0;
  if (e == cudaSuccess) e = cudaMemcpy(m, dm, sizeof(float) * 10 * (size_t)n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&err, derr, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(df);
  cudaFree(dm);
  cudaFree(derr);
  if (e != cudaSuccess) return bt_fail(RFLBM_ECUDA, "rflbm_testing_forward", e);
  if (err) return bt_fail(RFLBM_ETIMEOUT, "rflbm_testing_forward: a bounded wait for the MMA expired");
  return RFLBM_OK;
}

extern "C" int rflbm_testing_forward_time(int method, int64_t tiles, int reps, float* ms) {
  if ((method != 0 && method != 1) || tiles < 1 || reps < 1 || !ms)
    return bt_fail(RFLBM_EINVAL, "rflbm_testing_forward_time: invalid arguments");
  const int64_t n = tiles * kBtTile;
  float* dout = nullptr;
  int* derr = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&dout, sizeof(float) * 10 * (size_t)n);
  if (e == cudaSuccess) e = cudaMalloc(&derr, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(derr, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {  // warm-up, then timed
    if (pass == 1) e = cudaEventRecord(e0);
    if (method == 0) k_fw_fma<true><<<(unsigned)tiles, kBtTile>>>(nullptr, n, reps, dout);
    else k_fw_mma<true><<<(unsigned)tiles, kBtTile>>>(nullptr, n, reps, dout, derr);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (pass == 1 && e == cudaSuccess) e = cudaEventRecord(e1);
  }
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  int err = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&err, derr, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(dout);
  cudaFree(derr);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return bt_fail(RFLBM_ECUDA, "rflbm_testing_forward_time", e);
  if (err) return bt_fail(RFLBM_ETIMEOUT, "rflbm_testing_forward_time: a bounded wait for the MMA expired");
  return RFLBM_OK;
}

extern "C" int rflbm_testing_noise_time(int64_t nsites, float* ms) {
  if (nsites < 2 || nsites >= (int64_t(1) << 31) || !ms)
    return bt_fail(RFLBM_EINVAL, "rflbm_testing_noise_time: 2 <= nsites < 2^31");
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  const unsigned blocks = (unsigned)std::max(1, sms * 16);
  float* dout = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&dout, sizeof(float) * blocks * 128);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {  // warm-up, then timed
    if (pass == 1) e = cudaEventRecord(e0);
    k_noise_only<<<blocks, 128>>>((uint32_t)nsites, 7u, dout);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (pass == 1 && e == cudaSuccess) e = cudaEventRecord(e1);
  }
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaFree(dout);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return bt_fail(RFLBM_ECUDA, "rflbm_testing_noise_time", e);
  return RFLBM_OK;
}
