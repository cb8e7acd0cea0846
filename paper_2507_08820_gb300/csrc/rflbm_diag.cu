// Equilibrium-statistics diagnostics (off the timed path): per-mode sums for the
// fluctuation-dissipation check of every Table II mode, and the static structure factor
// S(|k|) of the hydrodynamic fields by FFT and spherical shell averaging (Sec. III).
#include <cufft.h>

#include "rflbm_diag.h"

namespace rflbm_dev {

constexpr int kDiagBlock = 256;

// All 27 Hermite moments of the shifted populations of one tile G[a][b][c] (Eq. 5 with
// the tensor-product basis of Table II): M[p][q][r] = sum g h_p(c_x) h_q(c_y) h_r(c_z).
__device__ __forceinline__ void all_moments(const float (&G)[3][3][3], float (&M)[3][3][3]) {
  float X[3][3][3];  // [p][b][c]
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float s0 = G[0][b][c] + G[1][b][c] + G[2][b][c];
      X[0][b][c] = s0;
      X[1][b][c] = G[2][b][c] - G[0][b][c];
      X[2][b][c] = fmaf(-1.0f / 3.0f, s0, G[2][b][c] + G[0][b][c]);
    }
  float Y[3][3][3];  // [p][q][c]
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float s0 = X[p][0][c] + X[p][1][c] + X[p][2][c];
      Y[p][0][c] = s0;
      Y[p][1][c] = X[p][2][c] - X[p][0][c];
      Y[p][2][c] = fmaf(-1.0f / 3.0f, s0, X[p][2][c] + X[p][0][c]);
    }
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float s0 = Y[p][q][0] + Y[p][q][1] + Y[p][q][2];
      M[p][q][0] = s0;
      M[p][q][1] = Y[p][q][2] - Y[p][q][0];
      M[p][q][2] = fmaf(-1.0f / 3.0f, s0, Y[p][q][2] + Y[p][q][0]);
    }
}

template <int kStore>
__device__ __forceinline__ void gather_tile(const typename Storage<kStore>::T* __restrict__ src,
                                            const Geometry& g, const StoreScale& ss, uint32_t s,
                                            float (&G)[3][3][3]) {
  const Neighbours nb = neighbours(s, g);
#pragma unroll
  for (int i = 0; i < kQ; ++i)
    G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1] =
        Storage<kStore>::load(src[pop_slot(g, nb, s, i)], class_of(i), ss);
}

// Each thread accumulates up to kDiagSitesPerThread sites in float32, then the block sums
// its 54 values in FP64 into one partial slot.
template <int kStore>
__global__ void __launch_bounds__(kDiagBlock) k_mode_sums(Geometry g, StoreScale ss,
                                                          const typename Storage<kStore>::T* __restrict__ src,
                                                          double* __restrict__ partials) {
  float acc[2 * kQ];
#pragma unroll
  for (int k = 0; k < 2 * kQ; ++k) acc[k] = 0.0f;
  const int64_t base = (int64_t)blockIdx.x * kDiagBlock * kDiagSitesPerThread;
  for (int j = 0; j < kDiagSitesPerThread; ++j) {
    const int64_t s = base + (int64_t)j * kDiagBlock + threadIdx.x;
    if (s >= g.n) break;
    float G[3][3][3], M[3][3][3];
    gather_tile<kStore>(src, g, ss, (uint32_t)s, G);
    all_moments(G, M);
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const int k = mode_of(p, q, r);
          acc[k] += M[p][q][r];
          acc[kQ + k] = fmaf(M[p][q][r], M[p][q][r], acc[kQ + k]);
        }
  }
  __shared__ double sh[kDiagBlock / 32][2 * kQ];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 2 * kQ; ++k) {
    double v = (double)acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[wid][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 2 * kQ) {
    double v = 0.0;
    for (int w = 0; w < kDiagBlock / 32; ++w) v += sh[w][threadIdx.x];
    partials[(int64_t)blockIdx.x * 2 * kQ + threadIdx.x] = v;
  }
}

__global__ void k_reduce_columns(const double* __restrict__ partials, int64_t rows, int cols,
                                 double* __restrict__ out) {
  // one warp per column, fixed order: lane l sums rows l, l + 32, ..., then a fixed tree
  const int col = blockIdx.x;
  double v = 0.0;
  for (int64_t r = threadIdx.x; r < rows; r += 32) v += partials[r * cols + col];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (threadIdx.x == 0) out[col] = v;
}

// Field value of one site, FP64 output from float32 sums of the shifted populations:
// 0 rho - rho0, 1..3 rho u, 4..9 Pi = a^(2) (xx, yy, zz, xy, xz, yz).
template <int kStore>
__global__ void k_field(Geometry g, StoreScale ss, const typename Storage<kStore>::T* __restrict__ src,
                        int field, double* __restrict__ out) {
  const int64_t s = (int64_t)blockIdx.x * kDiagBlock + threadIdx.x;
  if (s >= g.n) return;
  const Neighbours nb = neighbours((uint32_t)s, g);
  float v = 0.0f, drho = 0.0f;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const float x = Storage<kStore>::load(src[pop_slot(g, nb, (uint32_t)s, i)], class_of(i), ss);
    const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
    float w;
    switch (field) {
      case 0: w = 1.0f; break;
      case 1: w = (float)cx; break;
      case 2: w = (float)cy; break;
      case 3: w = (float)cz; break;
      case 4: w = (float)(cx * cx); break;
      case 5: w = (float)(cy * cy); break;
      case 6: w = (float)(cz * cz); break;
      case 7: w = (float)(cx * cy); break;
      case 8: w = (float)(cx * cz); break;
      default: w = (float)(cy * cz); break;
    }
    v = fmaf(w, x, v);
    drho += x;
  }
  // Pi_aa = sum g c_a^2 - drho / 3 (the rest state drops out)
  if (field >= 4 && field <= 6) v -= drho * (1.0f / 3.0f);
  out[s] = (double)v;
}

// Shell sums of |F(k)|^2 / N over the half spectrum of a D2Z transform (kx = 0 .. nx/2),
// each non-redundant vector counted twice. Shell n = round(|k| L / 2 pi) with
// L = max(nx, ny, nz). The sums are reproducible bit for bit: each warp owns a row of
// shell bins in shared memory and its lanes add to it one after another in lane order,
// over a fixed assignment of spectrum entries to warps; the rows are then summed in warp
// order into the block's partial row. (Counts are small integers, exact in any order.)
__global__ void k_shell_bins(Geometry g, const cufftDoubleComplex* __restrict__ spec, int nshell,
                             double* __restrict__ partials) {
  extern __shared__ double bins[];  // [nwarps][nshell] sums, then [nshell] counts
  const int nw = blockDim.x / 32, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int j = threadIdx.x; j < (nw + 1) * nshell; j += blockDim.x) bins[j] = 0.0;
  __syncthreads();
  double* const mine = bins + (size_t)wid * nshell;
  double* const counts = bins + (size_t)nw * nshell;
  const int nxh = g.nx / 2 + 1;
  const int64_t total = (int64_t)g.nz * g.ny * nxh;
  const double L = (double)max(g.nx, max(g.ny, g.nz));
  const double inv_n = 1.0 / (double)g.n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t wbase = (int64_t)blockIdx.x * blockDim.x + 32 * wid; wbase < total; wbase += stride) {
    const int64_t idx = wbase + lane;  // warp-uniform trip count
    int shell = nshell;
    double v = 0.0, w = 0.0;
    if (idx < total) {
      const int kx = (int)(idx % nxh);
      const int ky = (int)((idx / nxh) % g.ny);
      const int kz = (int)(idx / ((int64_t)nxh * g.ny));
      const double fx = (double)kx / g.nx;
      const double fy = (double)(ky <= (int)g.ny / 2 ? ky : ky - (int)g.ny) / g.ny;
      const double fz = (double)(kz <= (int)g.nz / 2 ? kz : kz - (int)g.nz) / g.nz;
      shell = (int)llrint(L * sqrt(fx * fx + fy * fy + fz * fz));
      const bool self = (kx == 0) || ((g.nx % 2 == 0) && kx == (int)g.nx / 2);
      w = self ? 1.0 : 2.0;
      const cufftDoubleComplex c = spec[idx];
      v = w * (c.x * c.x + c.y * c.y) * inv_n;
    }
    const bool ok = shell < nshell;
    if (ok) atomicAdd(&counts[shell], w);
    for (int src = 0; src < 32; ++src) {
      if (lane == src && ok) mine[shell] += v;
      __syncwarp();
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nshell; j += blockDim.x) {
    double sum = 0.0;
    for (int k = 0; k < nw; ++k) sum += bins[(size_t)k * nshell + j];
    partials[(int64_t)blockIdx.x * 2 * nshell + j] = sum;
    partials[(int64_t)blockIdx.x * 2 * nshell + nshell + j] = counts[j];
  }
}

int64_t mode_sum_blocks(const Geometry& g) {
  const int64_t per = (int64_t)kDiagBlock * kDiagSitesPerThread;
  return (g.n + per - 1) / per;
}

template <int K>
using DT = typename Storage<K>::T;

cudaError_t launch_mode_sums(const Geometry& g, const StoreScale& ss, int kind, const void* src,
                             double* partials, double* out54, cudaStream_t st) {
  const int64_t blocks = mode_sum_blocks(g);
  switch (kind) {
    case kStoreF32: k_mode_sums<kStoreF32><<<(unsigned)blocks, kDiagBlock, 0, st>>>(g, ss, (const DT<kStoreF32>*)src, partials); break;
    case kStoreF16: k_mode_sums<kStoreF16><<<(unsigned)blocks, kDiagBlock, 0, st>>>(g, ss, (const DT<kStoreF16>*)src, partials); break;
    case kStoreBF16: k_mode_sums<kStoreBF16><<<(unsigned)blocks, kDiagBlock, 0, st>>>(g, ss, (const DT<kStoreBF16>*)src, partials); break;
    default: return cudaErrorInvalidValue;
  }
  k_reduce_columns<<<2 * kQ, 32, 0, st>>>(partials, blocks, 2 * kQ, out54);
  return cudaGetLastError();
}

cudaError_t launch_field(const Geometry& g, const StoreScale& ss, int kind, const void* src,
                         int field, double* out, cudaStream_t st) {
  const unsigned blocks = (unsigned)((g.n + kDiagBlock - 1) / kDiagBlock);
  switch (kind) {
    case kStoreF32: k_field<kStoreF32><<<blocks, kDiagBlock, 0, st>>>(g, ss, (const DT<kStoreF32>*)src, field, out); break;
    case kStoreF16: k_field<kStoreF16><<<blocks, kDiagBlock, 0, st>>>(g, ss, (const DT<kStoreF16>*)src, field, out); break;
    case kStoreBF16: k_field<kStoreBF16><<<blocks, kDiagBlock, 0, st>>>(g, ss, (const DT<kStoreBF16>*)src, field, out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_shell_bins(const Geometry& g, const void* spec, int nshell, int blocks,
                              double* partials, double* out, cudaStream_t st) {
  // kDiagBlock / 32 rows of sums + one row of counts: up to 221 KB at nshell = 3072
  const size_t smem = sizeof(double) * (size_t)(kDiagBlock / 32 + 1) * (size_t)nshell;
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k_shell_bins, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_shell_bins<<<blocks, kDiagBlock, smem, st>>>(g, (const cufftDoubleComplex*)spec, nshell, partials);
  k_reduce_columns<<<2 * nshell, 32, 0, st>>>(partials, blocks, 2 * nshell, out);
  return cudaGetLastError();
}

}  // namespace rflbm_dev
