// Kernels around the step: initial states, population import/export in the pull layout,
// FP64 moments and global diagnostics, and the noise-source test kernels. Every kernel
// that touches the populations is instantiated for the three storage formats.
#include "rflbm_aux.h"

namespace rflbm_dev {

constexpr int kAuxBlock = 256;

__device__ __forceinline__ uint32_t site_of(int64_t t) { return (uint32_t)t; }

// One 1-D factor of the product-form equilibrium (Eq. 26 factorised over the axes):
// Psi(0, u) = 2/3 - u^2, Psi(+-1, u) = (1/3 +- u + u^2)/2.
__device__ __forceinline__ double psi(int c, double u) {
  return c == 0 ? (2.0 / 3.0 - u * u) : 0.5 * (1.0 / 3.0 + c * u + u * u);
}

// ---------------------------------------------------------------- initial states
template <int kStore>
__global__ void k_init_field(Geometry g, float rho0, StoreScale ss, const double* __restrict__ rho,
                             const double* __restrict__ u, typename Storage<kStore>::T* __restrict__ dst) {
  using S = Storage<kStore>;
  const int64_t s = (int64_t)blockIdx.x * kAuxBlock + threadIdx.x;
  if (s >= g.n) return;
  const double r = rho ? rho[s] : (double)rho0;
  const double ux = u ? u[s] : 0.0, uy = u ? u[g.n + s] : 0.0, uz = u ? u[2 * (int64_t)g.n + s] : 0.0;
  // scatter f_i(x) to plane i at x - c_i
  const Neighbours nb = neighbours(site_of(s), g);
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const double f = r * psi(cx_of(i), ux) * psi(cy_of(i), uy) * psi(cz_of(i), uz);
    dst[pop_slot(g, nb, site_of(s), i)] = S::store((float)(f - weight_of(i) * (double)rho0), class_of(i), ss);
  }
}

// Population with the velocity of tile entry (a, b, c) = (c_x + 1, c_y + 1, c_z + 1).
__host__ __device__ constexpr int pop_at(int a, int b, int c) {
  for (int k = 0; k < kQ; ++k)
    if (cx_of(k) == a - 1 && cy_of(k) == b - 1 && cz_of(k) == c - 1) return k;
  return 0;
}

// Thermal initial state: every mode of every site an independent normal of variance
// rho0 kT b_k / cs2 (the variance the amplitude of Eq. 10 maintains) around the rest
// state, drawn with Philox calls j = 6..12 of counter (site, 0, j, replica) (the step
// draws use j = 0..5). The scaled moments M = m_k / b_k = sqrt(3 rho0 kT / b_k) n_k go
// through the back transform of Eq. 11 (three sweeps of 1-D lines, then the weights).
template <int kStore>
__global__ void k_init_thermal(Geometry g, float rho0, float kT, StoreScale ss, uint32_t key0, uint32_t key1,
                               uint32_t replica, typename Storage<kStore>::T* __restrict__ dst) {
  using S = Storage<kStore>;
  const int64_t s = (int64_t)blockIdx.x * kAuxBlock + threadIdx.x;
  if (s >= g.n) return;
  float nrm[28];
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    const uint4 w = philox4x32_10(make_uint4(site_of(s) + g.site0, 0u, 6u + (uint32_t)j, replica), key0, key1);
    float r, c, sn;
    box_muller(w.x, w.y, r, c, sn);
    nrm[4 * j] = r * c;
    nrm[4 * j + 1] = r * sn;
    box_muller(w.z, w.w, r, c, sn);
    nrm[4 * j + 2] = r * c;
    nrm[4 * j + 3] = r * sn;
  }
  float M[3][3][3];
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
      for (int r = 0; r < 3; ++r)
        M[p][q][r] = sqrtf((float)(3.0 * (1.0 / bnorm(p, q, r))) * rho0 * kT) * nrm[mode_of(p, q, r)];
  float Z[3][3][3], Y[3][3][3];
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 3; ++q)
      line_inverse(M[p][q][0], M[p][q][1], M[p][q][2], Z[p][q][0], Z[p][q][1], Z[p][q][2]);
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      line_inverse(Z[p][0][c], Z[p][1][c], Z[p][2][c], Y[p][0][c], Y[p][1][c], Y[p][2][c]);
  const Neighbours nb = neighbours(site_of(s), g);
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float o[3];
      line_inverse(Y[0][b][c], Y[1][b][c], Y[2][b][c], o[0], o[1], o[2]);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        dst[pop_slot(g, nb, site_of(s), pop_at(a, b, c))] =
            S::store((float)(w1d(a) * w1d(b) * w1d(c)) * o[a], class_at(a, b, c), ss);
      }
    }
}

// Import of public-layout populations (double: exact shift in FP64; float: in FP32).
template <class Tin, int kStore>
__global__ void k_set_populations(Geometry g, float rho0, StoreScale ss, const Tin* __restrict__ f,
                                  typename Storage<kStore>::T* __restrict__ dst) {
  using S = Storage<kStore>;
  const int64_t s = (int64_t)blockIdx.x * kAuxBlock + threadIdx.x;
  if (s >= g.n) return;
  const Neighbours nb = neighbours(site_of(s), g);
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const Tin v = f[i * (int64_t)g.n + s] - (Tin)(weight_of(i) * (double)rho0);
    dst[pop_slot(g, nb, site_of(s), i)] = S::store((float)v, class_of(i), ss);
  }
}

template <class Tout, int kStore>
__global__ void k_get_populations(Geometry g, float rho0, StoreScale ss,
                                  const typename Storage<kStore>::T* __restrict__ src, Tout* __restrict__ f) {
  using S = Storage<kStore>;
  const int64_t s = (int64_t)blockIdx.x * kAuxBlock + threadIdx.x;
  if (s >= g.n) return;
  const Neighbours nb = neighbours(site_of(s), g);
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const float v = S::load(src[pop_slot(g, nb, site_of(s), i)], class_of(i), ss);
    f[i * (int64_t)g.n + s] = (Tout)v + (Tout)(weight_of(i) * (double)rho0);
  }
}

template <int kStore>
__global__ void k_get_sites(Geometry g, float rho0, StoreScale ss,
                            const typename Storage<kStore>::T* __restrict__ src,
                            const int64_t* __restrict__ sites, int64_t n, double* __restrict__ f) {
  using S = Storage<kStore>;
  const int64_t j = (int64_t)blockIdx.x * kAuxBlock + threadIdx.x;
  if (j >= n) return;
  const uint32_t s = site_of(sites[j]);
  const Neighbours nb = neighbours(s, g);
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    f[i * n + j] = (double)S::load(src[pop_slot(g, nb, s, i)], class_of(i), ss) +
                   weight_of(i) * (double)rho0;
  }
}

// Raw moments of order <= 2 of the shifted populations of one site, summed in Acc
// (double for the moments export; float for the global diagnostics, whose values are of
// order sqrt(kT) because the rest state is subtracted), returned in FP64.
struct SiteMoments {
  double drho, j[3], s[6];  // s: sum g c_a c_b for xx, yy, zz, xy, xz, yz
};

template <int kStore, class Acc>
__device__ __forceinline__ SiteMoments site_moments(const Geometry& g, uint32_t s,
                                                    const typename Storage<kStore>::T* src,
                                                    const StoreScale& ss) {
  const Neighbours nb = neighbours(s, g);
  using S = Storage<kStore>;
  Acc drho = 0, j0 = 0, j1 = 0, j2 = 0, s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0, s5 = 0;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const Acc v = (Acc)S::load(src[pop_slot(g, nb, s, i)], class_of(i), ss);
    const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
    drho += v;
    if (cx) j0 += cx * v;
    if (cy) j1 += cy * v;
    if (cz) j2 += cz * v;
    if (cx) s0 += v;
    if (cy) s1 += v;
    if (cz) s2 += v;
    if (cx * cy) s3 += cx * cy * v;
    if (cx * cz) s4 += cx * cz * v;
    if (cy * cz) s5 += cy * cz * v;
  }
  SiteMoments m;
  m.drho = drho;
  m.j[0] = j0; m.j[1] = j1; m.j[2] = j2;
  m.s[0] = s0; m.s[1] = s1; m.s[2] = s2; m.s[3] = s3; m.s[4] = s4; m.s[5] = s5;
  return m;
}

template <int kStore>
__global__ void k_moments(Geometry g, float rho0, StoreScale ss,
                          const typename Storage<kStore>::T* __restrict__ src,
                          double* __restrict__ rho, double* __restrict__ u, double* __restrict__ pi) {
  const int64_t s = (int64_t)blockIdx.x * kAuxBlock + threadIdx.x;
  if (s >= g.n) return;
  const SiteMoments m = site_moments<kStore, double>(g, site_of(s), src, ss);
  const double r = (double)rho0 + m.drho;
  if (rho) rho[s] = r;
  if (u) {
#pragma unroll
    for (int a = 0; a < 3; ++a) u[a * (int64_t)g.n + s] = m.j[a] / r;
  }
  if (pi) {
    // Pi_ab = sum_i f_i (c_a c_b - delta_ab/3) = sum_i g_i c_a c_b - delta_ab drho/3
#pragma unroll
    for (int a = 0; a < 6; ++a)
      pi[a * (int64_t)g.n + s] = m.s[a] - (a < 3 ? m.drho / 3.0 : 0.0);
  }
}

// Per-block partial sums: drho, j (3), max |u|, count of unstable sites (non-finite, or
// density not positive).
constexpr int kStatFields = 6;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

template <int kStore>
__global__ void k_stats_partial(Geometry g, float rho0, StoreScale ss,
                                const typename Storage<kStore>::T* __restrict__ src,
                                double* __restrict__ partials) {
  double acc[kStatFields] = {0, 0, 0, 0, 0, 0};
  for (int64_t s = (int64_t)blockIdx.x * kAuxBlock + threadIdx.x; s < g.n;
       s += (int64_t)gridDim.x * kAuxBlock) {
    const SiteMoments m = site_moments<kStore, float>(g, site_of(s), src, ss);
    const double r = (double)rho0 + m.drho;
    // a non-finite site, or one whose density is not positive, counts as unstable
    const bool stable = isfinite(m.drho) && isfinite(m.j[0]) && isfinite(m.j[1]) &&
                        isfinite(m.j[2]) && r > 0.0;
    if (stable) {
      acc[0] += m.drho;
      acc[1] += m.j[0]; acc[2] += m.j[1]; acc[3] += m.j[2];
      const float sp = sqrtf((float)(m.j[0] * m.j[0] + m.j[1] * m.j[1] + m.j[2] * m.j[2])) / fabsf((float)r);
      acc[4] = fmax(acc[4], (double)sp);
    } else {
      acc[5] += 1.0;
    }
  }
  __shared__ double sh[kAuxBlock / 32][kStatFields];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int f = 0; f < kStatFields; ++f) {
    const double v = (f == 4) ? warp_max(acc[f]) : warp_sum(acc[f]);
    if (lane == 0) sh[wid][f] = v;
  }
  __syncthreads();
  if (threadIdx.x < kStatFields) {
    const int f = threadIdx.x;
    double v = sh[0][f];
    for (int w = 1; w < kAuxBlock / 32; ++w) v = (f == 4) ? fmax(v, sh[w][f]) : v + sh[w][f];
    partials[(int64_t)blockIdx.x * kStatFields + f] = v;
  }
}

// Fixed-order final reduction (one warp per field; deterministic for a fixed grid).
__global__ void k_stats_final(const double* __restrict__ partials, int nblocks,
                              double* __restrict__ out) {
  const int f = blockIdx.x;
  double v = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += 32) {
    const double p = partials[(int64_t)b * kStatFields + f];
    v = (f == 4) ? fmax(v, p) : v + p;
  }
  v = (f == 4) ? warp_max(v) : warp_sum(v);
  if (threadIdx.x == 0) out[f] = v;
}

// ---------------------------------------------------------------- noise tests
__global__ void k_philox(const uint32_t* __restrict__ ctr, uint32_t k0, uint32_t k1,
                         uint32_t* __restrict__ out, int64_t n) {
  const int64_t j = (int64_t)blockIdx.x * kAuxBlock + threadIdx.x;
  if (j >= n) return;
  const uint4 w = philox4x32_10(make_uint4(ctr[4 * j], ctr[4 * j + 1], ctr[4 * j + 2], ctr[4 * j + 3]), k0, k1);
  out[4 * j] = w.x; out[4 * j + 1] = w.y; out[4 * j + 2] = w.z; out[4 * j + 3] = w.w;
}

__global__ void k_site_normals(uint32_t k0, uint32_t k1, uint32_t step, uint32_t replica,
                               const uint32_t* __restrict__ sites, int64_t n,
                               float* __restrict__ out) {
  const int64_t j = (int64_t)blockIdx.x * kAuxBlock + threadIdx.x;
  if (j >= n) return;
  SiteNoise nz;
  site_noise(sites[j], step, replica, k0, k1, nz);
#pragma unroll
  for (int m = 0; m < 24; ++m) out[24 * j + m] = normal_at(nz, m);
}

// ---------------------------------------------------------------- state images
// One plane of a state image (pull layout) from the plane of population i of a buffer in
// the natural view: out[y] = plane[y + c_i] under periodic wrap, zeros in the padding.
template <class E>
__global__ void k_image_plane(Geometry g, const E* __restrict__ plane, int cx, int cy, int cz,
                              E* __restrict__ out) {
  const int64_t y = (int64_t)blockIdx.x * kAuxBlock + threadIdx.x;
  if (y >= g.ps) return;
  if (y >= g.n) {
    out[y] = E(0);
    return;
  }
  const Neighbours nb = neighbours((uint32_t)y, g);  // X[a], Y[b], Z[c]: coordinate - (a - 1)
  out[y] = plane[nb.X[1 - cx] + nb.Y[1 - cy] + nb.Z[1 - cz]];
}

// ---------------------------------------------------------------- launchers
static unsigned blocks_for(int64_t n) { return (unsigned)((n + kAuxBlock - 1) / kAuxBlock); }

#define RFLBM_STORE_DISPATCH(kind, CALL)                                   \
  switch (kind) {                                                          \
    case kStoreF32: { constexpr int K = kStoreF32; CALL; } break;          \
    case kStoreF16: { constexpr int K = kStoreF16; CALL; } break;          \
    case kStoreBF16: { constexpr int K = kStoreBF16; CALL; } break;        \
    default: return cudaErrorInvalidValue;                                 \
  }

template <int K>
using ST = typename Storage<K>::T;

cudaError_t launch_init_field(const Geometry& g, float rho0, const StoreScale& ss, int kind,
                              const double* rho, const double* u, void* dst, cudaStream_t st) {
  RFLBM_STORE_DISPATCH(kind, (k_init_field<K><<<blocks_for(g.n), kAuxBlock, 0, st>>>(g, rho0, ss, rho, u, (ST<K>*)dst)));
  return cudaGetLastError();
}
cudaError_t launch_set_populations_f64(const Geometry& g, float rho0, const StoreScale& ss, int kind,
                                       const double* f, void* dst, cudaStream_t st) {
  RFLBM_STORE_DISPATCH(kind, (k_set_populations<double, K><<<blocks_for(g.n), kAuxBlock, 0, st>>>(g, rho0, ss, f, (ST<K>*)dst)));
  return cudaGetLastError();
}
cudaError_t launch_set_populations_f32(const Geometry& g, float rho0, const StoreScale& ss, int kind,
                                       const float* f, void* dst, cudaStream_t st) {
  RFLBM_STORE_DISPATCH(kind, (k_set_populations<float, K><<<blocks_for(g.n), kAuxBlock, 0, st>>>(g, rho0, ss, f, (ST<K>*)dst)));
  return cudaGetLastError();
}
cudaError_t launch_get_populations_f64(const Geometry& g, float rho0, const StoreScale& ss, int kind,
                                       const void* src, double* f, cudaStream_t st) {
  RFLBM_STORE_DISPATCH(kind, (k_get_populations<double, K><<<blocks_for(g.n), kAuxBlock, 0, st>>>(g, rho0, ss, (const ST<K>*)src, f)));
  return cudaGetLastError();
}
cudaError_t launch_get_populations_f32(const Geometry& g, float rho0, const StoreScale& ss, int kind,
                                       const void* src, float* f, cudaStream_t st) {
  RFLBM_STORE_DISPATCH(kind, (k_get_populations<float, K><<<blocks_for(g.n), kAuxBlock, 0, st>>>(g, rho0, ss, (const ST<K>*)src, f)));
  return cudaGetLastError();
}
cudaError_t launch_get_sites(const Geometry& g, float rho0, const StoreScale& ss, int kind,
                             const void* src, const int64_t* sites, int64_t n, double* f,
                             cudaStream_t st) {
  RFLBM_STORE_DISPATCH(kind, (k_get_sites<K><<<blocks_for(n), kAuxBlock, 0, st>>>(g, rho0, ss, (const ST<K>*)src, sites, n, f)));
  return cudaGetLastError();
}
cudaError_t launch_moments(const Geometry& g, float rho0, const StoreScale& ss, int kind,
                           const void* src, double* rho, double* u, double* pi, cudaStream_t st) {
  RFLBM_STORE_DISPATCH(kind, (k_moments<K><<<blocks_for(g.n), kAuxBlock, 0, st>>>(g, rho0, ss, (const ST<K>*)src, rho, u, pi)));
  return cudaGetLastError();
}
int stats_partial_blocks(const Geometry& g, int num_sms) {
  const int64_t want = (g.n + kAuxBlock - 1) / kAuxBlock;
  const int64_t cap = 4 * (int64_t)num_sms;
  return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}
cudaError_t launch_stats(const Geometry& g, float rho0, const StoreScale& ss, int kind,
                         const void* src, double* partials, int nblocks, double* out6,
                         cudaStream_t st) {
  RFLBM_STORE_DISPATCH(kind, (k_stats_partial<K><<<nblocks, kAuxBlock, 0, st>>>(g, rho0, ss, (const ST<K>*)src, partials)));
  k_stats_final<<<kStatFields, 32, 0, st>>>(partials, nblocks, out6);
  return cudaGetLastError();
}
cudaError_t launch_image_plane(const Geometry& g, size_t elem, const void* plane, int cx, int cy, int cz,
                               void* out, cudaStream_t st) {
  if (elem == 4)
    k_image_plane<uint32_t><<<blocks_for(g.ps), kAuxBlock, 0, st>>>(g, (const uint32_t*)plane, cx, cy, cz, (uint32_t*)out);
  else if (elem == 2)
    k_image_plane<uint16_t><<<blocks_for(g.ps), kAuxBlock, 0, st>>>(g, (const uint16_t*)plane, cx, cy, cz, (uint16_t*)out);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}
cudaError_t launch_init_thermal(const Geometry& g, float rho0, float kT, const StoreScale& ss, int kind,
                                uint32_t key0, uint32_t key1, uint32_t replica, void* dst, cudaStream_t st) {
  RFLBM_STORE_DISPATCH(kind, (k_init_thermal<K><<<blocks_for(g.n), kAuxBlock, 0, st>>>(g, rho0, kT, ss, key0, key1,
                                                                                        replica, (ST<K>*)dst)));
  return cudaGetLastError();
}
cudaError_t launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out,
                          int64_t n, cudaStream_t st) {
  k_philox<<<blocks_for(n), kAuxBlock, 0, st>>>(ctr, k0, k1, out, n);
  return cudaGetLastError();
}
cudaError_t launch_site_normals(uint32_t k0, uint32_t k1, uint32_t step, uint32_t replica,
                                const uint32_t* sites, int64_t n, float* out, cudaStream_t st) {
  k_site_normals<<<blocks_for(n), kAuxBlock, 0, st>>>(k0, k1, step, replica, sites, n, out);
  return cudaGetLastError();
}

}  // namespace rflbm_dev
