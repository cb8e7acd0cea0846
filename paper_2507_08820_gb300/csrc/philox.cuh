// Counter-based noise source of the step kernel: Philox4x32-10 (Salmon, Moraes, Dror,
// Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11) and Box-Muller (1958).
// The paper's Eq. 9 needs standard normals r_k and names no generator; this is the
// generator of the library's noise contract (rflbm.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace rflbm_dev {

// Philox4x32 multipliers and Weyl key increments (Salmon et al., SC'11).
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

// Full 64-bit product of two 32-bit words (one wide multiply gives both halves).
__device__ __forceinline__ void mulhilo(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo) {
  const unsigned long long p = (unsigned long long)a * b;
  hi = (uint32_t)(p >> 32);
  lo = (uint32_t)p;
}

// The ten round keys of key (k0, k1): round r uses (k0 + r W0, k1 + r W1) mod 2^32. Kernels
// that take them precomputed from their parameters spend no instructions on the schedule.
struct PhiloxRoundKeys {
  uint32_t k0[10], k1[10];
};
inline PhiloxRoundKeys philox_round_keys(uint32_t k0, uint32_t k1) {
  PhiloxRoundKeys rk;
  for (int r = 0; r < 10; ++r) {
    rk.k0[r] = k0 + (uint32_t)r * kPhiloxW0;
    rk.k1[r] = k1 + (uint32_t)r * kPhiloxW1;
  }
  return rk;
}

// Ten rounds of the Philox4x32 bijection on counter c under key (k0, k1).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo(kPhiloxM0, c.x, hi0, lo0);
    mulhilo(kPhiloxM1, c.z, hi1, lo1);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return c;
}

// Key (k0, k1) with its schedule computed in the rounds.
struct PhiloxKey {
  uint32_t k0, k1;
};
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKey& k) {
  return philox4x32_10(c, k.k0, k.k1);
}

// The same with the round keys given.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxRoundKeys& rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo(kPhiloxM0, c.x, hi0, lo0);
    mulhilo(kPhiloxM1, c.z, hi1, lo1);
    c = make_uint4(hi1 ^ c.y ^ rk.k0[r], lo1, hi0 ^ c.w ^ rk.k1[r], lo0);
  }
  return c;
}

// Single-instruction PTX approximations (relative error near 2^-23 for sqrt and rcp;
// lg2 has an absolute error near 2^-22 on [1/2, 2] and a small relative error elsewhere).
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// One Box-Muller pair from two uint32 draws, returned as radius and direction:
// n0 = r * c, n1 = r * s with r = sqrt(-2 ln u0), (c, s) = (cos 2 pi u1, sin 2 pi u1),
// u = (x + 1/2) 2^-32.
//
// -ln u0 is evaluated without cancellation: for x0 >= 2^31 it is -ln(1 - e) with
// e = 1 - u0 = (~x0 + 1/2) 2^-32 formed exactly from the integer, by the series
// e + e^2/2 + e^3/3 when e < 2^-8 (truncation below 2e-8 relative) and by log2 otherwise,
// so that radii near 0 keep their relative accuracy; log2 near 1 has an absolute error
// near 2^-22, which for e >= 2^-8 is a radius error below 2e-6 absolute.
// The angle is taken in (-pi, pi] where __sincosf is accurate: 2 pi u1 - pi, whose
// cosine and sine are the negatives of those of 2 pi u1.
__device__ __forceinline__ void box_muller(uint32_t x0, uint32_t x1, float& r, float& c,
                                           float& s) {
  const bool upper = (x0 >> 31) != 0u;
  const uint32_t xm = upper ? ~x0 : x0;  // < 2^31
  const float e = fmaf(__uint2float_rn(xm), 0x1p-32f, 0x1p-33f);  // (0, 1/2]
  const float arg = upper ? 1.0f - e : e;
  const float lg = -1.3862943611198906f * lg2_approx(arg);  // -2 ln(arg)
  const float ser = e * fmaf(e, fmaf(e, 0.66666667f, 1.0f), 2.0f);  // 2e + e^2 + 2e^3/3
  r = sqrt_approx((upper && e < 0.00390625f) ? ser : lg);
  const float t = fmaf(__uint2float_rn(x1), 6.283185307179586f * 0x1p-32f,
                       6.283185307179586f * 0x1p-33f - 3.14159265358979f);
  float st, ct;
  __sincosf(t, &st, &ct);
  c = -ct;
  s = -st;
}

// The 24 normals of one site at one step: Box-Muller pair m of call j (m = 2j, 2j + 1)
// gives n[2m] = r cos and n[2m + 1] = r sin, so n[4j .. 4j + 3] come from call j.
struct SiteNoise {
  float n[24];
};

// The two normals of one Box-Muller pair.
__device__ __forceinline__ void box_muller_normals(uint32_t x0, uint32_t x1, float& n0, float& n1) {
  float r, c, s;
  box_muller(x0, x1, r, c, s);
  n0 = __fmul_rn(r, c);
  n1 = __fmul_rn(r, s);
}

// Calls j0 <= j < j1 of site_noise (the draws can be split around other work).
template <int j0, int j1>
__device__ __forceinline__ void site_noise_part(uint32_t site, uint32_t step, uint32_t replica,
                                                uint32_t k0, uint32_t k1, SiteNoise& out) {
#pragma unroll
  for (int j = j0; j < j1; ++j) {
    const uint4 w = philox4x32_10(make_uint4(site, step, (uint32_t)j, replica), k0, k1);
    box_muller_normals(w.x, w.y, out.n[4 * j], out.n[4 * j + 1]);
    box_muller_normals(w.z, w.w, out.n[4 * j + 2], out.n[4 * j + 3]);
  }
}

// The same with the round keys given.
template <int j0, int j1>
__device__ __forceinline__ void site_noise_part(uint32_t site, uint32_t step, uint32_t replica,
                                                const PhiloxRoundKeys& rk, SiteNoise& out) {
#pragma unroll
  for (int j = j0; j < j1; ++j) {
    const uint4 w = philox4x32_10(make_uint4(site, step, (uint32_t)j, replica), rk);
    box_muller_normals(w.x, w.y, out.n[4 * j], out.n[4 * j + 1]);
    box_muller_normals(w.z, w.w, out.n[4 * j + 2], out.n[4 * j + 3]);
  }
}

__device__ __forceinline__ void site_noise(uint32_t site, uint32_t step, uint32_t replica,
                                           uint32_t k0, uint32_t k1, SiteNoise& out) {
  site_noise_part<0, 6>(site, step, replica, k0, k1, out);
}

// Normal n[m] (m = 0..23) of a SiteNoise.
__device__ __forceinline__ float normal_at(const SiteNoise& n, int m) { return n.n[m]; }

}  // namespace rflbm_dev
