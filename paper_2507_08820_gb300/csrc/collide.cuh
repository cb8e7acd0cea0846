// Per-site collision of the Reg-FLBM (Eq. 25) and BGK-FLBM (Eq. 12) in registers.
//
// Input: the 27 pre-collision populations of a site as a 3x3x3 tile G[a][b][c]
// (a = c_x + 1, ...), shifted by the rest state: g_i = f_i - w_i rho0. Output: the
// shifted post-collision populations g*_i = f*_i - w_i rho0 in the same tile, times an
// output weight per entry (the lattice weight, optionally with a storage scale folded in).
//
// Written once for one site per thread (V = float) and for two sites per thread
// (V = float2), whose lane-wise arithmetic issues as packed f32x2 instructions (sm_100
// family: one instruction updates both sites). Every operation is an explicitly rounded
// add, multiply or fused multiply-add, so that every kernel computes a site bit for bit the
// same way, whichever form it uses.
//
// Work per site (all FP32):
//  1. the ten moments of order <= 2 by three sum-factorised sweeps (Eqs. 3-5):
//     delta rho = rho - rho0, j = rho u, and the second Hermite moment
//     a^(2)_ab = sum_i f_i (c_ia c_ib - delta_ab/3);
//  2. the post-collision moments, divided by their norms b_k, in a tile M[p][q][r] of
//     Hermite exponents: the equilibrium coefficients rho u_x^p u_y^q u_z^r (Eq. 21);
//     Reg: the relaxed stress non-equilibrium a^(2) - rho u u (Eq. 20 with Eq. 15) for
//     k = 4..9 and the ghost non-equilibrium of Eq. 22 when omega_g != 1; BGK: omega times
//     the equilibrium coefficients; and phi_k r_k (Eqs. 9-10) for k = 4..26;
//  3. the back transform f_i = w_i sum_k b_k^-1 e_ki m_k (Eq. 11) by three
//     sum-factorised sweeps (4 operations per line of three) and the weights; BGK adds
//     (1 - omega) f (Eq. 12), re-read from shared memory by the kernels that stage their
//     inputs there.
#pragma once

#include <cuda_runtime.h>

#include "d3q27.cuh"
#include "philox.cuh"

namespace rflbm_dev {

enum : int { kModelReg = 0, kModelBgk = 1 };

// The noise amplitude of Eq. 10 for mode k, relative to sqrt(rho), factors into a rate part
// sqrt(kT omega (2 - omega)) shared by the modes of one relaxation rate and the mode part
// sqrt(1 / (cs2 b_k)) = sqrt(3 / b_k), a constant of the lattice (mode_amp).
struct CollideParams {
  float rho0;
  float omega;       // omega_h = 1/tau (the single rate of the BGK model)
  float neq_diag;    // (1 - omega_h) / b for the diagonal stress modes (b = 2/9)
  float neq_off;     // (1 - omega_h) / b for the off-diagonal stress modes (b = 1/9)
  float ghost_keep;  // 1 - omega_g (ghost non-equilibrium kept by the Eq. 22 recursion)
  float sqrt_rho0;   // sqrt(rho0), used when Eq. 10 takes the reference density
  float amp_h;       // sqrt(kT omega_h (2 - omega_h)): the rate part for k = 4..9
  float amp_g;       // sqrt(kT omega_g (2 - omega_g)) for k = 10..26 (BGK: omega_h)
};

// sqrt(3 / b_k) of mode k >= 1: with b = beta_p beta_q beta_r and beta = (1, 1/3, 2/9), every
// h_1 factor of the mode contributes sqrt(3) and every h_2 factor 3 / sqrt(2).
__host__ __device__ constexpr double mode_amp(int k) {
  double a = 1.7320508075688772;  // sqrt(3)
  const int e[3] = {p_of(k), q_of(k), r_of(k)};
  for (int d = 0; d < 3; ++d) a *= e[d] == 1 ? 1.7320508075688772 : (e[d] == 2 ? 2.1213203435596424 : 1.0);
  return a;
}

// e - 1 clamped at 0 (an exponent after one derivative; only used where e >= 1).
__host__ __device__ constexpr int lo(int e) { return e > 0 ? e - 1 : 0; }

// One line of the inverse 1-D transform: values at c = -1, 0, +1 of
// L0 h_0(c) + L1 h_1(c) + L2 h_2(c).
__device__ __forceinline__ void line_inverse(float L0, float L1, float L2, float& om,
                                             float& o0, float& op) {
  const float a = fmaf(2.0f / 3.0f, L2, L0);
  o0 = fmaf(-1.0f / 3.0f, L2, L0);
  om = a - L1;
  op = a + L1;
}

// ---- lane-wise arithmetic
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float vrcp(float a) { return rcp_approx(a); }
__device__ __forceinline__ float vsqrt(float a) { return sqrt_approx(a); }

__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) {
  return __fadd2_rn(a, make_float2(-b.x, -b.y));
}
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vrcp(float2 a) {
  return make_float2(rcp_approx(a.x), rcp_approx(a.y));
}
__device__ __forceinline__ float2 vsqrt(float2 a) {
  return make_float2(sqrt_approx(a.x), sqrt_approx(a.y));
}

template <class V>
__device__ __forceinline__ V splat(float k);
template <>
__device__ __forceinline__ float splat<float>(float k) { return k; }
template <>
__device__ __forceinline__ float2 splat<float2>(float k) { return make_float2(k, k); }

// k a, k a + c for a scalar k
template <class V>
__device__ __forceinline__ V kmul(float k, V a) { return vmul(splat<V>(k), a); }
template <class V>
__device__ __forceinline__ V kfma(float k, V a, V c) { return vfma(splat<V>(k), a, c); }

// One line of the inverse 1-D transform (see line_inverse).
template <class V>
__device__ __forceinline__ void line_inverse_v(V L0, V L1, V L2, V& om, V& o0, V& op) {
  const V a = kfma(2.0f / 3.0f, L2, L0);
  o0 = kfma(-1.0f / 3.0f, L2, L0);
  om = vsub(a, L1);
  op = vadd(a, L1);
}

// Noise sources of the collision: noise(j, n0, n1) gives the normals of the two Box-Muller
// pairs of Philox call j, n0[h] = r cos and n1[h] = r sin of pair h (the normals r_k of modes
// k = 4j + 2h + 4 and 4j + 2h + 5).

// One site per thread, the normals drawn beforehand (SiteNoise).
struct DrawnNoise {
  const SiteNoise& n;
  __device__ __forceinline__ void operator()(int j, float (&n0)[2], float (&n1)[2]) const {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      n0[h] = n.n[4 * j + 2 * h];
      n1[h] = n.n[4 * j + 2 * h + 1];
    }
  }
};

// Philox calls the two-site kernels draw before they wait for the previous step.
constexpr int kPairPreDrawn = 2;

// Two sites per thread (sites site0 and site0 + 1): Philox calls j < kPre drawn beforehand
// by draw() (raw words, while the previous step drains), the later calls when the collision
// needs them. Key: PhiloxKey or PhiloxRoundKeys.
template <int kPre, class Key>
struct PairNoise {
  uint32_t site0, step, replica;
  const Key& key;
  uint4 w[kPre > 0 ? kPre : 1][2];
  __device__ __forceinline__ uint4 call(uint32_t site, int j) const {
    return philox4x32_10(make_uint4(site, step, (uint32_t)j, replica), key);
  }
  __device__ __forceinline__ void draw() {
#pragma unroll
    for (int j = 0; j < kPre; ++j) {
      w[j][0] = call(site0, j);
      w[j][1] = call(site0 + 1u, j);
    }
  }
  __device__ __forceinline__ void operator()(int j, float2 (&n0)[2], float2 (&n1)[2]) const {
    uint4 a, b;
    if (j < kPre) {
      a = w[j < kPre ? j : 0][0];
      b = w[j < kPre ? j : 0][1];
    } else {
      a = call(site0, j);
      b = call(site0 + 1u, j);
    }
    // the radius times cosine and sine of both sites as packed products (rounded as the
    // scalar products of box_muller_normals)
    float2 r[2], c[2], s[2];
    box_muller(a.x, a.y, r[0].x, c[0].x, s[0].x);
    box_muller(b.x, b.y, r[0].y, c[0].y, s[0].y);
    box_muller(a.z, a.w, r[1].x, c[1].x, s[1].x);
    box_muller(b.z, b.w, r[1].y, c[1].y, s[1].y);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      n0[h] = __fmul2_rn(r[h], c[h]);
      n1[h] = __fmul2_rn(r[h], s[h]);
    }
  }
};

// Weight of the tile entry (a, b, c) applied after the back transform: the lattice weight,
// optionally times the storage scale of its velocity class.
struct LatticeWeight {
  __device__ __forceinline__ float operator()(int a, int b, int c) const {
    return float(w1d(a) * w1d(b) * w1d(c));
  }
};

// Adds phi_k r_k (Eqs. 9-10) to the scaled moments M of k = 4..26: M_k += sqrt(3 / b_k)
// sqrt(kT omega_k (2 - omega_k) rho) r_k, the factor of each mode formed once per site (modes
// of equal norm and rate share it).
template <bool kNoise, bool kPhiRho0, class V, class Noise>
__device__ __forceinline__ void inject_noise(V (&M)[3][3][3], V rho, const CollideParams& cp, const Noise& noise) {
  if (kNoise) {
    const V srho = kPhiRho0 ? splat<V>(cp.sqrt_rho0) : vsqrt(rho);
    const V sh = kmul(cp.amp_h, srho), sg = kmul(cp.amp_g, srho);
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      V n0[2], n1[2];
      noise(j, n0, n1);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        // pair m = 2j + h gives r_k of modes k = 2m + 4 (cosine) and 2m + 5 (sine, unused
        // for m = 11); a pair never mixes stress (k < 10) and ghost modes
        const int k0 = 4 * j + 2 * h + 4, k1 = k0 + 1;
        const V s = k0 < 10 ? sh : sg;
        V& M0 = M[p_of(k0)][q_of(k0)][r_of(k0)];
        M0 = vfma(kmul(float(mode_amp(k0)), s), n0[h], M0);
        if (k1 < kQ) {
          const int k1c = k1 < kQ ? k1 : 4;
          V& M1 = M[p_of(k1c)][q_of(k1c)][r_of(k1c)];
          M1 = vfma(kmul(float(mode_amp(k1c)), s), n1[h], M1);
        }
      }
    }
  }
}

// The back transform (Eq. 11; sweep z, then y, then x) of the scaled moments M into the
// tile G, times the output weights.
template <class V, class OutWeight>
__device__ __forceinline__ void back_transform(V (&M)[3][3][3], V (&G)[3][3][3], const OutWeight& outw) {
  V Z[3][3][3];  // [p][q][c]
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 3; ++q)
      line_inverse_v(M[p][q][0], M[p][q][1], M[p][q][2], Z[p][q][0], Z[p][q][1], Z[p][q][2]);
  V Y[3][3][3];  // [p][b][c]
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      line_inverse_v(Z[p][0][c], Z[p][1][c], Z[p][2][c], Y[p][0][c], Y[p][1][c], Y[p][2][c]);
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      V o[3];
      line_inverse_v(Y[0][b][c], Y[1][b][c], Y[2][b][c], o[0], o[1], o[2]);
#pragma unroll
      for (int a = 0; a < 3; ++a) G[a][b][c] = vmul(splat<V>(outw(a, b, c)), o[a]);
    }
}

// The moments of order <= 2 of the shifted populations by three sum-factorised sweeps
// (sweep x, then y, then z): delta rho, j = rho u, the off-diagonal second moments
// sum g c_a c_b and the diagonal second Hermite moments a^(2)_aa.
template <class V>
__device__ __forceinline__ void moments_order2(const V (&G)[3][3][3], V& drho, V& jx, V& jy, V& jz, V& sxy, V& sxz,
                                               V& syz, V& axx, V& ayy, V& azz) {
  V X0[3][3], X1[3][3], X2[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      X2[b][c] = vadd(G[2][b][c], G[0][b][c]);
      X1[b][c] = vsub(G[2][b][c], G[0][b][c]);
      X0[b][c] = vadd(X2[b][c], G[1][b][c]);
    }
  }
  V T00[3], T01[3], T02[3], T10[3], T11[3], T20[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    T02[c] = vadd(X0[2][c], X0[0][c]);
    T01[c] = vsub(X0[2][c], X0[0][c]);
    T00[c] = vadd(T02[c], X0[1][c]);
    T11[c] = vsub(X1[2][c], X1[0][c]);
    T10[c] = vadd(vadd(X1[2][c], X1[0][c]), X1[1][c]);
    T20[c] = vadd(vadd(X2[2][c], X2[0][c]), X2[1][c]);
  }
  const V s002 = vadd(T00[2], T00[0]);
  drho = vadd(s002, T00[1]);
  jz = vsub(T00[2], T00[0]);
  jy = vadd(vadd(T01[0], T01[1]), T01[2]);
  syz = vsub(T01[2], T01[0]);
  const V syy = vadd(vadd(T02[0], T02[1]), T02[2]);
  jx = vadd(vadd(T10[0], T10[1]), T10[2]);
  sxz = vsub(T10[2], T10[0]);
  sxy = vadd(vadd(T11[0], T11[1]), T11[2]);
  const V sxx = vadd(vadd(T20[0], T20[1]), T20[2]);
  const V szz = s002;
  // second Hermite moment of f: sum g (c c) - (drho / 3) delta (the rest state drops out)
  axx = kfma(-1.0f / 3.0f, drho, sxx);
  ayy = kfma(-1.0f / 3.0f, drho, syy);
  azz = kfma(-1.0f / 3.0f, drho, szz);

}

// Supplies the pre-collision value g of tile entry (a, b, c) to BGK-FLBM's (1 - omega) f
// term at the end of the collision. By default the tile itself, which keeps its 27 values in
// registers through the whole collision; kernels that still hold their inputs in shared
// memory pass a reader instead, and the registers are free in between.
struct KeepTile {
  template <class V>
  __device__ __forceinline__ V operator()(int, int, int, V g) const { return g; }
};

// BGK-FLBM (Eq. 12): f* = f^(0) + (1 - omega)(f - f^(0)) + noise, as the back transform of
// omega a_0 + noise (the shifted density mode is omega drho) plus (1 - omega) f.
template <bool kNoise, bool kPhiRho0, class V, class Noise, class OutWeight, class Reload>
__device__ __forceinline__ void collide_tile_bgk(V (&G)[3][3][3], const CollideParams& cp, const Noise& noise,
                                                 const OutWeight& outw, const Reload& reload) {
  V drho, jx, jy, jz, sxy, sxz, syz, axx, ayy, azz;
  moments_order2(G, drho, jx, jy, jz, sxy, sxz, syz, axx, ayy, azz);
  const V rho = vadd(splat<V>(cp.rho0), drho);
  const V inv_rho = vrcp(rho);
  const V ux = vmul(jx, inv_rho), uy = vmul(jy, inv_rho), uz = vmul(jz, inv_rho);
  const float om = cp.omega;
  const V Uy[3] = {splat<V>(1.0f), kmul(3.0f, uy), vmul(kmul(4.5f, uy), uy)};
  const V Uz[3] = {splat<V>(1.0f), kmul(3.0f, uz), vmul(kmul(4.5f, uz), uz)};
  // omega times the equilibrium moments; the shifted density mode is omega drho
  const V RX[3] = {kmul(om, rho), kmul(3.0f * om, jx), vmul(kmul(4.5f * om, jx), ux)};
  V M[3][3][3];
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const V yz = q == 0 ? Uz[r] : (r == 0 ? Uy[q] : vmul(Uy[q], Uz[r]));
        M[p][q][r] = (q == 0 && r == 0) ? RX[p] : vmul(RX[p], yz);
      }
  M[0][0][0] = kmul(om, drho);
  M[0][1][0] = kmul(3.0f * om, jy);
  M[0][0][1] = kmul(3.0f * om, jz);
  inject_noise<kNoise, kPhiRho0>(M, rho, cp, noise);
  // the back transform of Eq. 11 (as back_transform), each output combined with (1 - omega) g
  V Z[3][3][3];
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 3; ++q)
      line_inverse_v(M[p][q][0], M[p][q][1], M[p][q][2], Z[p][q][0], Z[p][q][1], Z[p][q][2]);
  V Y[3][3][3];
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      line_inverse_v(Z[p][0][c], Z[p][1][c], Z[p][2][c], Y[p][0][c], Y[p][1][c], Y[p][2][c]);
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      V o[3];
      line_inverse_v(Y[0][b][c], Y[1][b][c], Y[2][b][c], o[0], o[1], o[2]);
#pragma unroll
      for (int a = 0; a < 3; ++a)
        G[a][b][c] = vfma(splat<V>(1.0f - om), reload(a, b, c, G[a][b][c]), vmul(splat<V>(outw(a, b, c)), o[a]));
    }
}

template <int kModel, bool kNoise, bool kGhostNeq, bool kPhiRho0, class V, class Noise, class OutWeight,
          class Reload = KeepTile>
__device__ __forceinline__ void collide_tile(V (&G)[3][3][3], const CollideParams& cp,
                                          const Noise& noise, const OutWeight& outw,
                                          const Reload& reload = Reload()) {
  if (kModel == kModelBgk) {
    collide_tile_bgk<kNoise, kPhiRho0>(G, cp, noise, outw, reload);
    return;
  }
  // ---- 1. moments of order <= 2
  V drho, jx, jy, jz, sxy, sxz, syz, axx, ayy, azz;
  moments_order2(G, drho, jx, jy, jz, sxy, sxz, syz, axx, ayy, azz);

  // ---- 2. density, velocity and the scaled post-collision moments
  const V rho = vadd(splat<V>(cp.rho0), drho);
  const V inv_rho = vrcp(rho);
  const V ux = vmul(jx, inv_rho), uy = vmul(jy, inv_rho), uz = vmul(jz, inv_rho);
  // U[p] = u^p / beta_p: 1, 3u, 9u^2/2 (index 0 is the constant 1 and never multiplied)
  const V Uy[3] = {splat<V>(1.0f), kmul(3.0f, uy), vmul(kmul(4.5f, uy), uy)};
  const V Uz[3] = {splat<V>(1.0f), kmul(3.0f, uz), vmul(kmul(4.5f, uz), uz)};
  const float om = cp.omega;
  // RX[p] = rho U_x[p]
  const V RX[3] = {rho, kmul(3.0f, jx), vmul(kmul(4.5f, jx), ux)};
  V M[3][3][3];
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const V yz = q == 0 ? Uz[r] : (r == 0 ? Uy[q] : vmul(Uy[q], Uz[r]));
        M[p][q][r] = (q == 0 && r == 0) ? RX[p] : vmul(RX[p], yz);
      }

  const V vom = splat<V>(om);
  {
    // conserved modes are kept exactly
    M[0][0][0] = drho;
    M[0][1][0] = kmul(3.0f, jy);
    M[0][0][1] = kmul(3.0f, jz);
    // stress modes: omega a0/b + (1 - omega) m/b
    M[2][0][0] = vfma(vom, M[2][0][0], kmul(cp.neq_diag, axx));
    M[0][2][0] = vfma(vom, M[0][2][0], kmul(cp.neq_diag, ayy));
    M[0][0][2] = vfma(vom, M[0][0][2], kmul(cp.neq_diag, azz));
    M[1][1][0] = vfma(vom, M[1][1][0], kmul(cp.neq_off, sxy));
    M[1][0][1] = vfma(vom, M[1][0][1], kmul(cp.neq_off, sxz));
    M[0][1][1] = vfma(vom, M[0][1][1], kmul(cp.neq_off, syz));
    if (kGhostNeq) {
      // Eq. 22 closed form: a1 = 1/2 sum_ab a1_ab d^2(u_x^p u_y^q u_z^r)/du_a du_b
      const V rux = vmul(rho, ux), ruy = vmul(rho, uy), ruz = vmul(rho, uz);
      const V nxx = vsub(axx, vmul(rux, ux)), nyy = vsub(ayy, vmul(ruy, uy)),
              nzz = vsub(azz, vmul(ruz, uz));
      const V nxy = vsub(sxy, vmul(rux, uy)), nxz = vsub(sxz, vmul(rux, uz)),
              nyz = vsub(syz, vmul(ruy, uz));
      const V PX[3] = {splat<V>(1.0f), ux, vmul(ux, ux)}, PY[3] = {splat<V>(1.0f), uy, vmul(uy, uy)},
              PZ[3] = {splat<V>(1.0f), uz, vmul(uz, uz)};
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            if (p + q + r < 3) continue;
            V t = splat<V>(0.0f);
            if (p == 2) t = vfma(nxx, vmul(PY[q], PZ[r]), t);
            if (q == 2) t = vfma(nyy, vmul(PX[p], PZ[r]), t);
            if (r == 2) t = vfma(nzz, vmul(PX[p], PY[q]), t);
            if (p >= 1 && q >= 1)
              t = vfma(kmul(float(p * q), nxy), vmul(vmul(PX[lo(p)], PY[lo(q)]), PZ[r]), t);
            if (p >= 1 && r >= 1)
              t = vfma(kmul(float(p * r), nxz), vmul(vmul(PX[lo(p)], PY[q]), PZ[lo(r)]), t);
            if (q >= 1 && r >= 1)
              t = vfma(kmul(float(q * r), nyz), vmul(vmul(PX[p], PY[lo(q)]), PZ[lo(r)]), t);
            M[p][q][r] = kfma(cp.ghost_keep * float(1.0 / bnorm(p, q, r)), t, M[p][q][r]);
          }
    }
  }
  inject_noise<kNoise, kPhiRho0>(M, rho, cp, noise);
  back_transform(M, G, outw);
}

// The collision of one site per thread with its normals drawn beforehand and the lattice
// weights (the storage scale is applied by the caller).
template <int kModel, bool kNoise, bool kGhostNeq, bool kPhiRho0, class Reload = KeepTile>
__device__ __forceinline__ void collide_site(float (&G)[3][3][3], const CollideParams& cp,
                                             const SiteNoise& noise, const Reload& reload = Reload()) {
  collide_tile<kModel, kNoise, kGhostNeq, kPhiRho0>(G, cp, DrawnNoise{noise}, LatticeWeight(), reload);
}

}  // namespace rflbm_dev
