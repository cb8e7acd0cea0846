// Per-site collision of the Reg-FLBM (Eq. 25) and BGK-FLBM (Eq. 12) in registers.
//
// Input: the 27 pre-collision populations of one site as a 3x3x3 tile G[a][b][c]
// (a = c_x + 1, ...), shifted by the rest state: g_i = f_i - w_i rho0. Output: the
// shifted post-collision populations g*_i = f*_i - w_i rho0 in the same tile.
//
// Work per site (all FP32):
//  1. the ten moments of order <= 2 by three sum-factorised sweeps (Eqs. 3-5):
//     delta rho = rho - rho0, j = rho u, and the second Hermite moment
//     a^(2)_ab = sum_i f_i (c_ia c_ib - delta_ab/3);
//  2. the post-collision moments, divided by their norms b_k, in a tile M[p][q][r] of
//     Hermite exponents: the equilibrium coefficients rho u_x^p u_y^q u_z^r (Eq. 21),
//     the relaxed stress non-equilibrium a^(2) - rho u u (Eq. 20 with Eq. 15) for
//     k = 4..9, the ghost non-equilibrium of Eq. 22 when omega_g != 1, and
//     phi_k r_k (Eqs. 9-10) for k = 4..26;
//  3. the back transform f_i = w_i sum_k b_k^-1 e_ki m_k (Eq. 11) by three
//     sum-factorised sweeps (4 operations per line of three) and the weights.
#pragma once

#include "d3q27.cuh"
#include "philox.cuh"

namespace rflbm_dev {

enum : int { kModelReg = 0, kModelBgk = 1 };

struct CollideParams {
  float rho0;
  float omega;       // omega_h = 1/tau (the single rate of the BGK model)
  float neq_diag;    // (1 - omega_h) / b for the diagonal stress modes (b = 2/9)
  float neq_off;     // (1 - omega_h) / b for the off-diagonal stress modes (b = 1/9)
  float ghost_keep;  // 1 - omega_g (ghost non-equilibrium kept by the Eq. 22 recursion)
  float sqrt_rho0;   // sqrt(rho0), used when Eq. 10 takes the reference density
  float amp[23];     // sqrt(kT omega_k (2 - omega_k) / (cs2 b_k)) for k = 4..26
};

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

// Supplies the pre-collision value of tile entry (a, b, c) to the BGK update at the end of
// the collision. By default the tile itself, which keeps its 27 values live in registers
// through the whole collision; kernels that still hold the inputs in shared memory pass a
// reader instead, and the registers are free in between.
struct KeepTile {
  __device__ __forceinline__ float operator()(int, int, int, float g) const { return g; }
};

template <int kModel, bool kNoise, bool kGhostNeq, bool kPhiRho0, class Reload = KeepTile>
__device__ __forceinline__ void collide_site(float (&G)[3][3][3], const CollideParams& cp,
                                             const SiteNoise& noise, const Reload& reload = Reload()) {
  // ---- 1. moments of order <= 2 (sweep x, then y, then z)
  float X0[3][3], X1[3][3], X2[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      X2[b][c] = G[2][b][c] + G[0][b][c];
      X1[b][c] = G[2][b][c] - G[0][b][c];
      X0[b][c] = X2[b][c] + G[1][b][c];
    }
  }
  float T00[3], T01[3], T02[3], T10[3], T11[3], T20[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    T02[c] = X0[2][c] + X0[0][c];
    T01[c] = X0[2][c] - X0[0][c];
    T00[c] = T02[c] + X0[1][c];
    T11[c] = X1[2][c] - X1[0][c];
    T10[c] = X1[2][c] + X1[0][c] + X1[1][c];
    T20[c] = X2[2][c] + X2[0][c] + X2[1][c];
  }
  const float s002 = T00[2] + T00[0];
  const float drho = s002 + T00[1];
  const float jz = T00[2] - T00[0];
  const float jy = T01[0] + T01[1] + T01[2];
  const float syz = T01[2] - T01[0];
  const float syy = T02[0] + T02[1] + T02[2];
  const float jx = T10[0] + T10[1] + T10[2];
  const float sxz = T10[2] - T10[0];
  const float sxy = T11[0] + T11[1] + T11[2];
  const float sxx = T20[0] + T20[1] + T20[2];
  const float szz = s002;
  // second Hermite moment of f: sum g (c c) - (drho / 3) delta (the rest state drops out)
  const float third_drho = drho * (1.0f / 3.0f);
  const float axx = sxx - third_drho, ayy = syy - third_drho, azz = szz - third_drho;

  // ---- 2. density, velocity and the scaled post-collision moments
  const float rho = cp.rho0 + drho;
  const float inv_rho = rcp_approx(rho);
  const float ux = jx * inv_rho, uy = jy * inv_rho, uz = jz * inv_rho;
  // U[p] = u^p / beta_p: 1, 3u, 9u^2/2 ; RX[p] = rho U_x[p]
  const float Uy[3] = {1.0f, 3.0f * uy, 4.5f * uy * uy};
  const float Uz[3] = {1.0f, 3.0f * uz, 4.5f * uz * uz};
  // BGK scales every equilibrium moment by omega: fold it into the x factor
  const float om = cp.omega;
  const float rs = kModel == kModelBgk ? om * rho : rho;
  const float RX[3] = {rs, (3.0f * (kModel == kModelBgk ? om : 1.0f)) * jx, 4.5f * (kModel == kModelBgk ? om * jx : jx) * ux};
  float M[3][3][3];
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
      for (int r = 0; r < 3; ++r) M[p][q][r] = RX[p] * (Uy[q] * Uz[r]);

  if (kModel == kModelReg) {
    // conserved modes are kept exactly
    M[0][0][0] = drho;
    M[0][1][0] = 3.0f * jy;
    M[0][0][1] = 3.0f * jz;
    // stress modes: omega a0/b + (1 - omega) m/b
    M[2][0][0] = fmaf(om, M[2][0][0], cp.neq_diag * axx);
    M[0][2][0] = fmaf(om, M[0][2][0], cp.neq_diag * ayy);
    M[0][0][2] = fmaf(om, M[0][0][2], cp.neq_diag * azz);
    M[1][1][0] = fmaf(om, M[1][1][0], cp.neq_off * sxy);
    M[1][0][1] = fmaf(om, M[1][0][1], cp.neq_off * sxz);
    M[0][1][1] = fmaf(om, M[0][1][1], cp.neq_off * syz);
    if (kGhostNeq) {
      // Eq. 22 closed form: a1 = 1/2 sum_ab a1_ab d^2(u_x^p u_y^q u_z^r)/du_a du_b
      const float rux = rho * ux, ruy = rho * uy, ruz = rho * uz;
      const float nxx = axx - rux * ux, nyy = ayy - ruy * uy, nzz = azz - ruz * uz;
      const float nxy = sxy - rux * uy, nxz = sxz - rux * uz, nyz = syz - ruy * uz;
      const float PX[3] = {1.0f, ux, ux * ux}, PY[3] = {1.0f, uy, uy * uy},
                  PZ[3] = {1.0f, uz, uz * uz};
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            if (p + q + r < 3) continue;
            float t = 0.0f;
            if (p == 2) t = fmaf(nxx, PY[q] * PZ[r], t);
            if (q == 2) t = fmaf(nyy, PX[p] * PZ[r], t);
            if (r == 2) t = fmaf(nzz, PX[p] * PY[q], t);
            if (p >= 1 && q >= 1) t = fmaf(nxy * float(p * q), PX[lo(p)] * PY[lo(q)] * PZ[r], t);
            if (p >= 1 && r >= 1) t = fmaf(nxz * float(p * r), PX[lo(p)] * PY[q] * PZ[lo(r)], t);
            if (q >= 1 && r >= 1) t = fmaf(nyz * float(q * r), PX[p] * PY[lo(q)] * PZ[lo(r)], t);
            M[p][q][r] = fmaf(cp.ghost_keep * float(1.0 / bnorm(p, q, r)), t, M[p][q][r]);
          }
    }
  } else {
    // BGK: omega f^(0) here (omega is in RX), (1 - omega) f added after the back
    // transform; the shifted density mode is omega drho
    M[0][0][0] = om * drho;
    M[0][1][0] = om * (3.0f * jy);
    M[0][0][1] = om * (3.0f * jz);
  }
  if (kNoise) {
    // Box-Muller pair m gives the normals r_k of modes k = 2m + 4 (cosine) and 2m + 5 (sine)
    const float srho = kPhiRho0 ? cp.sqrt_rho0 : sqrt_approx(rho);
#pragma unroll
    for (int m = 0; m < 12; ++m) {
      const int k0 = 2 * m + 4, k1 = 2 * m + 5;
      float& M0 = M[p_of(k0)][q_of(k0)][r_of(k0)];
      const float rr = noise.r[m] * srho;
      if (k1 < kQ && same_amplitude(k0, k1)) {
        float& M1 = M[p_of(k1)][q_of(k1)][r_of(k1)];
        const float a = rr * cp.amp[k0 - 4];
        M0 = fmaf(a, noise.c[m], M0);
        M1 = fmaf(a, noise.s[m], M1);
      } else {
        M0 = fmaf(cp.amp[k0 - 4], rr * noise.c[m], M0);
        if (k1 < kQ) {
          float& M1 = M[p_of(k1 < kQ ? k1 : 0)][q_of(k1 < kQ ? k1 : 0)][r_of(k1 < kQ ? k1 : 0)];
          M1 = fmaf(cp.amp[(k1 < kQ ? k1 : 4) - 4], rr * noise.s[m], M1);
        }
      }
    }
  }

  // ---- 3. back transform (sweep z, then y, then x) and the lattice weights
  float Z[3][3][3];  // [p][q][c]
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 3; ++q)
      line_inverse(M[p][q][0], M[p][q][1], M[p][q][2], Z[p][q][0], Z[p][q][1], Z[p][q][2]);
  float Y[3][3][3];  // [p][b][c]
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      line_inverse(Z[p][0][c], Z[p][1][c], Z[p][2][c], Y[p][0][c], Y[p][1][c], Y[p][2][c]);
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float o[3];
      line_inverse(Y[0][b][c], Y[1][b][c], Y[2][b][c], o[0], o[1], o[2]);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float wt = float(w1d(a) * w1d(b) * w1d(c));
        if (kModel == kModelBgk) {
          G[a][b][c] = fmaf(1.0f - om, reload(a, b, c, G[a][b][c]), wt * o[a]);
        } else {
          G[a][b][c] = wt * o[a];
        }
      }
    }
}

}  // namespace rflbm_dev
