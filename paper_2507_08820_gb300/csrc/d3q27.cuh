// D3Q27 lattice constants for the device code (Table I, Table II of arXiv 2507.08820).
//
// The CUDA path never forms the 27x27 mode matrix. It uses the fact that every basis
// vector of Table II is a product h_p(c_x) h_q(c_y) h_r(c_z) of the 1-D Hermite
// polynomials h_0 = 1, h_1 = c, h_2 = c^2 - 1/3, that the weights factor as
// w_i = W(c_x) W(c_y) W(c_z) with W(0) = 2/3, W(+-1) = 1/6, and that the norms factor as
// b_k = beta_p beta_q beta_r with beta = (1, 1/3, 2/9) (Eq. 6). Populations are held in
// 3x3x3 register tiles G[a][b][c] with a = c_x + 1, b = c_y + 1, c = c_z + 1 and modes
// in tiles M[p][q][r] of Hermite exponents.
#pragma once

#include <cstdint>

namespace rflbm_dev {

constexpr int kQ = 27;

// Velocity components of population i (API order, see rflbm.h).
__host__ __device__ constexpr int cx_of(int i) {
  constexpr int t[kQ] = {0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1,
                         0, 0, 0, 0, 1, 1, 1, 1, -1, -1, -1, -1};
  return t[i];
}
__host__ __device__ constexpr int cy_of(int i) {
  constexpr int t[kQ] = {0, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, 0, 0, 0, 0,
                         1, 1, -1, -1, 1, 1, -1, -1, 1, 1, -1, -1};
  return t[i];
}
__host__ __device__ constexpr int cz_of(int i) {
  constexpr int t[kQ] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1,
                         1, -1, 1, -1, 1, -1, 1, -1, 1, -1, 1, -1};
  return t[i];
}

// Internal plane of population i in a population buffer: the populations that pull from
// the same source row (equal c_y, c_z) are adjacent, ordered by c_x = -1, 0, +1, so that
// one tensor copy moves all three. (The public API keeps the order of Table I.)
__host__ __device__ constexpr int plane_of(int i) {
  return 3 * (3 * (cy_of(i) + 1) + (cz_of(i) + 1)) + (cx_of(i) + 1);
}

// Population with the opposite velocity -c_i. Its plane is 26 - plane_of(i).
__host__ __device__ constexpr int opp_of(int i) {
  for (int j = 0; j < kQ; ++j)
    if (cx_of(j) == -cx_of(i) && cy_of(j) == -cy_of(i) && cz_of(j) == -cz_of(i)) return j;
  return -1;
}

// 1-D weight W(c) for a tile index a = c + 1.
__host__ __device__ constexpr double w1d(int a) { return a == 1 ? 2.0 / 3.0 : 1.0 / 6.0; }
// Lattice weight of population i.
__host__ __device__ constexpr double weight_of(int i) {
  return w1d(cx_of(i) + 1) * w1d(cy_of(i) + 1) * w1d(cz_of(i) + 1);
}
// 1-D Hermite norm beta_p and the mode norm b = beta_p beta_q beta_r.
__host__ __device__ constexpr double beta1d(int p) {
  return p == 0 ? 1.0 : (p == 1 ? 1.0 / 3.0 : 2.0 / 9.0);
}
__host__ __device__ constexpr double bnorm(int p, int q, int r) {
  return beta1d(p) * beta1d(q) * beta1d(r);
}
// Hermite exponents (p, q, r) of the Table II mode k.
__host__ __device__ constexpr int p_of(int k) {
  constexpr int t[kQ] = {0, 1, 0, 0, 2, 0, 0, 1, 1, 0, 2, 2, 1, 1, 0, 0, 1, 2, 2, 0, 1, 1, 2, 2, 2, 1, 2};
  return t[k];
}
__host__ __device__ constexpr int q_of(int k) {
  constexpr int t[kQ] = {0, 0, 1, 0, 0, 2, 0, 1, 0, 1, 1, 0, 2, 0, 1, 2, 1, 2, 0, 2, 1, 2, 1, 1, 2, 2, 2};
  return t[k];
}
__host__ __device__ constexpr int r_of(int k) {
  constexpr int t[kQ] = {0, 0, 0, 1, 0, 0, 2, 0, 1, 1, 0, 1, 0, 2, 2, 1, 1, 0, 2, 2, 2, 1, 1, 2, 1, 2, 2};
  return t[k];
}
// Table II index k of the mode with Hermite exponents (p, q, r).
__host__ __device__ constexpr int mode_of(int p, int q, int r) {
  constexpr int t[kQ] = {0, 3, 6, 2, 9, 14, 5, 15, 19, 1, 8, 13, 7, 16, 20,
                         12, 21, 25, 4, 11, 18, 10, 22, 23, 17, 24, 26};
  return t[9 * p + 3 * q + r];
}

// The two mode tables are inverse to each other, the weights sum to one, the plane map is
// a permutation and opposite populations occupy mirrored planes.
__host__ __device__ constexpr bool tables_consistent() {
  double wsum = 0.0;
  int seen = 0;
  for (int k = 0; k < kQ; ++k) {
    if (mode_of(p_of(k), q_of(k), r_of(k)) != k) return false;
    wsum += weight_of(k);
    seen |= 1 << plane_of(k);
    if (opp_of(opp_of(k)) != k || plane_of(opp_of(k)) != kQ - 1 - plane_of(k)) return false;
  }
  return wsum > 1.0 - 1e-12 && wsum < 1.0 + 1e-12 && seen == (1 << kQ) - 1;
}
static_assert(tables_consistent(), "D3Q27 tables are inconsistent");

}  // namespace rflbm_dev
