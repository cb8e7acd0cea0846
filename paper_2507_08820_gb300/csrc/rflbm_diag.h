// Launchers of the statistics diagnostics (rflbm_diag.cu).
#pragma once

#include "rflbm_internal.h"

namespace rflbm_dev {

constexpr int kDiagSitesPerThread = 16;

// Number of partial rows (blocks) of the mode-sum reduction; each row holds 54 doubles.
int64_t mode_sum_blocks(const Geometry& g);
// sum_s m_k(s) and sum_s m_k(s)^2 for the 27 modes of the shifted pre-collision state:
// out54[k] and out54[27 + k].
cudaError_t launch_mode_sums(const Geometry& g, const StoreScale& ss, int kind, const void* src,
                             double* partials, double* out54, cudaStream_t st);
// One FP64 field per site (0 rho - rho0, 1..3 rho u, 4..9 Pi: xx, yy, zz, xy, xz, yz).
cudaError_t launch_field(const Geometry& g, const StoreScale& ss, int kind, const void* src,
                         int field, double* out, cudaStream_t st);
// Shell sums of |F|^2 / N and vector counts of a D2Z spectrum: out[n], out[nshell + n].
cudaError_t launch_shell_bins(const Geometry& g, const void* spec, int nshell, int blocks,
                              double* partials, double* out, cudaStream_t st);

}  // namespace rflbm_dev
