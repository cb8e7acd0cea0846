// Launchers of the auxiliary kernels (rflbm_aux.cu). `kind` is the storage format
// (kStoreF32 / kStoreF16 / kStoreBF16) of the population buffer `src` / `dst`.
#pragma once

#include "rflbm_internal.h"

namespace rflbm_dev {

constexpr int kStatOutFields = 6;  // drho sum, momentum (3), max |u|, non-finite count

cudaError_t launch_init_field(const Geometry& g, float rho0, const StoreScale& ss, int kind,
                              const double* rho, const double* u, void* dst, cudaStream_t st);
// Thermal initial state (independent Gaussian modes with the FDT variances) in view g.view.
cudaError_t launch_init_thermal(const Geometry& g, float rho0, float kT, const StoreScale& ss, int kind,
                                uint32_t key0, uint32_t key1, uint32_t replica, void* dst, cudaStream_t st);
cudaError_t launch_set_populations_f64(const Geometry& g, float rho0, const StoreScale& ss, int kind,
                                       const double* f, void* dst, cudaStream_t st);
cudaError_t launch_set_populations_f32(const Geometry& g, float rho0, const StoreScale& ss, int kind,
                                       const float* f, void* dst, cudaStream_t st);
cudaError_t launch_get_populations_f64(const Geometry& g, float rho0, const StoreScale& ss, int kind,
                                       const void* src, double* f, cudaStream_t st);
cudaError_t launch_get_populations_f32(const Geometry& g, float rho0, const StoreScale& ss, int kind,
                                       const void* src, float* f, cudaStream_t st);
cudaError_t launch_get_sites(const Geometry& g, float rho0, const StoreScale& ss, int kind,
                             const void* src, const int64_t* sites, int64_t n, double* f,
                             cudaStream_t st);
cudaError_t launch_moments(const Geometry& g, float rho0, const StoreScale& ss, int kind,
                           const void* src, double* rho, double* u, double* pi, cudaStream_t st);
// Number of partial sums (blocks) the stats reduction uses for a box on a GPU with
// num_sms multiprocessors; the scratch buffer holds kStatOutFields doubles per block.
int stats_partial_blocks(const Geometry& g, int num_sms);
cudaError_t launch_stats(const Geometry& g, float rho0, const StoreScale& ss, int kind,
                         const void* src, double* partials, int nblocks, double* out6,
                         cudaStream_t st);
// One plane of a state image (pull layout) from the plane of a population with velocity
// (cx, cy, cz) held in the natural view; elem = 4 or 2 bytes per value.
cudaError_t launch_image_plane(const Geometry& g, size_t elem, const void* plane, int cx, int cy, int cz,
                               void* out, cudaStream_t st);
cudaError_t launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out,
                          int64_t n, cudaStream_t st);
cudaError_t launch_site_normals(uint32_t k0, uint32_t k1, uint32_t step, uint32_t replica,
                                const uint32_t* sites, int64_t n, float* out, cudaStream_t st);

}  // namespace rflbm_dev
