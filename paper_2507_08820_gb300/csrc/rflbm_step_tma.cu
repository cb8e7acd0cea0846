// The fused stream-and-collide step with TMA staging (boxes whose x edge is a multiple of
// the row-segment width kW in {32, 64, 128}).
//
// One CTA of kW threads updates one row segment [x0, x0 + kW) of one lattice row (y, z).
// The 27 populations of a site are pulled from 9 source rows (y - c_y, z - c_z), shifted
// by -c_x along x. Warp 0 issues, for every population i, one tiled TMA load of the
// source row segment [x0 - 4, x0 + kW + 4) of plane i into shared memory (27 loads of
// (kW + 8) floats, completion counted on one mbarrier); lanes whose segment touches the
// periodic x edge also fetch the wrapped neighbour with a plain load. While the copies are
// in flight every thread draws its 24 normals. Each thread then reads its 27 values from
// shared memory at fixed offsets (x - c_x within the row), collides in registers, writes
// its 27 results back to shared memory, and warp 0 issues 27 tiled TMA stores of the
// row segment into the destination planes.
//
// Every wait on the mbarrier is bounded; a CTA that gives up sets the handle's error flag,
// waits (again bounded) for its copies in flight and exits without storing.
#include "rflbm_internal.h"
#include "tma.cuh"

namespace rflbm_dev {

// Velocity component of population i for a run-time i (2 bits per population).
__host__ __device__ constexpr uint64_t pack_component(int axis) {
  uint64_t v = 0;
  for (int i = 0; i < kQ; ++i) {
    const int c = axis == 0 ? cx_of(i) : (axis == 1 ? cy_of(i) : cz_of(i));
    v |= (uint64_t)(c + 1) << (2 * i);
  }
  return v;
}
constexpr uint64_t kPackCx = pack_component(0), kPackCy = pack_component(1),
                   kPackCz = pack_component(2);
__device__ __forceinline__ int comp(uint64_t pack, int i) { return (int)((pack >> (2 * i)) & 3u) - 1; }

constexpr uint32_t kMaxPolls = 1u << 22;  // bounded mbarrier waits

template <int kW, int kModel, bool kNoise, bool kGhostNeq, bool kPhiRho0>
__global__ void __launch_bounds__(kW) step_tma_f32(const __grid_constant__ CUtensorMap load_map,
                                                   const __grid_constant__ CUtensorMap store_map,
                                                   const StepParams p) {
  constexpr int kSeg = kW + 8;                 // loaded segment: x0 - 4 .. x0 + kW + 3
  constexpr int kRow = (kSeg + 31) / 32 * 32;  // shared row stride (128-byte multiple)
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  // rows start on 128-byte boundaries of the shared window (the launch adds 128 bytes)
  float* const sm = reinterpret_cast<float*>(smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u));

  const int t = threadIdx.x;
  const uint32_t nseg = p.geo.nx / kW;
  const uint32_t row = blockIdx.x / nseg;            // y + ny * z
  const uint32_t x0 = (blockIdx.x - row * nseg) * kW;
  const uint32_t z = row / p.geo.ny, y = row - z * p.geo.ny;

  if (t == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();

  // warp 0: lane i loads the source row segment of population i
  float patch = 0.0f;
  int patch_at = -1;
  if (t < 32) {
    if (t == 0) mbar_arrive_expect_tx(&bar, (uint32_t)(kQ * kSeg * sizeof(float)));
    __syncwarp();
    if (t < kQ) {
      const int i = t;
      const int cx = comp(kPackCx, i), cy = comp(kPackCy, i), cz = comp(kPackCz, i);
      int ys = (int)y - cy, zs = (int)z - cz;
      ys += ys < 0 ? (int)p.geo.ny : 0;
      ys -= ys >= (int)p.geo.ny ? (int)p.geo.ny : 0;
      zs += zs < 0 ? (int)p.geo.nz : 0;
      zs -= zs >= (int)p.geo.nz ? (int)p.geo.nz : 0;
      tma_load_4d(sm + i * kRow, &load_map, (int)x0 - 4, ys, zs, i, &bar);
      // periodic x edge: the element left of x = 0 is x = nx - 1, right of nx - 1 is 0
      const int64_t rowoff = (int64_t)i * p.geo.ps + (int64_t)p.geo.nx * ((int64_t)ys + (int64_t)p.geo.ny * zs);
      if (cx == 1 && x0 == 0) {
        patch = __ldg(p.src + rowoff + (p.geo.nx - 1));
        patch_at = i * kRow + 3;
      } else if (cx == -1 && x0 + kW == p.geo.nx) {
        patch = __ldg(p.src + rowoff);
        patch_at = i * kRow + 4 + kW;
      }
    }
  }

  const uint32_t s = x0 + t + p.geo.nx * row;
  SiteNoise noise;
  if (kNoise) site_noise(s, p.step, p.replica, p.key0, p.key1, noise);

  const bool ok = mbar_wait_bounded(&bar, 0, kMaxPolls);
  if (__syncthreads_or(!ok)) {
    if (t == 0) atomicOr(p.err, 1);
    mbar_wait_bounded(&bar, 0, kMaxPolls);  // let copies in flight land before exiting
    return;
  }
  if (patch_at >= 0) sm[patch_at] = patch;
  __syncthreads();

  float G[3][3][3];
  const float* mine = sm + 4 + t;
#pragma unroll
  for (int i = 0; i < kQ; ++i) G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1] = mine[i * kRow - cx_of(i)];

  collide_site<kModel, kNoise, kGhostNeq, kPhiRho0>(G, p.cp, noise);

  __syncthreads();  // every thread has read its inputs: the rows can hold the outputs
  float* out = sm + t;  // output row i at the (128-byte aligned) start of shared row i
#pragma unroll
  for (int i = 0; i < kQ; ++i) out[i * kRow] = G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1];
  fence_proxy_async_smem();
  __syncthreads();
  if (t < kQ) {
    tma_store_4d(&store_map, sm + t * kRow, (int)x0, (int)y, (int)z, t);
    bulk_commit();
    bulk_wait_read();
  }
}

template <int kW, int kModel, bool kNoise, bool kGhostNeq, bool kPhiRho0>
static cudaError_t launch_w(const TmaMaps& m, const StepParams& p, cudaStream_t st) {
  const uint64_t blocks = (uint64_t)(p.geo.nx / kW) * p.geo.ny * p.geo.nz;
  const size_t smem = (size_t)kQ * ((kW + 8 + 31) / 32 * 32) * sizeof(float) + 128;
  step_tma_f32<kW, kModel, kNoise, kGhostNeq, kPhiRho0>
      <<<(unsigned)blocks, kW, smem, st>>>(*m.load, *m.store, p);
  return cudaGetLastError();
}

template <int kW>
static cudaError_t launch_variant(const TmaMaps& m, const StepParams& p, const StepVariant& v,
                                  cudaStream_t st) {
  if (v.model == kModelBgk) {
    if (!v.noise) return launch_w<kW, kModelBgk, false, false, false>(m, p, st);
    return v.phi_rho0 ? launch_w<kW, kModelBgk, true, false, true>(m, p, st)
                      : launch_w<kW, kModelBgk, true, false, false>(m, p, st);
  }
  if (!v.noise) {
    return v.ghost_neq ? launch_w<kW, kModelReg, false, true, false>(m, p, st)
                       : launch_w<kW, kModelReg, false, false, false>(m, p, st);
  }
  if (v.ghost_neq) {
    return v.phi_rho0 ? launch_w<kW, kModelReg, true, true, true>(m, p, st)
                      : launch_w<kW, kModelReg, true, true, false>(m, p, st);
  }
  return v.phi_rho0 ? launch_w<kW, kModelReg, true, false, true>(m, p, st)
                    : launch_w<kW, kModelReg, true, false, false>(m, p, st);
}

int tma_segment_width(uint32_t nx) {
  if (nx % 128 == 0) return 128;
  if (nx % 64 == 0) return 64;
  if (nx % 32 == 0) return 32;
  return 0;
}

cudaError_t launch_step_tma_f32(const TmaMaps& m, const StepParams& p, const StepVariant& v,
                                cudaStream_t stream) {
  switch (m.width) {
    case 128: return launch_variant<128>(m, p, v, stream);
    case 64: return launch_variant<64>(m, p, v, stream);
    case 32: return launch_variant<32>(m, p, v, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace rflbm_dev
