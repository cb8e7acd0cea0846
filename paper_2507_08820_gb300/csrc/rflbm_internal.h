// Internal declarations shared by the translation units of the library.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "collide.cuh"
#include "storage.cuh"

namespace rflbm_dev {

// Exact unsigned division n / d for n, d < 2^31 by one 32x32->64 multiply:
// m = floor(2^(31+l) / d) + 1 with l = ceil(log2 d) gives n / d = (n * m) >> (31 + l).
struct FastDiv {
  uint32_t d;
  uint32_t m;
  uint32_t shift;  // 31 + l
};

inline FastDiv make_fastdiv(uint32_t d) {
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;
  const unsigned long long m = ((1ull << (31 + l)) / d) + 1ull;
  return FastDiv{d, (uint32_t)m, 31u + l};
}

__device__ __forceinline__ uint32_t fastdiv(uint32_t n, const FastDiv& f) {
  return (uint32_t)(((unsigned long long)n * f.m) >> f.shift);
}

// Where the pre-collision value g_i(x, t) = f_i(x, t) - w_i rho0 of site x lives in a
// population buffer between steps (P = plane_of):
//  - kViewPull: plane P(i) at x - c_i (the post-collision value of step t - 1 at x - c_i).
//    The ping-pong pattern, and the layout of state images.
//  - kViewNatural: plane P(i) at x. The AA pattern after an even number of steps.
//  - kViewFlipped: plane P(opp(i)) = 26 - P(i) at x - c_i. The AA pattern after an odd
//    number of steps (the even form wrote each value into the opposite slot).
constexpr uint32_t kViewPull = 0;
constexpr uint32_t kViewNatural = 1;
constexpr uint32_t kViewFlipped = 2;

// Geometry of a box and the view of its buffer.
//
// A whole periodic box wraps in z. A z-slab (one part of a box split along z, Sec. IV)
// holds its nz local rows between two ghost rows: buffer row 0 is the row below the slab
// (global z0 - 1), rows 1..nz its own rows, row nz + 1 the row above; z does not wrap
// inside the slab, and the ghost rows are filled by the exchange between slabs.
struct Geometry {
  uint32_t nx, ny, nz, nxy, n;  // n = nx ny nz local sites
  uint32_t view;  // kViewPull / kViewNatural / kViewFlipped (read by the non-step kernels)
  int64_t ps;     // plane stride in elements ((nz + 2 zlo) nx ny rounded up to 64)
  FastDiv div_nx, div_nxy;
  uint32_t zlo = 0;    // buffer row of local row 0: 0 (periodic box) or 1 (z-slab)
  uint32_t site0 = 0;  // global index of local site 0 (the Philox site counter): nx ny z0
};

// Buffer row of local row z moved by dz in {-1, 0, +1}: periodic wrap for a whole box;
// for a z-slab the rows beyond its faces are its ghost rows.
__host__ __device__ __forceinline__ int zrow(const Geometry& g, int z, int dz) {
  int zs = z + dz;
  if (g.zlo) return zs + 1;
  zs += zs < 0 ? (int)g.nz : 0;
  zs -= zs >= (int)g.nz ? (int)g.nz : 0;
  return zs;
}

// Periodic neighbour coordinates of site s: X[a] is the x coordinate of x - (a - 1),
// Y[b] and Z[c] the row and slab offsets of y - (b - 1), z - (c - 1).
struct Neighbours {
  uint32_t X[3], Y[3], Z[3];
};

// (Z offsets are buffer rows: for a z-slab they include its ghost row below.)
__device__ __forceinline__ Neighbours neighbours(uint32_t s, const Geometry& g) {
  const uint32_t z = fastdiv(s, g.div_nxy);
  const uint32_t rem = s - z * g.nxy;
  const uint32_t y = fastdiv(rem, g.div_nx);
  const uint32_t x = rem - y * g.nx;
  const uint32_t xm = (x == 0 ? g.nx : x) - 1, xp = (x + 1 == g.nx) ? 0 : x + 1;
  const uint32_t ym = (y == 0 ? g.ny : y) - 1, yp = (y + 1 == g.ny) ? 0 : y + 1;
  const uint32_t zm = (uint32_t)zrow(g, (int)z, -1), zp = (uint32_t)zrow(g, (int)z, 1);
  Neighbours nb;
  nb.X[0] = xp; nb.X[1] = x; nb.X[2] = xm;
  nb.Y[0] = yp * g.nx; nb.Y[1] = y * g.nx; nb.Y[2] = ym * g.nx;
  nb.Z[0] = zp * g.nxy; nb.Z[1] = (z + g.zlo) * g.nxy; nb.Z[2] = zm * g.nxy;
  return nb;
}

// Site that population i of site x is pulled from: x - c_i.
__device__ __forceinline__ uint32_t pull_site(const Neighbours& nb, int i) {
  return nb.X[cx_of(i) + 1] + nb.Y[cy_of(i) + 1] + nb.Z[cz_of(i) + 1];
}

// Element offset of g_i(s, t) in a buffer of view g.view (nb = neighbours(s, g)).
__device__ __forceinline__ int64_t pop_slot(const Geometry& g, const Neighbours& nb, uint32_t s, int i) {
  if (g.view == kViewNatural) return plane_of(i) * g.ps + s + g.zlo * g.nxy;
  const int plane = g.view == kViewFlipped ? kQ - 1 - plane_of(i) : plane_of(i);
  return plane * g.ps + pull_site(nb, i);
}

// Signed offsets from site s to its periodic neighbours, per axis and per direction of
// the pulled population: D?[a] is the offset of the coordinate minus (a - 1), so the
// pull source x - c_i of population i is s + DX[cx+1] + DY[cy+1] + DZ[cz+1].
struct PullDeltas {
  int32_t DX[3], DY[3], DZ[3];
};

__device__ __forceinline__ PullDeltas deltas_at(uint32_t x, uint32_t y, uint32_t z, const Geometry& g) {
  const int32_t nx = (int32_t)g.nx, nxy = (int32_t)g.nxy, nyz = nxy * ((int32_t)g.nz - 1);
  PullDeltas d;
  d.DX[1] = 0;
  d.DX[0] = (x + 1 == g.nx) ? 1 - nx : 1;            // x + 1 (pulled when c_x = -1)
  d.DX[2] = (x == 0) ? nx - 1 : -1;                  // x - 1 (pulled when c_x = +1)
  d.DY[1] = 0;
  d.DY[0] = (y + 1 == g.ny) ? nx - nxy : nx;
  d.DY[2] = (y == 0) ? nxy - nx : -nx;
  d.DZ[1] = 0;
  d.DZ[0] = (!g.zlo && z + 1 == g.nz) ? -nyz : nxy;  // a z-slab reaches its ghost rows
  d.DZ[2] = (!g.zlo && z == 0) ? nyz : -nxy;
  return d;
}

__device__ __forceinline__ PullDeltas pull_deltas(uint32_t s, const Geometry& g) {
  const uint32_t z = fastdiv(s, g.div_nxy);
  const uint32_t rem = s - z * g.nxy;
  const uint32_t y = fastdiv(rem, g.div_nx);
  return deltas_at(rem - y * g.nx, y, z, g);
}

__device__ __forceinline__ int32_t pull_delta(const PullDeltas& d, int i) {
  return d.DX[cx_of(i) + 1] + d.DY[cy_of(i) + 1] + d.DZ[cz_of(i) + 1];
}

// Offset to x + c_i, the site that receives population i of x (push).
__device__ __forceinline__ int32_t push_delta(const PullDeltas& d, int i) {
  return d.DX[1 - cx_of(i)] + d.DY[1 - cy_of(i)] + d.DZ[1 - cz_of(i)];
}

struct StepParams {
  Geometry geo;
  // The launch updates nrows rows (row = y + ny z): rows row0 .. row0 + row_split - 1, then
  // from row0 + row_split + row_gap on (row_gap 0: one contiguous range).
  uint32_t row0, nrows, row_split, row_gap;
  CollideParams cp;
  StoreScale ss;    // 16-bit storage scales (unused for float32)
  const void* src;  // population buffers in the handle's storage format
  void* dst;
  int* err;  // device error flag (bit 0: a bounded wait expired)
  uint32_t key0, key1, step, replica;
  PhiloxRoundKeys rk;  // the round keys of (key0, key1)
  uint32_t test_extra_tx;  // testing hook: bytes a TMA step expects beyond its copies (0)
};

// TMA descriptors of a source buffer (the three planes of a source row, row segment plus
// a 16-byte halo on each side) and of a destination buffer (all planes of a row segment).
struct TmaMaps {
  const CUtensorMap* load;   // box: (width + 2 halo) x 1 x 1 x 3 planes
  const CUtensorMap* store;  // box: width x 1 x 1 x 27 planes
  int width;
  const CUtensorMap* row3 = nullptr;  // AA, width == nx: box width x 1 x 1 x 3 planes
};

constexpr int kStepBlock = 256;

// Variant flags of the step kernel.
struct StepVariant {
  int model;        // kModelReg / kModelBgk
  bool noise;       // kT > 0
  bool ghost_neq;   // omega_g != 1 (Reg only)
  bool phi_rho0;    // Eq. 10 with rho0
  int storage;      // kStoreF32 / kStoreF16 / kStoreBF16 (16-bit: no ghost_neq, no phi_rho0)
};

// Encodes the population buffer at `base` (4-D: x, y, z, plane; planes ps apart) for tiled
// TMA copies of (box_x, box_y, 1, box_planes) boxes; false if the driver refuses.
bool encode_population_map(CUtensorMap* map, void* base, const Geometry& g, uint32_t box_x,
                           uint32_t box_y, uint32_t box_planes, int storage);

// Records `msg` (and `detail`, if not NULL) as the calling thread's last error
// (rflbm_last_error) and returns `code`.
int record_error(int code, const char* msg, const char* detail);

// Launches one step of the general gather kernel (any box) on `stream`.
cudaError_t launch_step_gather(const StepParams& p, const StepVariant& v, cudaStream_t stream);
// One in-place AA step of the general kernel on the buffer p.dst (== p.src): the even form
// (odd = false) or the odd form. Paper configuration only (no ghost_neq, no phi_rho0).
cudaError_t launch_step_aa_gather(const StepParams& p, const StepVariant& v, bool odd, cudaStream_t stream);
// One in-place AA step of the TMA kernels: the even form uses m.store (27-plane box) for
// its load and its store; the odd form uses m.load (three-plane boxes with halo).
cudaError_t launch_step_aa_tma(const TmaMaps& m, const StepParams& p, const StepVariant& v, bool odd,
                               cudaStream_t stream);

// True when the TMA step of variant v updates two sites per thread (step_tma_pair; the AA
// steps of such variants likewise).
bool tma_uses_pairs(const StepVariant& v);
// True when an AA step (odd: from the flipped view; full_row: its segments are whole rows,
// stored as rotated rows) runs in the two-site form.
bool aa_uses_pairs(const StepVariant& v, bool odd, bool full_row);

// Row-segment width of the TMA step kernels for a box of x edge nx (0: not supported).
int tma_segment_width(uint32_t nx);
// Launches one step of a TMA-staged kernel on `stream` (any storage format).
cudaError_t launch_step_tma(const TmaMaps& m, const StepParams& p, const StepVariant& v,
                            cudaStream_t stream);
// The 16-bit storage part of launch_step_tma (rflbm_step_tma16.cu).
cudaError_t launch_step_tma_16(const TmaMaps& m, const StepParams& p, const StepVariant& v,
                               cudaStream_t stream);

}  // namespace rflbm_dev
