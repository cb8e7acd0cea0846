// The fused stream-and-collide step in the AA pattern: one population buffer updated in
// place, with TMA staging; for boxes whose rows are whole 16-byte units, in row segments
// of width kW in {32, 64, 96, 128, 192}; templated on the storage format. Where kW does not
// divide the x edge, the last segment of each row ends past it: the copies fill its missing
// sites with zeros, the even form's store is clipped at the row's end, and the odd form's
// excess threads store nothing.
//
// Between steps the buffer alternates between two views of the same populations
// (P = plane_of, opp(i) the population with velocity -c_i, P(opp(i)) = 26 - P(i)):
//   after an even number of steps g_i(x) sits in plane P(i) at x        (natural view),
//   after an odd number              g_i(x) sits in plane 26 - P(i) at x - c_i (flipped).
// Even form: a site reads its 27 values from its own slots and writes its post-collision
// value of population i into its own slot of plane 26 - P(i). Streaming is deferred: that
// is where the next (odd) step of site x + c_i looks for it.
// Odd form: a site reads g_i from plane 26 - P(i) at x - c_i and writes its post-collision
// value of population i into plane P(i) at x + c_i, where the next (even) step of that
// site reads it as its own. The 27 locations a site reads are the 27 it writes (with
// j = opp(i): plane P(j) at x - c_j), so each step is race-free in place.
//
// Each step computes exactly what the ping-pong kernel computes (same tile order, same
// arithmetic, same Philox counters (site, step)): the two patterns give bit-identical
// populations. One CTA of kW threads updates one row segment [x0, x0 + kW) of row (y, z).
//  - Even: one TMA load and one TMA store of the 27-plane box (x0, y, z, 0..26).
//  - Odd: 9 three-plane TMA loads with a 16-byte halo, one per source row
//    (y - c_y, z - c_z), as in the ping-pong kernel but of the mirrored plane group. When
//    the segment is a whole row (nx == kW) the results are rotated by c_x in shared memory
//    and leave as 9 three-plane row stores, one per destination row (y + c_y, z + c_z).
//    Otherwise they go straight to the neighbours x + c_i with coalesced stores: the x
//    shift of one element rules out aligned tensor stores of a segment, and a wider box
//    would overwrite slots of the neighbouring segments. (Two staged alternatives measured
//    slower: tensor stores of each segment's aligned interior with plain stores at its
//    edges, and the segments of a row as one thread-block cluster handing the edge values
//    to their neighbours through distributed shared memory.)
// Reg-FLBM forms are held to 9 CTAs of 128 threads per SM (56 registers; 8 CTAs at the 60
// registers the compiler would take measured 93.0 % against 94.0 % of the copy bandwidth at
// 128^3), BGK forms to 8. Both forms use programmatic dependent launch and bounded mbarrier
// waits like the ping-pong kernel: global memory is touched only after griddepcontrol.wait, so an in-place
// step never overlaps the previous one.
#pragma once

#include "step_tma.cuh"

namespace rflbm_dev {

template <int kStore, int kW>
struct AaEvenLayout {
  using T = typename Storage<kStore>::T;
  static constexpr size_t kTileBytes = (size_t)kQ * kW * sizeof(T);
  static constexpr size_t kBytes = kTileBytes + 128;  // + alignment slack
};

template <int kStore, int kW, int kModel, bool kNoise>
__global__ void __launch_bounds__(kW, kModel == kModelBgk ? 1024 / kW : 1152 / kW) step_aa_even(const __grid_constant__ CUtensorMap map,
                                                   const StepParams p) {
  using S = Storage<kStore>;
  using T = typename S::T;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  T* const sm = reinterpret_cast<T*>(smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u));

  const int t = threadIdx.x;
  const uint32_t nseg = (p.geo.nx + kW - 1) / kW;  // the last segment of a row may end past x = nx - 1
  const uint32_t rb = blockIdx.x / nseg;
  const uint32_t row = p.row0 + rb + (rb >= p.row_split ? p.row_gap : 0u);  // y + ny * z
  const uint32_t x0 = (blockIdx.x - rb * nseg) * kW;
  const uint32_t z = row / p.geo.ny, y = row - z * p.geo.ny;

  grid_launch_dependents();
  const uint32_t s = x0 + t + p.geo.nx * row + p.geo.site0;  // global site (Philox counter)
  SiteNoise noise;
  if (kNoise) site_noise_part<0, kPreWaitCalls>(s, p.step, p.replica, p.rk, noise);

  if (t == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  grid_dependency_wait();

  if (t == 0) {
    mbar_arrive_expect_tx(&bar, (uint32_t)AaEvenLayout<kStore, kW>::kTileBytes + p.test_extra_tx);
    tma_load_4d(sm, &map, (int)x0, (int)y, (int)(z + p.geo.zlo), 0, &bar);
  }

  if (kNoise) site_noise_part<kPreWaitCalls, 6>(s, p.step, p.replica, p.rk, noise);

  const bool ok = mbar_wait_bounded(&bar, 0, kMaxPolls);
  if (__syncthreads_or(!ok)) {
    if (t == 0) atomicOr(p.err, 1);
    mbar_wait_bounded(&bar, 0, kMaxPolls);
    return;
  }

  float G[3][3][3];
#pragma unroll
  for (int i = 0; i < kQ; ++i)
    G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1] = S::load(sm[plane_of(i) * kW + t], class_of(i), p.ss);

  if (kModel == kModelBgk) {
    const auto reload = [&](int a, int b, int c, float) {
      return S::load(sm[(9 * b + 3 * c + a) * kW + t], class_at(a, b, c), p.ss);
    };
    collide_site<kModel, kNoise, false, false>(G, p.cp, noise, reload);
  } else {
    collide_site<kModel, kNoise, false, false>(G, p.cp, noise);
  }

  __syncthreads();  // all inputs are read: the tile can take the outputs
#pragma unroll
  for (int i = 0; i < kQ; ++i)
    sm[(kQ - 1 - plane_of(i)) * kW + t] =
        S::store(G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1], class_of(i), p.ss);
  fence_proxy_async_smem();
  __syncthreads();
  if (t == 0) {
    tma_store_4d(&map, sm, (int)x0, (int)y, (int)(z + p.geo.zlo), 0);
    bulk_commit();
    bulk_wait_read();
  }
}

// Output tile of the odd form when one CTA covers a whole row (nx == kW): per destination
// row (group) the three planes, each rotated by its c_x, at 128-byte aligned group starts.
template <int kStore, int kW>
struct AaRowOut {
  using T = typename Storage<kStore>::T;
  static constexpr int kGroupBytes = (3 * kW * (int)sizeof(T) + 127) / 128 * 128;
  static constexpr int kGroup = kGroupBytes / (int)sizeof(T);
  static_assert((size_t)kGroups * kGroupBytes <= (size_t)kGroups * TmaLayout<kStore, kW>::kGroupBytes,
                "the rotated output tile must fit in the input tile");
};

template <int kStore, int kW, int kModel, bool kNoise, bool kFullRow>
__global__ void __launch_bounds__(kW, kModel == kModelBgk ? 1024 / kW : 1152 / kW) step_aa_odd(const __grid_constant__ CUtensorMap load_map,
                                                  const __grid_constant__ CUtensorMap row_map,
                                                  const StepParams p) {
  using S = Storage<kStore>;
  using L = TmaLayout<kStore, kW>;
  using T = typename L::T;
  constexpr int kH = L::kH;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  T* const sm = reinterpret_cast<T*>(smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u));

  const int t = threadIdx.x;
  const uint32_t nseg = (p.geo.nx + kW - 1) / kW;  // the last segment of a row may end past x = nx - 1
  const uint32_t rb = blockIdx.x / nseg;
  const uint32_t row = p.row0 + rb + (rb >= p.row_split ? p.row_gap : 0u);  // y + ny * z
  const uint32_t x0 = (blockIdx.x - rb * nseg) * kW;
  const uint32_t z = row / p.geo.ny, y = row - z * p.geo.ny;

  grid_launch_dependents();
  const uint32_t x = x0 + t;
  const uint32_t s = x + p.geo.nx * row;  // local site; the buffer holds it at s + zlo nx ny
  SiteNoise noise;
  if (kNoise) site_noise_part<0, kPreWaitCalls>(s + p.geo.site0, p.step, p.replica, p.rk, noise);

  if (t == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  grid_dependency_wait();

  // lane g of warp 0 loads source row (y - c_y, z - c_z) of group g = 3 (c_y + 1) + (c_z + 1):
  // the populations with velocity -c live in the mirrored group 8 - g, in-group order
  // -c_x = -1, 0, +1, i.e. position 1 - c_x for the population with x velocity c_x
  T* const buf = static_cast<T*>(p.dst);
  T patch_l = T(), patch_r = T();
  int at_l = -1, at_r = -1;
  if (t < kGroups) {
    if (t == 0) mbar_arrive_expect_tx(&bar, (uint32_t)(kGroups * 3 * L::kSeg * sizeof(T)) + p.test_extra_tx);
    const int cy = t / 3 - 1, cz = t % 3 - 1;
    int ys = (int)y - cy;
    ys += ys < 0 ? (int)p.geo.ny : 0;
    ys -= ys >= (int)p.geo.ny ? (int)p.geo.ny : 0;
    const int zs = zrow(p.geo, (int)z, -cz);  // buffer row (a z-slab's ghost rows at its faces)
    const int mirror = kGroups - 1 - t;
    tma_load_4d(sm + t * L::kGroup, &load_map, (int)x0 - kH, ys, zs, 3 * mirror, &bar);
    // periodic x edge: c_x = +1 (position 0) needs x = nx - 1 left of x = 0; c_x = -1
    // (position 2) needs x = 0 right of x = nx - 1. These slots belong to this segment.
    const int64_t rowoff = (int64_t)p.geo.nx * ((int64_t)ys + (int64_t)p.geo.ny * zs);
    if (x0 == 0) {
      patch_l = buf[(int64_t)(3 * mirror) * p.geo.ps + rowoff + (p.geo.nx - 1)];
      at_l = t * L::kGroup + kH - 1;
    }
    if (x0 + kW >= p.geo.nx) {  // right of the row's last site, at x0 + kW or inside the segment
      patch_r = buf[(int64_t)(3 * mirror + 2) * p.geo.ps + rowoff];
      at_r = t * L::kGroup + 2 * L::kSeg + kH + (int)(p.geo.nx - x0);
    }
  }

  if (kNoise) site_noise_part<kPreWaitCalls, 6>(s + p.geo.site0, p.step, p.replica, p.rk, noise);
  const PullDeltas d = deltas_at(x, y, z, p.geo);

  const bool ok = mbar_wait_bounded(&bar, 0, kMaxPolls);
  if (__syncthreads_or(!ok)) {
    if (t == 0) atomicOr(p.err, 1);
    mbar_wait_bounded(&bar, 0, kMaxPolls);
    return;
  }
  if (at_l >= 0) sm[at_l] = patch_l;
  if (at_r >= 0) sm[at_r] = patch_r;
  __syncthreads();

  float G[3][3][3];
  const T* mine = sm + kH + t;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const int gi = 3 * (cy_of(i) + 1) + (cz_of(i) + 1);
    G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1] =
        S::load(mine[gi * L::kGroup + (1 - cx_of(i)) * L::kSeg - cx_of(i)], class_of(i), p.ss);
  }

  if (kModel == kModelBgk) {
    const auto reload = [&](int a, int b, int c, float) {
      return S::load(mine[(3 * b + c) * L::kGroup + (2 - a) * L::kSeg + (1 - a)], class_at(a, b, c), p.ss);
    };
    collide_site<kModel, kNoise, false, false>(G, p.cp, noise, reload);
  } else {
    collide_site<kModel, kNoise, false, false>(G, p.cp, noise);
  }

  if (kFullRow) {
    // the segment is the whole row: population i of x goes to position (x + c_x) mod nx of
    // plane P(i) in row (y + c_y, z + c_z). Rotate each plane row in shared memory, then
    // lane g of warp 0 stores destination group g (three planes, one row) with one copy.
    using O = AaRowOut<kStore, kW>;
    __syncthreads();  // all inputs are read: the tile can take the outputs
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const int g = 3 * (cy_of(i) + 1) + (cz_of(i) + 1);
      const int pos = t + cx_of(i);  // x + c_x, wrapped within the row
      const int wrapped = (kW & (kW - 1)) == 0 ? (pos & (kW - 1))
                                                : (pos < 0 ? pos + kW : (pos >= kW ? pos - kW : pos));
      sm[g * O::kGroup + (cx_of(i) + 1) * kW + wrapped] =
          S::store(G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1], class_of(i), p.ss);
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (t < kGroups) {
      const int cy = t / 3 - 1, cz = t % 3 - 1;
      int yd = (int)y + cy;
      yd += yd < 0 ? (int)p.geo.ny : 0;
      yd -= yd >= (int)p.geo.ny ? (int)p.geo.ny : 0;
      const int zd = zrow(p.geo, (int)z, cz);
      tma_store_4d(&row_map, sm + t * O::kGroup, 0, yd, zd, 3 * t);
      bulk_commit();
      bulk_wait_read();
    }
    return;
  }

  // population i of x goes to plane P(i) at x + c_i (coalesced: a warp writes 32
  // consecutive positions of each plane); the excess threads of a ragged segment store nothing
  if (x >= p.geo.nx) return;
  T* const dst = buf + s + (int64_t)p.geo.zlo * p.geo.nxy;
#pragma unroll
  for (int i = 0; i < kQ; ++i)
    dst[plane_of(i) * p.geo.ps + push_delta(d, i)] =
        S::store(G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1], class_of(i), p.ss);
}

// ---- two sites per thread (x0 + 2t, x0 + 2t + 1), the collision in packed f32x2
// arithmetic, Reg-FLBM: the same copies, waits and addresses as the one-site forms above;
// the storage scale is folded into the lattice weights as in step_tma_pair.

template <int kStore, int kW, bool kNoise>
__global__ void __launch_bounds__(kW / 2) step_aa_even_pair(const __grid_constant__ CUtensorMap map,
                                                            const StepParams p) {
  using S = Storage<kStore>;
  using T = typename S::T;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  T* const sm = reinterpret_cast<T*>(smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u));

  const int t = threadIdx.x;
  const uint32_t nseg = (p.geo.nx + kW - 1) / kW;  // the last segment of a row may end past x = nx - 1
  const uint32_t rb = blockIdx.x / nseg;
  const uint32_t row = p.row0 + rb + (rb >= p.row_split ? p.row_gap : 0u);  // y + ny * z
  const uint32_t x0 = (blockIdx.x - rb * nseg) * kW;
  const uint32_t z = row / p.geo.ny, y = row - z * p.geo.ny;

  grid_launch_dependents();
  const PhiloxKey key{p.key0, p.key1};
  PairNoise<kPairPreDrawn, PhiloxKey> noise{x0 + 2u * t + p.geo.nx * row + p.geo.site0, p.step, p.replica, key};
  if (kNoise) noise.draw();
  if (t == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  grid_dependency_wait();

  if (t == 0) {
    mbar_arrive_expect_tx(&bar, (uint32_t)AaEvenLayout<kStore, kW>::kTileBytes + p.test_extra_tx);
    tma_load_4d(sm, &map, (int)x0, (int)y, (int)(z + p.geo.zlo), 0, &bar);
  }
  const bool ok = mbar_wait_bounded(&bar, 0, kMaxPolls);
  if (__syncthreads_or(!ok)) {
    if (t == 0) atomicOr(p.err, 1);
    mbar_wait_bounded(&bar, 0, kMaxPolls);
    return;
  }

  float2 G[3][3][3];
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    float2 v = S::load2(sm + plane_of(i) * kW + 2 * t);
    if (S::kScaled) v = kmul(p.ss.inv_scale[class_of(i)], v);
    G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1] = v;
  }
  collide_tile<kModelReg, kNoise, false, false>(G, p.cp, noise, ScaledWeight<kStore>{p.ss});

  __syncthreads();  // all inputs are read: the tile can take the outputs
#pragma unroll
  for (int i = 0; i < kQ; ++i)
    S::store2(sm + (kQ - 1 - plane_of(i)) * kW + 2 * t, G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1]);
  fence_proxy_async_smem();
  __syncthreads();
  if (t == 0) {
    tma_store_4d(&map, sm, (int)x0, (int)y, (int)(z + p.geo.zlo), 0);
    bulk_commit();
    bulk_wait_read();
  }
}

template <int kStore, int kW, bool kNoise, bool kFullRow>
__global__ void __launch_bounds__(kW / 2) step_aa_odd_pair(const __grid_constant__ CUtensorMap load_map,
                                                           const __grid_constant__ CUtensorMap row_map,
                                                           const StepParams p) {
  using S = Storage<kStore>;
  using L = TmaLayout<kStore, kW>;
  using T = typename L::T;
  constexpr int kH = L::kH;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  T* const sm = reinterpret_cast<T*>(smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u));

  const int t = threadIdx.x;
  const uint32_t nseg = (p.geo.nx + kW - 1) / kW;  // the last segment of a row may end past x = nx - 1
  const uint32_t rb = blockIdx.x / nseg;
  const uint32_t row = p.row0 + rb + (rb >= p.row_split ? p.row_gap : 0u);  // y + ny * z
  const uint32_t x0 = (blockIdx.x - rb * nseg) * kW;
  const uint32_t z = row / p.geo.ny, y = row - z * p.geo.ny;

  grid_launch_dependents();
  const uint32_t x = x0 + 2u * t;  // and x + 1
  const uint32_t s = x + p.geo.nx * row;  // local site; the buffer holds it at s + zlo nx ny
  const PhiloxKey key{p.key0, p.key1};
  PairNoise<kPairPreDrawn, PhiloxKey> noise{s + p.geo.site0, p.step, p.replica, key};
  if (kNoise) noise.draw();
  if (t == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  grid_dependency_wait();

  // the loads of the one-site odd form: mirrored group 8 - g of source row g
  T* const buf = static_cast<T*>(p.dst);
  T patch_l = T(), patch_r = T();
  int at_l = -1, at_r = -1;
  if (t < kGroups) {
    if (t == 0) mbar_arrive_expect_tx(&bar, (uint32_t)(kGroups * 3 * L::kSeg * sizeof(T)) + p.test_extra_tx);
    const int cy = t / 3 - 1, cz = t % 3 - 1;
    int ys = (int)y - cy;
    ys += ys < 0 ? (int)p.geo.ny : 0;
    ys -= ys >= (int)p.geo.ny ? (int)p.geo.ny : 0;
    const int zs = zrow(p.geo, (int)z, -cz);  // buffer row (a z-slab's ghost rows at its faces)
    const int mirror = kGroups - 1 - t;
    tma_load_4d(sm + t * L::kGroup, &load_map, (int)x0 - kH, ys, zs, 3 * mirror, &bar);
    const int64_t rowoff = (int64_t)p.geo.nx * ((int64_t)ys + (int64_t)p.geo.ny * zs);
    if (x0 == 0) {
      patch_l = buf[(int64_t)(3 * mirror) * p.geo.ps + rowoff + (p.geo.nx - 1)];
      at_l = t * L::kGroup + kH - 1;
    }
    if (x0 + kW >= p.geo.nx) {  // right of the row's last site, at x0 + kW or inside the segment
      patch_r = buf[(int64_t)(3 * mirror + 2) * p.geo.ps + rowoff];
      at_r = t * L::kGroup + 2 * L::kSeg + kH + (int)(p.geo.nx - x0);
    }
  }
  const PullDeltas d = deltas_at(x, y, z, p.geo);

  const bool ok = mbar_wait_bounded(&bar, 0, kMaxPolls);
  if (__syncthreads_or(!ok)) {
    if (t == 0) atomicOr(p.err, 1);
    mbar_wait_bounded(&bar, 0, kMaxPolls);
    return;
  }
  if (at_l >= 0) sm[at_l] = patch_l;
  if (at_r >= 0) sm[at_r] = patch_r;
  __syncthreads();

  float2 G[3][3][3];
  const T* mine = sm + kH + 2 * t;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const int gi = 3 * (cy_of(i) + 1) + (cz_of(i) + 1);
    const T* at = mine + gi * L::kGroup + (1 - cx_of(i)) * L::kSeg - cx_of(i);
    float2 v = cx_of(i) == 0 ? S::load2(at) : S::load1x2(at);
    if (S::kScaled) v = kmul(p.ss.inv_scale[class_of(i)], v);
    G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1] = v;
  }
  collide_tile<kModelReg, kNoise, false, false>(G, p.cp, noise, ScaledWeight<kStore>{p.ss});

  if (kFullRow) {
    using O = AaRowOut<kStore, kW>;
    __syncthreads();  // all inputs are read: the tile can take the outputs
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
      const int g = 3 * (cy_of(i) + 1) + (cz_of(i) + 1);
      T* const prow = sm + g * O::kGroup + (cx_of(i) + 1) * kW;
      const float2 v = G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1];
      if (cx_of(i) == 0) {
        S::store2(prow + 2 * t, v);
      } else {
        // positions x + c_x and x + 1 + c_x, wrapped within the row
        const int p0 = 2 * t + cx_of(i), p1 = p0 + 1;
        prow[p0 < 0 ? p0 + kW : p0] = S::pack(v.x);
        prow[p1 >= kW ? p1 - kW : p1] = S::pack(v.y);
      }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (t < kGroups) {
      const int cy = t / 3 - 1, cz = t % 3 - 1;
      int yd = (int)y + cy;
      yd += yd < 0 ? (int)p.geo.ny : 0;
      yd -= yd >= (int)p.geo.ny ? (int)p.geo.ny : 0;
      const int zd = zrow(p.geo, (int)z, cz);
      tma_store_4d(&row_map, sm + t * O::kGroup, 0, yd, zd, 3 * t);
      bulk_commit();
      bulk_wait_read();
    }
    return;
  }

  // population i of x and x + 1 goes to plane P(i) at x + c_i and x + 1 + c_i: the rows
  // (y, z) shifts are shared; along x, x + 1 never wraps from x (x is even, nx is even),
  // x - 1 wraps when x = 0, and x + 2 wraps when x + 2 = nx; the excess threads of a ragged
  // segment store nothing
  if (x >= p.geo.nx) return;
  T* const dst = buf + s + (int64_t)p.geo.zlo * p.geo.nxy;
  const int32_t dxb_plus = (x + 2u == p.geo.nx) ? 1 - (int32_t)p.geo.nx : 1;
#pragma unroll
  for (int i = 0; i < kQ; ++i) {
    const float2 v = G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1];
    const int64_t base = plane_of(i) * p.geo.ps + d.DY[1 - cy_of(i)] + d.DZ[1 - cz_of(i)];
    if (cx_of(i) == 0) {
      S::store2(dst + base, v);
    } else if (cx_of(i) > 0) {
      dst[base + 1] = S::pack(v.x);
      dst[base + 1 + dxb_plus] = S::pack(v.y);
    } else {
      dst[base + d.DX[2]] = S::pack(v.x);
      dst[base] = S::pack(v.y);  // x + 1 - 1
    }
  }
}

template <int kStore, int kW, bool kNoise>
cudaError_t launch_aa_pair(const TmaMaps& m, const StepParams& p, bool odd, cudaStream_t st) {
  const uint64_t blocks = (uint64_t)((p.geo.nx + kW - 1) / kW) * p.nrows;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(kW / 2);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (odd) {
    cfg.dynamicSmemBytes = TmaLayout<kStore, kW>::kBytes;
    if (m.row3 && p.geo.nx == (uint32_t)kW)
      return cudaLaunchKernelEx(&cfg, step_aa_odd_pair<kStore, kW, kNoise, true>, *m.load, *m.row3, p);
    return cudaLaunchKernelEx(&cfg, step_aa_odd_pair<kStore, kW, kNoise, false>, *m.load, *m.load, p);
  }
  cfg.dynamicSmemBytes = AaEvenLayout<kStore, kW>::kBytes;
  return cudaLaunchKernelEx(&cfg, step_aa_even_pair<kStore, kW, kNoise>, *m.store, p);
}

template <int kStore, int kW, int kModel, bool kNoise>
cudaError_t launch_aa_segment(const TmaMaps& m, const StepParams& p, bool odd, cudaStream_t st) {
  const uint64_t blocks = (uint64_t)((p.geo.nx + kW - 1) / kW) * p.nrows;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(kW);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (odd) {
    cfg.dynamicSmemBytes = TmaLayout<kStore, kW>::kBytes;
    if (m.row3 && p.geo.nx == (uint32_t)kW)
      return cudaLaunchKernelEx(&cfg, step_aa_odd<kStore, kW, kModel, kNoise, true>, *m.load, *m.row3, p);
    return cudaLaunchKernelEx(&cfg, step_aa_odd<kStore, kW, kModel, kNoise, false>, *m.load, *m.load, p);
  }
  cfg.dynamicSmemBytes = AaEvenLayout<kStore, kW>::kBytes;
  return cudaLaunchKernelEx(&cfg, step_aa_even<kStore, kW, kModel, kNoise>, *m.store, p);
}

template <int kStore, int kW>
cudaError_t launch_aa_variant(const TmaMaps& m, const StepParams& p, const StepVariant& v, bool odd,
                              cudaStream_t st) {
  if (v.ghost_neq || v.phi_rho0) return cudaErrorInvalidValue;
  if (aa_uses_pairs(v, odd, m.row3 && p.geo.nx == (uint32_t)kW))
    return v.noise ? launch_aa_pair<kStore, kW, true>(m, p, odd, st) : launch_aa_pair<kStore, kW, false>(m, p, odd, st);
  if (v.model == kModelBgk)
    return v.noise ? launch_aa_segment<kStore, kW, kModelBgk, true>(m, p, odd, st)
                   : launch_aa_segment<kStore, kW, kModelBgk, false>(m, p, odd, st);
  return v.noise ? launch_aa_segment<kStore, kW, kModelReg, true>(m, p, odd, st)
                 : launch_aa_segment<kStore, kW, kModelReg, false>(m, p, odd, st);
}

template <int kStore>
cudaError_t launch_aa_storage(const TmaMaps& m, const StepParams& p, const StepVariant& v, bool odd,
                              cudaStream_t st) {
  switch (m.width) {
    case 128: return launch_aa_variant<kStore, 128>(m, p, v, odd, st);
    case 192: return launch_aa_variant<kStore, 192>(m, p, v, odd, st);
    case 96: return launch_aa_variant<kStore, 96>(m, p, v, odd, st);
    case 64: return launch_aa_variant<kStore, 64>(m, p, v, odd, st);
    case 32: return launch_aa_variant<kStore, 32>(m, p, v, odd, st);
    default: return cudaErrorInvalidValue;
  }
}

// Per-storage entry points (one translation unit each).
cudaError_t launch_step_aa_tma_f32(const TmaMaps& m, const StepParams& p, const StepVariant& v, bool odd,
                                   cudaStream_t st);
cudaError_t launch_step_aa_tma_f16(const TmaMaps& m, const StepParams& p, const StepVariant& v, bool odd,
                                   cudaStream_t st);
cudaError_t launch_step_aa_tma_bf16(const TmaMaps& m, const StepParams& p, const StepVariant& v, bool odd,
                                    cudaStream_t st);

}  // namespace rflbm_dev
