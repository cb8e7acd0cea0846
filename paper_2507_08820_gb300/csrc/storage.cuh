// Population storage formats.
//
// The shifted populations g_i = f_i - w_i rho0 are stored as float32, or as float16 /
// bfloat16 scaled by a power of two per velocity class |c_i|^2 (stored value
// h_i = g_i 2^(e_class)); all arithmetic is float32. The scale maps the thermal amplitude
// sqrt(w_i rho0 kT / cs2) of g_i to order one, so that float16 keeps full relative
// precision (no subnormals) and the rounding error stays a fixed fraction of the
// fluctuation; powers of two make the scaling exact.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

#include "d3q27.cuh"

namespace rflbm_dev {

enum : int { kStoreF32 = 0, kStoreF16 = 1, kStoreBF16 = 2 };

// Velocity class |c_i|^2 of population i (0 rest, 1 face, 2 edge, 3 corner).
__host__ __device__ constexpr int class_of(int i) {
  return (i == 0) ? 0 : (i <= 6 ? 1 : (i <= 18 ? 2 : 3));
}

// Velocity class of the tile entry (a, b, c) = (c_x + 1, c_y + 1, c_z + 1).
__host__ __device__ constexpr int class_at(int a, int b, int c) {
  return (a != 1) + (b != 1) + (c != 1);
}

// Per-class scale factors of 16-bit storage: stored = g * scale, g = stored * inv_scale.
struct StoreScale {
  float scale[4];
  float inv_scale[4];
};

template <int kStore>
struct Storage;

template <>
struct Storage<kStoreF32> {
  using T = float;
  static constexpr int kHalo = 4;  // halo elements per side: 16 bytes
  static __device__ __forceinline__ float load(T v, int, const StoreScale&) { return v; }
  static __device__ __forceinline__ T store(float g, int, const StoreScale&) { return g; }
  // two adjacent elements (8-byte aligned), unscaled
  static __device__ __forceinline__ float2 load2(const T* p) {
    return *reinterpret_cast<const float2*>(p);
  }
  static __device__ __forceinline__ float2 load1x2(const T* p) { return make_float2(p[0], p[1]); }
  static __device__ __forceinline__ void store2(T* p, float2 v) {
    *reinterpret_cast<float2*>(p) = v;
  }
  static __device__ __forceinline__ T pack(float v) { return v; }  // already scaled
  static __device__ __forceinline__ float to_float(T v) { return v; }  // not scaled
  static constexpr bool kScaled = false;
};

template <>
struct Storage<kStoreF16> {
  using T = __half;
  static constexpr int kHalo = 8;
  static __device__ __forceinline__ float load(T v, int cls, const StoreScale& s) {
    return __half2float(v) * s.inv_scale[cls];
  }
  static __device__ __forceinline__ T store(float g, int cls, const StoreScale& s) {
    return __float2half_rn(g * s.scale[cls]);
  }
  // two adjacent elements (4-byte aligned), converted but not scaled; store2 and pack
  // convert values whose scale the caller has applied
  static __device__ __forceinline__ float2 load2(const T* p) {
    return __half22float2(*reinterpret_cast<const __half2*>(p));
  }
  static __device__ __forceinline__ float2 load1x2(const T* p) {
    return make_float2(__half2float(p[0]), __half2float(p[1]));
  }
  static __device__ __forceinline__ void store2(T* p, float2 v) {
    *reinterpret_cast<__half2*>(p) = __float22half2_rn(v);
  }
  static __device__ __forceinline__ T pack(float v) { return __float2half_rn(v); }
  static __device__ __forceinline__ float to_float(T v) { return __half2float(v); }
  static constexpr bool kScaled = true;
};

template <>
struct Storage<kStoreBF16> {
  using T = __nv_bfloat16;
  static constexpr int kHalo = 8;
  static __device__ __forceinline__ float load(T v, int cls, const StoreScale& s) {
    return __bfloat162float(v) * s.inv_scale[cls];
  }
  static __device__ __forceinline__ T store(float g, int cls, const StoreScale& s) {
    return __float2bfloat16_rn(g * s.scale[cls]);
  }
  static __device__ __forceinline__ float2 load2(const T* p) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
  }
  static __device__ __forceinline__ float2 load1x2(const T* p) {
    return make_float2(__bfloat162float(p[0]), __bfloat162float(p[1]));
  }
  static __device__ __forceinline__ void store2(T* p, float2 v) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __float22bfloat162_rn(v);
  }
  static __device__ __forceinline__ T pack(float v) { return __float2bfloat16_rn(v); }
  static __device__ __forceinline__ float to_float(T v) { return __bfloat162float(v); }
  static constexpr bool kScaled = true;
};

inline size_t storage_bytes(int kind) { return kind == kStoreF32 ? 4 : 2; }

// Output weight of the two-site kernels (collide_tile's OutWeight): the lattice weight of
// tile entry (a, b, c) times the storage scale of its velocity class. The scale is a power
// of two, so the product rounds exactly as scaling after the weighting would.
template <int kStore>
struct ScaledWeight {
  const StoreScale& ss;
  __device__ __forceinline__ float operator()(int a, int b, int c) const {
    const float wt = float(w1d(a) * w1d(b) * w1d(c));
    return Storage<kStore>::kScaled ? wt * ss.scale[class_at(a, b, c)] : wt;
  }
};

}  // namespace rflbm_dev
