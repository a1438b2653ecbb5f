// Half-precision storage (BF16 or FP16) of links, clover blocks and spinors,
// with FP32 arithmetic.
//
// A half field keeps the unit structure of the FP32 block-major layout
// (common.cuh): four values per unit, [block][unit][site in block], but a
// unit is 8 bytes (uint2) instead of 16.  Links, clover blocks and test
// vectors are stored as they are; a spinor is stored divided by its site
// norm m = max |component| (so every stored value lies in [-1, 1], where
// FP16 keeps its full 11-bit precision), with m in a separate FP32 array
// indexed by the device site.  A site of zeros stores m = 0.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace ddamg {

// two values <-> one 32-bit word of the storage type
template <class S>
struct H2;
template <>
struct H2<__half> {
  __device__ __forceinline__ static float2 unpack(uint32_t w) {
    __half2 h = *reinterpret_cast<const __half2*>(&w);
    return __half22float2(h);
  }
  __device__ __forceinline__ static uint32_t pack(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
};
template <>
struct H2<__nv_bfloat16> {
  __device__ __forceinline__ static float2 unpack(uint32_t w) {
    __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&w);
    return __bfloat1622float2(h);
  }
  __device__ __forceinline__ static uint32_t pack(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
};

template <class S>
__device__ __forceinline__ void unpack4(uint2 w, float* v) {
  const float2 a = H2<S>::unpack(w.x), b = H2<S>::unpack(w.y);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
template <class S>
__device__ __forceinline__ uint2 pack4(const float* v) {
  return make_uint2(H2<S>::pack(v[0], v[1]), H2<S>::pack(v[2], v[3]));
}

// unit `off` (8 bytes, four values) of a half field
template <class S>
__device__ __forceinline__ void ld4(const S* p, size_t off, float* v) {
  unpack4<S>(__ldg(reinterpret_cast<const uint2*>(p) + off), v);
}
template <class S>
__device__ __forceinline__ void ld4_cg(const S* p, size_t off, float* v) {
  unpack4<S>(__ldcg(reinterpret_cast<const uint2*>(p) + off), v);
}
template <class S>
__device__ __forceinline__ void st4(S* p, size_t off, const float* v) {
  reinterpret_cast<uint2*>(p)[off] = pack4<S>(v);
}

// NR values of site d (unit indexing of the FP32 layout)
template <class S, int NR>
__device__ __forceinline__ void load_site_h(const S* f, int d, int Vb, float* v) {
  using LY = Layout<float, NR>;
  const size_t b = LY::base(d, Vb);
#pragma unroll
  for (int u = 0; u < LY::NU; ++u) ld4<S>(f, b + (size_t)u * Vb, v + 4 * u);
}
template <class S, int NR>
__device__ __forceinline__ void load_site_h_cg(const S* f, int d, int Vb, float* v) {
  using LY = Layout<float, NR>;
  const size_t b = LY::base(d, Vb);
#pragma unroll
  for (int u = 0; u < LY::NU; ++u) ld4_cg<S>(f, b + (size_t)u * Vb, v + 4 * u);
}
template <class S, int NR>
__device__ __forceinline__ void store_site_h(S* f, int d, int Vb, const float* v) {
  using LY = Layout<float, NR>;
  const size_t b = LY::base(d, Vb);
#pragma unroll
  for (int u = 0; u < LY::NU; ++u) st4<S>(f, b + (size_t)u * Vb, v + 4 * u);
}

// spinor of site d: stored values times the site norm
template <class S>
__device__ __forceinline__ void load_spinor_h(const S* f, const float* nrm, int d, int Vb, Spinor<float>& s) {
  float* v = reinterpret_cast<float*>(s.c);
  load_site_h<S, SPINOR_NR>(f, d, Vb, v);
  const float m = __ldg(nrm + d);
#pragma unroll
  for (int k = 0; k < SPINOR_NR; ++k) v[k] *= m;
}
// the same for data written earlier in the same kernel launch sequence
template <class S>
__device__ __forceinline__ void load_spinor_h_cg(const S* f, const float* nrm, int d, int Vb, Spinor<float>& s) {
  float* v = reinterpret_cast<float*>(s.c);
  load_site_h_cg<S, SPINOR_NR>(f, d, Vb, v);
  const float m = __ldcg(nrm + d);
#pragma unroll
  for (int k = 0; k < SPINOR_NR; ++k) v[k] *= m;
}
template <class S>
__device__ __forceinline__ void store_spinor_h(S* f, float* nrm, int d, int Vb, const Spinor<float>& s) {
  const float* v = reinterpret_cast<const float*>(s.c);
  float m = 0.f;
#pragma unroll
  for (int k = 0; k < SPINOR_NR; ++k) m = fmaxf(m, fabsf(v[k]));
  const float inv = m > 0.f ? 1.f / m : 0.f;
  float w[SPINOR_NR];
#pragma unroll
  for (int k = 0; k < SPINOR_NR; ++k) w[k] = v[k] * inv;
  store_site_h<S, SPINOR_NR>(f, d, Vb, w);
  nrm[d] = m;
}

// link mu of site d (two rows, the third rebuilt)
template <class S>
__device__ __forceinline__ void load_link_h(const S* g, int d, int Vb, int mu, Link<float>& U) {
  using LY = Layout<float, GAUGE_NR>;
  float v[LINK_NR];
  const size_t b = LY::base(d, Vb) + (size_t)(mu * 3) * Vb;
#pragma unroll
  for (int u = 0; u < 3; ++u) ld4<S>(g, b + (size_t)u * Vb, v + 4 * u);
#pragma unroll
  for (int k = 0; k < 6; ++k) U.m[k / 3][k % 3] = mk(v[2 * k], v[2 * k + 1]);
  complete_link(U);
}

// y = A(site) v with the two packed chiral blocks of a half clover field
template <class S>
__device__ __forceinline__ void clover_mul_h(const S* clov, int d, int Vb, const Spinor<float>& v, Spinor<float>& y) {
  using LY = Layout<float, CLOVER_NR>;
  const size_t b = LY::base(d, Vb);
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    float P[36];
#pragma unroll
    for (int u = 0; u < 9; ++u) ld4<S>(clov, b + (size_t)(9 * s + u) * Vb, P + 4 * u);
    herm6<float>(P, v.c + 6 * s, y.c + 6 * s);
  }
}

}  // namespace ddamg
