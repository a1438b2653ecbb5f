// Half-precision storage (BF16 or FP16) of links, clover blocks and spinors,
// with FP32 arithmetic.
//
// Operator and spinor fields in half storage are block-major structures of
// arrays like the FP32 fields (common.cuh), [block][unit][site in block],
// with 16-byte units of eight values: a spinor is 3 units per site, the four
// two-row links 6, the two packed clover blocks 9.  A spinor is stored
// divided by its site norm m = max |component| (so every stored value lies
// in [-1, 1], where FP16 keeps its full 11-bit precision), with m in a
// separate FP32 array indexed by the device site; a site of zeros stores
// m = 0.  Test vectors in half keep the FP32 unit structure instead (8-byte
// units of four values, see load_site_h4).
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

// NR values of site d from a field with the FP32 unit structure and 8-byte
// units of four values (half test vectors)
template <class S, int NR>
__device__ __forceinline__ void load_site_h4(const S* f, int d, int Vb, float* v) {
  using LY = Layout<float, NR>;
  const size_t b = LY::base(d, Vb);
#pragma unroll
  for (int u = 0; u < LY::NU; ++u) ld4<S>(f, b + (size_t)u * Vb, v + 4 * u);
}

// ---- 16-byte units of eight values ---------------------------------------------
template <class S>
__device__ __forceinline__ void unpack8(const uint4& w, float* v) {
  float2 a = H2<S>::unpack(w.x), b = H2<S>::unpack(w.y), c = H2<S>::unpack(w.z), e = H2<S>::unpack(w.w);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y; v[6] = e.x; v[7] = e.y;
}
template <class S>
__device__ __forceinline__ uint4 pack8(const float* v) {
  return make_uint4(H2<S>::pack(v[0], v[1]), H2<S>::pack(v[2], v[3]), H2<S>::pack(v[4], v[5]),
                    H2<S>::pack(v[6], v[7]));
}
template <class S>
__device__ __forceinline__ void ld8(const S* p, size_t off, float* v) {
  unpack8<S>(__ldg(reinterpret_cast<const uint4*>(p) + off), v);
}
template <class S>
__device__ __forceinline__ void ld8_cg(const S* p, size_t off, float* v) {
  unpack8<S>(__ldcg(reinterpret_cast<const uint4*>(p) + off), v);
}
template <class S>
__device__ __forceinline__ void st8(S* p, size_t off, const float* v) {
  reinterpret_cast<uint4*>(p)[off] = pack8<S>(v);
}

// unit u of site d in a half field of NU units per site
template <int NU>
__device__ __forceinline__ size_t hunit(int d, int Vb, int u) {
  const int B = d / Vb, q = d - B * Vb;
  return ((size_t)B * NU + u) * Vb + q;
}
constexpr int HSPIN_NU = 3;    // units per site: spinor
constexpr int HGAUGE_NU = 6;   // four two-row links
constexpr int HCLOV_NU = 9;    // two packed Hermitian 6x6 blocks

// spinor of site d: stored values times the site norm
template <class S>
__device__ __forceinline__ void load_spinor_h(const S* f, const float* nrm, int d, int Vb, Spinor<float>& s) {
  float* v = reinterpret_cast<float*>(s.c);
#pragma unroll
  for (int u = 0; u < HSPIN_NU; ++u) ld8<S>(f, hunit<HSPIN_NU>(d, Vb, u), v + 8 * u);
  const float m = __ldg(nrm + d);
#pragma unroll
  for (int k = 0; k < SPINOR_NR; ++k) v[k] *= m;
}
// the stored values of site d's spinor, not yet multiplied by the site norm
template <class S>
__device__ __forceinline__ void load_spinor_h_raw(const S* f, int d, int Vb, Spinor<float>& s) {
  float* v = reinterpret_cast<float*>(s.c);
#pragma unroll
  for (int u = 0; u < HSPIN_NU; ++u) ld8<S>(f, hunit<HSPIN_NU>(d, Vb, u), v + 8 * u);
}
// the same for data written by an earlier kernel of the same sequence
template <class S>
__device__ __forceinline__ void load_spinor_h_cg(const S* f, const float* nrm, int d, int Vb, Spinor<float>& s) {
  float* v = reinterpret_cast<float*>(s.c);
#pragma unroll
  for (int u = 0; u < HSPIN_NU; ++u) ld8_cg<S>(f, hunit<HSPIN_NU>(d, Vb, u), v + 8 * u);
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
#pragma unroll
  for (int u = 0; u < HSPIN_NU; ++u) st8<S>(f, hunit<HSPIN_NU>(d, Vb, u), w + 8 * u);
  nrm[d] = m;
}

// the 12 values of link mu (two rows) within the 16 values of units
// (12 mu) / 8 and the next one, at offset (12 mu) % 8 = 4 (mu & 1)
__device__ __forceinline__ void link_rows_from16(const float* v16, int mu, Link<float>& U) {
  const bool odd = mu & 1;
#pragma unroll
  for (int k = 0; k < 6; ++k)
    U.m[k / 3][k % 3] = mk(odd ? v16[4 + 2 * k] : v16[2 * k], odd ? v16[5 + 2 * k] : v16[2 * k + 1]);
}
__device__ __forceinline__ void link_from16(const float* v16, int mu, Link<float>& U) {
  link_rows_from16(v16, mu, U);
  complete_link(U);
}
__device__ __forceinline__ int link_unit(int mu) { return (12 * mu) / 8; }

template <class S>
__device__ __forceinline__ void load_link_h(const S* g, int d, int Vb, int mu, Link<float>& U) {
  float v[16];
  const int u0 = link_unit(mu);
  ld8<S>(g, hunit<HGAUGE_NU>(d, Vb, u0), v);
  ld8<S>(g, hunit<HGAUGE_NU>(d, Vb, u0 + 1), v + 8);
  link_from16(v, mu, U);
}

// the 36 values of chiral block cb: units 4 cb .. 4 cb + 4, offset 4 cb
template <class S>
__device__ __forceinline__ void load_block36_h(const S* c, int d, int Vb, int cb, float* P) {
  float v[40];
  const int u0 = 4 * cb;
#pragma unroll
  for (int u = 0; u < 5; ++u) ld8<S>(c, hunit<HCLOV_NU>(d, Vb, u0 + u), v + 8 * u);
#pragma unroll
  for (int k = 0; k < 36; ++k) P[k] = cb ? v[4 + k] : v[k];
}

// y = A(site) v with the two packed chiral blocks of a half clover field
// (block 0: values 0..35, block 1: 36..71; unit 4 holds the end of block 0
// and the start of block 1)
template <class S>
__device__ __forceinline__ void clover_mul_h(const S* clov, int d, int Vb, const Spinor<float>& v, Spinor<float>& y) {
  float P[40];
#pragma unroll
  for (int u = 0; u < 5; ++u) ld8<S>(clov, hunit<HCLOV_NU>(d, Vb, u), P + 8 * u);
  herm6<float>(P, v.c, y.c);
  float Q[36];
#pragma unroll
  for (int k = 0; k < 4; ++k) Q[k] = P[36 + k];
#pragma unroll
  for (int u = 0; u < 4; ++u) ld8<S>(clov, hunit<HCLOV_NU>(d, Vb, 5 + u), Q + 4 + 8 * u);
  herm6<float>(Q, v.c + 6, y.c + 6);
}

}  // namespace ddamg
