// Wilson-clover stencil and layout conversions for half-precision storage
// (BF16 or FP16, see half.cuh) with FP32 arithmetic.
//
// D x = A x - 1/2 sum_mu [(1-g_mu) U_mu(x) x(x+mu) + (1+g_mu) U_mu(x-mu)^H x(x-mu)]
// (paper Sec. 1 and 3) with links, the two packed clover blocks and the
// spinors read from half fields (16-byte units of eight values): per site
// 48 + 4 bytes of input spinor, 96 of links (two rows of four links), 144 of
// clover, 48 + 4 of output.
#include "half.cuh"
#include "kernels.h"

namespace ddamg {

namespace {

constexpr int TPB = 128;

inline unsigned nblk(size_t n, int tpb) { return (unsigned)((n + tpb - 1) / tpb); }

// The hop is linear in the neighbour spinor, so its site norm m rides on the
// boundary sign: the stored values are projected and multiplied as they are
// and the result is accumulated with the factor +-m.
template <int MU, class S>
__device__ __forceinline__ void hop_dir_h(const Geom& g, const S* __restrict__ x, const float* __restrict__ xn,
                                          const S* __restrict__ gauge, int d, Spinor<float>& acc) {
  cpx<float> h[2][3], y[2][3];
  Spinor<float> nb;
  {  // forward: (1 - g_mu) U_mu(x) x(x+mu)
    const uint32_t e = __ldg(g.nbr + (size_t)(2 * MU) * g.V + d);
    const int n = (int)(e & ~NEG_BIT);
    const float m = __ldg(xn + n);
    const float sc = (e & NEG_BIT) ? -m : m;
    load_spinor_h_raw<S>(x, n, g.Vb, nb);
    project<MU, -1>(nb, h);
    Link<float> U;
    load_link_h<S>(gauge, d, g.Vb, MU, U);
    su3_mul(U, h, y);
    accumulate<MU, -1>(acc, y, sc);
  }
  {  // backward: (1 + g_mu) U_mu(x-mu)^H x(x-mu)
    const uint32_t e = __ldg(g.nbr + (size_t)(2 * MU + 1) * g.V + d);
    const int n = (int)(e & ~NEG_BIT);
    const float m = __ldg(xn + n);
    const float sc = (e & NEG_BIT) ? -m : m;
    load_spinor_h_raw<S>(x, n, g.Vb, nb);
    project<MU, +1>(nb, h);
    Link<float> U;
    load_link_h<S>(gauge, n, g.Vb, MU, U);
    su3_mul_dag(U, h, y);
    accumulate<MU, +1>(acc, y, sc);
  }
}

// one thread per site; right-hand side blockIdx.y (fields V sites apart)
// at most 80 registers: six CTAs per SM keep more loads in flight than the
// unbounded 96, and unlike 64 (eight CTAs) leave almost nothing to spill
template <class S, int MODE>
__global__ void __launch_bounds__(TPB, 6) k_dslash_h(Geom g, const S* __restrict__ x, const float* __restrict__ xn,
                                                  const S* __restrict__ b, const float* __restrict__ bn,
                                                  S* __restrict__ y, float* __restrict__ yn,
                                                  const S* __restrict__ gauge, const S* __restrict__ clover) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= g.V) return;
  const size_t off = (size_t)blockIdx.y * g.V * SPINOR_NR;
  const size_t noff = (size_t)blockIdx.y * g.V;
  x += off;
  xn += noff;
  y += off;
  yn += noff;
  Spinor<float> out;
  {  // A x on the stored values, then the site norm
    Spinor<float> xs;
    load_spinor_h_raw<S>(x, d, g.Vb, xs);
    clover_mul_h<S>(clover, d, g.Vb, xs, out);
    const float m = __ldg(xn + d);
#pragma unroll
    for (int k = 0; k < 12; ++k) out.c[k] = m * out.c[k];
  }
  if (MODE != DSLASH_CLOVER) {
    Spinor<float> acc;
#pragma unroll
    for (int k = 0; k < 12; ++k) acc.c[k] = mk(0.f, 0.f);
    hop_dir_h<0>(g, x, xn, gauge, d, acc);
    hop_dir_h<1>(g, x, xn, gauge, d, acc);
    hop_dir_h<2>(g, x, xn, gauge, d, acc);
    hop_dir_h<3>(g, x, xn, gauge, d, acc);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      out.c[k].re = fmaf(-0.5f, acc.c[k].re, out.c[k].re);
      out.c[k].im = fmaf(-0.5f, acc.c[k].im, out.c[k].im);
    }
  }
  if (MODE == DSLASH_RES) {
    Spinor<float> bs;
    load_spinor_h<S>(b + off, bn + noff, d, g.Vb, bs);
#pragma unroll
    for (int k = 0; k < 12; ++k) out.c[k] = bs.c[k] - out.c[k];
  }
  store_spinor_h<S>(y, yn, d, g.Vb, out);
}

// FP32 spinor fields -> half fields with site norms (nf fields)
template <class S>
__global__ void k_spinor_to_half(Geom g, const float* __restrict__ src, S* __restrict__ dst, float* __restrict__ nrm) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= g.V) return;
  const size_t off = (size_t)blockIdx.y * g.V * SPINOR_NR;
  Spinor<float> s;
  load_spinor<float>(src + off, d, g.Vb, s);
  store_spinor_h<S>(dst + off, nrm + (size_t)blockIdx.y * g.V, d, g.Vb, s);
}

// half fields -> FP32 fields (dst = value, or dst += value)
template <class S>
__global__ void k_spinor_from_half(Geom g, const S* __restrict__ src, const float* __restrict__ nrm,
                                   float* __restrict__ dst, int accumulate) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= g.V) return;
  const size_t off = (size_t)blockIdx.y * g.V * SPINOR_NR;
  Spinor<float> s;
  load_spinor_h<S>(src + off, nrm + (size_t)blockIdx.y * g.V, d, g.Vb, s);
  if (accumulate) {
    Spinor<float> o;
    load_spinor<float>(dst + off, d, g.Vb, o);
#pragma unroll
    for (int k = 0; k < 12; ++k) s.c[k] = s.c[k] + o.c[k];
  }
  store_spinor<float>(dst + off, d, g.Vb, s);
}

// an FP32 field of nr reals per site (FP32 layout, 16-byte units of four)
// -> the half layout (16-byte units of eight): half unit j of a site holds
// FP32 units 2 j and 2 j + 1
template <class S>
__global__ void k_to_half(Geom g, const float* __restrict__ src, S* __restrict__ dst, int nu8) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)g.V * nu8) return;
  const int d = (int)(i % g.V), j = (int)(i / g.V);
  const int B = d / g.Vb, q = d - B * g.Vb;
  const float4* s4 = reinterpret_cast<const float4*>(src);
  const size_t b4 = (size_t)B * (2 * nu8) * g.Vb + q;
  const float4 a = __ldg(s4 + b4 + (size_t)(2 * j) * g.Vb), c = __ldg(s4 + b4 + (size_t)(2 * j + 1) * g.Vb);
  const float w[8] = {a.x, a.y, a.z, a.w, c.x, c.y, c.z, c.w};
  st8<S>(dst, ((size_t)B * nu8 + j) * g.Vb + q, w);
}

}  // namespace

template <class S>
cudaError_t dslash_h(const Geom& g, int mode, const void* x, const float* xn, const void* b, const float* bn,
                     void* y, float* yn, const void* gauge, const void* clover, int nrhs, cudaStream_t st) {
  const dim3 grid(nblk(g.V, TPB), nrhs);
  const S* xs = static_cast<const S*>(x);
  const S* bs = static_cast<const S*>(b);
  S* ys = static_cast<S*>(y);
  const S* gs = static_cast<const S*>(gauge);
  const S* cs = static_cast<const S*>(clover);
  if (mode == DSLASH_D)
    k_dslash_h<S, DSLASH_D><<<grid, TPB, 0, st>>>(g, xs, xn, bs, bn, ys, yn, gs, cs);
  else if (mode == DSLASH_RES)
    k_dslash_h<S, DSLASH_RES><<<grid, TPB, 0, st>>>(g, xs, xn, bs, bn, ys, yn, gs, cs);
  else
    k_dslash_h<S, DSLASH_CLOVER><<<grid, TPB, 0, st>>>(g, xs, xn, bs, bn, ys, yn, gs, cs);
  ++g_launches;
  return cudaGetLastError();
}

template <class S>
cudaError_t spinor_to_half(const Geom& g, const float* src, void* dst, float* nrm, int nf, cudaStream_t st) {
  if (nf < 1) return cudaSuccess;
  k_spinor_to_half<S><<<dim3(nblk(g.V, TPB), nf), TPB, 0, st>>>(g, src, static_cast<S*>(dst), nrm);
  ++g_launches;
  return cudaGetLastError();
}

template <class S>
cudaError_t spinor_from_half(const Geom& g, const void* src, const float* nrm, float* dst, int nf, bool accumulate,
                             cudaStream_t st) {
  if (nf < 1) return cudaSuccess;
  k_spinor_from_half<S><<<dim3(nblk(g.V, TPB), nf), TPB, 0, st>>>(g, static_cast<const S*>(src), nrm, dst,
                                                                   accumulate ? 1 : 0);
  ++g_launches;
  return cudaGetLastError();
}

template <class S>
cudaError_t to_half(const Geom& g, const float* src, void* dst, int nr, cudaStream_t st) {
  const int nu8 = nr / 8;
  const size_t n = (size_t)g.V * nu8;
  if (!n) return cudaSuccess;
  k_to_half<S><<<nblk(n, 256), 256, 0, st>>>(g, src, static_cast<S*>(dst), nu8);
  ++g_launches;
  return cudaGetLastError();
}

#define INST_H(S)                                                                                              \
  template cudaError_t dslash_h<S>(const Geom&, int, const void*, const float*, const void*, const float*, void*, \
                                   float*, const void*, const void*, int, cudaStream_t);                      \
  template cudaError_t spinor_to_half<S>(const Geom&, const float*, void*, float*, int, cudaStream_t);         \
  template cudaError_t spinor_from_half<S>(const Geom&, const void*, const float*, float*, int, bool,           \
                                           cudaStream_t);                                                      \
  template cudaError_t to_half<S>(const Geom&, const float*, void*, int, cudaStream_t);

INST_H(__half)
INST_H(__nv_bfloat16)
#undef INST_H

}  // namespace ddamg
