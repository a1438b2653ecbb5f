// Coarse-grid kernels of the 2-level method (paper Sec. 2, Eq. 1-4, Fig. 1):
//   * orthonormalisation of the test vectors inside every aggregate X and
//     chirality s (classical Gram-Schmidt twice, FP64);
//   * restriction  b_c(X,s,i) = <lambda_i(X,s)|b>            (Eq. 3)
//   * prolongation x = sum x_c(X,s,i) lambda_i(X,s)             (Eq. 4)
//   * coarse operator D_c(X,s,i;Y,t,j) = <lambda_i(X,s)|D|lambda_j(Y,t)> (Eq. 2)
//     stored per coarse site as nine 2n x 2n blocks (self, then +mu / -mu);
//   * the 9-point coarse stencil and its even-odd preconditioned GMRES,
//     stopped at a relative residual of the even-site Schur system (Sec. 2).
// Aggregates coincide with the Schwarz blocks: aggregate X owns the device
// sites [X Vb, (X+1) Vb).
#include <cuda_fp16.h>

#include <mutex>

#include "common.cuh"
#include "half.cuh"
#include "kernels.h"

namespace ddamg {

namespace {

inline unsigned nblk(size_t n, int tpb) { return (unsigned)((n + tpb - 1) / tpb); }

template <class R>
__device__ __forceinline__ R warp_sum_t(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum of (a, b) over the CTA, broadcast to every thread; sh >= 2 * warps values
template <class R>
__device__ __forceinline__ void block_sum2_all(R& a, R& b, R* sh) {
  a = warp_sum_t<R>(a);
  b = warp_sum_t<R>(b);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) { sh[2 * w] = a; sh[2 * w + 1] = b; }
  __syncthreads();
  a = R(0); b = R(0);
  for (int i = 0; i < nw; ++i) { a += sh[2 * i]; b += sh[2 * i + 1]; }
  __syncthreads();
}

// sum of (a, b) over a warp with five additions per lane instead of ten:
// the halves trade one value each first.  Lane 0 returns the sum of a, lane
// 16 the sum of b.
template <class R>
__device__ __forceinline__ R warp_sum_pair(R a, R b) {
  const bool up = (threadIdx.x & 16) != 0;
  R keep = up ? b : a;
  keep += __shfl_xor_sync(0xffffffffu, up ? a : b, 16);
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) keep += __shfl_xor_sync(0xffffffffu, keep, o);
  return keep;
}

// ---------------------------------------------------------------------------
// orthonormalisation: CTA per (aggregate, chirality), SITES sites per thread.
// Classical Gram-Schmidt, two passes, in FP64 or FP32: for vector i every
// thread forms its partial products with all earlier vectors j < i at once,
// and the CTA reduces the i coefficients together (one barrier per pass, not
// per j).  In FP64 several sites per thread cut the share of additions spent
// in the cross-thread sums, FP64 being GB300's scarce arithmetic; in FP32 one
// site per thread keeps more loads in flight.
// ---------------------------------------------------------------------------
// the six complex components 6 s .. 6 s + 5 (chirality s) of the site whose
// unit 0 is at b: one component per FP64 unit, two per FP32 unit
template <class R>
struct Chiral6;
template <>
struct Chiral6<double> {
  __device__ __forceinline__ static void load(const double* f, size_t b, int Vb, int s, cpx<double>* v) {
    const double2* p = reinterpret_cast<const double2*>(f) + b + (size_t)6 * s * Vb;
#pragma unroll
    for (int u = 0; u < 6; ++u) {
      const double2 a = p[(size_t)u * Vb];
      v[u] = mk(a.x, a.y);
    }
  }
  __device__ __forceinline__ static void store(double* f, size_t b, int Vb, int s, const cpx<double>* v) {
    double2* p = reinterpret_cast<double2*>(f) + b + (size_t)6 * s * Vb;
#pragma unroll
    for (int u = 0; u < 6; ++u) p[(size_t)u * Vb] = make_double2(v[u].re, v[u].im);
  }
};
template <>
struct Chiral6<float> {
  __device__ __forceinline__ static void load(const float* f, size_t b, int Vb, int s, cpx<float>* v) {
    const float4* p = reinterpret_cast<const float4*>(f) + b + (size_t)3 * s * Vb;
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const float4 a = p[(size_t)u * Vb];
      v[2 * u] = mk(a.x, a.y);
      v[2 * u + 1] = mk(a.z, a.w);
    }
  }
  __device__ __forceinline__ static void store(float* f, size_t b, int Vb, int s, const cpx<float>* v) {
    float4* p = reinterpret_cast<float4*>(f) + b + (size_t)3 * s * Vb;
#pragma unroll
    for (int u = 0; u < 3; ++u) p[(size_t)u * Vb] = make_float4(v[2 * u].re, v[2 * u].im, v[2 * u + 1].re, v[2 * u + 1].im);
  }
};

template <class R, int SITES>
__global__ void k_orthonormalise(Geom g, R* __restrict__ lam, int n) {
  extern __shared__ __align__(16) unsigned char osh_raw[];   // red [warps][n][2], coef [n][2]
  R* osh = reinterpret_cast<R*>(osh_raw);
  const int nw = blockDim.x >> 5, w = threadIdx.x >> 5, l = threadIdx.x & 31;
  R* red = osh;
  R* coef = osh + (size_t)2 * nw * n;
  const int X = blockIdx.x, s = blockIdx.y;
  const size_t fstride = (size_t)g.V * SPINOR_NR / U16<R>::N;    // units per field
  using LY = Layout<R, SPINOR_NR>;
  using C6 = Chiral6<R>;
  bool own[SITES];
  size_t base[SITES];
#pragma unroll
  for (int e = 0; e < SITES; ++e) {
    const int q = threadIdx.x + e * blockDim.x;
    own[e] = q < g.Vb;
    base[e] = LY::base(X * g.Vb + (own[e] ? q : 0), g.Vb);
  }
  for (int i = 0; i < n; ++i) {
    cpx<R> v[SITES][6];
#pragma unroll
    for (int e = 0; e < SITES; ++e) {
      if (own[e]) C6::load(lam, base[e] + i * fstride, g.Vb, s, v[e]);
      else
#pragma unroll
        for (int u = 0; u < 6; ++u) v[e][u] = mk(R(0), R(0));
    }
    for (int pass = 0; pass < 2 && i > 0; ++pass) {
      for (int j = 0; j < i; ++j) {
        R re = R(0), im = R(0);
#pragma unroll
        for (int e = 0; e < SITES; ++e) {
          if (own[e]) {
            cpx<R> a[6];
            C6::load(lam, base[e] + j * fstride, g.Vb, s, a);
#pragma unroll
            for (int u = 0; u < 6; ++u) {
              re = ::fma(a[u].re, v[e][u].re, ::fma(a[u].im, v[e][u].im, re));
              im = ::fma(a[u].re, v[e][u].im, ::fma(-a[u].im, v[e][u].re, im));
            }
          }
        }
        const R r = warp_sum_pair<R>(re, im);
        if ((l & 15) == 0) red[(w * n + j) * 2 + (l >> 4)] = r;
      }
      __syncthreads();
      for (int j = threadIdx.x; j < i; j += blockDim.x) {
        R re = R(0), im = R(0);
        for (int ww = 0; ww < nw; ++ww) { re += red[(ww * n + j) * 2]; im += red[(ww * n + j) * 2 + 1]; }
        coef[2 * j] = re;
        coef[2 * j + 1] = im;
      }
      __syncthreads();
      for (int j = 0; j < i; ++j) {
        const R cr = coef[2 * j], ci = coef[2 * j + 1];
#pragma unroll
        for (int e = 0; e < SITES; ++e) {
          if (own[e]) {
            cpx<R> a[6];
            C6::load(lam, base[e] + j * fstride, g.Vb, s, a);
#pragma unroll
            for (int u = 0; u < 6; ++u) {
              v[e][u].re = ::fma(-cr, a[u].re, ::fma(ci, a[u].im, v[e][u].re));
              v[e][u].im = ::fma(-cr, a[u].im, ::fma(-ci, a[u].re, v[e][u].im));
            }
          }
        }
      }
      __syncthreads();
    }
    R nn = R(0), dummy = R(0);
#pragma unroll
    for (int e = 0; e < SITES; ++e)
#pragma unroll
      for (int u = 0; u < 6; ++u) nn = ::fma(v[e][u].re, v[e][u].re, ::fma(v[e][u].im, v[e][u].im, nn));
    block_sum2_all<R>(nn, dummy, red);
    const R f = R(1) / sqrt(nn);
#pragma unroll
    for (int e = 0; e < SITES; ++e)
      if (own[e]) {
#pragma unroll
        for (int u = 0; u < 6; ++u) v[e][u] = mk(v[e][u].re * f, v[e][u].im * f);
        C6::store(lam, base[e] + i * fstride, g.Vb, s, v[e]);
      }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// test vectors as R and P read them: in the field's precision, or (FP32
// arithmetic) stored in FP16 in the FP32 field layout with 8-byte units
// (four halves, two complex numbers, per unit)
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void load_lam(const R* lam, int d, int Vb, Spinor<R>& s) {
  load_spinor<R>(lam, d, Vb, s);
}
template <class S>
__device__ __forceinline__ void load_lam_h(const S* lam, int d, int Vb, Spinor<float>& s) {
  load_site_h4<S, SPINOR_NR>(lam, d, Vb, reinterpret_cast<float*>(s.c));
}
__device__ __forceinline__ void load_lam(const __half* lam, int d, int Vb, Spinor<float>& s) {
  load_lam_h<__half>(lam, d, Vb, s);
}
__device__ __forceinline__ void load_lam(const __nv_bfloat16* lam, int d, int Vb, Spinor<float>& s) {
  load_lam_h<__nv_bfloat16>(lam, d, Vb, s);
}

// half copy of FP32 test vectors, and the FP32 vectors rounded to the same
// values (so that D_c is assembled from exactly the P that R and P apply)
template <class S>
__global__ void k_round_half(float* __restrict__ lam32, S* __restrict__ lam16, size_t n4) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; i < n4; i += stride) {
    float4 v = reinterpret_cast<const float4*>(lam32)[i];
    float w[4] = {v.x, v.y, v.z, v.w};
    const uint2 p = pack4<S>(w);
    reinterpret_cast<uint2*>(lam16)[i] = p;
    unpack4<S>(p, w);
    reinterpret_cast<float4*>(lam32)[i] = make_float4(w[0], w[1], w[2], w[3]);
  }
}

// ---------------------------------------------------------------------------
// restriction: CTA per (aggregate, rhs)
// ---------------------------------------------------------------------------
// sum of 16 values over a warp as a reduce-scatter: 16 shuffles instead of
// 80; lane l ends with the total of value (l >> 1) & 15
template <class R>
__device__ __forceinline__ R warp_reduce_scatter16(R (&v)[16]) {
  const int l = threadIdx.x & 31;
#pragma unroll
  for (int lev = 0; lev < 4; ++lev) {
    const int half = 8 >> lev, off = 16 >> lev;
    const bool up = (l & off) != 0;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const R send = up ? v[k] : v[k + half];
      const R keep = up ? v[k + half] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// restriction b_c(X, s, i) = <lambda_i restricted to (X, s), b> (Eq. 3): CTA
// per (aggregate, rhs, slice); test vectors in groups of four, the groups
// dealt round-robin to gridDim.z slices (more CTAs for a single right-hand
// side), each site's b loaded once per group, the group's 16 sums reduced by
// a reduce-scatter
template <class R, class S>
__global__ void k_restrict(Geom g, const S* __restrict__ lam, int n, const R* __restrict__ b,
                           cpx<R>* __restrict__ bc) {
  extern __shared__ double rsh[];    // [warps][2n][2]
  const int X = blockIdx.x, rhs = blockIdx.y;
  const int nw = blockDim.x >> 5, w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const size_t fstride = (size_t)g.V * SPINOR_NR;
  const R* bb = b + rhs * fstride;
  for (int i0 = 4 * blockIdx.z; i0 < n; i0 += 4 * gridDim.z) {
    R acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = R(0);
    for (int q = threadIdx.x; q < g.Vb; q += blockDim.x) {
      const int d = X * g.Vb + q;
      Spinor<R> B;
      load_spinor<R>(bb, d, g.Vb, B);
#pragma unroll
      for (int ii = 0; ii < 4; ++ii) {
        if (i0 + ii < n) {
          Spinor<R> L;
          load_lam(lam + (i0 + ii) * fstride, d, g.Vb, L);
          cpx<R> a0 = mk(R(0), R(0)), a1 = mk(R(0), R(0));
#pragma unroll
          for (int k = 0; k < 6; ++k) fmac(a0, L.c[k], B.c[k]);
#pragma unroll
          for (int k = 6; k < 12; ++k) fmac(a1, L.c[k], B.c[k]);
          acc[4 * ii] += a0.re;
          acc[4 * ii + 1] += a0.im;
          acc[4 * ii + 2] += a1.re;
          acc[4 * ii + 3] += a1.im;
        }
      }
    }
    const R tot = warp_reduce_scatter16<R>(acc);
    const int vi = (l >> 1) & 15, ii = vi >> 2, sc = (vi >> 1) & 1, ri = vi & 1;
    if ((l & 1) == 0 && i0 + ii < n) rsh[(w * 2 * n + sc * n + i0 + ii) * 2 + ri] = (double)tot;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < 2 * n; r += blockDim.x) {
    const int i = r < n ? r : r - n;
    if (((i >> 2) % gridDim.z) != blockIdx.z) continue;   // another slice's vector
    double re = 0.0, im = 0.0;
    for (int ww = 0; ww < nw; ++ww) {
      re += rsh[(ww * 2 * n + r) * 2];
      im += rsh[(ww * 2 * n + r) * 2 + 1];
    }
    bc[((size_t)rhs * g.nb + X) * 2 * n + r] = mk((R)re, (R)im);
  }
}

// ---------------------------------------------------------------------------
// prolongation: thread per (site, rhs)
// ---------------------------------------------------------------------------
template <class R, class S>
__global__ void k_prolong(Geom g, const S* __restrict__ lam, int n, const cpx<R>* __restrict__ xc,
                          R* __restrict__ x, int accumulate) {
  int d = blockIdx.x * blockDim.x + threadIdx.x;
  int rhs = blockIdx.y;
  if (d >= g.V) return;
  const size_t fstride = (size_t)g.V * SPINOR_NR;
  int X = d / g.Vb;
  const cpx<R>* c = xc + ((size_t)rhs * g.nb + X) * 2 * n;
  Spinor<R> acc;
#pragma unroll
  for (int k = 0; k < 12; ++k) acc.c[k] = mk(R(0), R(0));
#pragma unroll 4
  for (int i = 0; i < n; ++i) {
    Spinor<R> L;
    load_lam(lam + i * fstride, d, g.Vb, L);
    cpx<R> c0 = c[i], c1 = c[n + i];
#pragma unroll
    for (int k = 0; k < 12; ++k) fma(acc.c[k], k < 6 ? c0 : c1, L.c[k]);
  }
  R* xx = x + rhs * fstride;
  if (accumulate) {
    Spinor<R> o;
    load_spinor<R>(xx, d, g.Vb, o);
#pragma unroll
    for (int k = 0; k < 12; ++k) acc.c[k] = acc.c[k] + o.c[k];
  }
  store_spinor<R>(xx, d, g.Vb, acc);
}

// ---------------------------------------------------------------------------
// coarse operator assembly: CTA per aggregate
//   smem: Lc[CH][12][n] = conj(lambda_i(x)), W[CH][12][2n] = term applied to
//   P_t lambda_j at the chunk's sites (column t n + j)
// ---------------------------------------------------------------------------
template <int MU, int SIGN, class R>
__device__ __forceinline__ void hop_term(const Spinor<R>& src, const Link<R>& U, R sc, Spinor<R>& acc) {
  cpx<R> h[2][3], y[2][3];
  project<MU, SIGN>(src, h);
  if (SIGN < 0) su3_mul(U, h, y);
  else su3_mul_dag(U, h, y);
  accumulate<MU, SIGN>(acc, y, sc);
}

template <class R>
__device__ void apply_term(const Geom& g, int dir, int MUv, int sgn, const Spinor<R>& src,
                           const Link<R>& U, R sc, Spinor<R>& acc) {
  // dispatch on the run-time direction to the compile-time projectors
  if (sgn < 0) {
    switch (MUv) {
      case 0: hop_term<0, -1>(src, U, sc, acc); break;
      case 1: hop_term<1, -1>(src, U, sc, acc); break;
      case 2: hop_term<2, -1>(src, U, sc, acc); break;
      default: hop_term<3, -1>(src, U, sc, acc); break;
    }
  } else {
    switch (MUv) {
      case 0: hop_term<0, +1>(src, U, sc, acc); break;
      case 1: hop_term<1, +1>(src, U, sc, acc); break;
      case 2: hop_term<2, +1>(src, U, sc, acc); break;
      default: hop_term<3, +1>(src, U, sc, acc); break;
    }
  }
}

// load lambda_j at device site d projected on chirality t
template <class R>
__device__ __forceinline__ void load_proj(const R* lam_j, int d, int Vb, int t, Spinor<R>& s) {
  load_spinor<R>(lam_j, d, Vb, s);
#pragma unroll
  for (int k = 0; k < 12; ++k)
    if ((k / 6) != t) s.c[k] = mk(R(0), R(0));
}

template <class R>
__global__ void k_assemble(Geom g, const R* __restrict__ lam, int n, const R* __restrict__ gauge,
                           const R* __restrict__ clover, cpx<R>* __restrict__ Dc, int CH) {
  extern __shared__ __align__(16) unsigned char ash[];
  const int X = blockIdx.x;
  const int n2 = 2 * n, NE = n2 * n2;
  cpx<R>* Lc = reinterpret_cast<cpx<R>*>(ash);            // [CH][12][n]
  cpx<R>* W = Lc + (size_t)CH * 12 * n;                   // [CH][12][2n]
  int* sites = reinterpret_cast<int*>(W + (size_t)CH * 12 * n2);   // [CH]
  const size_t fstride = (size_t)g.V * SPINOR_NR;
  constexpr int MAXE = 16;   // entries per thread (4 n^2 <= 16 * blockDim)
  for (int dd = 0; dd < 9; ++dd) {
    cpx<R> acc[MAXE];
#pragma unroll
    for (int e = 0; e < MAXE; ++e) acc[e] = mk(R(0), R(0));
    const int mu = dd == 0 ? 0 : (dd - 1) / 2;
    const int nsite = dd == 0 ? g.Vb : g.Vb / g.b[mu];
    for (int c0 = 0; c0 < nsite; c0 += CH) {
      const int cn = min(CH, nsite - c0);
      if (threadIdx.x < cn) {
        int q = dd == 0 ? c0 + threadIdx.x : g.face[(dd - 1) * g.Vb + c0 + threadIdx.x];
        sites[threadIdx.x] = X * g.Vb + q;
      }
      __syncthreads();
      // conj(lambda_i) at the chunk's sites
      for (int it = threadIdx.x; it < cn * n; it += blockDim.x) {
        int si = it / n, i = it - si * n;
        Spinor<R> L;
        load_spinor<R>(lam + i * fstride, sites[si], g.Vb, L);
#pragma unroll
        for (int k = 0; k < 12; ++k) Lc[((size_t)si * 12 + k) * n + i] = conj(L.c[k]);
      }
      // terms applied to P_t lambda_j
      for (int it = threadIdx.x; it < cn * n2; it += blockDim.x) {
        int si = it / n2, col = it - si * n2;
        int t = col / n, j = col - t * n;
        int d = sites[si];
        const R* lj = lam + j * fstride;
        Spinor<R> out;
#pragma unroll
        for (int k = 0; k < 12; ++k) out.c[k] = mk(R(0), R(0));
        if (dd == 0) {
          // A(x) + hops that stay inside the aggregate
          Spinor<R> v, hacc;
          load_proj<R>(lj, d, g.Vb, t, v);
          clover_mul<R>(clover, d, g.Vb, v, out);
#pragma unroll
          for (int k = 0; k < 12; ++k) hacc.c[k] = mk(R(0), R(0));
          for (int m = 0; m < 4; ++m) {
            uint32_t ef = __ldg(g.nbr + (size_t)(2 * m) * g.V + d);
            int nf = (int)(ef & ~NEG_BIT);
            if (nf / g.Vb == X) {
              Link<R> U;
              load_link<R>(gauge, d, g.Vb, m, U);
              load_proj<R>(lj, nf, g.Vb, t, v);
              apply_term<R>(g, 0, m, -1, v, U, (ef & NEG_BIT) ? R(-1) : R(1), hacc);
            }
            uint32_t eb = __ldg(g.nbr + (size_t)(2 * m + 1) * g.V + d);
            int nbk = (int)(eb & ~NEG_BIT);
            if (nbk / g.Vb == X) {
              Link<R> U;
              load_link<R>(gauge, nbk, g.Vb, m, U);
              load_proj<R>(lj, nbk, g.Vb, t, v);
              apply_term<R>(g, 0, m, +1, v, U, (eb & NEG_BIT) ? R(-1) : R(1), hacc);
            }
          }
#pragma unroll
          for (int k = 0; k < 12; ++k) {
            out.c[k].re = fma_r(R(-0.5), hacc.c[k].re, out.c[k].re);
            out.c[k].im = fma_r(R(-0.5), hacc.c[k].im, out.c[k].im);
          }
        } else {
          const int fwd = ((dd - 1) & 1) == 0;
          uint32_t e = __ldg(g.nbr + (size_t)(dd - 1) * g.V + d);
          int nbd = (int)(e & ~NEG_BIT);
          Spinor<R> v, hacc;
#pragma unroll
          for (int k = 0; k < 12; ++k) hacc.c[k] = mk(R(0), R(0));
          Link<R> U;
          load_link<R>(gauge, fwd ? d : nbd, g.Vb, mu, U);
          load_proj<R>(lj, nbd, g.Vb, t, v);
          apply_term<R>(g, 0, mu, fwd ? -1 : +1, v, U, (e & NEG_BIT) ? R(-1) : R(1), hacc);
#pragma unroll
          for (int k = 0; k < 12; ++k) out.c[k] = R(-0.5) * hacc.c[k];
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) W[((size_t)si * 12 + k) * n2 + col] = out.c[k];
      }
      __syncthreads();
      // contraction
#pragma unroll
      for (int e = 0; e < MAXE; ++e) {
        int idx = threadIdx.x + e * blockDim.x;
        if (idx < NE) {
          int r = idx / n2, c = idx - r * n2;
          int s = r / n, i = r - s * n;
          cpx<R> a = acc[e];
          for (int si = 0; si < cn; ++si)
#pragma unroll
            for (int k = 0; k < 6; ++k) {
              int kk = 6 * s + k;
              fma(a, Lc[((size_t)si * 12 + kk) * n + i], W[((size_t)si * 12 + kk) * n2 + c]);
            }
          acc[e] = a;
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int e = 0; e < MAXE; ++e) {
      int idx = threadIdx.x + e * blockDim.x;
      if (idx < NE) {
        int r = idx / n2, c = idx - r * n2;
        Dc[((size_t)X * 9 + dd) * NE + (size_t)c * n2 + r] = acc[e];   // column-major block
      }
    }
  }
}

// ---------------------------------------------------------------------------
// self-block inversion: CTA per coarse site, Gauss-Jordan in FP64 smem
// ---------------------------------------------------------------------------
template <class R>
__global__ void k_invert_self(Geom g, const cpx<R>* __restrict__ Dc, int n2, cpx<R>* __restrict__ Ainv,
                              int* singular) {
  extern __shared__ double ish[];
  cpx<double>* M = reinterpret_cast<cpx<double>*>(ish);   // [n2][2 n2]
  __shared__ int piv_s;
  const int X = blockIdx.x;
  const int W2 = 2 * n2;
  const cpx<R>* A = Dc + (size_t)X * 9 * n2 * n2;
  for (int idx = threadIdx.x; idx < n2 * W2; idx += blockDim.x) {
    int r = idx / W2, c = idx - r * W2;
    cpx<double> v;
    if (c < n2) v = mk((double)A[c * n2 + r].re, (double)A[c * n2 + r].im);
    else v = mk(c - n2 == r ? 1.0 : 0.0, 0.0);
    M[idx] = v;
  }
  __syncthreads();
  for (int col = 0; col < n2; ++col) {
    if (threadIdx.x == 0) {
      int p = col;
      double best = norm2(M[col * W2 + col]);
      for (int r = col + 1; r < n2; ++r) {
        double v = norm2(M[r * W2 + col]);
        if (v > best) { best = v; p = r; }
      }
      piv_s = best > 0.0 ? p : -1;
      if (best == 0.0) atomicExch(singular, 1);
    }
    __syncthreads();
    int p = piv_s;
    if (p < 0) return;
    if (p != col) {
      for (int c = threadIdx.x; c < W2; c += blockDim.x) {
        cpx<double> t = M[col * W2 + c];
        M[col * W2 + c] = M[p * W2 + c];
        M[p * W2 + c] = t;
      }
      __syncthreads();
    }
    cpx<double> pv = M[col * W2 + col];
    double pn = norm2(pv);
    cpx<double> pinv = mk(pv.re / pn, -pv.im / pn);
    __syncthreads();
    for (int c = threadIdx.x; c < W2; c += blockDim.x) M[col * W2 + c] = M[col * W2 + c] * pinv;
    __syncthreads();
    for (int idx = threadIdx.x; idx < n2 * W2; idx += blockDim.x) {
      int r = idx / W2, c = idx - r * W2;
      if (r == col || c == col) continue;
      cpx<double> f = M[r * W2 + col];
      M[idx] = M[idx] - f * M[col * W2 + c];
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n2; r += blockDim.x)
      if (r != col) M[r * W2 + col] = mk(0.0, 0.0);
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < n2 * n2; idx += blockDim.x) {
    int r = idx / n2, c = idx - r * n2;
    cpx<double> v = M[r * W2 + n2 + c];
    Ainv[(size_t)X * n2 * n2 + (size_t)c * n2 + r] = mk((R)v.re, (R)v.im);   // column-major
  }
}

// ---------------------------------------------------------------------------
// coarse 9-point stencil (Eq. 2 applied): y(X) = sum_d D_c(X,d) x(nbr_d(X)).
// The nine 2n x 2n blocks of a site are stored column-major and back to back,
// so together they form one 2n x 18n matrix whose column dc = d*2n + c
// multiplies x(nbr_d(X))[c].  A team of NP = 2n / RPU threads owns a site;
// a thread owns RPU rows (two in FP32, one in FP64), streams them down all
// 18n columns with 16-byte loads (neighbouring threads read neighbouring rows
// of a column) and accumulates in registers.  Every byte of D_c is read once,
// no partial sums go through shared memory and no thread idles while others
// stream.  The gathered neighbour vectors sit in shared memory, one padded
// copy per team so that the teams' broadcasts fall in different banks.  The
// sum runs in a fixed order, so the result is bitwise reproducible.
// ---------------------------------------------------------------------------
template <class R>
__global__ void k_coarse_apply(Geom g, const cpx<R>* __restrict__ Dc, int n2, int S,
                               const cpx<R>* __restrict__ x, cpx<R>* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char csh[];
  using T = typename U16<R>::T;
  constexpr int RPU = 16 / (2 * sizeof(R));      // rows per 16-byte load
  const int NP = n2 / RPU;
  const int NC = 9 * n2;                         // columns of the site's 2n x 18n matrix
  const int team = threadIdx.x / NP, j = threadIdx.x - team * NP;
  const int X = blockIdx.x * S + team;
  const bool live = team < S && X < g.nb;
  cpx<R>* sv = reinterpret_cast<cpx<R>*>(csh) + team * (NC + 1);
  const size_t roff = (size_t)blockIdx.y * g.nb * n2;
  if (live) {
    const cpx<R>* xr = x + roff;
    for (int idx = j; idx < NC; idx += NP) {
      const int d = idx / n2, c = idx - d * n2;
      sv[idx] = xr[(size_t)g.cnbr[d * g.nb + X] * n2 + c];
    }
  }
  __syncthreads();
  if (!live) return;
  const T* col = reinterpret_cast<const T*>(Dc + (size_t)X * NC * n2) + j;
  cpx<R> a0 = mk(R(0), R(0)), a1 = mk(R(0), R(0));
#pragma unroll 8
  for (int c = 0; c < NC; ++c) {
    const T m = __ldg(col + (size_t)c * NP);
    const cpx<R> vc = sv[c];
    if constexpr (RPU == 2) {
      fma(a0, mk((R)m.x, (R)m.y), vc);
      fma(a1, mk((R)m.z, (R)m.w), vc);
    } else {
      fma(a0, mk((R)m.x, (R)m.y), vc);
    }
  }
  cpx<R>* out = y + roff + (size_t)X * n2 + RPU * j;
  out[0] = a0;
  if constexpr (RPU == 2) out[1] = a1;
}

// The same stencil from five of the nine blocks.  D is gamma5-hermitian term
// by term (the backward hop x+mu -> x is gamma5 T^H gamma5 of the forward hop
// T: x -> x+mu), and P keeps chirality, so every backward block of D_c is
// the conjugate of its neighbour's forward block:
//   D_c(X, d = 2 + 2 mu) = G5 D_c(X - mu, d = 1 + 2 mu)^H G5,
// G5 = diag(1_n, -1_n) on a coarse site.  A team reads the self block and the
// four forward blocks of its site as above, and for the backward terms the
// neighbour's forward block M: (G5 M^H G5 v)[r] = g_r sum_c conj(M(c, r)) g_c
// v[c], where M(c, r), column r of the column-major M, is contiguous, so a
// thread streams the columns of its own rows.  The signs g_c ride on the
// staged neighbour vectors, g_r on the backward sum.  Valid for a D_c that
// was assembled from a gamma5-hermitian D (not for an arbitrary stencil).
template <class R>
__global__ void k_coarse_apply_g5(Geom g, const cpx<R>* __restrict__ Dc, int n2, int S,
                                  const cpx<R>* __restrict__ x, cpx<R>* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char csh[];
  using T = typename U16<R>::T;
  constexpr int RPU = 16 / (2 * sizeof(R));      // rows per 16-byte load
  const int NP = n2 / RPU, n = n2 / 2;
  const int NC = 9 * n2;
  const int team = threadIdx.x / NP, j = threadIdx.x - team * NP;
  const int X = blockIdx.x * S + team;
  const bool live = team < S && X < g.nb;
  cpx<R>* sv = reinterpret_cast<cpx<R>*>(csh) + team * (NC + 1);
  const size_t roff = (size_t)blockIdx.y * g.nb * n2;
  if (live) {
    const cpx<R>* xr = x + roff;
    for (int idx = j; idx < NC; idx += NP) {
      const int d = idx / n2, c = idx - d * n2;
      const cpx<R> v = xr[(size_t)g.cnbr[d * g.nb + X] * n2 + c];
      sv[idx] = (d >= 2 && (d & 1) == 0 && c >= n) ? mk(-v.re, -v.im) : v;
    }
  }
  __syncthreads();
  if (!live) return;
  // self and forward blocks (d = 0, 1, 3, 5, 7) of the site
  cpx<R> a[RPU];
#pragma unroll
  for (int q = 0; q < RPU; ++q) a[q] = mk(R(0), R(0));
  const T* site = reinterpret_cast<const T*>(Dc + (size_t)X * NC * n2) + j;
  for (int t = 0; t < 5; ++t) {
    const int d = t == 0 ? 0 : 2 * t - 1;
    const T* col = site + (size_t)d * n2 * NP;
    const cpx<R>* vs = sv + d * n2;
#pragma unroll 8
    for (int c = 0; c < n2; ++c) {
      const T m = __ldg(col + (size_t)c * NP);
      const cpx<R> vc = vs[c];
      if constexpr (RPU == 2) {
        fma(a[0], mk((R)m.x, (R)m.y), vc);
        fma(a[1], mk((R)m.z, (R)m.w), vc);
      } else {
        fma(a[0], mk((R)m.x, (R)m.y), vc);
      }
    }
  }
  // backward blocks from the neighbours' forward blocks
  cpx<R> b[RPU];
#pragma unroll
  for (int q = 0; q < RPU; ++q) b[q] = mk(R(0), R(0));
  for (int mu = 0; mu < 4; ++mu) {
    const int Y = g.cnbr[(2 + 2 * mu) * g.nb + X];
    const cpx<R>* M = Dc + ((size_t)Y * 9 + 1 + 2 * mu) * n2 * n2;
    const cpx<R>* vs = sv + (2 + 2 * mu) * n2;
#pragma unroll
    for (int q = 0; q < RPU; ++q) {
      const T* colr = reinterpret_cast<const T*>(M + (size_t)(RPU * j + q) * n2);
      cpx<R> s = mk(R(0), R(0));
#pragma unroll 4
      for (int u = 0; u < NP; ++u) {
        const T m = __ldg(colr + u);
        if constexpr (RPU == 2) {
          fma(s, mk((R)m.x, (R)-m.y), vs[2 * u]);
          fma(s, mk((R)m.z, (R)-m.w), vs[2 * u + 1]);
        } else {
          fma(s, mk((R)m.x, (R)-m.y), vs[u]);
        }
      }
      b[q] = b[q] + s;
    }
  }
  cpx<R>* out = y + roff + (size_t)X * n2 + RPU * j;
#pragma unroll
  for (int q = 0; q < RPU; ++q) out[q] = (RPU * j + q < n) ? a[q] + b[q] : a[q] - b[q];
}

// C = A B for one odd site X and direction d (column-major 2n x 2n blocks)
template <class R>
__global__ void k_premultiply_odd(Geom g, const cpx<R>* __restrict__ Dc, const cpx<R>* __restrict__ Ainv, int n2,
                                  cpx<R>* __restrict__ AD) {
  extern __shared__ __align__(16) unsigned char psh[];
  cpx<R>* As = reinterpret_cast<cpx<R>*>(psh);
  cpx<R>* Bs = As + n2 * n2;
  const int ko = blockIdx.x, d = blockIdx.y + 1;
  const int X = g.codd[ko];
  const cpx<R>* A = Ainv + (size_t)X * n2 * n2;
  const cpx<R>* B = Dc + ((size_t)X * 9 + d) * n2 * n2;
  for (int i = threadIdx.x; i < n2 * n2; i += blockDim.x) {
    As[i] = A[i];
    Bs[i] = B[i];
  }
  __syncthreads();
  cpx<R>* C = AD + ((size_t)ko * 8 + (d - 1)) * n2 * n2;
  // accumulated in the blocks' own precision (FP32 blocks stay off the FP64 pipe)
  for (int i = threadIdx.x; i < n2 * n2; i += blockDim.x) {
    const int r = i % n2, c = i / n2;
    cpx<R> acc = mk(R(0), R(0));
    for (int k = 0; k < n2; ++k) fma(acc, As[k * n2 + r], Bs[c * n2 + k]);
    C[i] = acc;
  }
}

template <class R>
__global__ void k_coarse_export(const cpx<R>* __restrict__ src, double* __restrict__ dst, int n2, size_t nblocks) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t total = nblocks * n2 * n2;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; i < total; i += stride) {
    size_t blk = i / ((size_t)n2 * n2);
    int e = (int)(i - blk * n2 * n2);
    int r = e / n2, c = e - r * n2;
    cpx<R> v = src[blk * n2 * n2 + (size_t)c * n2 + r];
    dst[2 * i] = (double)v.re;
    dst[2 * i + 1] = (double)v.im;
  }
}

// row-major complex doubles (host layout) -> column-major blocks in R
template <class R>
__global__ void k_coarse_import(const double* __restrict__ src, cpx<R>* __restrict__ dst, int n2, size_t nblocks) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t total = nblocks * n2 * n2;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; i < total; i += stride) {
    size_t blk = i / ((size_t)n2 * n2);
    int e = (int)(i - blk * n2 * n2);
    int r = e / n2, c = e - r * n2;
    dst[blk * n2 * n2 + (size_t)c * n2 + r] = mk((R)src[2 * i], (R)src[2 * i + 1]);
  }
}

template <class RD, class RS>
__global__ void k_conv_c(const RS* __restrict__ s, RD* __restrict__ d, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) d[i] = (RD)s[i];
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <class R, int SITES>
static cudaError_t ortho_launch(const Geom& g, R* lam, int n, cudaStream_t st) {
  const int threads = (((g.Vb + SITES - 1) / SITES + 31) / 32) * 32;
  if (threads > 1024) return cudaErrorInvalidValue;
  const size_t smem = ((size_t)2 * (threads / 32) * (n > 1 ? n : 1) + 2 * n) * sizeof(R);
  k_orthonormalise<R, SITES><<<dim3(g.nb, 2), threads, smem, st>>>(g, lam, n);
  ++g_launches;
  return cudaGetLastError();
}
cudaError_t orthonormalise(const Geom& g, double* lam, int n, cudaStream_t st) {
  return ortho_launch<double, 4>(g, lam, n, st);
}
cudaError_t orthonormalise(const Geom& g, float* lam, int n, cudaStream_t st) {
  if (g.Vb <= 1024) return ortho_launch<float, 1>(g, lam, n, st);
  return ortho_launch<float, 4>(g, lam, n, st);
}

template <class R, class S>
static cudaError_t restrict_launch(const Geom& g, const S* lam, int n, const R* b, R* bc, int nrhs,
                                   cudaStream_t st) {
  int threads = g.Vb >= 256 ? 256 : ((g.Vb + 31) / 32) * 32;
  size_t smem = (size_t)(threads / 32) * 2 * n * 2 * sizeof(double);
  // a single right-hand side leaves SMs idle with one CTA per aggregate
  const int slices = (nrhs == 1 && n >= 8) ? 2 : 1;
  k_restrict<R, S><<<dim3(g.nb, nrhs, slices), threads, smem, st>>>(g, lam, n, b, reinterpret_cast<cpx<R>*>(bc));
  ++g_launches;
  return cudaGetLastError();
}
template <class R, class S>
static cudaError_t prolong_launch(const Geom& g, const S* lam, int n, const R* xc, R* x, int nrhs, bool accumulate,
                                  cudaStream_t st) {
  k_prolong<R, S><<<dim3(nblk(g.V, 128), nrhs), 128, 0, st>>>(
      g, lam, n, reinterpret_cast<const cpx<R>*>(xc), x, accumulate ? 1 : 0);
  ++g_launches;
  return cudaGetLastError();
}

template <class R>
cudaError_t restrict_op(const Geom& g, const R* lam, int n, const R* b, R* bc, int nrhs, cudaStream_t st) {
  return restrict_launch<R, R>(g, lam, n, b, bc, nrhs, st);
}
template <class R>
cudaError_t prolong_op(const Geom& g, const R* lam, int n, const R* xc, R* x, int nrhs, bool accumulate,
                       cudaStream_t st) {
  return prolong_launch<R, R>(g, lam, n, xc, x, nrhs, accumulate, st);
}
cudaError_t restrict_op_h(const Geom& g, int bf16, const void* lam16, int n, const float* b, float* bc, int nrhs,
                          cudaStream_t st) {
  if (bf16)
    return restrict_launch<float, __nv_bfloat16>(g, static_cast<const __nv_bfloat16*>(lam16), n, b, bc, nrhs, st);
  return restrict_launch<float, __half>(g, static_cast<const __half*>(lam16), n, b, bc, nrhs, st);
}
cudaError_t prolong_op_h(const Geom& g, int bf16, const void* lam16, int n, const float* xc, float* x, int nrhs,
                         bool accumulate, cudaStream_t st) {
  if (bf16)
    return prolong_launch<float, __nv_bfloat16>(g, static_cast<const __nv_bfloat16*>(lam16), n, xc, x, nrhs,
                                                accumulate, st);
  return prolong_launch<float, __half>(g, static_cast<const __half*>(lam16), n, xc, x, nrhs, accumulate, st);
}
cudaError_t round_vectors_half(int bf16, float* lam32, void* lam16, size_t n, cudaStream_t st) {
  const size_t n4 = n / 4;
  unsigned nb = nblk(n4, 256);
  if (nb > 4096) nb = 4096;
  if (!nb) return cudaSuccess;
  if (bf16) k_round_half<__nv_bfloat16><<<nb, 256, 0, st>>>(lam32, static_cast<__nv_bfloat16*>(lam16), n4);
  else k_round_half<__half><<<nb, 256, 0, st>>>(lam32, static_cast<__half*>(lam16), n4);
  ++g_launches;
  return cudaGetLastError();
}

static int assemble_chunk(int n, int real_size) {
  size_t per_site = (size_t)12 * 3 * n * 2 * real_size + sizeof(int);
  int ch = (int)((160 * 1024) / per_site);
  if (ch > 32) ch = 32;
  if (ch < 1) ch = 1;
  return ch;
}

template <class R>
cudaError_t assemble_coarse(const Geom& g, const R* lam, int n, const R* gauge, const R* clover, R* Dc,
                            cudaStream_t st) {
  const int threads = 256;
  if (4 * n * n > 16 * threads) return cudaErrorInvalidValue;
  int ch = assemble_chunk(n, sizeof(R));
  size_t smem = (size_t)ch * 12 * 3 * n * 2 * sizeof(R) + ch * sizeof(int) + 16;
  cudaError_t e = raise_smem_limit((const void*)k_assemble<R>, smem);
  if (e != cudaSuccess) return e;
  k_assemble<R><<<g.nb, threads, smem, st>>>(g, lam, n, gauge, clover, reinterpret_cast<cpx<R>*>(Dc), ch);
  ++g_launches;
  return cudaGetLastError();
}

template <class R>
cudaError_t invert_self_blocks(const Geom& g, const R* Dc, int n, R* Ainv, int* singular, cudaStream_t st) {
  int n2 = 2 * n;
  size_t smem = (size_t)n2 * 2 * n2 * sizeof(cpx<double>);
  cudaError_t e = raise_smem_limit((const void*)k_invert_self<R>, smem);
  if (e != cudaSuccess) return e;
  k_invert_self<R><<<g.nb, 256, smem, st>>>(g, reinterpret_cast<const cpx<R>*>(Dc), n2,
                                            reinterpret_cast<cpx<R>*>(Ainv), singular);
  ++g_launches;
  return cudaGetLastError();
}

template <class R>
cudaError_t premultiply_odd(const Geom& g, const R* Dc, const R* Ainv, int n, R* AD, cudaStream_t st) {
  const int n2 = 2 * n;
  const size_t smem = (size_t)2 * n2 * n2 * sizeof(cpx<R>);
  cudaError_t e = raise_smem_limit((const void*)k_premultiply_odd<R>, smem);
  if (e != cudaSuccess) return e;
  k_premultiply_odd<R><<<dim3(g.nb / 2, 8), 256, smem, st>>>(g, reinterpret_cast<const cpx<R>*>(Dc),
                                                           reinterpret_cast<const cpx<R>*>(Ainv), n2,
                                                           reinterpret_cast<cpx<R>*>(AD));
  ++g_launches;
  return cudaGetLastError();
}

template <class R>
cudaError_t coarse_apply(const Geom& g, const R* Dc, int n, const R* x, R* y, int nrhs, cudaStream_t st,
                         bool g5) {
  const int n2 = 2 * n;
  const int NP = n2 / (16 / (2 * (int)sizeof(R)));
  // sites per CTA: the fewest that fill whole warps, at most 1024 threads
  int S = 32;
  while (S > 1 && (S / 2) * NP % 32 == 0) S /= 2;
  while (S > 1 && S * NP > 1024) S /= 2;
  const size_t smem = (size_t)S * (9 * n2 + 1) * sizeof(cpx<R>);
  const void* fn = g5 ? (const void*)k_coarse_apply_g5<R> : (const void*)k_coarse_apply<R>;
  if (smem > 48 * 1024) {
    cudaError_t e = raise_smem_limit(fn, smem);
    if (e != cudaSuccess) return e;
  }
  if (g5) {
    // the backward terms read each thread's own columns: keep half of the
    // unified L1 / shared memory as L1 so that their lines stay resident
    // (a hint; measured 293 us against 311 with the default split)
    static std::once_flag once;
    std::call_once(once, [] {
      cudaFuncSetAttribute(k_coarse_apply_g5<R>, cudaFuncAttributePreferredSharedMemoryCarveout, 50);
      cudaGetLastError();
    });
  }
  const dim3 grid((g.nb + S - 1) / S, nrhs);
  const auto* Dcc = reinterpret_cast<const cpx<R>*>(Dc);
  const auto* xc = reinterpret_cast<const cpx<R>*>(x);
  auto* yc = reinterpret_cast<cpx<R>*>(y);
  if (g5) k_coarse_apply_g5<R><<<grid, S * NP, smem, st>>>(g, Dcc, n2, S, xc, yc);
  else k_coarse_apply<R><<<grid, S * NP, smem, st>>>(g, Dcc, n2, S, xc, yc);
  ++g_launches;
  return cudaGetLastError();
}

template <class R>
cudaError_t coarse_from_f64(const double* src, R* dst, size_t ncomplex, cudaStream_t st) {
  size_t n = 2 * ncomplex;
  unsigned nb = nblk(n, 256);
  if (nb > 4096) nb = 4096;
  if (!nb) return cudaSuccess;
  k_conv_c<R, double><<<nb, 256, 0, st>>>(src, dst, n);
  ++g_launches;
  return cudaGetLastError();
}
template <class R>
cudaError_t coarse_to_f64(const R* src, double* dst, size_t ncomplex, cudaStream_t st) {
  size_t n = 2 * ncomplex;
  unsigned nb = nblk(n, 256);
  if (nb > 4096) nb = 4096;
  if (!nb) return cudaSuccess;
  k_conv_c<double, R><<<nb, 256, 0, st>>>(src, dst, n);
  ++g_launches;
  return cudaGetLastError();
}

template <class R>
cudaError_t coarse_export(const R* Dc, int n, size_t nblocks, double* out, cudaStream_t st) {
  k_coarse_export<R><<<4096, 256, 0, st>>>(reinterpret_cast<const cpx<R>*>(Dc), out, 2 * n, nblocks);
  ++g_launches;
  return cudaGetLastError();
}
template <class R>
cudaError_t coarse_import(const double* src, int n, size_t nblocks, R* Dc, cudaStream_t st) {
  k_coarse_import<R><<<4096, 256, 0, st>>>(src, reinterpret_cast<cpx<R>*>(Dc), 2 * n, nblocks);
  ++g_launches;
  return cudaGetLastError();
}
template cudaError_t coarse_import<float>(const double*, int, size_t, float*, cudaStream_t);
template cudaError_t coarse_import<double>(const double*, int, size_t, double*, cudaStream_t);
template cudaError_t coarse_export<float>(const float*, int, size_t, double*, cudaStream_t);
template cudaError_t coarse_export<double>(const double*, int, size_t, double*, cudaStream_t);

// instantiations
#define INST(R)                                                                                          \
  template cudaError_t restrict_op<R>(const Geom&, const R*, int, const R*, R*, int, cudaStream_t);     \
  template cudaError_t prolong_op<R>(const Geom&, const R*, int, const R*, R*, int, bool, cudaStream_t); \
  template cudaError_t assemble_coarse<R>(const Geom&, const R*, int, const R*, const R*, R*,           \
                                          cudaStream_t);                                                \
  template cudaError_t invert_self_blocks<R>(const Geom&, const R*, int, R*, int*, cudaStream_t);       \
  template cudaError_t premultiply_odd<R>(const Geom&, const R*, const R*, int, R*, cudaStream_t);      \
  template cudaError_t coarse_apply<R>(const Geom&, const R*, int, const R*, R*, int, cudaStream_t, bool); \
  template cudaError_t coarse_from_f64<R>(const double*, R*, size_t, cudaStream_t);                     \
  template cudaError_t coarse_to_f64<R>(const R*, double*, size_t, cudaStream_t);                       \

INST(float)
INST(double)
#undef INST

}  // namespace ddamg
