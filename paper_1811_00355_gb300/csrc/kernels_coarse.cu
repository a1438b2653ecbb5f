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
#include "common.cuh"
#include "kernels.h"

namespace ddamg {

namespace {

inline unsigned nblk(size_t n, int tpb) { return (unsigned)((n + tpb - 1) / tpb); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum of (a, b) over the CTA, broadcast to every thread; sh >= 2 * warps doubles
__device__ __forceinline__ void block_sum2_all(double& a, double& b, double* sh) {
  a = warp_sum(a);
  b = warp_sum(b);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) { sh[2 * w] = a; sh[2 * w + 1] = b; }
  __syncthreads();
  a = 0.0; b = 0.0;
  for (int i = 0; i < nw; ++i) { a += sh[2 * i]; b += sh[2 * i + 1]; }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// orthonormalisation: CTA per (aggregate, chirality), thread per site
// ---------------------------------------------------------------------------
__global__ void k_orthonormalise(Geom g, double* __restrict__ lam, int n) {
  extern __shared__ double osh[];          // [2 * warps] + [2 * n] coefficients
  double* red = osh;
  double* coef = osh + 2 * (blockDim.x >> 5);
  const int X = blockIdx.x, s = blockIdx.y;
  const size_t fstride = (size_t)g.V * SPINOR_NR;
  using LY = Layout<double, SPINOR_NR>;
  for (int i = 0; i < n; ++i) {
    for (int pass = 0; pass < 2; ++pass) {
      // coefficients <lambda_j, lambda_i> for j < i, from the same lambda_i
      for (int j = 0; j < i; ++j) {
        double re = 0.0, im = 0.0;
        for (int q = threadIdx.x; q < g.Vb; q += blockDim.x) {
          size_t b = LY::base(X * g.Vb + q, g.Vb);
          for (int u = 6 * s; u < 6 * s + 6; ++u) {
            double2 a = reinterpret_cast<const double2*>(lam + j * fstride)[b + (size_t)u * g.Vb];
            double2 c = reinterpret_cast<const double2*>(lam + i * fstride)[b + (size_t)u * g.Vb];
            re += a.x * c.x + a.y * c.y;
            im += a.x * c.y - a.y * c.x;
          }
        }
        block_sum2_all(re, im, red);
        if (threadIdx.x == 0) { coef[2 * j] = re; coef[2 * j + 1] = im; }
      }
      __syncthreads();
      for (int q = threadIdx.x; q < g.Vb; q += blockDim.x) {
        size_t b = LY::base(X * g.Vb + q, g.Vb);
        for (int u = 6 * s; u < 6 * s + 6; ++u) {
          double2* pi = reinterpret_cast<double2*>(lam + i * fstride) + b + (size_t)u * g.Vb;
          double2 v = *pi;
          for (int j = 0; j < i; ++j) {
            double2 a = reinterpret_cast<const double2*>(lam + j * fstride)[b + (size_t)u * g.Vb];
            double cr = coef[2 * j], ci = coef[2 * j + 1];
            v.x -= cr * a.x - ci * a.y;
            v.y -= cr * a.y + ci * a.x;
          }
          *pi = v;
        }
      }
      __syncthreads();
    }
    double nn = 0.0, dummy = 0.0;
    for (int q = threadIdx.x; q < g.Vb; q += blockDim.x) {
      size_t b = LY::base(X * g.Vb + q, g.Vb);
      for (int u = 6 * s; u < 6 * s + 6; ++u) {
        double2 v = reinterpret_cast<const double2*>(lam + i * fstride)[b + (size_t)u * g.Vb];
        nn += v.x * v.x + v.y * v.y;
      }
    }
    block_sum2_all(nn, dummy, red);
    double f = 1.0 / sqrt(nn);
    for (int q = threadIdx.x; q < g.Vb; q += blockDim.x) {
      size_t b = LY::base(X * g.Vb + q, g.Vb);
      for (int u = 6 * s; u < 6 * s + 6; ++u) {
        double2* pi = reinterpret_cast<double2*>(lam + i * fstride) + b + (size_t)u * g.Vb;
        double2 v = *pi;
        v.x *= f;
        v.y *= f;
        *pi = v;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// restriction: CTA per (aggregate, rhs)
// ---------------------------------------------------------------------------
template <class R>
__global__ void k_restrict(Geom g, const R* __restrict__ lam, int n, const R* __restrict__ b,
                           cpx<R>* __restrict__ bc) {
  extern __shared__ double rsh[];    // [warps][2n][2]
  const int X = blockIdx.x, rhs = blockIdx.y;
  const int nw = blockDim.x >> 5, w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const size_t fstride = (size_t)g.V * SPINOR_NR;
  const R* bb = b + rhs * fstride;
  for (int i = 0; i < n; ++i) {
    double a[4] = {0.0, 0.0, 0.0, 0.0};   // (re, im) for s = 0, 1
    for (int q = threadIdx.x; q < g.Vb; q += blockDim.x) {
      int d = X * g.Vb + q;
      Spinor<R> L, B;
      load_spinor<R>(lam + i * fstride, d, g.Vb, L);
      load_spinor<R>(bb, d, g.Vb, B);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        int s = k / 6;
        a[2 * s] += (double)L.c[k].re * B.c[k].re + (double)L.c[k].im * B.c[k].im;
        a[2 * s + 1] += (double)L.c[k].re * B.c[k].im - (double)L.c[k].im * B.c[k].re;
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] = warp_sum(a[k]);
    if (l == 0) {
      for (int s = 0; s < 2; ++s) {
        rsh[(w * 2 * n + s * n + i) * 2] = a[2 * s];
        rsh[(w * 2 * n + s * n + i) * 2 + 1] = a[2 * s + 1];
      }
    }
  }
  __syncthreads();
  for (int r = threadIdx.x; r < 2 * n; r += blockDim.x) {
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
template <class R>
__global__ void k_prolong(Geom g, const R* __restrict__ lam, int n, const cpx<R>* __restrict__ xc,
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
  for (int i = 0; i < n; ++i) {
    Spinor<R> L;
    load_spinor<R>(lam + i * fstride, d, g.Vb, L);
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
      if (idx < NE) Dc[((size_t)X * 9 + dd) * NE + idx] = acc[e];
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
    if (c < n2) v = mk((double)A[r * n2 + c].re, (double)A[r * n2 + c].im);
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
    Ainv[(size_t)X * n2 * n2 + idx] = mk((R)v.re, (R)v.im);
  }
}

// ---------------------------------------------------------------------------
// coarse stencil building block: out[r] = sum_{d in [d0,d1)} M_d[r][:] . v_d[:]
// computed by the whole CTA (warp per row), v_d staged in smem
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void cta_matvec(const cpx<R>* __restrict__ M, const cpx<R>* sv, int d0,
                                           int d1, int n2, cpx<R>* out, R scale, bool add) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int r = w; r < n2; r += nw) {
    double re = 0.0, im = 0.0;
    for (int d = d0; d < d1; ++d) {
      const cpx<R>* row = M + ((size_t)d * n2 + r) * n2;
      const cpx<R>* v = sv + d * n2;
      for (int c = l; c < n2; c += 32) {
        cpx<R> a = row[c], b = v[c];
        re += (double)a.re * b.re - (double)a.im * b.im;
        im += (double)a.re * b.im + (double)a.im * b.re;
      }
    }
    re = warp_sum(re);
    im = warp_sum(im);
    if (l == 0) {
      cpx<R> o = mk((R)(scale * re), (R)(scale * im));
      out[r] = add ? out[r] + o : o;
    }
  }
}

template <class R>
__global__ void k_coarse_apply(Geom g, const cpx<R>* __restrict__ Dc, int n2, const cpx<R>* __restrict__ x,
                               cpx<R>* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char csh[];
  cpx<R>* sv = reinterpret_cast<cpx<R>*>(csh);   // [9][n2]
  const int X = blockIdx.x, rhs = blockIdx.y;
  const cpx<R>* xr = x + (size_t)rhs * g.nb * n2;
  for (int idx = threadIdx.x; idx < 9 * n2; idx += blockDim.x) {
    int d = idx / n2, c = idx - d * n2;
    sv[idx] = xr[(size_t)g.cnbr[d * g.nb + X] * n2 + c];
  }
  __syncthreads();
  cta_matvec<R>(Dc + (size_t)X * 9 * n2 * n2, sv, 0, 9, n2, y + ((size_t)rhs * g.nb + X) * n2, R(1), false);
}

template <class RD, class RS>
__global__ void k_conv_c(const RS* __restrict__ s, RD* __restrict__ d, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) d[i] = (RD)s[i];
}

// ---------------------------------------------------------------------------
// even-odd preconditioned GMRES, persistent cooperative kernel
// Work vectors written by one CTA and read by others are loaded with ld.cg
// (L2), never through the non-coherent L1.
// ---------------------------------------------------------------------------
__device__ __forceinline__ cpx<float> ldc(const cpx<float>* p) {
  float2 t = __ldcg(reinterpret_cast<const float2*>(p));
  return mk(t.x, t.y);
}
__device__ __forceinline__ cpx<double> ldc(const cpx<double>* p) {
  double2 t = __ldcg(reinterpret_cast<const double2*>(p));
  return mk(t.x, t.y);
}
constexpr int CG_TPB = 256;
constexpr int CG_MAXM = 64;
constexpr long long BARRIER_SPIN_LIMIT = 1ll << 24;   // ~ seconds with nanosleep

template <class R>
struct CGArgs {
  Geom g;
  const cpx<R>* Dc;
  const cpx<R>* Ainv;
  int n2;
  double tol;
  int m;
  int max_iter;
  const cpx<R>* b;
  cpx<R>* x;
  int nrhs;
  int NE;           // sites per parity
  cpx<R>* V;        // [(m+1)][NE][n2]
  cpx<R>* w;        // [NE][n2]
  cpx<R>* to;       // [NE][n2] (odd sites)
  cpx<R>* xe;       // [NE][n2]
  cpx<R>* rhs_e;    // [NE][n2]
  double* part;     // [G][m+1][2]
  unsigned* bar;    // [2] count, generation
  int* iters;       // [nrhs] iteration counts (nullable)
  int* iters_acc;   // running total over calls (nullable)
  int* status;
};

__device__ bool grid_barrier(unsigned* bar, int* status) {
  __syncthreads();
  __shared__ int ok_s;
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    unsigned my = *gen;
    __threadfence();
    unsigned arrived = atomicAdd(bar, 1u);
    int ok = 1;
    if (arrived == gridDim.x - 1) {
      bar[0] = 0;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*gen == my) {
        if (++spins > BARRIER_SPIN_LIMIT) { atomicExch(status, 6); ok = 0; break; }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*(volatile int*)status != 0) ok = 0;
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// owned range [lo, hi) of parity positions for this CTA
__device__ __forceinline__ void owned(int NE, int& lo, int& hi) {
  int per = (NE + gridDim.x - 1) / gridDim.x;
  lo = blockIdx.x * per;
  hi = min(lo + per, NE);
  if (lo > NE) lo = NE;
}

// odd phase: to[k_o] = Ainv (sum_{d>=1} Dc[O][d] v[nbr]) for owned odd sites
template <class R>
__device__ void phase_odd(const CGArgs<R>& a, const cpx<R>* v, cpx<R>* sv, cpx<R>* tmp) {
  int lo, hi;
  owned(a.NE, lo, hi);
  const int n2 = a.n2;
  for (int k = lo; k < hi; ++k) {
    int X = a.g.codd[k];
    for (int idx = threadIdx.x; idx < 9 * n2; idx += blockDim.x) {
      int d = idx / n2, c = idx - d * n2;
      sv[idx] = d == 0 ? mk(R(0), R(0)) : ldc(v + (size_t)a.g.cpos[a.g.cnbr[d * a.g.nb + X]] * n2 + c);
    }
    __syncthreads();
    cta_matvec<R>(a.Dc + (size_t)X * 9 * n2 * n2, sv, 1, 9, n2, tmp, R(1), false);
    __syncthreads();
    cta_matvec<R>(a.Ainv + (size_t)X * n2 * n2, tmp, 0, 1, n2, a.to + (size_t)k * n2, R(1), false);
    __syncthreads();
  }
}

// even phase: out[k_e] = (sv0 ? A_ee v : 0) - sum_{d>=1} Dc[E][d] to[nbr] + (addb ? bvec : 0)
template <class R>
__device__ void phase_even(const CGArgs<R>& a, const cpx<R>* v, bool use_self, const cpx<R>* bvec,
                           cpx<R>* out, cpx<R>* sv) {
  int lo, hi;
  owned(a.NE, lo, hi);
  const int n2 = a.n2;
  for (int k = lo; k < hi; ++k) {
    int X = a.g.ceven[k];
    for (int idx = threadIdx.x; idx < 9 * n2; idx += blockDim.x) {
      int d = idx / n2, c = idx - d * n2;
      cpx<R> val;
      if (d == 0) val = use_self ? ldc(v + (size_t)k * n2 + c) : mk(R(0), R(0));
      else val = ldc(a.to + (size_t)a.g.cpos[a.g.cnbr[d * a.g.nb + X]] * n2 + c);
      sv[idx] = val;
    }
    __syncthreads();
    const cpx<R>* M = a.Dc + (size_t)X * 9 * n2 * n2;
    cpx<R>* o = out + (size_t)k * n2;
    if (use_self) cta_matvec<R>(M, sv, 0, 1, n2, o, R(1), false);
    else
      for (int r = threadIdx.x; r < n2; r += blockDim.x) o[r] = mk(R(0), R(0));
    __syncthreads();
    cta_matvec<R>(M, sv, 1, 9, n2, o, R(-1), true);
    __syncthreads();
    if (bvec)
      for (int r = threadIdx.x; r < n2; r += blockDim.x) o[r] = ldc(o + r) + bvec[(size_t)X * n2 + r];
    __syncthreads();
  }
}

// CTA partial dots <V_j, w> (j < k) or ||w||^2 over owned even sites -> part
template <class R>
__device__ void partial_dots(const CGArgs<R>& a, int k, const cpx<R>* const* vs, const cpx<R>* w,
                             double* red) {
  int lo, hi;
  owned(a.NE, lo, hi);
  const size_t e0 = (size_t)lo * a.n2, e1 = (size_t)hi * a.n2;
  for (int j = 0; j < k; ++j) {
    double re = 0.0, im = 0.0;
    const cpx<R>* vj = vs[j];
    for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      cpx<R> p = ldc(vj + e), q = ldc(w + e);
      re += (double)p.re * q.re + (double)p.im * q.im;
      im += (double)p.re * q.im - (double)p.im * q.re;
    }
    block_sum2_all(re, im, red);
    if (threadIdx.x == 0) {
      a.part[((size_t)blockIdx.x * (CG_MAXM + 1) + j) * 2] = re;
      a.part[((size_t)blockIdx.x * (CG_MAXM + 1) + j) * 2 + 1] = im;
    }
  }
}

// after a barrier: h[j] = sum over CTAs (fixed order) -> smem
__device__ void gather_dots(int k, double* part, double* h) {
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int c = 0; c < (int)gridDim.x; ++c) {
      re += __ldcg(part + ((size_t)c * (CG_MAXM + 1) + j) * 2);
      im += __ldcg(part + ((size_t)c * (CG_MAXM + 1) + j) * 2 + 1);
    }
    h[2 * j] = re;
    h[2 * j + 1] = im;
  }
  __syncthreads();
}

template <class R>
__global__ void __launch_bounds__(CG_TPB) k_coarse_gmres(CGArgs<R> a) {
  extern __shared__ __align__(16) unsigned char gsh[];
  const int n2 = a.n2, m = a.m;
  cpx<R>* sv = reinterpret_cast<cpx<R>*>(gsh);                 // [9][n2]
  cpx<R>* tmp = sv + 9 * n2;                                   // [n2]
  double* red = reinterpret_cast<double*>(tmp + n2);           // [2 * warps]
  double* h = red + 2 * (CG_TPB / 32);                         // [2 (m+1)]
  double* Rf = h + 2 * (CG_MAXM + 1);                          // [m][m+1] complex (col-major)
  double* cs = Rf + 2 * CG_MAXM * (CG_MAXM + 1);               // [m]
  double* sn = cs + CG_MAXM;                                   // [2 m]
  double* gv = sn + 2 * CG_MAXM;                               // [2 (m+1)]
  double* yv = gv + 2 * (CG_MAXM + 1);                         // [2 m]
  __shared__ int flag_s;
  __shared__ const cpx<R>* vptr[CG_MAXM + 1];

  int lo, hi;
  owned(a.NE, lo, hi);
  const size_t e0 = (size_t)lo * n2, e1 = (size_t)hi * n2;
  const size_t vstride = (size_t)a.NE * n2;
  for (int j = threadIdx.x; j <= m; j += blockDim.x) vptr[j] = a.V + j * vstride;

  for (int rhs = 0; rhs < a.nrhs; ++rhs) {
    const cpx<R>* b = a.b + (size_t)rhs * a.g.nb * n2;
    cpx<R>* x = a.x + (size_t)rhs * a.g.nb * n2;
    // to = A_oo^-1 b_o
    {
      for (int k = lo; k < hi; ++k) {
        int X = a.g.codd[k];
        for (int r = threadIdx.x; r < n2; r += blockDim.x) tmp[r] = b[(size_t)X * n2 + r];
        __syncthreads();
        cta_matvec<R>(a.Ainv + (size_t)X * n2 * n2, tmp, 0, 1, n2, a.to + (size_t)k * n2, R(1), false);
        __syncthreads();
      }
    }
    if (!grid_barrier(a.bar, a.status)) return;
    // rhs_e = b_e - D_eo to
    phase_even<R>(a, nullptr, false, b, a.rhs_e, sv);
    // x_e = 0, V0 = rhs_e (unnormalised for now)
    for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      a.xe[e] = mk(R(0), R(0));
      a.w[e] = ldc(a.rhs_e + e);
    }
    __syncthreads();
    partial_dots<R>(a, 1, &a.w, a.w, red);   // ||rhs_e||^2 (vs = {w})
    if (!grid_barrier(a.bar, a.status)) return;
    gather_dots(1, a.part, h);
    const double bnorm = sqrt(h[0]);
    double beta = bnorm;
    int total = 0;
    bool done = !(bnorm > 0.0) || beta <= a.tol * bnorm;
    while (!done) {
      if (total >= a.max_iter) break;
      // V0 = w / beta  (w holds the current residual)
      {
        double f = 1.0 / beta;
        for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
          cpx<R> v = ldc(a.w + e);
          a.V[e] = mk((R)(v.re * f), (R)(v.im * f));
        }
      }
      if (threadIdx.x == 0) {
        gv[0] = beta; gv[1] = 0.0;
      }
      if (!grid_barrier(a.bar, a.status)) return;
      int kdone = 0;
      for (int k = 0; k < m; ++k) {
        const cpx<R>* vk = a.V + k * vstride;
        // w = S V_k
        phase_odd<R>(a, vk, sv, tmp);
        if (!grid_barrier(a.bar, a.status)) return;
        phase_even<R>(a, vk, true, nullptr, a.w, sv);
        // classical Gram-Schmidt, two passes
        for (int pass = 0; pass < 2; ++pass) {
          partial_dots<R>(a, k + 1, vptr, a.w, red);
          if (!grid_barrier(a.bar, a.status)) return;
          double* hh = pass == 0 ? h : yv;    // reuse yv as second-pass buffer
          gather_dots(k + 1, a.part, hh);
          for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            cpx<R> w0 = ldc(a.w + e);
            double re = w0.re, im = w0.im;
            for (int j = 0; j <= k; ++j) {
              cpx<R> v = ldc(vptr[j] + e);
              double cr = hh[2 * j], ci = hh[2 * j + 1];
              re -= cr * v.re - ci * v.im;
              im -= cr * v.im + ci * v.re;
            }
            a.w[e] = mk((R)re, (R)im);
          }
          if (pass == 1 && threadIdx.x == 0)
            for (int j = 0; j <= k; ++j) { h[2 * j] += yv[2 * j]; h[2 * j + 1] += yv[2 * j + 1]; }
          __syncthreads();
          if (!grid_barrier(a.bar, a.status)) return;
        }
        partial_dots<R>(a, 1, &a.w, a.w, red);
        if (!grid_barrier(a.bar, a.status)) return;
        gather_dots(1, a.part, yv);
        const double hn = sqrt(yv[0]);
        // V_{k+1} = w / hn
        {
          double f = hn > 0.0 ? 1.0 / hn : 0.0;
          cpx<R>* vn = a.V + (k + 1) * vstride;
          for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            cpx<R> v = ldc(a.w + e);
            vn[e] = mk((R)(v.re * f), (R)(v.im * f));
          }
        }
        // Givens (identical in every CTA)
        if (threadIdx.x == 0) {
          double col[2 * (CG_MAXM + 1)];
          for (int j = 0; j <= k; ++j) { col[2 * j] = h[2 * j]; col[2 * j + 1] = h[2 * j + 1]; }
          col[2 * (k + 1)] = hn; col[2 * (k + 1) + 1] = 0.0;
          for (int j = 0; j < k; ++j) {
            double c = cs[j], sr = sn[2 * j], si = sn[2 * j + 1];
            double ar = col[2 * j], ai = col[2 * j + 1], br = col[2 * j + 2], bi = col[2 * j + 3];
            // t = c a + s b ; b' = -conj(s) a + c b
            double tr = c * ar + (sr * br - si * bi), ti = c * ai + (sr * bi + si * br);
            double ur = -(sr * ar + si * ai) + c * br, ui = -(sr * ai - si * ar) + c * bi;
            col[2 * j] = tr; col[2 * j + 1] = ti; col[2 * j + 2] = ur; col[2 * j + 3] = ui;
          }
          double ar = col[2 * k], ai = col[2 * k + 1], br = col[2 * k + 2], bi = col[2 * k + 3];
          double a1 = sqrt(ar * ar + ai * ai), a2 = sqrt(br * br + bi * bi);
          double c, sr, si, rr, ri;
          if (a2 == 0.0) { c = 1.0; sr = 0.0; si = 0.0; rr = ar; ri = ai; }
          else if (a1 == 0.0) { c = 0.0; sr = br / a2; si = -bi / a2; rr = a2; ri = 0.0; }
          else {
            double rho = hypot(a1, a2);
            double pr = ar / a1, pi = ai / a1;
            c = a1 / rho;
            sr = (pr * br + pi * bi) / rho;      // ph * conj(b) / rho
            si = (pi * br - pr * bi) / rho;
            rr = pr * rho; ri = pi * rho;
          }
          cs[k] = c; sn[2 * k] = sr; sn[2 * k + 1] = si;
          col[2 * k] = rr; col[2 * k + 1] = ri;
          for (int j = 0; j <= k; ++j) {
            Rf[2 * (k * (CG_MAXM + 1) + j)] = col[2 * j];
            Rf[2 * (k * (CG_MAXM + 1) + j) + 1] = col[2 * j + 1];
          }
          double gr = gv[2 * k], gi = gv[2 * k + 1];
          gv[2 * (k + 1)] = -(sr * gr + si * gi);      // -conj(s) g
          gv[2 * (k + 1) + 1] = -(sr * gi - si * gr);
          gv[2 * k] = c * gr;
          gv[2 * k + 1] = c * gi;
          double res = sqrt(gv[2 * (k + 1)] * gv[2 * (k + 1)] + gv[2 * (k + 1) + 1] * gv[2 * (k + 1) + 1]);
          flag_s = (res <= a.tol * bnorm || hn == 0.0) ? 1 : 0;
        }
        __syncthreads();
        ++total;
        kdone = k + 1;
        if (flag_s || total >= a.max_iter) break;
        if (!grid_barrier(a.bar, a.status)) return;
      }
      // y = R^-1 g ; x_e += sum y_j V_j
      if (threadIdx.x == 0) {
        for (int i = kdone - 1; i >= 0; --i) {
          double accr = gv[2 * i], acci = gv[2 * i + 1];
          for (int j = i + 1; j < kdone; ++j) {
            double rr = Rf[2 * (j * (CG_MAXM + 1) + i)], ri = Rf[2 * (j * (CG_MAXM + 1) + i) + 1];
            accr -= rr * yv[2 * j] - ri * yv[2 * j + 1];
            acci -= rr * yv[2 * j + 1] + ri * yv[2 * j];
          }
          double dr = Rf[2 * (i * (CG_MAXM + 1) + i)], di = Rf[2 * (i * (CG_MAXM + 1) + i) + 1];
          double dn = dr * dr + di * di;
          yv[2 * i] = (accr * dr + acci * di) / dn;
          yv[2 * i + 1] = (acci * dr - accr * di) / dn;
        }
      }
      __syncthreads();
      for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        cpx<R> x0 = ldc(a.xe + e);
        double re = x0.re, im = x0.im;
        for (int j = 0; j < kdone; ++j) {
          cpx<R> v = ldc(vptr[j] + e);
          re += yv[2 * j] * v.re - yv[2 * j + 1] * v.im;
          im += yv[2 * j] * v.im + yv[2 * j + 1] * v.re;
        }
        a.xe[e] = mk((R)re, (R)im);
      }
      if (!grid_barrier(a.bar, a.status)) return;
      // true residual w = rhs_e - S x_e
      phase_odd<R>(a, a.xe, sv, tmp);
      if (!grid_barrier(a.bar, a.status)) return;
      phase_even<R>(a, a.xe, true, nullptr, a.w, sv);
      for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) a.w[e] = ldc(a.rhs_e + e) - ldc(a.w + e);
      __syncthreads();
      partial_dots<R>(a, 1, &a.w, a.w, red);
      if (!grid_barrier(a.bar, a.status)) return;
      gather_dots(1, a.part, yv);
      beta = sqrt(yv[0]);
      done = beta <= a.tol * bnorm;
      if (!grid_barrier(a.bar, a.status)) return;
    }
    // x_o = A_oo^-1 (b_o - D_oe x_e); x_e out
    {
      int X;
      for (int k = lo; k < hi; ++k) {
        X = a.g.codd[k];
        for (int idx = threadIdx.x; idx < 9 * n2; idx += blockDim.x) {
          int d = idx / n2, c = idx - d * n2;
          sv[idx] = d == 0 ? mk(R(0), R(0)) : ldc(a.xe + (size_t)a.g.cpos[a.g.cnbr[d * a.g.nb + X]] * n2 + c);
        }
        __syncthreads();
        cta_matvec<R>(a.Dc + (size_t)X * 9 * n2 * n2, sv, 1, 9, n2, tmp, R(-1), false);
        __syncthreads();
        for (int r = threadIdx.x; r < n2; r += blockDim.x) tmp[r] = tmp[r] + b[(size_t)X * n2 + r];
        __syncthreads();
        cta_matvec<R>(a.Ainv + (size_t)X * n2 * n2, tmp, 0, 1, n2, x + (size_t)X * n2, R(1), false);
        __syncthreads();
      }
      for (int k = lo; k < hi; ++k) {
        X = a.g.ceven[k];
        for (int r = threadIdx.x; r < n2; r += blockDim.x) x[(size_t)X * n2 + r] = ldc(a.xe + (size_t)k * n2 + r);
      }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      if (a.iters) a.iters[rhs] = total;
      if (a.iters_acc) atomicAdd(a.iters_acc, total);
    }
    if (!grid_barrier(a.bar, a.status)) return;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t orthonormalise(const Geom& g, double* lam, int n, cudaStream_t st) {
  int threads = g.Vb >= 256 ? 256 : ((g.Vb + 31) / 32) * 32;
  size_t smem = (2 * (threads / 32) + 2 * n) * sizeof(double);
  k_orthonormalise<<<dim3(g.nb, 2), threads, smem, st>>>(g, lam, n);
  ++g_launches;
  return cudaGetLastError();
}

template <class R>
cudaError_t restrict_op(const Geom& g, const R* lam, int n, const R* b, R* bc, int nrhs, cudaStream_t st) {
  int threads = g.Vb >= 256 ? 256 : ((g.Vb + 31) / 32) * 32;
  size_t smem = (size_t)(threads / 32) * 2 * n * 2 * sizeof(double);
  k_restrict<R><<<dim3(g.nb, nrhs), threads, smem, st>>>(g, lam, n, b, reinterpret_cast<cpx<R>*>(bc));
  ++g_launches;
  return cudaGetLastError();
}

template <class R>
cudaError_t prolong_op(const Geom& g, const R* lam, int n, const R* xc, R* x, int nrhs, bool accumulate,
                       cudaStream_t st) {
  k_prolong<R><<<dim3(nblk(g.V, 128), nrhs), 128, 0, st>>>(
      g, lam, n, reinterpret_cast<const cpx<R>*>(xc), x, accumulate ? 1 : 0);
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
  cudaError_t e = cudaFuncSetAttribute(k_assemble<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_assemble<R><<<g.nb, threads, smem, st>>>(g, lam, n, gauge, clover, reinterpret_cast<cpx<R>*>(Dc), ch);
  ++g_launches;
  return cudaGetLastError();
}

template <class R>
cudaError_t invert_self_blocks(const Geom& g, const R* Dc, int n, R* Ainv, int* singular, cudaStream_t st) {
  int n2 = 2 * n;
  size_t smem = (size_t)n2 * 2 * n2 * sizeof(cpx<double>);
  cudaError_t e = cudaFuncSetAttribute(k_invert_self<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_invert_self<R><<<g.nb, 256, smem, st>>>(g, reinterpret_cast<const cpx<R>*>(Dc), n2,
                                            reinterpret_cast<cpx<R>*>(Ainv), singular);
  ++g_launches;
  return cudaGetLastError();
}

template <class R>
cudaError_t coarse_apply(const Geom& g, const R* Dc, int n, const R* x, R* y, int nrhs, cudaStream_t st) {
  int n2 = 2 * n;
  size_t smem = (size_t)9 * n2 * sizeof(cpx<R>);
  k_coarse_apply<R><<<dim3(g.nb, nrhs), 128, smem, st>>>(g, reinterpret_cast<const cpx<R>*>(Dc), n2,
                                                         reinterpret_cast<const cpx<R>*>(x),
                                                         reinterpret_cast<cpx<R>*>(y));
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

static size_t cg_smem_bytes(int n2, int real_size) {
  size_t s = (size_t)10 * n2 * 2 * real_size;                    // sv + tmp
  s = (s + 15) / 16 * 16;
  s += sizeof(double) * (2 * (CG_TPB / 32) + 2 * (CG_MAXM + 1) + 2 * CG_MAXM * (CG_MAXM + 1) +
                         CG_MAXM + 2 * CG_MAXM + 2 * (CG_MAXM + 1) + 2 * CG_MAXM);
  return s;
}

static int cg_grid(const Geom& g, int n2, int real_size, const void* fn) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, CG_TPB, cg_smem_bytes(n2, real_size));
  int maxg = sms * (per > 0 ? per : 1);
  int NE = g.nb / 2;
  return NE < maxg ? NE : maxg;
}

size_t coarse_gmres_work_bytes(const Geom& g, int n, int restart, int real_size) {
  size_t NE = g.nb / 2, n2 = 2 * n;
  size_t cplx = (size_t)2 * real_size;
  size_t vec = NE * n2 * cplx;
  size_t bytes = (restart + 1) * vec + 4 * vec;   // V, w, to, xe, rhs_e
  bytes = (bytes + 255) / 256 * 256;
  bytes += (size_t)NE * (CG_MAXM + 1) * 2 * sizeof(double);   // partials (grid <= NE)
  bytes += 256;                                                  // barrier
  return bytes;
}

template <class R>
cudaError_t coarse_gmres(const Geom& g, const CoarseSolveArgs& ca, const R* b, R* x, int nrhs, void* work,
                         int* iters, int* iters_acc, int* status, cudaStream_t st) {
  if (ca.restart > CG_MAXM || ca.restart < 1) return cudaErrorInvalidValue;
  CGArgs<R> a;
  a.g = g;
  a.Dc = reinterpret_cast<const cpx<R>*>(ca.Dc);
  a.Ainv = reinterpret_cast<const cpx<R>*>(ca.Ainv);
  a.n2 = 2 * ca.n;
  a.tol = ca.tol;
  a.m = ca.restart;
  a.max_iter = ca.max_iter;
  a.b = reinterpret_cast<const cpx<R>*>(b);
  a.x = reinterpret_cast<cpx<R>*>(x);
  a.nrhs = nrhs;
  a.NE = g.nb / 2;
  size_t vec = (size_t)a.NE * a.n2;
  cpx<R>* base = reinterpret_cast<cpx<R>*>(work);
  a.V = base;
  a.w = a.V + (ca.restart + 1) * vec;
  a.to = a.w + vec;
  a.xe = a.to + vec;
  a.rhs_e = a.xe + vec;
  size_t off = ((size_t)(ca.restart + 5) * vec * sizeof(cpx<R>) + 255) / 256 * 256;
  a.part = reinterpret_cast<double*>(reinterpret_cast<char*>(work) + off);
  off += (size_t)a.NE * (CG_MAXM + 1) * 2 * sizeof(double);
  a.bar = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(work) + off);
  a.iters = iters;
  a.iters_acc = iters_acc;
  a.status = status;
  cudaError_t e = cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  size_t smem = cg_smem_bytes(a.n2, sizeof(R));
  e = cudaFuncSetAttribute(k_coarse_gmres<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int grid = cg_grid(g, a.n2, sizeof(R), (const void*)k_coarse_gmres<R>);
  void* args[] = {&a};
  e = cudaLaunchCooperativeKernel((const void*)k_coarse_gmres<R>, dim3(grid), dim3(CG_TPB), args, smem, st);
  ++g_launches;
  return e;
}

// instantiations
#define INST(R)                                                                                          \
  template cudaError_t restrict_op<R>(const Geom&, const R*, int, const R*, R*, int, cudaStream_t);     \
  template cudaError_t prolong_op<R>(const Geom&, const R*, int, const R*, R*, int, bool, cudaStream_t); \
  template cudaError_t assemble_coarse<R>(const Geom&, const R*, int, const R*, const R*, R*,           \
                                          cudaStream_t);                                                \
  template cudaError_t invert_self_blocks<R>(const Geom&, const R*, int, R*, int*, cudaStream_t);       \
  template cudaError_t coarse_apply<R>(const Geom&, const R*, int, const R*, R*, int, cudaStream_t);    \
  template cudaError_t coarse_from_f64<R>(const double*, R*, size_t, cudaStream_t);                     \
  template cudaError_t coarse_to_f64<R>(const R*, double*, size_t, cudaStream_t);                       \
  template cudaError_t coarse_gmres<R>(const Geom&, const CoarseSolveArgs&, const R*, R*, int, void*,   \
                                       int*, int*, int*, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace ddamg
