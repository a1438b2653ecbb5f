// Schwarz alternating procedure (SAP) smoother, paper Sec. 2: a
// multiplicative Schwarz sweep over the blocks of one colour, the block
// system solved approximately by site even-odd preconditioned minimal
// residual with a fixed number of iterations.  Loops over blocks are the
// parallel dimension (Sec. 4); here one CTA owns one block and one
// right-hand side, with the block's links staged in shared memory.
//
// Per CTA (block B of colour c):
//   r   = b - D x on the block's sites (full operator, neighbours from global
//         memory; r = b when x is known to be zero)
//   rhs = r_e - D_eo A_oo^-1 r_o                      (D_B restricted to B)
//   MR on S = A_ee - D_eo A_oo^-1 D_oe from e_e = 0:
//         p = S res; alpha = <p,res>/<p,p>; e_e += alpha res; res -= alpha p
//   e_o = A_oo^-1 (r_o - D_oe e_e)
//   x  += e
// with D_eo, D_oe the hops that stay inside the block (-1/2 (1 -+ g) U).
#include <mutex>
#include <type_traits>

#include "common.cuh"
#include "half.cuh"
#include "kernels.h"

namespace ddamg {

namespace {

// Four threads per site: thread sub = 0..3 of a site applies the two hops
// of direction mu = sub and owns the three colour components of spin sub of
// every site vector (res, e, p, ...).  Hop partial sums of the four threads
// are combined by a reduce-scatter of warp shuffles.

constexpr int LPAD = 2;   // padding of the staged link rows (bank groups)

template <class R>
using T16 = typename U16<R>::T;

// link mu of local site q from the staged block links (rows of Vb + LPAD units)
template <class R>
__device__ __forceinline__ void smem_link(const T16<R>* sl, int Vbp, int q, int mu, Link<R>& U) {
  using LY = Layout<R, GAUGE_NR>;
  constexpr int NUL = LINK_NR / LY::PER;
  R v[LINK_NR];
#pragma unroll
  for (int u = 0; u < NUL; ++u) {
    T16<R> t = sl[(mu * NUL + u) * Vbp + q];
    if constexpr (LY::PER == 4) {
      v[4 * u] = t.x; v[4 * u + 1] = t.y; v[4 * u + 2] = t.z; v[4 * u + 3] = t.w;
    } else {
      v[2 * u] = t.x; v[2 * u + 1] = t.y;
    }
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) U.m[k / 3][k % 3] = mk(v[2 * k], v[2 * k + 1]);
  complete_link(U);
}

template <class R>
__device__ __forceinline__ void smem_spinor(const cpx<R>* buf, int Vh, int h, Spinor<R>& s) {
#pragma unroll
  for (int k = 0; k < 12; ++k) s.c[k] = buf[k * Vh + h];
}

// one complex component k of site d in a global spinor field
template <class R>
__device__ __forceinline__ size_t comp_off(int d, int Vb, int k) {
  using LY = Layout<R, SPINOR_NR>;
  constexpr int CPU = LY::PER / 2;   // complex numbers per 16-byte unit
  int B = d / Vb, q = d - B * Vb;
  return (((size_t)B * LY::NU + k / CPU) * Vb + q) * LY::PER + (k % CPU) * 2;
}
__device__ __forceinline__ cpx<float> ld_comp(const float* f, size_t off) {
  float2 t = __ldcg(reinterpret_cast<const float2*>(f + off));
  return mk(t.x, t.y);
}
__device__ __forceinline__ cpx<double> ld_comp(const double* f, size_t off) {
  double2 t = __ldcg(reinterpret_cast<const double2*>(f + off));
  return mk(t.x, t.y);
}
__device__ __forceinline__ void st_comp(float* f, size_t off, cpx<float> v) {
  *reinterpret_cast<float2*>(f + off) = make_float2(v.re, v.im);
}
__device__ __forceinline__ void st_comp(double* f, size_t off, cpx<double> v) {
  *reinterpret_cast<double2*>(f + off) = make_double2(v.re, v.im);
}

template <class R>
__device__ __forceinline__ cpx<R> shfl_x(cpx<R> v, int m) {
  return mk(__shfl_xor_sync(0xffffffffu, v.re, m), __shfl_xor_sync(0xffffffffu, v.im, m));
}

// reduce-scatter of a 12-component partial sum over the 4 threads of a site:
// thread sub receives the full sum of components 3 sub .. 3 sub + 2
template <class R>
__device__ __forceinline__ void reduce_scatter(const Spinor<R>& acc, int sub, cpx<R> out[3]) {
  const bool hi = sub >= 2;      // chirality block of this thread
  cpx<R> keep[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    cpx<R> send = hi ? acc.c[i] : acc.c[6 + i];
    keep[i] = (hi ? acc.c[6 + i] : acc.c[i]) + shfl_x(send, 2);
  }
  const bool odd = sub & 1;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    cpx<R> send = odd ? keep[i] : keep[3 + i];
    out[i] = (odd ? keep[3 + i] : keep[i]) + shfl_x(send, 1);
  }
}

// the 6 components of this thread's chirality block: own 3 + partner's 3
template <class R>
__device__ __forceinline__ void chiral6(const cpx<R> own[3], int sub, cpx<R> v6[6]) {
  const bool odd = sub & 1;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    cpx<R> other = shfl_x(own[i], 1);
    v6[i] = odd ? other : own[i];
    v6[3 + i] = odd ? own[i] : other;
  }
}

// own 3 rows of the packed Hermitian block (chirality sub / 2) times v6
template <class R>
__device__ __forceinline__ void clover_rows(const R* __restrict__ clov, int d, int Vb, int sub,
                                            const cpx<R> v6[6], cpx<R> y[3]) {
  using LY = Layout<R, CLOVER_NR>;
  constexpr int NUB = 36 / LY::PER;
  R P[36];
  load_units<R, CLOVER_NR>(clov, d, Vb, (sub >> 1) * NUB, NUB, P);
  cpx<R> y6[6];
  herm6<R>(P, v6, y6);
  const bool odd = sub & 1;
#pragma unroll
  for (int i = 0; i < 3; ++i) y[i] = odd ? y6[3 + i] : y6[i];
}

// Runtime direction: with g_mu = [[0, B], [B^H, 0]] every B_mu has one
// non-zero per row, B[r][pi(r)] = c_r with pi the identity (z, t) or the
// swap (x, y) and c_r in {+-1, +-i}.  Writing the projector this way keeps
// the four threads of a site (four directions) in one instruction stream.
// A factor c in {+-1, +-i} is held as (rot, a): c = a when rot is false and
// c = -i a when it is true, so c t = rot ? (a t.im, -a t.re) : (a t.re, a t.im)
// costs two selects and no multiplications.
template <class R>
struct Dir {
  bool swp;          // pi swaps the spin pairs
  bool rot0, rot1;   // c_0, c_1 imaginary
  R a0, a1;
};
template <class R>
__device__ __forceinline__ Dir<R> make_dir(int mu) {
  Dir<R> d;
  d.swp = mu < 2;
  d.rot0 = d.rot1 = (mu == 0 || mu == 2);
  d.a0 = (mu == 1) ? R(-1) : R(1);      // c_0: -i, -1, -i, 1
  d.a1 = (mu == 2) ? R(-1) : R(1);      // c_1: -i,  1,  i, 1
  return d;
}
// acc += s c t for c = (rot, a) and a real scale s (sa = s a)
template <class R>
__device__ __forceinline__ void add_ct(cpx<R>& acc, bool rot, R sa, cpx<R> t) {
  const R u = rot ? t.im : t.re, v = rot ? t.re : t.im;
  const R sb = rot ? -sa : sa;
  acc.re += sa * u;
  acc.im += sb * v;
}
// h_r = s_r + sigma c_r s_{2 + pi(r)}
template <class R>
__device__ __forceinline__ void project_rt(const Spinor<R>& p, const Dir<R>& dr, R sigma, cpx<R> h[2][3]) {
  const R s0 = sigma * dr.a0, s1 = sigma * dr.a1;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cpx<R> s2 = p.c[6 + a], s3 = p.c[9 + a];
    cpx<R> t0 = dr.swp ? s3 : s2, t1 = dr.swp ? s2 : s3;
    h[0][a] = p.c[a];
    h[1][a] = p.c[3 + a];
    add_ct(h[0][a], dr.rot0, s0, t0);
    add_ct(h[1][a], dr.rot1, s1, t1);
  }
}
// acc += sc [y; sigma B^H y],  (B^H y)_r = conj(c_pi(r)) y_pi(r); the
// conjugate of (rot, a) is (rot, -a) when rot is true
template <class R>
__device__ __forceinline__ void accumulate_rt(Spinor<R>& acc, const cpx<R> y[2][3], const Dir<R>& dr,
                                              R sigma, R sc) {
  const bool r2 = dr.swp ? dr.rot1 : dr.rot0, r3 = dr.swp ? dr.rot0 : dr.rot1;
  R a2 = dr.swp ? dr.a1 : dr.a0, a3 = dr.swp ? dr.a0 : dr.a1;
  if (r2) a2 = -a2;
  if (r3) a3 = -a3;
  const R s2 = sigma * sc * a2, s3 = sigma * sc * a3;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const cpx<R> y0 = y[0][a], y1 = y[1][a];
    acc.c[a].re += sc * y0.re;
    acc.c[a].im += sc * y0.im;
    acc.c[3 + a].re += sc * y1.re;
    acc.c[3 + a].im += sc * y1.im;
    add_ct(acc.c[6 + a], r2, s2, dr.swp ? y1 : y0);
    add_ct(acc.c[9 + a], r3, s3, dr.swp ? y0 : y1);
  }
}

// own 3 components of the sum of the block-internal hops at local site q;
// this thread applies the two hops of direction mu = sub
template <class R>
__device__ __forceinline__ void hop_block(const int16_t* __restrict__ bnbr, const T16<R>* sl,
                                          const cpx<R>* buf, int Vb, int Vbp, int Vh, int q, int sub,
                                          cpx<R> out[3]) {
  Spinor<R> acc;
#pragma unroll
  for (int k = 0; k < 12; ++k) acc.c[k] = mk(R(0), R(0));
  const Dir<R> dr = make_dir<R>(sub);
  cpx<R> hh[2][3], y[2][3];
  Spinor<R> nb;
  int qf = __ldg(bnbr + (2 * sub) * Vb + q);
  if (qf >= 0) {   // (1 - g_mu) U_mu(x) x(x + mu)
    smem_spinor<R>(buf, Vh, qf >= Vh ? qf - Vh : qf, nb);
    project_rt<R>(nb, dr, R(-1), hh);
    Link<R> U;
    smem_link<R>(sl, Vbp, q, sub, U);
    su3_mul(U, hh, y);
    accumulate_rt<R>(acc, y, dr, R(-1), R(1));
  }
  int qb = __ldg(bnbr + (2 * sub + 1) * Vb + q);
  if (qb >= 0) {   // (1 + g_mu) U_mu(x - mu)^H x(x - mu)
    smem_spinor<R>(buf, Vh, qb >= Vh ? qb - Vh : qb, nb);
    project_rt<R>(nb, dr, R(1), hh);
    Link<R> U;
    smem_link<R>(sl, Vbp, qb, sub, U);
    su3_mul_dag(U, hh, y);
    accumulate_rt<R>(acc, y, dr, R(1), R(1));
  }
  reduce_scatter<R>(acc, sub, out);
}

// own 3 components of the full (global) hopping sum at device site d
template <class R>
__device__ __forceinline__ void hop_global(const Geom& g, const R* x, const R* gauge, int d, int sub,
                                           cpx<R> out[3]) {
  Spinor<R> acc;
#pragma unroll
  for (int k = 0; k < 12; ++k) acc.c[k] = mk(R(0), R(0));
  const Dir<R> dr = make_dir<R>(sub);
  cpx<R> hh[2][3], y[2][3];
  Spinor<R> nb;
  {
    uint32_t e = __ldg(g.nbr + (size_t)(2 * sub) * g.V + d);
    int n = (int)(e & ~NEG_BIT);
    load_spinor_cg<R>(x, n, g.Vb, nb);
    project_rt<R>(nb, dr, R(-1), hh);
    Link<R> U;
    load_link<R>(gauge, d, g.Vb, sub, U);
    su3_mul(U, hh, y);
    accumulate_rt<R>(acc, y, dr, R(-1), (e & NEG_BIT) ? R(-1) : R(1));
  }
  {
    uint32_t e = __ldg(g.nbr + (size_t)(2 * sub + 1) * g.V + d);
    int n = (int)(e & ~NEG_BIT);
    load_spinor_cg<R>(x, n, g.Vb, nb);
    project_rt<R>(nb, dr, R(1), hh);
    Link<R> U;
    load_link<R>(gauge, n, g.Vb, sub, U);
    su3_mul_dag(U, hh, y);
    accumulate_rt<R>(acc, y, dr, R(1), (e & NEG_BIT) ? R(-1) : R(1));
  }
  reduce_scatter<R>(acc, sub, out);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <class R>
__device__ __forceinline__ R warp_sum_r(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block sum of three per-thread partials in the working precision (warp
// trees, then one warp over the per-warp sums), broadcast to every thread
template <class R>
__device__ __forceinline__ void block_sum3(R ra, R rb, R rc, R& a, R& b, R& c, R* sh) {
  ra = warp_sum_r<R>(ra);
  rb = warp_sum_r<R>(rb);
  rc = warp_sum_r<R>(rc);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  if (l == 0) { sh[3 * w] = ra; sh[3 * w + 1] = rb; sh[3 * w + 2] = rc; }
  __syncthreads();
  if (w == 0) {
    R x = l < nw ? sh[3 * l] : R(0), y = l < nw ? sh[3 * l + 1] : R(0), z = l < nw ? sh[3 * l + 2] : R(0);
    x = warp_sum_r<R>(x);
    y = warp_sum_r<R>(y);
    z = warp_sum_r<R>(z);
    if (l == 0) { sh[96] = x; sh[97] = y; sh[98] = z; }
  }
  __syncthreads();
  a = sh[96];
  b = sh[97];
  c = sh[98];
}

// block index of the k-th block of colour c (block-grid extent 0 even)
__device__ __forceinline__ int block_of_colour(const Geom& g, int c, int k) {
  int t = 2 * k;
  int b0 = t % g.grid[0];
  int r = t / g.grid[0];
  int b1 = r % g.grid[1];
  r /= g.grid[1];
  int b2 = r % g.grid[2];
  int b3 = r / g.grid[2];
  b0 += (c + b1 + b2 + b3) & 1;
  return b0 + g.grid[0] * (b1 + g.grid[1] * (b2 + g.grid[2] * b3));
}

template <class R>
__global__ void __launch_bounds__(512) k_sap_sweep(Geom g, int colour, int mr_iters, int x_is_zero,
                                                   const R* __restrict__ b, R* __restrict__ x,
                                                   const R* __restrict__ gauge, const R* __restrict__ clov,
                                                   const R* __restrict__ clov_inv) {
  using LYG = Layout<R, GAUGE_NR>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Vb = g.Vb, Vh = Vb / 2, Vbp = Vb + LPAD;
  T16<R>* sl = reinterpret_cast<T16<R>*>(smem_raw);                      // [NU][Vb + LPAD]
  cpx<R>* E = reinterpret_cast<cpx<R>*>(sl + (size_t)LYG::NU * Vbp);      // [12][Vh]
  cpx<R>* O = E + 12 * Vh;                                                // [12][Vh]
  R* red = reinterpret_cast<R*>(O + 12 * Vh);                             // [3 * warps + 3]

  const int B = block_of_colour(g, colour, blockIdx.x);
  const size_t off = (size_t)blockIdx.y * g.V * SPINOR_NR;
  b += off;
  x += off;
  const int h = threadIdx.x >> 2, sub = threadIdx.x & 3;
  const bool act = h < Vh;
  const int hs = act ? h : 0;                 // inactive lanes shadow site 0 (no stores)
  const int de = B * Vb + hs, dO = B * Vb + Vh + hs;

  // stage the block's links (contiguous in the block-major layout)
  {
    const T16<R>* src = reinterpret_cast<const T16<R>*>(gauge) + (size_t)B * LYG::NU * Vb;
    for (int i = threadIdx.x; i < LYG::NU * Vb; i += blockDim.x) {
      int u = i / Vb, q = i - u * Vb;
      sl[u * Vbp + q] = __ldg(src + i);
    }
  }

  // residual r = b - D x on the own components of both sites
  cpx<R> re[3], ro[3];
  {
#pragma unroll
    for (int par = 0; par < 2; ++par) {
      const int d = par ? dO : de;
      cpx<R> r[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) r[i] = ld_comp(b, comp_off<R>(d, Vb, 3 * sub + i));
      if (!x_is_zero) {
        cpx<R> hop[3], x6[6], ax[3];
        hop_global<R>(g, x, gauge, d, sub, hop);
        const int c0 = 6 * (sub >> 1);
#pragma unroll
        for (int i = 0; i < 6; ++i) x6[i] = ld_comp(x, comp_off<R>(d, Vb, c0 + i));
        clover_rows<R>(clov, d, Vb, sub, x6, ax);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          r[i].re -= ax[i].re - R(0.5) * hop[i].re;
          r[i].im -= ax[i].im - R(0.5) * hop[i].im;
        }
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        if (par) ro[i] = r[i];
        else re[i] = r[i];
      }
    }
    // u_o = A_oo^-1 r_o
    cpx<R> v6[6], u[3];
    chiral6<R>(ro, sub, v6);
    clover_rows<R>(clov_inv, dO, Vb, sub, v6, u);
    if (act)
#pragma unroll
      for (int i = 0; i < 3; ++i) O[(3 * sub + i) * Vh + h] = u[i];
  }
  __syncthreads();

  // rhs_e = r_e - D_eo u_o = r_e + 1/2 hop(u_o)
  cpx<R> res[3], xe[3];
  {
    cpx<R> t[3];
    hop_block<R>(g.bnbr, sl, O, Vb, Vbp, Vh, hs, sub, t);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      res[i].re = fma_r(R(0.5), t[i].re, re[i].re);
      res[i].im = fma_r(R(0.5), t[i].im, re[i].im);
      xe[i] = mk(R(0), R(0));
    }
  }

  for (int it = 0; it < mr_iters; ++it) {
    __syncthreads();       // readers of E / O from the previous step are done
    if (act)
#pragma unroll
      for (int i = 0; i < 3; ++i) E[(3 * sub + i) * Vh + h] = res[i];
    __syncthreads();
    {  // odd: w = A_oo^-1 D_oe res = A_oo^-1 (-1/2 hop(res))
      cpx<R> t[3], v6[6], w[3];
      hop_block<R>(g.bnbr, sl, E, Vb, Vbp, Vh, Vh + hs, sub, t);
#pragma unroll
      for (int i = 0; i < 3; ++i) t[i] = R(-0.5) * t[i];
      chiral6<R>(t, sub, v6);
      clover_rows<R>(clov_inv, dO, Vb, sub, v6, w);
      if (act)
#pragma unroll
        for (int i = 0; i < 3; ++i) O[(3 * sub + i) * Vh + h] = w[i];
    }
    __syncthreads();
    R pr_re = 0, pr_im = 0, pp_r = 0;
    cpx<R> p[3];
    {  // even: p = A_ee res - D_eo w = A_ee res + 1/2 hop(w)
      cpx<R> t[3], v6[6];
      chiral6<R>(res, sub, v6);
      clover_rows<R>(clov, de, Vb, sub, v6, p);
      hop_block<R>(g.bnbr, sl, O, Vb, Vbp, Vh, hs, sub, t);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        p[i].re = fma_r(R(0.5), t[i].re, p[i].re);
        p[i].im = fma_r(R(0.5), t[i].im, p[i].im);
        if (act) {
          pr_re += p[i].re * res[i].re + p[i].im * res[i].im;
          pr_im += p[i].re * res[i].im - p[i].im * res[i].re;
          pp_r += p[i].re * p[i].re + p[i].im * p[i].im;
        }
      }
    }
    R dpr_re, dpr_im, pp;
    block_sum3<R>(pr_re, pr_im, pp_r, dpr_re, dpr_im, pp, red);
    if (pp > R(0)) {
      cpx<R> a = mk(dpr_re / pp, dpr_im / pp);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        fma(xe[i], a, res[i]);
        res[i] = res[i] - a * p[i];
      }
    }
  }

  // e_o = A_oo^-1 (r_o - D_oe e_e) = A_oo^-1 (r_o + 1/2 hop(e_e))
  __syncthreads();
  if (act)
#pragma unroll
    for (int i = 0; i < 3; ++i) E[(3 * sub + i) * Vh + h] = xe[i];
  __syncthreads();
  cpx<R> eo[3];
  {
    cpx<R> t[3], v6[6];
    hop_block<R>(g.bnbr, sl, E, Vb, Vbp, Vh, Vh + hs, sub, t);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      t[i].re = fma_r(R(0.5), t[i].re, ro[i].re);
      t[i].im = fma_r(R(0.5), t[i].im, ro[i].im);
    }
    chiral6<R>(t, sub, v6);
    clover_rows<R>(clov_inv, dO, Vb, sub, v6, eo);
  }
  if (act) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      size_t oe = comp_off<R>(de, Vb, 3 * sub + i), oo = comp_off<R>(dO, Vb, 3 * sub + i);
      cpx<R> ve = xe[i], vo = eo[i];
      if (!x_is_zero) {
        ve = ve + ld_comp(x, oe);
        vo = vo + ld_comp(x, oo);
      }
      st_comp(x, oe, ve);
      st_comp(x, oo, vo);
    }
  }
}

// ---------------------------------------------------------------------------
// Staged sweep (FP32 arithmetic) for Schwarz blocks whose half volume is a
// multiple of 32: the thread layout and hop code of k_sap_sweep (four
// threads per site, one runtime direction each, partial sums combined by
// warp shuffles), with
//  * the block's links, A_ee and A_oo^-1 staged into shared memory by bulk
//    asynchronous copies (cp.async.bulk + mbarrier) that land while the
//    residual is computed from global memory;
//  * each thread's block-internal neighbour indices held in registers;
//  * a programmatic-dependent-launch prologue: barrier set-up and the staging
//    copies (links and clover are read-only during a solve) are issued before
//    griddepcontrol.wait, so they overlap the previous sweep's tail.
// Storage S: FP32 (16-byte units), or BF16 / FP16 (half.cuh: 8-byte units of
// the same four values, spinors divided by their site norms).
// ---------------------------------------------------------------------------
namespace stg {

using f2 = cpx<float>;

// storage traits: unit type of the staged arrays and global loads / stores
template <class S>
struct IO;
template <>
struct IO<float> {
  using T = float4;
  static constexpr int LINK_U = 12;   // 16-byte units per site: links
  static constexpr int CLOV_U = 18;   // clover blocks
  __device__ __forceinline__ static void unpack(const T& t, float* v) {
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
  // 36 values of chiral block cb from a staged clover array ([units][Vh], site h)
  __device__ __forceinline__ static void block_smem(const T* A, int Vh, int h, int cb, float* P) {
#pragma unroll
    for (int u = 0; u < 9; ++u) unpack(A[(9 * cb + u) * Vh + h], P + 4 * u);
  }
  // rows 0 and 1 of link mu of local site q from the staged links (rows of
  // Vbp units); link_smem also rebuilds row 2
  __device__ __forceinline__ static void link2_smem(const T* sl, int Vbp, int q, int mu, Link<float>& U) {
    float v[LINK_NR];
#pragma unroll
    for (int u = 0; u < 3; ++u) unpack(sl[(mu * 3 + u) * Vbp + q], v + 4 * u);
#pragma unroll
    for (int k = 0; k < 6; ++k) U.m[k / 3][k % 3] = mk(v[2 * k], v[2 * k + 1]);
  }
  __device__ __forceinline__ static void link_smem(const T* sl, int Vbp, int q, int mu, Link<float>& U) {
    link2_smem(sl, Vbp, q, mu, U);
    complete_link(U);
  }
  // complex component k of the spinor at site d
  __device__ __forceinline__ static f2 comp(const float* f, const float*, int d, int Vb, int k) {
    return ld_comp(f, comp_off<float>(d, Vb, k));
  }
  __device__ __forceinline__ static void spinor(const float* f, const float*, int d, int Vb, Spinor<float>& s) {
    load_spinor_cg<float>(f, d, Vb, s);
  }
  __device__ __forceinline__ static void link(const float* g, int d, int Vb, int mu, Link<float>& U) {
    load_link<float>(g, d, Vb, mu, U);
  }
  // 36 values of chirality block cb of site d of a clover field
  __device__ __forceinline__ static void block36(const float* c, int d, int Vb, int cb, float* P) {
    load_units<float, CLOVER_NR>(c, d, Vb, cb * 9, 9, P);
  }
  // write this thread's 3 components (k0 = 3 sub) of site d
  __device__ __forceinline__ static void store3(float* f, float*, int d, int Vb, int sub, const f2 v[3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i) st_comp(f, comp_off<float>(d, Vb, 3 * sub + i), v[i]);
  }
};

template <class S>
struct IOH {
  using T = uint4;
  static constexpr int LINK_U = HGAUGE_NU;
  static constexpr int CLOV_U = HCLOV_NU;
  __device__ __forceinline__ static void unpack(const T& t, float* v) { unpack8<S>(t, v); }
  // chiral block cb: units 4 cb .. 4 cb + 4, offset 4 cb
  __device__ __forceinline__ static void block_smem(const T* A, int Vh, int h, int cb, float* P) {
    float v[40];
#pragma unroll
    for (int u = 0; u < 5; ++u) unpack(A[(4 * cb + u) * Vh + h], v + 8 * u);
#pragma unroll
    for (int k = 0; k < 36; ++k) P[k] = cb ? v[4 + k] : v[k];
  }
  __device__ __forceinline__ static void link2_smem(const T* sl, int Vbp, int q, int mu, Link<float>& U) {
    float v[16];
    const int u0 = link_unit(mu);
    unpack(sl[u0 * Vbp + q], v);
    unpack(sl[(u0 + 1) * Vbp + q], v + 8);
    link_rows_from16(v, mu, U);
  }
  __device__ __forceinline__ static void link_smem(const T* sl, int Vbp, int q, int mu, Link<float>& U) {
    link2_smem(sl, Vbp, q, mu, U);
    complete_link(U);
  }
  // 32-bit word of complex component k: unit k / 4, position k % 4
  __device__ __forceinline__ static size_t word(int d, int Vb, int k) {
    return hunit<HSPIN_NU>(d, Vb, k >> 2) * 4 + (k & 3);
  }
  __device__ __forceinline__ static f2 comp(const S* f, const float* nrm, int d, int Vb, int k) {
    const uint32_t w = __ldcg(reinterpret_cast<const unsigned int*>(f) + word(d, Vb, k));
    const float2 v = H2<S>::unpack(w);
    const float m = __ldcg(nrm + d);
    return mk(v.x * m, v.y * m);
  }
  __device__ __forceinline__ static void spinor(const S* f, const float* nrm, int d, int Vb, Spinor<float>& s) {
    load_spinor_h_cg<S>(f, nrm, d, Vb, s);
  }
  __device__ __forceinline__ static void link(const S* g, int d, int Vb, int mu, Link<float>& U) {
    load_link_h<S>(g, d, Vb, mu, U);
  }
  __device__ __forceinline__ static void block36(const S* c, int d, int Vb, int cb, float* P) {
    load_block36_h<S>(c, d, Vb, cb, P);
  }
  // the site norm is the largest magnitude over the four threads of the
  // site (adjacent lanes, combined by shuffles); thread 0 of the site
  // writes it.  Every lane of the warp must call this.
  __device__ __forceinline__ static void store3(S* f, float* nrm, int d, int Vb, int sub, const f2 v[3]) {
    float m = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) m = fmaxf(m, fmaxf(fabsf(v[i].re), fabsf(v[i].im)));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
    const float inv = m > 0.f ? 1.f / m : 0.f;
    unsigned int* w = reinterpret_cast<unsigned int*>(f);
#pragma unroll
    for (int i = 0; i < 3; ++i) w[word(d, Vb, 3 * sub + i)] = H2<S>::pack(v[i].re * inv, v[i].im * inv);
    if (sub == 0) nrm[d] = m;
  }
};
template <>
struct IO<__half> : IOH<__half> {};
template <>
struct IO<__nv_bfloat16> : IOH<__nv_bfloat16> {};

// block sum of three per-thread partials with one barrier: every warp
// leaves its three warp sums in sh[3 w ..], and after the barrier every warp
// adds all of them up itself, in the same fixed order, so every thread holds
// the same bits.  Two calls must be separated by another barrier of the CTA
// (all reads of one call are done before the next call writes).
__device__ __forceinline__ void block_sum3_1(float ra, float rb, float rc, float& a, float& b, float& c,
                                             float* sh) {
  ra = warp_sum_r<float>(ra);
  rb = warp_sum_r<float>(rb);
  rc = warp_sum_r<float>(rc);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (l == 0) { sh[3 * w] = ra; sh[3 * w + 1] = rb; sh[3 * w + 2] = rc; }
  __syncthreads();
  const float x = l < nw ? sh[3 * l] : 0.f, y = l < nw ? sh[3 * l + 1] : 0.f, z = l < nw ? sh[3 * l + 2] : 0.f;
  a = warp_sum_r<float>(x);
  b = warp_sum_r<float>(y);
  c = warp_sum_r<float>(z);
}

// own 3 rows of a staged chiral block (site h) times v6
template <class S>
__device__ __forceinline__ void rows3(const typename IO<S>::T* A, int Vh, int h, int cb, int half, const f2 v6[6],
                                      f2 y[3]) {
  float P[36];
  IO<S>::block_smem(A, Vh, h, cb, P);
  f2 y6[6];
  herm6<float>(P, v6, y6);
#pragma unroll
  for (int i = 0; i < 3; ++i) y[i] = half ? y6[3 + i] : y6[i];
}

// link mu of local site q from the staged block links, its third row from
// the rows rebuilt once per sweep (row3[(3 mu + c) Vbp + q])
template <class S>
__device__ __forceinline__ void slink(const typename IO<S>::T* sl, const f2* row3, int Vbp, int q, int mu,
                                      Link<float>& U) {
  IO<S>::link2_smem(sl, Vbp, q, mu, U);
#pragma unroll
  for (int c = 0; c < 3; ++c) U.m[2][c] = row3[(3 * mu + c) * Vbp + q];
}

// hop_block with the neighbour indices already known (-1: outside the block)
template <class S>
__device__ __forceinline__ void hop_block_q(int qf, int qb, const typename IO<S>::T* sl, const f2* row3, const f2* buf,
                                            int Vbp,
                                            int Vh, int q, int sub, f2 out[3]) {
  Spinor<float> acc;
#pragma unroll
  for (int k = 0; k < 12; ++k) acc.c[k] = mk(0.f, 0.f);
  const Dir<float> dr = make_dir<float>(sub);
  f2 hh[2][3], y[2][3];
  Spinor<float> nb;
  if (qf >= 0) {
    smem_spinor<float>(buf, Vh, qf >= Vh ? qf - Vh : qf, nb);
    project_rt<float>(nb, dr, -1.f, hh);
    Link<float> U;
    slink<S>(sl, row3, Vbp, q, sub, U);
    su3_mul(U, hh, y);
    accumulate_rt<float>(acc, y, dr, -1.f, 1.f);
  }
  if (qb >= 0) {
    smem_spinor<float>(buf, Vh, qb >= Vh ? qb - Vh : qb, nb);
    project_rt<float>(nb, dr, 1.f, hh);
    Link<float> U;
    slink<S>(sl, row3, Vbp, qb, sub, U);
    su3_mul_dag(U, hh, y);
    accumulate_rt<float>(acc, y, dr, 1.f, 1.f);
  }
  reduce_scatter<float>(acc, sub, out);
}

// own 3 components of the full (global) hopping sum at device site d
template <class S>
__device__ __forceinline__ void hop_global_s(const Geom& g, const S* x, const float* xn, const S* gauge, int d,
                                             int sub, f2 out[3]) {
  Spinor<float> acc;
#pragma unroll
  for (int k = 0; k < 12; ++k) acc.c[k] = mk(0.f, 0.f);
  const Dir<float> dr = make_dir<float>(sub);
  f2 hh[2][3], y[2][3];
  Spinor<float> nb;
  {
    const uint32_t e = __ldg(g.nbr + (size_t)(2 * sub) * g.V + d);
    const int n = (int)(e & ~NEG_BIT);
    IO<S>::spinor(x, xn, n, g.Vb, nb);
    project_rt<float>(nb, dr, -1.f, hh);
    Link<float> U;
    IO<S>::link(gauge, d, g.Vb, sub, U);
    su3_mul(U, hh, y);
    accumulate_rt<float>(acc, y, dr, -1.f, (e & NEG_BIT) ? -1.f : 1.f);
  }
  {
    const uint32_t e = __ldg(g.nbr + (size_t)(2 * sub + 1) * g.V + d);
    const int n = (int)(e & ~NEG_BIT);
    IO<S>::spinor(x, xn, n, g.Vb, nb);
    project_rt<float>(nb, dr, 1.f, hh);
    Link<float> U;
    IO<S>::link(gauge, n, g.Vb, sub, U);
    su3_mul_dag(U, hh, y);
    accumulate_rt<float>(acc, y, dr, 1.f, (e & NEG_BIT) ? -1.f : 1.f);
  }
  reduce_scatter<float>(acc, sub, out);
}

__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// bn / xn: site norms of b and x (half storage only; ignored for FP32).
// SM is the type the staged block operators are kept in: the storage type S,
// or FP32 for half storage (SM = float, S half): the half units are staged
// into the upper half of each FP32 array and widened in place once per
// sweep, so that the block solve's many reads of the staged links and
// clover blocks need no unpacking.
template <class S, class SM>
__global__ void __launch_bounds__(512) k_sap_stg(Geom g, int colour, int mr_iters, int x_is_zero,
                                                 const S* __restrict__ b, const float* __restrict__ bn,
                                                 S* __restrict__ x, float* __restrict__ xn,
                                                 const S* __restrict__ gauge, const S* __restrict__ clov,
                                                 const S* __restrict__ clov_inv, int* status, long long wait_limit) {
  using T = typename IO<SM>::T;
  constexpr bool WIDEN = !std::is_same<S, SM>::value;
  static_assert(sizeof(T) == sizeof(typename IO<S>::T), "16-byte units in both types");
  constexpr unsigned UB = sizeof(T);            // bytes per unit
  constexpr int LU = IO<SM>::LINK_U, CU = IO<SM>::CLOV_U;     // staged units per site
  constexpr int LG = IO<S>::LINK_U, CG = IO<S>::CLOV_U;       // units per site in global memory
  static_assert(!WIDEN || (LU == 2 * LG && CU == 2 * CG), "a half unit widens into two FP32 units");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Vb = g.Vb, Vh = Vb / 2, Vbp = Vb + LPAD;
  T* sl = reinterpret_cast<T*>(smem_raw);                               // [LU][Vb + LPAD]
  T* Aee = sl + (size_t)LU * Vbp;                                       // [CU][Vh]
  T* Aoi = Aee + CU * Vh;                                               // [CU][Vh]
  f2* E = reinterpret_cast<f2*>(Aoi + CU * Vh);                         // [12][Vh]
  f2* O = E + 12 * Vh;                                                  // [12][Vh]
  float* red = reinterpret_cast<float*>(O + 12 * Vh);                   // [3 * warps + 3]
  f2* row3 = reinterpret_cast<f2*>(red + 200);                          // [12][Vb + LPAD]

  // CTA c handles right-hand side c % nrhs of block c / nrhs of the colour:
  // the CTAs of one block run side by side, so the block's links and clover
  // blocks come from DRAM once and from L2 for the other right-hand sides
  const int nrhs = gridDim.x / (g.nb / 2);
  const int rhs = blockIdx.x % nrhs;
  const int B = block_of_colour(g, colour, blockIdx.x / nrhs);
  const size_t off = (size_t)rhs * g.V * SPINOR_NR;
  const size_t noff = (size_t)rhs * g.V;
  b += off;
  x += off;
  if (bn) bn += noff;       // site norms exist for half storage only
  if (xn) xn += noff;
  const int t = threadIdx.x;
  const int h = t >> 2, sub = t & 3;
  const int cb = sub >> 1, half = sub & 1;
  const int de = B * Vb + h, dO = B * Vb + Vh + h;
  // block-internal neighbours of this thread's direction, even and odd site
  const int qf_e = __ldg(g.bnbr + (2 * sub) * Vb + h), qb_e = __ldg(g.bnbr + (2 * sub + 1) * Vb + h);
  const int qf_o = __ldg(g.bnbr + (2 * sub) * Vb + Vh + h), qb_o = __ldg(g.bnbr + (2 * sub + 1) * Vb + Vh + h);

  // stage the block's links (and A_ee, A_oo^-1) with bulk asynchronous
  // copies: global unit row u lands in staged row u, or in row LU - LG + u
  // (CU - CG + u) when it is widened afterwards
  __shared__ __align__(8) uint64_t mbar;
  if (t == 0) {
    mbar_init(&mbar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  {
    const unsigned link_row = (unsigned)Vb * UB, half_row = (unsigned)Vh * UB;
    if (t == 0) mbar_expect_tx(&mbar, (unsigned)LG * link_row + 2u * CG * half_row);
    __syncthreads();
    if (t < LG) {
      const T* src = reinterpret_cast<const T*>(gauge) + (size_t)B * LG * Vb;
      bulk_g2s(sl + (size_t)(LU - LG + t) * Vbp, src + (size_t)t * Vb, link_row, &mbar);
    } else if (t < LG + CG) {
      const int u = t - LG;
      const T* ca = reinterpret_cast<const T*>(clov) + (size_t)B * CG * Vb;
      bulk_g2s(Aee + (size_t)(CU - CG + u) * Vh, ca + (size_t)u * Vb, half_row, &mbar);
    } else if (t < LG + 2 * CG) {
      const int u = t - LG - CG;
      const T* ci = reinterpret_cast<const T*>(clov_inv) + (size_t)B * CG * Vb;
      bulk_g2s(Aoi + (size_t)(CU - CG + u) * Vh, ci + (size_t)u * Vb + Vh, half_row, &mbar);
    }
  }
  // b and x may still be written by the previous kernel of the stream
  grid_dependency_wait();

  // residual r = b - D x on the own components of both sites: the hops and
  // the odd site's clover product from global memory while the block is
  // staged, the even site's clover product from the staged A_ee after it
  f2 re[3], ro[3], xe6[6];
#pragma unroll
  for (int par = 0; par < 2; ++par) {
    const int d = par ? dO : de;
    f2 r[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) r[i] = IO<S>::comp(b, bn, d, Vb, 3 * sub + i);
    if (!x_is_zero) {
      f2 hop[3], x6[6];
      hop_global_s<S>(g, x, xn, gauge, d, sub, hop);
#pragma unroll
      for (int i = 0; i < 6; ++i) x6[i] = IO<S>::comp(x, xn, d, Vb, 6 * cb + i);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        r[i].re += 0.5f * hop[i].re;
        r[i].im += 0.5f * hop[i].im;
      }
      if (par) {
        float P[36];
        IO<S>::block36(clov, d, Vb, cb, P);
        f2 y6[6];
        herm6<float>(P, x6, y6);
#pragma unroll
        for (int i = 0; i < 3; ++i) r[i] = r[i] - (half ? y6[3 + i] : y6[i]);
      } else {
#pragma unroll
        for (int i = 0; i < 6; ++i) xe6[i] = x6[i];
      }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if (par) ro[i] = r[i];
      else re[i] = r[i];
    }
  }
  // the staged block must have landed (bounded wait; on time-out record
  // DDAMG_ETIMEOUT, wait again for the copies in flight, and leave x alone)
  {
    const bool ok = mbar_wait_bounded(&mbar, 0, wait_limit);
    if (__syncthreads_or(!ok)) {
      if (t == 0) atomicExch(status, 6);
      mbar_wait_bounded(&mbar, 0, MBAR_POLL_LIMIT);
      return;
    }
  }
  if constexpr (WIDEN) {
    // half unit k of a site (staged row n + k of an array of 2 n rows) holds
    // the values of FP32 units 2 k and 2 k + 1.  One thread widens one site
    // of one array in increasing k: the rows 2 k, 2 k + 1 it writes are
    // half rows n + k' with k' <= k, already read by the same thread, and
    // no other thread touches the site's column.
    for (int s = t; s < Vb + 2 * Vh; s += blockDim.x) {
      T* a;
      int n, stride, q;
      if (s < Vb) { a = sl; n = LG; stride = Vbp; q = s; }
      else if (s < Vb + Vh) { a = Aee; n = CG; stride = Vh; q = s - Vb; }
      else { a = Aoi; n = CG; stride = Vh; q = s - Vb - Vh; }
      for (int k = 0; k < n; ++k) {
        float v[8];
        unpack8<S>(*reinterpret_cast<const uint4*>(a + (size_t)(n + k) * stride + q), v);
        a[(size_t)(2 * k) * stride + q] = make_float4(v[0], v[1], v[2], v[3]);
        a[(size_t)(2 * k + 1) * stride + q] = make_float4(v[4], v[5], v[6], v[7]);
      }
    }
    __syncthreads();
  }
  if (!x_is_zero) {     // r_e -= A_ee x_e, A_ee staged
    f2 ax[3];
    rows3<SM>(Aee, Vh, h, cb, half, xe6, ax);
#pragma unroll
    for (int i = 0; i < 3; ++i) re[i] = re[i] - ax[i];
  }
  // the third rows of the staged links, rebuilt once per sweep instead of
  // at every hop (visible to the hops after the barrier below)
  for (int k = t; k < 4 * Vb; k += blockDim.x) {
    const int mu = k / Vb, q = k - mu * Vb;
    Link<float> U;
    IO<SM>::link_smem(sl, Vbp, q, mu, U);
#pragma unroll
    for (int c = 0; c < 3; ++c) row3[(3 * mu + c) * Vbp + q] = U.m[2][c];
  }
  auto ainv_rows = [&](const f2 v6[6], f2 y[3]) { rows3<SM>(Aoi, Vh, h, cb, half, v6, y); };
  auto aee_rows = [&](const f2 v6[6], f2 y[3]) { rows3<SM>(Aee, Vh, h, cb, half, v6, y); };
  // u_o = A_oo^-1 r_o
  {
    f2 v6[6], u[3];
    chiral6<float>(ro, sub, v6);
    ainv_rows(v6, u);
#pragma unroll
    for (int i = 0; i < 3; ++i) O[(3 * sub + i) * Vh + h] = u[i];
  }
  __syncthreads();
  // rhs_e = r_e + 1/2 hop(u_o)
  f2 res[3], xe[3];
  {
    f2 tt[3];
    hop_block_q<SM>(qf_e, qb_e, sl, row3, O, Vbp, Vh, h, sub, tt);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      res[i] = mk(fmaf(0.5f, tt[i].re, re[i].re), fmaf(0.5f, tt[i].im, re[i].im));
      xe[i] = mk(0.f, 0.f);
    }
  }
  for (int it = 0; it < mr_iters; ++it) {
#pragma unroll
    for (int i = 0; i < 3; ++i) E[(3 * sub + i) * Vh + h] = res[i];
    // A_ee res needs only this site's res: formed while the barrier waits
    f2 p[3];
    {
      f2 v6[6];
      chiral6<float>(res, sub, v6);
      aee_rows(v6, p);
    }
    __syncthreads();
    {  // odd: w = A_oo^-1 (-1/2 hop(res))
      f2 tt[3], v6[6], w[3];
      hop_block_q<SM>(qf_o, qb_o, sl, row3, E, Vbp, Vh, Vh + h, sub, tt);
#pragma unroll
      for (int i = 0; i < 3; ++i) tt[i] = -0.5f * tt[i];
      chiral6<float>(tt, sub, v6);
      ainv_rows(v6, w);
#pragma unroll
      for (int i = 0; i < 3; ++i) O[(3 * sub + i) * Vh + h] = w[i];
    }
    __syncthreads();
    float pr_re = 0.f, pr_im = 0.f, pp_r = 0.f;
    {  // even: p = A_ee res + 1/2 hop(w)
      f2 tt[3];
      hop_block_q<SM>(qf_e, qb_e, sl, row3, O, Vbp, Vh, h, sub, tt);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        p[i] = mk(fmaf(0.5f, tt[i].re, p[i].re), fmaf(0.5f, tt[i].im, p[i].im));
        pr_re += p[i].re * res[i].re + p[i].im * res[i].im;
        pr_im += p[i].re * res[i].im - p[i].im * res[i].re;
        pp_r += p[i].re * p[i].re + p[i].im * p[i].im;
      }
    }
    float dre, dim, pp;
    block_sum3_1(pr_re, pr_im, pp_r, dre, dim, pp, red);
    if (pp > 0.f) {
      const f2 a = mk(dre / pp, dim / pp);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        fma(xe[i], a, res[i]);
        res[i] = res[i] - a * p[i];
      }
    }
  }
  // the next sweep may start its prologue
  launch_dependents();
  // e_o = A_oo^-1 (r_o + 1/2 hop(e_e))
#pragma unroll
  for (int i = 0; i < 3; ++i) E[(3 * sub + i) * Vh + h] = xe[i];
  __syncthreads();
  f2 eo[3];
  {
    f2 tt[3], v6[6];
    hop_block_q<SM>(qf_o, qb_o, sl, row3, E, Vbp, Vh, Vh + h, sub, tt);
#pragma unroll
    for (int i = 0; i < 3; ++i) tt[i] = mk(fmaf(0.5f, tt[i].re, ro[i].re), fmaf(0.5f, tt[i].im, ro[i].im));
    chiral6<float>(tt, sub, v6);
    ainv_rows(v6, eo);
  }
  f2 ve[3], vo[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    ve[i] = xe[i];
    vo[i] = eo[i];
    if (!x_is_zero) {
      ve[i] = ve[i] + IO<S>::comp(x, xn, de, Vb, 3 * sub + i);
      vo[i] = vo[i] + IO<S>::comp(x, xn, dO, Vb, 3 * sub + i);
    }
  }
  IO<S>::store3(x, xn, de, Vb, sub, ve);
  IO<S>::store3(x, xn, dO, Vb, sub, vo);
}

// ---------------------------------------------------------------------------
// Wilson-clover D on the whole lattice with four threads per site (the
// thread layout of the SAP kernel): thread sub applies the two hops of
// direction mu = sub and the three rows of its chiral clover block that it
// owns; the hop sums are combined by warp shuffles.  A quarter of the
// loads per thread and four times the threads of the one-thread-per-site
// kernel keep more memory requests in flight.
//   y = A x - 1/2 hop(x)                       (DSLASH_D)
// ---------------------------------------------------------------------------
template <class S>
__global__ void __launch_bounds__(256) k_dslash4(Geom g, const S* __restrict__ x, const float* __restrict__ xn,
                                                 S* __restrict__ y, float* __restrict__ yn,
                                                 const S* __restrict__ gauge, const S* __restrict__ clov) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)4 * g.V) return;        // whole warps (4 V is a multiple of 32)
  const int d = (int)(t >> 2), sub = (int)(t & 3);
  const int cb = sub >> 1, half = sub & 1;
  const size_t off = (size_t)blockIdx.y * g.V * SPINOR_NR;
  const size_t noff = (size_t)blockIdx.y * g.V;
  x += off;
  y += off;
  if (xn) xn += noff;        // site norms exist for half storage only
  if (yn) yn += noff;
  f2 hop[3];
  hop_global_s<S>(g, x, xn, gauge, d, sub, hop);
  f2 x6[6], ax[3];
#pragma unroll
  for (int i = 0; i < 6; ++i) x6[i] = IO<S>::comp(x, xn, d, g.Vb, 6 * cb + i);
  {
    float P[36];
    IO<S>::block36(clov, d, g.Vb, cb, P);
    f2 y6[6];
    herm6<float>(P, x6, y6);
#pragma unroll
    for (int i = 0; i < 3; ++i) ax[i] = half ? y6[3 + i] : y6[i];
  }
  f2 out[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) out[i] = mk(fmaf(-0.5f, hop[i].re, ax[i].re), fmaf(-0.5f, hop[i].im, ax[i].im));
  IO<S>::store3(y, yn, d, g.Vb, sub, out);
}

}  // namespace stg

}  // namespace

static int sap_threads(const Geom& g) { return ((4 * (g.Vb / 2) + 31) / 32) * 32; }

size_t sap_smem_bytes(const Geom& g, int real_size) {
  size_t units = (size_t)GAUGE_NR * real_size / 16 * (g.Vb + LPAD);   // staged links
  size_t bufs = 2 * 12 * (size_t)(g.Vb / 2) * 2 * real_size;          // E, O
  return units * 16 + bufs + 100 * sizeof(double);
}

// shared memory of the staged kernel: link rows (LU units per site, padded),
// the even half of A and the odd half of A^-1 (CU units per site each), the
// even and odd work vectors, the reduction slots and the third rows of the
// staged links; 16-byte units
static size_t sap_stg_smem(const Geom& g, int LU, int CU) {
  const int Vh = g.Vb / 2;
  size_t bytes = (size_t)LU * (g.Vb + LPAD) * 16;
  bytes += (size_t)2 * CU * Vh * 16;
  bytes += (size_t)24 * Vh * 8;
  bytes += 100 * sizeof(double);
  bytes += (size_t)12 * (g.Vb + LPAD) * 8;     // third link rows (FP32 complex)
  return bytes;
}

static bool sap_stg_ok(const Geom& g, int LU, int CU) {
  const int Vh = g.Vb / 2;
  return Vh % 32 == 0 && 4 * Vh <= 512 && sap_stg_smem(g, LU, CU) <= 226 * 1024;
}

bool sap_half_ok(const Geom& g) { return sap_stg_ok(g, HGAUGE_NU, HCLOV_NU); }
bool sap_staged_ok(const Geom& g) { return sap_stg_ok(g, 12, 18); }

template <class S, class SM>
static cudaError_t launch_stg(const Geom& g, int colour, int mr_iters, bool x_is_zero, const S* b, const float* bn,
                              S* x, float* xn, const S* gauge, const S* clover, const S* clover_inv, int nrhs,
                              int* status, long long wait_limit, cudaStream_t st) {
  const size_t need = sap_stg_smem(g, stg::IO<SM>::LINK_U, stg::IO<SM>::CLOV_U);
  {
    // the attribute is per device and per instance; set it on every launch
    // whose size exceeds what this device's instance was given
    static std::mutex mu;
    static size_t cfg[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (cfg[dev] < need) {
      cudaError_t e =
          cudaFuncSetAttribute(stg::k_sap_stg<S, SM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
      if (e != cudaSuccess) return e;
      cfg[dev] = need;
    }
  }
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)(g.nb / 2) * (unsigned)nrhs);
  lc.blockDim = dim3(2 * g.Vb);
  lc.dynamicSmemBytes = need;
  lc.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;   // prologue overlaps the previous kernel
  at[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  const int zero = x_is_zero ? 1 : 0;
  cudaError_t e = cudaLaunchKernelEx(&lc, stg::k_sap_stg<S, SM>, g, colour, mr_iters, zero, b, bn, x, xn, gauge,
                                     clover, clover_inv, status, wait_limit);
  ++g_launches;
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <class S>
cudaError_t sap_sweep_h(const Geom& g, int colour, int mr_iters, bool x_is_zero, const void* b, const float* bn,
                        void* x, float* xn, const void* gauge, const void* clover, const void* clover_inv, int nrhs,
                        int* status, long long wait_limit, cudaStream_t st, bool widen) {
  if (!sap_half_ok(g)) return cudaErrorInvalidValue;
  if (widen && sap_staged_ok(g))
    return launch_stg<S, float>(g, colour, mr_iters, x_is_zero, static_cast<const S*>(b), bn, static_cast<S*>(x), xn,
                                static_cast<const S*>(gauge), static_cast<const S*>(clover),
                                static_cast<const S*>(clover_inv), nrhs, status, wait_limit, st);
  return launch_stg<S, S>(g, colour, mr_iters, x_is_zero, static_cast<const S*>(b), bn, static_cast<S*>(x), xn,
                          static_cast<const S*>(gauge), static_cast<const S*>(clover),
                          static_cast<const S*>(clover_inv), nrhs, status, wait_limit, st);
}
template cudaError_t sap_sweep_h<__half>(const Geom&, int, int, bool, const void*, const float*, void*, float*,
                                         const void*, const void*, const void*, int, int*, long long, cudaStream_t,
                                         bool);
template cudaError_t sap_sweep_h<__nv_bfloat16>(const Geom&, int, int, bool, const void*, const float*, void*,
                                                float*, const void*, const void*, const void*, int, int*, long long,
                                                cudaStream_t, bool);

template <class S>
cudaError_t dslash4(const Geom& g, const void* x, const float* xn, void* y, float* yn, const void* gauge,
                    const void* clover, int nrhs, cudaStream_t st) {
  if (g.V % 8) return cudaErrorInvalidValue;
  const size_t threads = (size_t)4 * g.V;
  stg::k_dslash4<S><<<dim3((unsigned)((threads + 255) / 256), nrhs), 256, 0, st>>>(
      g, static_cast<const S*>(x), xn, static_cast<S*>(y), yn, static_cast<const S*>(gauge),
      static_cast<const S*>(clover));
  ++g_launches;
  return cudaGetLastError();
}
template cudaError_t dslash4<float>(const Geom&, const void*, const float*, void*, float*, const void*, const void*,
                                    int, cudaStream_t);
template cudaError_t dslash4<__half>(const Geom&, const void*, const float*, void*, float*, const void*, const void*,
                                     int, cudaStream_t);
template cudaError_t dslash4<__nv_bfloat16>(const Geom&, const void*, const float*, void*, float*, const void*,
                                            const void*, int, cudaStream_t);

template <class R>
cudaError_t sap_sweep(const Geom& g, int colour, int mr_iters, bool x_is_zero, const R* b, R* x,
                      const R* gauge, const R* clover, const R* clover_inv, int nrhs, int* status,
                      long long wait_limit, cudaStream_t st, bool staged) {
  if constexpr (sizeof(R) == 4) {
    if (staged && sap_stg_ok(g, 12, 18)) {
      return launch_stg<float, float>(g, colour, mr_iters, x_is_zero, b, nullptr, x, nullptr, gauge, clover,
                                      clover_inv, nrhs, status, wait_limit, st);
    }
  }
  int threads = sap_threads(g);
  size_t smem = sap_smem_bytes(g, sizeof(R));
  {
    static std::mutex mu;
    static size_t configured[64][2] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (configured[dev][sizeof(R) == 8] < smem) {
      cudaError_t e = cudaFuncSetAttribute(k_sap_sweep<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      configured[dev][sizeof(R) == 8] = smem;
    }
  }
  dim3 grid(g.nb / 2, nrhs);
  k_sap_sweep<R><<<grid, threads, smem, st>>>(g, colour, mr_iters, x_is_zero ? 1 : 0, b, x, gauge,
                                               clover, clover_inv);
  ++g_launches;
  return cudaGetLastError();
}

template cudaError_t sap_sweep<float>(const Geom&, int, int, bool, const float*, float*, const float*,
                                      const float*, const float*, int, int*, long long, cudaStream_t, bool);
template cudaError_t sap_sweep<double>(const Geom&, int, int, bool, const double*, double*,
                                       const double*, const double*, const double*, int, int*, long long,
                                       cudaStream_t, bool);

}  // namespace ddamg
