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
#include "common.cuh"
#include "kernels.h"

namespace ddamg {

namespace {

template <class R>
struct Sh {
  using T = typename U16<R>::T;
};

// link mu of local site q from the staged block links ([unit][Vb] in smem)
template <class R>
__device__ __forceinline__ void smem_link(const typename U16<R>::T* sl, int Vb, int q, int mu,
                                          Link<R>& U) {
  using LY = Layout<R, GAUGE_NR>;
  constexpr int NUL = LINK_NR / LY::PER;
  R v[LINK_NR];
#pragma unroll
  for (int u = 0; u < NUL; ++u) {
    typename U16<R>::T t = sl[(mu * NUL + u) * Vb + q];
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

// spinor of half-index h from a shared SoA buffer buf[12][Vh]
template <class R>
__device__ __forceinline__ void smem_spinor(const cpx<R>* buf, int Vh, int h, Spinor<R>& s) {
#pragma unroll
  for (int k = 0; k < 12; ++k) s.c[k] = buf[k * Vh + h];
}
template <class R>
__device__ __forceinline__ void smem_store(cpx<R>* buf, int Vh, int h, const Spinor<R>& s) {
#pragma unroll
  for (int k = 0; k < 12; ++k) buf[k * Vh + h] = s.c[k];
}

// block-local hop of one direction at local site q; the neighbour values
// (other parity) come from buf
template <int MU, class R>
__device__ __forceinline__ void hop_block_dir(const int16_t* __restrict__ bnbr,
                                              const typename U16<R>::T* sl, const cpx<R>* buf,
                                              int Vb, int Vh, int q, Spinor<R>& acc) {
  cpx<R> h[2][3], y[2][3];
  Spinor<R> nb;
  int qf = __ldg(bnbr + (2 * MU) * Vb + q);
  if (qf >= 0) {
    smem_spinor<R>(buf, Vh, qf >= Vh ? qf - Vh : qf, nb);
    project<MU, -1>(nb, h);
    Link<R> U;
    smem_link<R>(sl, Vb, q, MU, U);
    su3_mul(U, h, y);
    accumulate<MU, -1>(acc, y, R(1));
  }
  int qb = __ldg(bnbr + (2 * MU + 1) * Vb + q);
  if (qb >= 0) {
    smem_spinor<R>(buf, Vh, qb >= Vh ? qb - Vh : qb, nb);
    project<MU, +1>(nb, h);
    Link<R> U;
    smem_link<R>(sl, Vb, qb, MU, U);
    su3_mul_dag(U, h, y);
    accumulate<MU, +1>(acc, y, R(1));
  }
}

template <class R>
__device__ __forceinline__ void hop_block(const int16_t* bnbr, const typename U16<R>::T* sl,
                                          const cpx<R>* buf, int Vb, int Vh, int q,
                                          Spinor<R>& acc) {
#pragma unroll
  for (int k = 0; k < 12; ++k) acc.c[k] = mk(R(0), R(0));
  hop_block_dir<0>(bnbr, sl, buf, Vb, Vh, q, acc);
  hop_block_dir<1>(bnbr, sl, buf, Vb, Vh, q, acc);
  hop_block_dir<2>(bnbr, sl, buf, Vb, Vh, q, acc);
  hop_block_dir<3>(bnbr, sl, buf, Vb, Vh, q, acc);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block sum of three doubles, result broadcast to all threads
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c, double* sh) {
  a = warp_sum(a);
  b = warp_sum(b);
  c = warp_sum(c);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  int nw = blockDim.x >> 5;
  if (l == 0) { sh[3 * w] = a; sh[3 * w + 1] = b; sh[3 * w + 2] = c; }
  __syncthreads();
  a = b = c = 0.0;
  for (int i = 0; i < nw; ++i) { a += sh[3 * i]; b += sh[3 * i + 1]; c += sh[3 * i + 2]; }
  __syncthreads();
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
__global__ void k_sap_sweep(Geom g, int colour, int mr_iters, int x_is_zero,
                            const R* __restrict__ b, R* __restrict__ x,
                            const R* __restrict__ gauge, const R* __restrict__ clov,
                            const R* __restrict__ clov_inv) {
  using T = typename U16<R>::T;
  using LYG = Layout<R, GAUGE_NR>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Vb = g.Vb, Vh = Vb / 2;
  T* sl = reinterpret_cast<T*>(smem_raw);                               // [NU][Vb]
  cpx<R>* E = reinterpret_cast<cpx<R>*>(sl + (size_t)LYG::NU * Vb);      // [12][Vh]
  cpx<R>* O = E + 12 * Vh;                                               // [12][Vh]
  cpx<R>* Ro = O + 12 * Vh;                                              // [12][Vh]
  double* red = reinterpret_cast<double*>(Ro + 12 * Vh);                 // [3 * warps]

  const int B = block_of_colour(g, colour, blockIdx.x);
  const size_t off = (size_t)blockIdx.y * g.V * SPINOR_NR;
  b += off;
  x += off;
  const int h = threadIdx.x;
  const bool act = h < Vh;
  const int de = B * Vb + h, dO = B * Vb + Vh + h;

  // stage the block's links (contiguous in the block-major layout)
  {
    const T* src = reinterpret_cast<const T*>(gauge) + (size_t)B * LYG::NU * Vb;
    for (int i = threadIdx.x; i < LYG::NU * Vb; i += blockDim.x) sl[i] = __ldg(src + i);
  }

  // residual on the block
  Spinor<R> re;    // even-site residual
  if (act) {
    Spinor<R> ro;
    for (int par = 0; par < 2; ++par) {
      int d = par ? dO : de;
      Spinor<R> r;
      load_spinor<R>(b, d, Vb, r);
      if (!x_is_zero) {
        Spinor<R> xs, ax, acc;
        load_spinor_cg<R>(x, d, Vb, xs);
        clover_mul<R>(clov, d, Vb, xs, ax);
#pragma unroll
        for (int k = 0; k < 12; ++k) acc.c[k] = mk(R(0), R(0));
        hop_dir<0>(g, x, gauge, d, acc);
        hop_dir<1>(g, x, gauge, d, acc);
        hop_dir<2>(g, x, gauge, d, acc);
        hop_dir<3>(g, x, gauge, d, acc);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          r.c[k].re -= ax.c[k].re - R(0.5) * acc.c[k].re;
          r.c[k].im -= ax.c[k].im - R(0.5) * acc.c[k].im;
        }
      }
      if (par) ro = r; else re = r;
    }
    smem_store<R>(Ro, Vh, h, ro);
    // u_o = A_oo^-1 r_o
    Spinor<R> u;
    clover_mul<R>(clov_inv, dO, Vb, ro, u);
    smem_store<R>(O, Vh, h, u);
  }
  __syncthreads();

  // rhs_e = r_e - D_eo u_o = r_e + 1/2 hop(u_o)
  Spinor<R> res, xe;
  if (act) {
    Spinor<R> t;
    hop_block<R>(g.bnbr, sl, O, Vb, Vh, h, t);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      res.c[k].re = fma_r(R(0.5), t.c[k].re, re.c[k].re);
      res.c[k].im = fma_r(R(0.5), t.c[k].im, re.c[k].im);
      xe.c[k] = mk(R(0), R(0));
    }
  }

  for (int it = 0; it < mr_iters; ++it) {
    if (act) smem_store<R>(E, Vh, h, res);
    __syncthreads();
    if (act) {  // odd: w = A_oo^-1 D_oe res = A_oo^-1 (-1/2 hop(res))
      Spinor<R> t, w;
      hop_block<R>(g.bnbr, sl, E, Vb, Vh, Vh + h, t);
#pragma unroll
      for (int k = 0; k < 12; ++k) t.c[k] = R(-0.5) * t.c[k];
      clover_mul<R>(clov_inv, dO, Vb, t, w);
      smem_store<R>(O, Vh, h, w);
    }
    __syncthreads();
    double pr_re = 0.0, pr_im = 0.0, pp = 0.0;
    Spinor<R> p;
    if (act) {  // even: p = A_ee res - D_eo w = A_ee res + 1/2 hop(w)
      Spinor<R> t;
      clover_mul<R>(clov, de, Vb, res, p);
      hop_block<R>(g.bnbr, sl, O, Vb, Vh, h, t);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        p.c[k].re = fma_r(R(0.5), t.c[k].re, p.c[k].re);
        p.c[k].im = fma_r(R(0.5), t.c[k].im, p.c[k].im);
        pr_re += (double)p.c[k].re * res.c[k].re + (double)p.c[k].im * res.c[k].im;
        pr_im += (double)p.c[k].re * res.c[k].im - (double)p.c[k].im * res.c[k].re;
        pp += (double)p.c[k].re * p.c[k].re + (double)p.c[k].im * p.c[k].im;
      }
    }
    block_sum3(pr_re, pr_im, pp, red);
    if (act && pp > 0.0) {
      R are = (R)(pr_re / pp), aim = (R)(pr_im / pp);
      cpx<R> a = mk(are, aim);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        fma(xe.c[k], a, res.c[k]);
        cpx<R> ap = a * p.c[k];
        res.c[k] = res.c[k] - ap;
      }
    }
  }

  // e_o = A_oo^-1 (r_o - D_oe e_e) = A_oo^-1 (r_o + 1/2 hop(e_e))
  if (act) smem_store<R>(E, Vh, h, xe);
  __syncthreads();
  if (act) {
    Spinor<R> t, ro, eo;
    hop_block<R>(g.bnbr, sl, E, Vb, Vh, Vh + h, t);
    smem_spinor<R>(Ro, Vh, h, ro);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      ro.c[k].re = fma_r(R(0.5), t.c[k].re, ro.c[k].re);
      ro.c[k].im = fma_r(R(0.5), t.c[k].im, ro.c[k].im);
    }
    clover_mul<R>(clov_inv, dO, Vb, ro, eo);
    if (!x_is_zero) {
      Spinor<R> xo, xev;
      load_spinor_cg<R>(x, de, Vb, xev);
      load_spinor_cg<R>(x, dO, Vb, xo);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        xe.c[k] = xe.c[k] + xev.c[k];
        eo.c[k] = eo.c[k] + xo.c[k];
      }
    }
    store_spinor<R>(x, de, Vb, xe);
    store_spinor<R>(x, dO, Vb, eo);
  }
}

}  // namespace

size_t sap_smem_bytes(const Geom& g, int real_size) {
  size_t units = (size_t)GAUGE_NR * real_size / 16 * g.Vb;        // staged links
  size_t bufs = 3 * 12 * (size_t)(g.Vb / 2) * 2 * real_size;       // E, O, Ro
  int threads = ((g.Vb / 2 + 31) / 32) * 32;
  return units * 16 + bufs + 3 * sizeof(double) * (threads / 32);
}

template <class R>
cudaError_t sap_sweep(const Geom& g, int colour, int mr_iters, bool x_is_zero, const R* b, R* x,
                      const R* gauge, const R* clover, const R* clover_inv, int nrhs,
                      cudaStream_t st) {
  int threads = ((g.Vb / 2 + 31) / 32) * 32;
  size_t smem = sap_smem_bytes(g, sizeof(R));
  static bool configured[2] = {false, false};
  cudaError_t e;
  if (!configured[sizeof(R) == 8]) {
    e = cudaFuncSetAttribute(k_sap_sweep<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    configured[sizeof(R) == 8] = true;
  }
  dim3 grid(g.nb / 2, nrhs);
  k_sap_sweep<R><<<grid, threads, smem, st>>>(g, colour, mr_iters, x_is_zero ? 1 : 0, b, x, gauge,
                                               clover, clover_inv);
  ++g_launches;
  return cudaGetLastError();
}

template cudaError_t sap_sweep<float>(const Geom&, int, int, bool, const float*, float*, const float*,
                                      const float*, const float*, int, cudaStream_t);
template cudaError_t sap_sweep<double>(const Geom&, int, int, bool, const double*, double*,
                                       const double*, const double*, const double*, int, cudaStream_t);

}  // namespace ddamg
