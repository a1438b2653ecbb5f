// Kernels of the third level (paper Sec. 1: the coarse-grid solver can be
// given a coarse grid of its own, recursively): the construction of Sec. 2
// and Eq. 1-5 applied once more, to the coarse operator D_c instead of D.
//
// Level 2 is the coarse lattice of level 1 with D_c as its 9-point operator
// (2n components per coarse site, coarse chirality G5 = diag(1_n, -1_n)):
//   * a multiplicative Schwarz sweep over blocks of coarse sites (colour =
//     parity of the block coordinates), each block solved by even-odd MR on
//     S = A_ee - D_eo A_oo^-1 D_oe with the self blocks of D_c as A;
//   * aggregates of coarse sites (equal to those blocks) with n2 test vectors
//     split by coarse chirality: R2 (Eq. 3), P2 (Eq. 4), their classical
//     Gram-Schmidt orthonormalisation per (aggregate, chirality), and the
//     Galerkin operator D_cc = P2^H D_c P2 (Eq. 2), assembled term by term
//     of the coarse stencil with forward and backward links kept apart.
// Coarse fields are [X][2n] complex (X the lexicographic coarse site), test
// vectors [i][X][2n], D_c and D_cc blocks column-major (entry (r, c) at
// c * 2n + r), as on level 1.
#include "common.cuh"
#include "kernels.h"

namespace ddamg {

namespace {

// CTA sum of three partials (every thread gets the same bits: fixed order)
template <class R>
__device__ __forceinline__ void cta_sum3(R& a, R& b, R& c, R* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (l == 0) { sh[3 * w] = a; sh[3 * w + 1] = b; sh[3 * w + 2] = c; }
  __syncthreads();
  a = R(0); b = R(0); c = R(0);
  for (int i = 0; i < nw; ++i) { a += sh[3 * i]; b += sh[3 * i + 1]; c += sh[3 * i + 2]; }
  __syncthreads();
}

// row `row` of the column-major n2 x n2 block M times v
template <class R>
__device__ __forceinline__ cpx<R> blk_row(const cpx<R>* __restrict__ M, const cpx<R>* v, int n2, int row) {
  cpx<R> acc = mk(R(0), R(0));
  for (int c = 0; c < n2; ++c) fma(acc, M[(size_t)c * n2 + row], v[c]);
  return acc;
}

// ---------------------------------------------------------------------------
// one colour of the level-2 Schwarz sweep: CTA per block of that colour (and
// right-hand side blockIdx.y), thread per (site of the block, row):
//   r = b - D_c x on the block's sites (r = b if x is zero)
//   rhs = r_e - D_eo A_oo^-1 r_o; MR on S from e_e = 0, mr_iters steps:
//     p = S res; alpha = <p, res> / <p, p>; e_e += alpha res; res -= alpha p
//   e_o = A_oo^-1 (r_o - D_oe e_e); x += e
// with D_eo, D_oe the hops of D_c that stay inside the block.
// ---------------------------------------------------------------------------
template <class R>
__global__ void k_l2_sap(L2Geom d, const cpx<R>* __restrict__ Dc, const cpx<R>* __restrict__ Ainv, int n2,
                         int colour, int mr_iters, int x_is_zero, const cpx<R>* __restrict__ b,
                         cpx<R>* __restrict__ x) {
  extern __shared__ __align__(16) unsigned char l2sh[];
  const int Vb = d.Vb, nvec = Vb * n2;
  cpx<R>* Rr = reinterpret_cast<cpx<R>*>(l2sh);      // r, every site of the block
  cpx<R>* U = Rr + nvec;                             // even sites: res
  cpx<R>* W = U + nvec;                              // odd sites: temporaries
  cpx<R>* Z = W + nvec;
  cpx<R>* E = Z + nvec;                              // even: e_e; odd (at the end): e_o
  R* red = reinterpret_cast<R*>(E + nvec);           // 3 per warp
  const int Bk = d.bcol[colour * (d.NXp / 2) + blockIdx.x];
  const size_t roff = (size_t)blockIdx.y * d.NX * n2;
  b += roff;
  x += roff;
  const int t = threadIdx.x;
  const bool live = t < nvec;
  const int s = live ? t / n2 : 0, row = live ? t - s * n2 : 0;
  const int X = d.sites[(size_t)Bk * Vb + s];
  const int par = d.par[X];
  const size_t NN = (size_t)n2 * n2;
  // sum over the block-internal hops of site X applied to the block vector src
  auto hop_in = [&](const cpx<R>* src) {
    cpx<R> acc = mk(R(0), R(0));
    for (int dd = 1; dd < 9; ++dd) {
      const int nb = d.cnbr[dd * d.NX + X];
      if (d.blk[nb] != Bk) continue;
      acc = acc + blk_row<R>(Dc + ((size_t)X * 9 + dd) * NN, src + (size_t)d.loc[nb] * n2, n2, row);
    }
    return acc;
  };
  if (live) {
    cpx<R> r = b[(size_t)X * n2 + row];
    if (!x_is_zero)
      for (int dd = 0; dd < 9; ++dd) {
        const int nb = d.cnbr[dd * d.NX + X];
        r = r - blk_row<R>(Dc + ((size_t)X * 9 + dd) * NN, x + (size_t)nb * n2, n2, row);
      }
    Rr[t] = r;
    E[t] = mk(R(0), R(0));
  }
  __syncthreads();
  if (live && par == 1) W[t] = blk_row<R>(Ainv + (size_t)X * NN, Rr + (size_t)s * n2, n2, row);
  __syncthreads();
  if (live && par == 0) U[t] = Rr[t] - hop_in(W);
  __syncthreads();
  for (int it = 0; it < mr_iters; ++it) {
    if (live && par == 1) W[t] = hop_in(U);
    __syncthreads();
    if (live && par == 1) Z[t] = blk_row<R>(Ainv + (size_t)X * NN, W + (size_t)s * n2, n2, row);
    __syncthreads();
    cpx<R> pv = mk(R(0), R(0));
    R pr_re = R(0), pr_im = R(0), pp = R(0);
    if (live && par == 0) {
      pv = blk_row<R>(Dc + (size_t)X * 9 * NN, U + (size_t)s * n2, n2, row) - hop_in(Z);
      const cpx<R> rs = U[t];
      pr_re = pv.re * rs.re + pv.im * rs.im;       // <p, res> = sum conj(p) res
      pr_im = pv.re * rs.im - pv.im * rs.re;
      pp = pv.re * pv.re + pv.im * pv.im;
    }
    cta_sum3<R>(pr_re, pr_im, pp, red);
    const bool ok = pp > (sizeof(R) == 8 ? R(2.2250738585072014e-308) : R(1.17549435e-38));
    const cpx<R> alpha = ok ? mk(pr_re / pp, pr_im / pp) : mk(R(0), R(0));
    if (live && par == 0) {
      E[t] = E[t] + alpha * U[t];
      U[t] = U[t] - alpha * pv;
    }
    __syncthreads();
  }
  if (live && par == 1) W[t] = Rr[t] - hop_in(E);
  __syncthreads();
  if (live && par == 1) E[t] = blk_row<R>(Ainv + (size_t)X * NN, W + (size_t)s * n2, n2, row);
  if (live) {
    const size_t o = (size_t)X * n2 + row;
    x[o] = x_is_zero ? E[t] : x[o] + E[t];
  }
}

// b2[r][X'][s n2v + i] = sum over the sites x of X' and c < n1 of
// conj(lam2[i][x][s n1 + c]) v[r][x][s n1 + c]   (Eq. 3 on level 2)
template <class R>
__global__ void k_l2_restrict(L2Geom d, const cpx<R>* __restrict__ lam2, int n1, int n2v,
                              const cpx<R>* __restrict__ v, cpx<R>* __restrict__ b2) {
  extern __shared__ __align__(16) unsigned char l2sh[];
  cpx<R>* part = reinterpret_cast<cpx<R>*>(l2sh);
  const int Xp = blockIdx.x, O = 2 * n2v, Q = blockDim.x / O;
  const int n2 = 2 * n1, E = d.Vb * n1;
  v += (size_t)blockIdx.y * d.NX * n2;
  const int o = threadIdx.x % O, q = threadIdx.x / O;
  if (q < Q) {
    const int s = o / n2v, i = o - s * n2v;
    cpx<R> acc = mk(R(0), R(0));
    for (int e = q; e < E; e += Q) {
      const int k = e / n1, c = e - k * n1;
      const int X = d.sites[(size_t)Xp * d.Vb + k];
      const size_t a = (size_t)X * n2 + s * n1 + c;
      fmac(acc, lam2[(size_t)i * d.NX * n2 + a], v[a]);
    }
    part[q * O + o] = acc;
  }
  __syncthreads();
  if (threadIdx.x < O) {
    cpx<R> acc = mk(R(0), R(0));
    for (int qq = 0; qq < Q; ++qq) acc = acc + part[qq * O + threadIdx.x];
    b2[((size_t)blockIdx.y * d.NXp + Xp) * O + threadIdx.x] = acc;
  }
}

// x[r][x][s n1 + c] (+)= sum_i x2[r][X'(x)][s n2v + i] lam2[i][x][s n1 + c]   (Eq. 4)
template <class R>
__global__ void k_l2_prolong(L2Geom d, const cpx<R>* __restrict__ lam2, int n1, int n2v,
                             const cpx<R>* __restrict__ x2, cpx<R>* __restrict__ x, int accumulate) {
  const int n2 = 2 * n1;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)d.NX * n2) return;
  const int X = (int)(idx / n2), a = (int)(idx - (size_t)X * n2);
  const int s = a / n1;
  const cpx<R>* c2 = x2 + ((size_t)blockIdx.y * d.NXp + d.blk[X]) * 2 * n2v + s * n2v;
  cpx<R> acc = mk(R(0), R(0));
  for (int i = 0; i < n2v; ++i) fma(acc, c2[i], lam2[((size_t)i * d.NX + X) * n2 + a]);
  cpx<R>* out = x + (size_t)blockIdx.y * d.NX * n2 + idx;
  *out = accumulate ? *out + acc : acc;
}

// classical Gram-Schmidt, twice, of the n2v vectors inside (aggregate X',
// chirality s = blockIdx.y), i = 0 .. n2v - 1, in FP64: CTA per (X', s),
// thread per element (site of X', component c < n1)
__global__ void k_l2_ortho(L2Geom d, cpx<double>* __restrict__ lam2, int n1, int n2v) {
  extern __shared__ __align__(16) unsigned char l2sh[];
  const int nw = (blockDim.x + 31) >> 5, w = threadIdx.x >> 5, l = threadIdx.x & 31;
  double* red = reinterpret_cast<double*>(l2sh);             // [warps][n2v][2]
  double* coef = red + (size_t)nw * n2v * 2;                 // [n2v][2]
  double* red3 = coef + 2 * n2v;                             // [3 * warps]
  const int Xp = blockIdx.x, s = blockIdx.y, n2 = 2 * n1;
  const int e = threadIdx.x;
  const bool live = e < d.Vb * n1;
  size_t a = 0;
  if (live) {
    const int k = e / n1, c = e - k * n1;
    a = (size_t)d.sites[(size_t)Xp * d.Vb + k] * n2 + s * n1 + c;
  }
  const size_t vs = (size_t)d.NX * n2;
  for (int i = 0; i < n2v; ++i) {
    cpx<double> v = live ? lam2[(size_t)i * vs + a] : mk(0.0, 0.0);
    for (int pass = 0; pass < 2 && i > 0; ++pass) {
      for (int j = 0; j < i; ++j) {
        double re = 0.0, im = 0.0;
        if (live) {
          const cpx<double> u = lam2[(size_t)j * vs + a];
          re = u.re * v.re + u.im * v.im;
          im = u.re * v.im - u.im * v.re;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          re += __shfl_xor_sync(0xffffffffu, re, o);
          im += __shfl_xor_sync(0xffffffffu, im, o);
        }
        if (l == 0) { red[(w * n2v + j) * 2] = re; red[(w * n2v + j) * 2 + 1] = im; }
      }
      __syncthreads();
      if (threadIdx.x < i) {
        double re = 0.0, im = 0.0;
        for (int ww = 0; ww < nw; ++ww) { re += red[(ww * n2v + threadIdx.x) * 2]; im += red[(ww * n2v + threadIdx.x) * 2 + 1]; }
        coef[2 * threadIdx.x] = re;
        coef[2 * threadIdx.x + 1] = im;
      }
      __syncthreads();
      if (live)
        for (int j = 0; j < i; ++j) {
          const cpx<double> u = lam2[(size_t)j * vs + a];
          v = v - mk(coef[2 * j], coef[2 * j + 1]) * u;
        }
      __syncthreads();
    }
    double nn = live ? v.re * v.re + v.im * v.im : 0.0, z0 = 0.0, z1 = 0.0;
    cta_sum3<double>(nn, z0, z1, red3);
    const double f = 1.0 / sqrt(nn);
    if (live) lam2[(size_t)i * vs + a] = mk(v.re * f, v.im * f);
    __syncthreads();
  }
}

// D_cc[X'][T] (Eq. 2 on level 2): for every site x of X' and term d of the
// coarse stencil (y its neighbour), W_t[j] = D_c[x][d] P_t lam2_j(y) and
// G[s n2v + i][t n2v + j] += <P_s lam2_i(x) | W_t[j]>; the self term and links
// that stay inside X' go to block T = 0, a link that leaves X' to T = d.
// CTA per aggregate; blocks accumulated in shared memory, column-major.
template <class R>
__global__ void k_l2_assemble(L2Geom d, const cpx<R>* __restrict__ Dc, const cpx<R>* __restrict__ lam2, int n1,
                              int n2v, cpx<R>* __restrict__ Dcc) {
  extern __shared__ __align__(16) unsigned char l2sh[];
  const int n2 = 2 * n1, m2 = 2 * n2v, NE2 = m2 * m2;
  cpx<R>* Acc = reinterpret_cast<cpx<R>*>(l2sh);             // [9][NE2]
  cpx<R>* W = Acc + 9 * NE2;                                 // [2][n2v][n2]
  const int Xp = blockIdx.x;
  const size_t NN = (size_t)n2 * n2, vs = (size_t)d.NX * n2;
  for (int e = threadIdx.x; e < 9 * NE2; e += blockDim.x) Acc[e] = mk(R(0), R(0));
  for (int k = 0; k < d.Vb; ++k) {
    const int X = d.sites[(size_t)Xp * d.Vb + k];
    for (int dd = 0; dd < 9; ++dd) {
      const int Y = d.cnbr[dd * d.NX + X];
      const int T = (dd == 0 || d.blk[Y] == Xp) ? 0 : dd;
      const cpx<R>* M = Dc + ((size_t)X * 9 + dd) * NN;
      __syncthreads();               // the previous term's W is consumed
      for (int idx = threadIdx.x; idx < 2 * n2v * n2; idx += blockDim.x) {
        const int t = idx / (n2v * n2), rem = idx - t * n2v * n2, j = rem / n2, a = rem - j * n2;
        const cpx<R>* lj = lam2 + (size_t)j * vs + (size_t)Y * n2;
        cpx<R> acc = mk(R(0), R(0));
        for (int bb = 0; bb < n1; ++bb) {
          const int bcol = t * n1 + bb;
          fma(acc, M[(size_t)bcol * n2 + a], lj[bcol]);
        }
        W[idx] = acc;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < NE2; e += blockDim.x) {
        const int col = e / m2, rw = e - col * m2;
        const int s = rw / n2v, i = rw - s * n2v, t = col / n2v, j = col - t * n2v;
        const cpx<R>* li = lam2 + (size_t)i * vs + (size_t)X * n2 + s * n1;
        const cpx<R>* wt = W + (size_t)(t * n2v + j) * n2 + s * n1;
        cpx<R> acc = mk(R(0), R(0));
        for (int aa = 0; aa < n1; ++aa) fmac(acc, li[aa], wt[aa]);
        Acc[T * NE2 + e] = Acc[T * NE2 + e] + acc;
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 9 * NE2; e += blockDim.x) Dcc[(size_t)Xp * 9 * NE2 + e] = Acc[e];
}

inline unsigned nblk(size_t n, int tpb) { return (unsigned)((n + tpb - 1) / tpb); }

}  // namespace

template <class R>
cudaError_t l2_sap_sweep(const L2Geom& d, const R* Dc, const R* Ainv, int n1, int colour, int mr_iters,
                         bool x_is_zero, const R* b, R* x, int nrhs, cudaStream_t st) {
  const int n2 = 2 * n1, threads = ((d.Vb * n2 + 31) / 32) * 32;
  if (threads > 1024 || d.NXp % 2) return cudaErrorInvalidValue;
  const size_t smem = (size_t)5 * d.Vb * n2 * sizeof(cpx<R>) + 3 * 32 * sizeof(R);
  cudaError_t e = raise_smem_limit((const void*)k_l2_sap<R>, smem);
  if (e != cudaSuccess) return e;
  k_l2_sap<R><<<dim3(d.NXp / 2, nrhs), threads, smem, st>>>(
      d, reinterpret_cast<const cpx<R>*>(Dc), reinterpret_cast<const cpx<R>*>(Ainv), n2, colour, mr_iters,
      x_is_zero ? 1 : 0, reinterpret_cast<const cpx<R>*>(b), reinterpret_cast<cpx<R>*>(x));
  ++g_launches;
  return cudaGetLastError();
}

template <class R>
cudaError_t l2_restrict(const L2Geom& d, const R* lam2, int n1, int n2v, const R* v, R* b2, int nrhs,
                        cudaStream_t st) {
  const int O = 2 * n2v;
  if (O > 256) return cudaErrorInvalidValue;
  const int threads = 256;
  const size_t smem = (size_t)(threads / O) * O * sizeof(cpx<R>);
  k_l2_restrict<R><<<dim3(d.NXp, nrhs), threads, smem, st>>>(d, reinterpret_cast<const cpx<R>*>(lam2), n1, n2v,
                                                            reinterpret_cast<const cpx<R>*>(v),
                                                            reinterpret_cast<cpx<R>*>(b2));
  ++g_launches;
  return cudaGetLastError();
}

template <class R>
cudaError_t l2_prolong(const L2Geom& d, const R* lam2, int n1, int n2v, const R* x2, R* x, int nrhs, bool accumulate,
                       cudaStream_t st) {
  k_l2_prolong<R><<<dim3(nblk((size_t)d.NX * 2 * n1, 128), nrhs), 128, 0, st>>>(
      d, reinterpret_cast<const cpx<R>*>(lam2), n1, n2v, reinterpret_cast<const cpx<R>*>(x2),
      reinterpret_cast<cpx<R>*>(x), accumulate ? 1 : 0);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t l2_orthonormalise(const L2Geom& d, double* lam2, int n1, int n2v, cudaStream_t st) {
  const int threads = ((d.Vb * n1 + 31) / 32) * 32;
  if (threads > 1024) return cudaErrorInvalidValue;
  const size_t smem = ((size_t)(threads / 32) * n2v * 2 + 2 * n2v + 3 * 32) * sizeof(double);
  k_l2_ortho<<<dim3(d.NXp, 2), threads, smem, st>>>(d, reinterpret_cast<cpx<double>*>(lam2), n1, n2v);
  ++g_launches;
  return cudaGetLastError();
}

template <class R>
cudaError_t l2_assemble(const L2Geom& d, const R* Dc, const R* lam2, int n1, int n2v, R* Dcc, cudaStream_t st) {
  const size_t smem = ((size_t)9 * 4 * n2v * n2v + (size_t)2 * n2v * 2 * n1) * sizeof(cpx<R>);
  cudaError_t e = raise_smem_limit((const void*)k_l2_assemble<R>, smem);
  if (e != cudaSuccess) return e;
  k_l2_assemble<R><<<d.NXp, 256, smem, st>>>(d, reinterpret_cast<const cpx<R>*>(Dc),
                                              reinterpret_cast<const cpx<R>*>(lam2), n1, n2v,
                                              reinterpret_cast<cpx<R>*>(Dcc));
  ++g_launches;
  return cudaGetLastError();
}

size_t l2_assemble_smem(int n1, int n2v, int real_size) {
  return ((size_t)9 * 4 * n2v * n2v + (size_t)2 * n2v * 2 * n1) * 2 * real_size;
}

#define INST_L2(R)                                                                                               \
  template cudaError_t l2_sap_sweep<R>(const L2Geom&, const R*, const R*, int, int, int, bool, const R*, R*, int, \
                                       cudaStream_t);                                                            \
  template cudaError_t l2_restrict<R>(const L2Geom&, const R*, int, int, const R*, R*, int, cudaStream_t);       \
  template cudaError_t l2_prolong<R>(const L2Geom&, const R*, int, int, const R*, R*, int, bool, cudaStream_t);  \
  template cudaError_t l2_assemble<R>(const L2Geom&, const R*, const R*, int, int, R*, cudaStream_t);

INST_L2(float)
INST_L2(double)
#undef INST_L2

}  // namespace ddamg
