// Fine-lattice kernels: layout conversion, gauge import, clover term and its
// inverse, the Wilson-clover stencil, BLAS-1 reductions, random vectors.
//
// Wilson-clover operator (paper Sec. 1 and 3; formula in include/ddamg.h):
//   D x = A x - 1/2 sum_mu [(1-g_mu) U_mu(x) x(x+mu) + (1+g_mu) U_mu(x-mu)^H x(x-mu)]
// with A = (4 + m0) + C stored as two packed Hermitian 6x6 chiral blocks.
#include "common.cuh"
#include "kernels.h"

#include <map>
#include <mutex>

namespace ddamg {

LaunchCount g_launches;

cudaError_t raise_smem_limit(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> limit;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = limit[{dev, fn}];
  if (cur >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

namespace {

constexpr int TPB = 128;

inline unsigned nblk(size_t n, int tpb) { return (unsigned)((n + tpb - 1) / tpb); }

// ---------------------------------------------------------------------------
// layout conversion
// ---------------------------------------------------------------------------
template <class R>
__global__ void k_pack_spinor(Geom g, const double* __restrict__ lex, R* __restrict__ dev) {
  int d = blockIdx.x * blockDim.x + threadIdx.x;
  int rhs = blockIdx.y;
  if (d >= g.V) return;
  int x = g.lex_of_dev[d];
  const double* src = lex + ((size_t)rhs * g.V + x) * SPINOR_NR;
  R v[SPINOR_NR];
#pragma unroll
  for (int k = 0; k < SPINOR_NR; ++k) v[k] = (R)src[k];
  store_site<R, SPINOR_NR>(dev + (size_t)rhs * g.V * SPINOR_NR, d, g.Vb, v);
}

template <class R>
__global__ void k_unpack_spinor(Geom g, const R* __restrict__ dev, double* __restrict__ lex) {
  int d = blockIdx.x * blockDim.x + threadIdx.x;
  int rhs = blockIdx.y;
  if (d >= g.V) return;
  int x = g.lex_of_dev[d];
  R v[SPINOR_NR];
  load_site<R, SPINOR_NR>(dev + (size_t)rhs * g.V * SPINOR_NR, d, g.Vb, v);
  double* dst = lex + ((size_t)rhs * g.V + x) * SPINOR_NR;
#pragma unroll
  for (int k = 0; k < SPINOR_NR; ++k) dst[k] = (double)v[k];
}

// spinor fields of different precision have different unit widths, so the
// conversion goes site by site through the layout
template <class RD, class RS>
__global__ void k_convert_spinor(Geom g, const RS* __restrict__ s, RD* __restrict__ d) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= g.V) return;
  size_t off = (size_t)blockIdx.y * g.V * SPINOR_NR;
  RS v[SPINOR_NR];
  load_site<RS, SPINOR_NR>(s + off, x, g.Vb, v);
  RD w[SPINOR_NR];
#pragma unroll
  for (int k = 0; k < SPINOR_NR; ++k) w[k] = (RD)v[k];
  store_site<RD, SPINOR_NR>(d + off, x, g.Vb, w);
}

template <class RD, class RS>
__global__ void k_convert(const RS* __restrict__ s, RD* __restrict__ d, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) d[i] = (RD)s[i];
}

// ---------------------------------------------------------------------------
// 3x3 complex helpers (FP64, setup only)
// ---------------------------------------------------------------------------
using c64 = cpx<double>;
struct M3 {
  c64 a[3][3];
};

__device__ __forceinline__ M3 ld_lex_link(const double* __restrict__ lex, int site, int mu) {
  M3 U;
  const double* p = lex + ((size_t)site * 4 + mu) * 18;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) U.a[i][j] = mk(p[(i * 3 + j) * 2], p[(i * 3 + j) * 2 + 1]);
  return U;
}
__device__ __forceinline__ M3 mul(const M3& A, const M3& B) {
  M3 C;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      c64 s = A.a[i][0] * B.a[0][j];
      fma(s, A.a[i][1], B.a[1][j]);
      fma(s, A.a[i][2], B.a[2][j]);
      C.a[i][j] = s;
    }
  return C;
}
__device__ __forceinline__ M3 dag(const M3& A) {
  M3 C;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) C.a[i][j] = conj(A.a[j][i]);
  return C;
}
__device__ __forceinline__ M3 add(const M3& A, const M3& B) {
  M3 C;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) C.a[i][j] = A.a[i][j] + B.a[i][j];
  return C;
}

__device__ __forceinline__ int lex_shift(int site, int mu, int step, const int* L) {
  int c[4];
  int r = site;
  c[0] = r % L[0]; r /= L[0];
  c[1] = r % L[1]; r /= L[1];
  c[2] = r % L[2]; r /= L[2];
  c[3] = r;
  c[mu] = (c[mu] + step + L[mu]) % L[mu];
  return c[0] + L[0] * (c[1] + L[1] * (c[2] + L[2] * c[3]));
}

// B_mu of g_mu = [[0, B], [B^H, 0]]
__device__ __forceinline__ c64 Bmat(int mu, int r, int c) {
  // x: [[0,-i],[-i,0]]  y: [[0,-1],[1,0]]  z: [[-i,0],[0,i]]  t: [[1,0],[0,1]]
  if (mu == 0) return (r != c) ? mk(0.0, -1.0) : mk(0.0, 0.0);
  if (mu == 1) return (r == c) ? mk(0.0, 0.0) : (r == 0 ? mk(-1.0, 0.0) : mk(1.0, 0.0));
  if (mu == 2) return (r != c) ? mk(0.0, 0.0) : (r == 0 ? mk(0.0, -1.0) : mk(0.0, 1.0));
  return (r == c) ? mk(1.0, 0.0) : mk(0.0, 0.0);
}

// Gauss-Jordan inverse with partial pivoting of an N x N complex matrix
template <int N>
__device__ bool gj_invert(c64 (&a)[N][N], c64 (&inv)[N][N]) {
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) inv[i][j] = mk(i == j ? 1.0 : 0.0, 0.0);
  for (int col = 0; col < N; ++col) {
    int piv = col;
    double best = norm2(a[col][col]);
    for (int r = col + 1; r < N; ++r) {
      double v = norm2(a[r][col]);
      if (v > best) { best = v; piv = r; }
    }
    if (best == 0.0) return false;
    if (piv != col) {
      for (int j = 0; j < N; ++j) {
        c64 t = a[col][j]; a[col][j] = a[piv][j]; a[piv][j] = t;
        t = inv[col][j]; inv[col][j] = inv[piv][j]; inv[piv][j] = t;
      }
    }
    c64 p = a[col][col];
    double pn = norm2(p);
    c64 pi = mk(p.re / pn, -p.im / pn);
    for (int j = 0; j < N; ++j) {
      a[col][j] = a[col][j] * pi;
      inv[col][j] = inv[col][j] * pi;
    }
    for (int r = 0; r < N; ++r) {
      if (r == col) continue;
      c64 f = a[r][col];
      if (f.re == 0.0 && f.im == 0.0) continue;
      for (int j = 0; j < N; ++j) {
        a[r][j] = a[r][j] - f * a[col][j];
        inv[r][j] = inv[r][j] - f * inv[col][j];
      }
    }
  }
  return true;
}

template <class R>
__device__ __forceinline__ void store_packed(R* f, int d, int Vb, const double (&P)[CLOVER_NR]) {
  R v[CLOVER_NR];
#pragma unroll
  for (int k = 0; k < CLOVER_NR; ++k) v[k] = (R)P[k];
  store_site<R, CLOVER_NR>(f, d, Vb, v);
}

__device__ __forceinline__ void pack6(const c64 (&m)[6][6], double* P) {
  for (int i = 0; i < 6; ++i) P[i] = m[i][i].re;
  int k = 0;
  for (int i = 0; i < 6; ++i)
    for (int j = i + 1; j < 6; ++j) {
      P[6 + 2 * k] = m[i][j].re;
      P[7 + 2 * k] = m[i][j].im;
      ++k;
    }
}

// ---------------------------------------------------------------------------
// gauge import: two rows of each link in both precisions + SU(3) check
// ---------------------------------------------------------------------------
__global__ void k_import_gauge(Geom g, const double* __restrict__ lex, double* __restrict__ g64,
                               float* __restrict__ g32, unsigned long long* dev_dev) {
  int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= g.V) return;
  int x = g.lex_of_dev[d];
  double v64[GAUGE_NR];
  double worst = 0.0;
  for (int mu = 0; mu < 4; ++mu) {
    M3 U = ld_lex_link(lex, x, mu);
    // unitarity
    M3 UU = mul(U, dag(U));
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        c64 e = UU.a[i][j] - mk(i == j ? 1.0 : 0.0, 0.0);
        worst = fmax(worst, sqrt(norm2(e)));
      }
    c64 det = U.a[0][0] * (U.a[1][1] * U.a[2][2] - U.a[1][2] * U.a[2][1]) -
              U.a[0][1] * (U.a[1][0] * U.a[2][2] - U.a[1][2] * U.a[2][0]) +
              U.a[0][2] * (U.a[1][0] * U.a[2][1] - U.a[1][1] * U.a[2][0]);
    worst = fmax(worst, sqrt(norm2(det - mk(1.0, 0.0))));
    if (!(worst == worst)) worst = 1e300;   // NaN
    for (int k = 0; k < 6; ++k) {
      v64[mu * 12 + 2 * k] = U.a[k / 3][k % 3].re;
      v64[mu * 12 + 2 * k + 1] = U.a[k / 3][k % 3].im;
    }
  }
  store_site<double, GAUGE_NR>(g64, d, g.Vb, v64);
  float v32[GAUGE_NR];
  for (int k = 0; k < GAUGE_NR; ++k) v32[k] = (float)v64[k];
  store_site<float, GAUGE_NR>(g32, d, g.Vb, v32);
  atomicMax(dev_dev, (unsigned long long)__double_as_longlong(worst));
}

// ---------------------------------------------------------------------------
// clover term C = -(csw/16) sum_{mu<nu} g_mu g_nu (x) (Q_munu - Q_munu^H),
// chiral blocks: g_mu g_nu = diag(B_mu B_nu^H, B_mu^H B_nu)
// ---------------------------------------------------------------------------
__global__ void k_build_clover(Geom g, const double* __restrict__ lex, double m0, double csw,
                               double* A64, double* Ai64, float* A32, float* Ai32) {
  int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= g.V) return;
  int x = g.lex_of_dev[d];
  c64 blk[2][6][6];
  for (int s = 0; s < 2; ++s)
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) blk[s][i][j] = mk(0.0, 0.0);
  const double coef = -csw / 16.0;
  for (int mu = 0; mu < 4; ++mu) {
    for (int nu = mu + 1; nu < 4; ++nu) {
      int xpm = lex_shift(x, mu, 1, g.L), xpn = lex_shift(x, nu, 1, g.L);
      int xmm = lex_shift(x, mu, -1, g.L), xmn = lex_shift(x, nu, -1, g.L);
      int xmm_pn = lex_shift(xmm, nu, 1, g.L), xmm_mn = lex_shift(xmm, nu, -1, g.L);
      int xmn_pm = lex_shift(xmn, mu, 1, g.L);
      M3 Umx = ld_lex_link(lex, x, mu), Unx = ld_lex_link(lex, x, nu);
      M3 l1 = mul(mul(Umx, ld_lex_link(lex, xpm, nu)), mul(dag(ld_lex_link(lex, xpn, mu)), dag(Unx)));
      M3 Umm = ld_lex_link(lex, xmm, mu);
      M3 l2 = mul(mul(Unx, dag(ld_lex_link(lex, xmm_pn, mu))),
                  mul(dag(ld_lex_link(lex, xmm, nu)), Umm));
      M3 l3 = mul(mul(dag(Umm), dag(ld_lex_link(lex, xmm_mn, nu))),
                  mul(ld_lex_link(lex, xmm_mn, mu), ld_lex_link(lex, xmn, nu)));
      M3 Unm = ld_lex_link(lex, xmn, nu);
      M3 l4 = mul(mul(dag(Unm), ld_lex_link(lex, xmn, mu)),
                  mul(ld_lex_link(lex, xmn_pm, nu), dag(Umx)));
      M3 Q = add(add(l1, l2), add(l3, l4));
      M3 Qd = dag(Q);
      for (int s = 0; s < 2; ++s) {
        for (int si = 0; si < 2; ++si)
          for (int sj = 0; sj < 2; ++sj) {
            // G^+ = B_mu B_nu^H, G^- = B_mu^H B_nu
            c64 G = mk(0.0, 0.0);
            for (int k = 0; k < 2; ++k) {
              if (s == 0) G = G + Bmat(mu, si, k) * conj(Bmat(nu, sj, k));
              else        G = G + conj(Bmat(mu, k, si)) * Bmat(nu, k, sj);
            }
            if (G.re == 0.0 && G.im == 0.0) continue;
            G = coef * G;
            for (int a = 0; a < 3; ++a)
              for (int b = 0; b < 3; ++b)
                blk[s][si * 3 + a][sj * 3 + b] =
                    blk[s][si * 3 + a][sj * 3 + b] + G * (Q.a[a][b] - Qd.a[a][b]);
          }
      }
    }
  }
  double PA[CLOVER_NR], PI[CLOVER_NR];
  for (int s = 0; s < 2; ++s) {
    c64 a[6][6], inv[6][6];
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) a[i][j] = blk[s][i][j] + mk(i == j ? 4.0 + m0 : 0.0, 0.0);
    pack6(a, PA + 36 * s);
    if (!gj_invert<6>(a, inv)) {
      for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) inv[i][j] = mk(__longlong_as_double(0x7ff8000000000000ll), 0.0);
    }
    pack6(inv, PI + 36 * s);
  }
  store_packed<double>(A64, d, g.Vb, PA);
  store_packed<double>(Ai64, d, g.Vb, PI);
  store_packed<float>(A32, d, g.Vb, PA);
  store_packed<float>(Ai32, d, g.Vb, PI);
}

__global__ void k_export_clover(Geom g, const double* __restrict__ dev, double* __restrict__ lex) {
  int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= g.V) return;
  double v[CLOVER_NR];
  load_site<double, CLOVER_NR>(dev, d, g.Vb, v);
  double* dst = lex + (size_t)g.lex_of_dev[d] * CLOVER_NR;
  for (int k = 0; k < CLOVER_NR; ++k) dst[k] = v[k];
}

// ---------------------------------------------------------------------------
// Wilson-clover stencil, one thread per site
// ---------------------------------------------------------------------------
template <class R, int MODE>
__global__ void __launch_bounds__(TPB) k_dslash(Geom g, const R* __restrict__ x,
                                                const R* __restrict__ b, R* __restrict__ y,
                                                const R* __restrict__ gauge,
                                                const R* __restrict__ clover) {
  int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= g.V) return;
  size_t off = (size_t)blockIdx.y * g.V * SPINOR_NR;
  x += off;
  y += off;
  Spinor<R> out;
  {
    Spinor<R> xs;
    load_spinor<R>(x, d, g.Vb, xs);
    clover_mul<R>(clover, d, g.Vb, xs, out);
  }
  if (MODE != DSLASH_CLOVER) {
    Spinor<R> acc;
#pragma unroll
    for (int k = 0; k < 12; ++k) acc.c[k] = mk(R(0), R(0));
    hop_dir<0>(g, x, gauge, d, acc);
    hop_dir<1>(g, x, gauge, d, acc);
    hop_dir<2>(g, x, gauge, d, acc);
    hop_dir<3>(g, x, gauge, d, acc);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      out.c[k].re = fma_r(R(-0.5), acc.c[k].re, out.c[k].re);
      out.c[k].im = fma_r(R(-0.5), acc.c[k].im, out.c[k].im);
    }
  }
  if (MODE == DSLASH_RES) {
    Spinor<R> bs;
    load_spinor<R>(b + off, d, g.Vb, bs);
#pragma unroll
    for (int k = 0; k < 12; ++k) out.c[k] = bs.c[k] - out.c[k];
  }
  store_spinor<R>(y, d, g.Vb, out);
}

// ---------------------------------------------------------------------------
// BLAS-1: deterministic two-pass reductions
// ---------------------------------------------------------------------------
constexpr int RED_CTAS = 304;   // 2 x 152 SMs
constexpr int RED_TPB = 256;
constexpr int MAXK = 64;

template <class R>
struct PtrList {
  const R* p[MAXK];
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block sum of (a, b) pairs; result valid in thread 0
__device__ __forceinline__ void block_sum2(double& a, double& b, double* sh) {
  a = warp_sum(a);
  b = warp_sum(b);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sh[2 * w] = a; sh[2 * w + 1] = b; }
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    a = (l < nw) ? sh[2 * l] : 0.0;
    b = (l < nw) ? sh[2 * l + 1] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
  }
  __syncthreads();
}

// FP64 arithmetic is the scarce resource of these kernels (GB300 issues two
// FP64 lanes per clock per SM against 128 FP32 lanes), so they are written to
// spend it on the products: vectors are taken in groups of DOT_J, each
// thread sums many elements before any cross-thread step, and the CTA
// reduction transposes the partial sums through shared memory so that every
// value is reduced by one warp instead of every warp reducing every value.
constexpr int DOT_J = 4;

// acc[2 jj + (0, 1)] += <v_{j0 + jj}, w> over this thread's elements, jj < NJ
template <class R, int NJ>
__device__ __forceinline__ void dot_group(const PtrList<R>& v, int j0, const cpx<R>* __restrict__ wc, size_t lo,
                                          size_t hi, double (&acc)[2 * DOT_J]) {
  for (size_t i = lo + threadIdx.x; i < hi; i += RED_TPB) {
    const cpx<R> b = wc[i];
    const double br = (double)b.re, bi = (double)b.im;
#pragma unroll
    for (int jj = 0; jj < NJ; ++jj) {
      const cpx<R> a = reinterpret_cast<const cpx<R>*>(v.p[j0 + jj])[i];
      const double ar = (double)a.re, ai = (double)a.im;
      acc[2 * jj] = ::fma(ar, br, ::fma(ai, bi, acc[2 * jj]));
      acc[2 * jj + 1] = ::fma(ar, bi, ::fma(-ai, br, acc[2 * jj + 1]));
    }
  }
}

// right-hand side r = blockIdx.y of a batch: vectors and w start r * rstride
// complex numbers further, its partial sums k * gridDim.x slots further
template <class R>
__global__ void __launch_bounds__(RED_TPB) k_multi_dot_partial(PtrList<R> v, int k,
                                                               const R* __restrict__ w, size_t n,
                                                               double* __restrict__ part, size_t rstride) {
  __shared__ double sh[2 * DOT_J][RED_TPB];
  const size_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const size_t lo = blockIdx.x * chunk;
  const size_t hi = lo + chunk < n ? lo + chunk : n;
  const size_t roff = blockIdx.y * rstride;
  if (roff)
    for (int j = 0; j < k; ++j) v.p[j] += 2 * roff;
  part += (size_t)blockIdx.y * k * gridDim.x * 2;
  const cpx<R>* wc = reinterpret_cast<const cpx<R>*>(w) + roff;
  const int t = threadIdx.x, wid = t >> 5, lane = t & 31;
  for (int j0 = 0; j0 < k; j0 += DOT_J) {
    const int nj = k - j0 < DOT_J ? k - j0 : DOT_J;
    double acc[2 * DOT_J];
#pragma unroll
    for (int q = 0; q < 2 * DOT_J; ++q) acc[q] = 0.0;
    static_assert(DOT_J == 4, "the dispatch below covers groups of up to four");
    switch (nj) {
      case 4: dot_group<R, 4>(v, j0, wc, lo, hi, acc); break;
      case 3: dot_group<R, 3>(v, j0, wc, lo, hi, acc); break;
      case 2: dot_group<R, 2>(v, j0, wc, lo, hi, acc); break;
      default: dot_group<R, 1>(v, j0, wc, lo, hi, acc); break;
    }
#pragma unroll
    for (int q = 0; q < 2 * DOT_J; ++q) sh[q][t] = acc[q];
    __syncthreads();
    for (int q = wid; q < 2 * nj; q += RED_TPB / 32) {
      double sum = 0.0;
#pragma unroll
      for (int u = 0; u < RED_TPB / 32; ++u) sum += sh[q][lane + 32 * u];
      sum = warp_sum(sum);
      if (lane == 0) part[((size_t)(j0 + (q >> 1)) * gridDim.x + blockIdx.x) * 2 + (q & 1)] = sum;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(RED_TPB) k_reduce_final(const double* __restrict__ part, int ncta,
                                                          double* __restrict__ out) {
  __shared__ double sh[2 * (RED_TPB / 32)];
  int j = blockIdx.x;
  double re = 0.0, im = 0.0;
  for (int i = threadIdx.x; i < ncta; i += blockDim.x) {
    re += part[((size_t)j * ncta + i) * 2];
    im += part[((size_t)j * ncta + i) * 2 + 1];
  }
  block_sum2(re, im, sh);
  if (threadIdx.x == 0) {
    out[2 * j] = re;
    out[2 * j + 1] = im;
  }
}

// w -= sum_j coef_j v_j (coef scaled by sign); with part != nullptr also the
// CTA partial sums of ||w_new||^2 (slot layout of k_multi_dot_partial, k = 1)
// batched as k_multi_dot_partial: right-hand side r = blockIdx.y takes its
// coefficients r * cstride doubles further and its norm partials gridDim.x
// slots further
template <class R>
__global__ void __launch_bounds__(RED_TPB) k_multi_axpy(PtrList<R> v, int k, const double* __restrict__ coef,
                                                        double sign, R* __restrict__ w, size_t n,
                                                        double* __restrict__ part, size_t rstride, int cstride) {
  __shared__ double cs[2 * MAXK];            // signed coefficients, loaded once per CTA
  __shared__ double sh[RED_TPB / 32];
  coef += (size_t)blockIdx.y * cstride;
  for (int j = threadIdx.x; j < 2 * k; j += blockDim.x) cs[j] = sign * coef[j];
  __syncthreads();
  const size_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const size_t lo = blockIdx.x * chunk;
  const size_t hi = lo + chunk < n ? lo + chunk : n;
  const size_t roff = blockIdx.y * rstride;
  if (roff)
    for (int j = 0; j < k; ++j) v.p[j] += 2 * roff;
  if (part) part += (size_t)blockIdx.y * gridDim.x * 2;
  cpx<R>* wc = reinterpret_cast<cpx<R>*>(w) + roff;
  double nn = 0.0;
  for (size_t i = lo + threadIdx.x; i < hi; i += RED_TPB) {
    double re = (double)wc[i].re, im = (double)wc[i].im;
    int j = 0;
    for (; j + 4 <= k; j += 4) {
      cpx<R> a[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = reinterpret_cast<const cpx<R>*>(v.p[j + u])[i];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const double cr = cs[2 * (j + u)], ci = cs[2 * (j + u) + 1];
        const double ar = (double)a[u].re, ai = (double)a[u].im;
        re = ::fma(cr, ar, ::fma(-ci, ai, re));
        im = ::fma(cr, ai, ::fma(ci, ar, im));
      }
    }
    for (; j < k; ++j) {
      const cpx<R> a = reinterpret_cast<const cpx<R>*>(v.p[j])[i];
      const double cr = cs[2 * j], ci = cs[2 * j + 1];
      const double ar = (double)a.re, ai = (double)a.im;
      re = ::fma(cr, ar, ::fma(-ci, ai, re));
      im = ::fma(cr, ai, ::fma(ci, ar, im));
    }
    const cpx<R> o = mk((R)re, (R)im);
    wc[i] = o;
    if (part) nn = ::fma((double)o.re, (double)o.re, ::fma((double)o.im, (double)o.im, nn));
  }
  if (part) {
    nn = warp_sum(nn);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = nn;
    __syncthreads();
    if (threadIdx.x < 32) {
      double s2 = threadIdx.x < RED_TPB / 32 ? sh[threadIdx.x] : 0.0;
      s2 = warp_sum(s2);
      if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s2;
        part[2 * blockIdx.x + 1] = 0.0;
      }
    }
  }
}

// FP64 spinor fields w += sum_j coef_j v_j with FP32 spinor fields v_j.  The
// two precisions lay a block out in 16-byte units of different width (12
// double2 or 6 float4 per site), so complex component c of local site q of
// block B sits at (B 12 + c) Vb + q in w and at 2 ((B 6 + c / 2) Vb + q) + c % 2
// in v_j.
// (field r = blockIdx.y of a batch: its own coefficients, cstride apart)
__global__ void __launch_bounds__(RED_TPB) k_multi_axpy_f32(PtrList<float> v, int k, const double* __restrict__ coef,
                                                            double sign, double* __restrict__ w, size_t n, int Vb,
                                                            int cstride) {
  __shared__ double cs[2 * MAXK];
  coef += (size_t)blockIdx.y * cstride;
  for (int j = threadIdx.x; j < 2 * k; j += blockDim.x) cs[j] = sign * coef[j];
  __syncthreads();
  const size_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const size_t lo = blockIdx.x * chunk;
  const size_t hi = lo + chunk < n ? lo + chunk : n;
  const size_t roff = (size_t)blockIdx.y * n;          // complex numbers per field
  for (int j = 0; j < k; ++j) v.p[j] += 2 * roff;
  cpx<double>* wc = reinterpret_cast<cpx<double>*>(w) + roff;
  const size_t per_block = (size_t)12 * Vb;
  for (size_t i = lo + threadIdx.x; i < hi; i += RED_TPB) {
    const size_t B = i / per_block;
    const int rem = (int)(i - B * per_block);
    const int c = rem / Vb, q = rem - c * Vb;
    const size_t i32 = 2 * ((B * 6 + (size_t)(c >> 1)) * Vb + q) + (c & 1);
    double re = wc[i].re, im = wc[i].im;
    int j = 0;
    for (; j + 4 <= k; j += 4) {
      cpx<float> a[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = reinterpret_cast<const cpx<float>*>(v.p[j + u])[i32];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const double cr = cs[2 * (j + u)], ci = cs[2 * (j + u) + 1];
        re = ::fma(cr, (double)a[u].re, ::fma(-ci, (double)a[u].im, re));
        im = ::fma(cr, (double)a[u].im, ::fma(ci, (double)a[u].re, im));
      }
    }
    for (; j < k; ++j) {
      const cpx<float> a = reinterpret_cast<const cpx<float>*>(v.p[j])[i32];
      const double cr = cs[2 * j], ci = cs[2 * j + 1];
      re = ::fma(cr, (double)a.re, ::fma(-ci, (double)a.im, re));
      im = ::fma(cr, (double)a.im, ::fma(ci, (double)a.re, im));
    }
    wc[i] = mk(re, im);
  }
}

// y = a x + b y in the field's own precision (FP32 fields stay off the
// narrow FP64 pipe)
template <class R>
__global__ void k_axpby(R a, const R* __restrict__ x, R b, R* __restrict__ y, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) y[i] = a * x[i] + b * y[i];
}

// y = x / sqrt(s) for field r = blockIdx.y of a batch (n reals per field,
// s[2 r]); a zero norm gives y = 0
template <class R>
__global__ void k_scale_inv_norm(const R* __restrict__ x, R* __restrict__ y, const double* s, size_t n) {
  __shared__ double fs;                      // 1/sqrt(s) once per CTA (FP64 division is scarce)
  if (threadIdx.x == 0) {
    const double q = s[2 * blockIdx.y];
    fs = q > 0.0 ? 1.0 / sqrt(q) : 0.0;
  }
  __syncthreads();
  const double f = fs;
  x += (size_t)blockIdx.y * n;
  y += (size_t)blockIdx.y * n;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) y[i] = (R)((double)x[i] * f);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11) and Box-Muller
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
    uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
    uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += W0; k1 += W1;
  }
}

__global__ void k_random_spinors(Geom g, uint64_t seed, int n, double* __restrict__ out) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;   // lexicographic site
  int i = blockIdx.y;                              // vector
  if (x >= g.V) return;
  double* dst = out + ((size_t)i * g.V + x) * SPINOR_NR;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int blk = 0; blk < 6; ++blk) {
    uint32_t c[4] = {(uint32_t)x, (uint32_t)i, (uint32_t)blk, 0u};
    philox(c, k0, k1);
    for (int pr = 0; pr < 2; ++pr) {
      double u1 = ((double)c[2 * pr] + 1.0) * 2.3283064365386963e-10;   // (0, 1]
      double u2 = (double)c[2 * pr + 1] * 2.3283064365386963e-10;       // [0, 1)
      double r = sqrt(-2.0 * log(u1));
      double sn, cs;
      sincospi(2.0 * u2, &sn, &cs);
      dst[blk * 4 + pr * 2] = r * cs;
      dst[blk * 4 + pr * 2 + 1] = r * sn;
    }
  }
}

__global__ void k_index_maps(Geom g, int* parity, int* block, int* colour) {
  int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= g.V) return;
  int x = g.lex_of_dev[d];
  int B = d / g.Vb;
  int q = d - B * g.Vb;
  int bc0 = B % g.grid[0], r = B / g.grid[0];
  int bc1 = r % g.grid[1]; r /= g.grid[1];
  int bc2 = r % g.grid[2];
  int bc3 = r / g.grid[2];
  if (parity) parity[x] = q >= g.Vb / 2 ? 1 : 0;
  if (block) block[x] = B;
  if (colour) colour[x] = (bc0 + bc1 + bc2 + bc3) & 1;
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <class R>
cudaError_t pack_spinor(const Geom& g, const double* lex, R* dev, int nrhs, cudaStream_t st) {
  k_pack_spinor<R><<<dim3(nblk(g.V, TPB), nrhs), TPB, 0, st>>>(g, lex, dev);
  ++g_launches;
  return cudaGetLastError();
}
template <class R>
cudaError_t unpack_spinor(const Geom& g, const R* dev, double* lex, int nrhs, cudaStream_t st) {
  k_unpack_spinor<R><<<dim3(nblk(g.V, TPB), nrhs), TPB, 0, st>>>(g, dev, lex);
  ++g_launches;
  return cudaGetLastError();
}
template <class RD, class RS>
cudaError_t convert_field(const RS* src, RD* dst, size_t nreal, cudaStream_t st) {
  unsigned nb = nblk(nreal, 256);
  if (nb > 4096) nb = 4096;
  if (nb == 0) return cudaSuccess;
  k_convert<RD, RS><<<nb, 256, 0, st>>>(src, dst, nreal);
  ++g_launches;
  return cudaGetLastError();
}

template <class RD, class RS>
cudaError_t convert_spinor(const Geom& g, const RS* src, RD* dst, int nf, cudaStream_t st) {
  k_convert_spinor<RD, RS><<<dim3(nblk(g.V, TPB), nf), TPB, 0, st>>>(g, src, dst);
  ++g_launches;
  return cudaGetLastError();
}
template cudaError_t convert_spinor<float, double>(const Geom&, const double*, float*, int, cudaStream_t);
template cudaError_t convert_spinor<double, float>(const Geom&, const float*, double*, int, cudaStream_t);

cudaError_t import_gauge(const Geom& g, const double* lex, double* g64, float* g32,
                         unsigned long long* dev_dev, cudaStream_t st) {
  k_import_gauge<<<nblk(g.V, TPB), TPB, 0, st>>>(g, lex, g64, g32, dev_dev);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t build_clover(const Geom& g, const double* lex_gauge, double m0, double csw,
                         double* A64, double* Ai64, float* A32, float* Ai32, cudaStream_t st) {
  k_build_clover<<<nblk(g.V, 64), 64, 0, st>>>(g, lex_gauge, m0, csw, A64, Ai64, A32, Ai32);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t export_clover(const Geom& g, const double* dev, double* lex, cudaStream_t st) {
  k_export_clover<<<nblk(g.V, TPB), TPB, 0, st>>>(g, dev, lex);
  ++g_launches;
  return cudaGetLastError();
}

template <class R>
cudaError_t dslash(const Geom& g, int mode, const R* x, const R* b, R* y, const R* gauge,
                   const R* clover, int nrhs, cudaStream_t st) {
  dim3 grid(nblk(g.V, TPB), nrhs);
  if (mode == DSLASH_D)
    k_dslash<R, DSLASH_D><<<grid, TPB, 0, st>>>(g, x, b, y, gauge, clover);
  else if (mode == DSLASH_RES)
    k_dslash<R, DSLASH_RES><<<grid, TPB, 0, st>>>(g, x, b, y, gauge, clover);
  else
    k_dslash<R, DSLASH_CLOVER><<<grid, TPB, 0, st>>>(g, x, b, y, gauge, clover);
  ++g_launches;
  return cudaGetLastError();
}

size_t reduce_scratch_len(int k) { return (size_t)k * RED_CTAS * 2; }

static unsigned batch_ctas(int nb) {
  const int c = RED_CTAS / (nb > 0 ? nb : 1);
  return (unsigned)(c > 0 ? c : 1);
}

template <class R>
cudaError_t multi_dot_batched(const R* const* v, int k, const R* w, size_t n, int nb, size_t rstride,
                              double* scratch, double* out, cudaStream_t st) {
  if (k > MAXK || k < 1 || nb < 1) return cudaErrorInvalidValue;
  PtrList<R> pl;
  for (int j = 0; j < k; ++j) pl.p[j] = v[j];
  const unsigned C = batch_ctas(nb);
  k_multi_dot_partial<R><<<dim3(C, nb), RED_TPB, 0, st>>>(pl, k, w, n, scratch, rstride);
  k_reduce_final<<<nb * k, RED_TPB, 0, st>>>(scratch, (int)C, out);
  g_launches += 2;
  return cudaGetLastError();
}
template <class R>
cudaError_t multi_dot(const R* const* v, int k, const R* w, size_t n, double* scratch, double* out,
                      cudaStream_t st) {
  return multi_dot_batched<R>(v, k, w, n, 1, 0, scratch, out, st);
}
template <class R>
cudaError_t norm2(const R* w, size_t n, double* scratch, double* out, cudaStream_t st) {
  const R* v[1] = {w};
  return multi_dot<R>(v, 1, w, n, scratch, out, st);
}
template <class R>
cudaError_t norm2_batched(const R* w, size_t n, int nb, size_t rstride, double* scratch, double* out,
                          cudaStream_t st) {
  const R* v[1] = {w};
  return multi_dot_batched<R>(v, 1, w, n, nb, rstride, scratch, out, st);
}
template <class R>
cudaError_t multi_axpy_batched(const R* const* v, int k, const double* coef, int cstride, double sign, R* w,
                               size_t n, int nb, size_t rstride, double* scratch, double* norms,
                               cudaStream_t st) {
  if (k > MAXK || k < 1 || nb < 1) return cudaErrorInvalidValue;
  PtrList<R> pl;
  for (int j = 0; j < k; ++j) pl.p[j] = v[j];
  const unsigned C = batch_ctas(nb);
  k_multi_axpy<R><<<dim3(C, nb), RED_TPB, 0, st>>>(pl, k, coef, sign, w, n, norms ? scratch : nullptr, rstride,
                                                   cstride);
  ++g_launches;
  if (norms) {
    k_reduce_final<<<nb, RED_TPB, 0, st>>>(scratch, (int)C, norms);
    ++g_launches;
  }
  return cudaGetLastError();
}
template <class R>
cudaError_t multi_axpy(const R* const* v, int k, const double* coef, double sign, R* w, size_t n,
                       cudaStream_t st) {
  return multi_axpy_batched<R>(v, k, coef, 0, sign, w, n, 1, 0, nullptr, nullptr, st);
}
template <class R>
cudaError_t multi_axpy_norm(const R* const* v, int k, const double* coef, double sign, R* w, size_t n,
                            double* scratch, double* out, cudaStream_t st) {
  return multi_axpy_batched<R>(v, k, coef, 0, sign, w, n, 1, 0, scratch, out, st);
}
cudaError_t multi_axpy_f32_into_f64(const Geom& g, const float* const* v, int k, const double* coef, int cstride,
                                    double sign, double* w, int nf, cudaStream_t st) {
  if (k > MAXK || k < 1 || nf < 1) return cudaErrorInvalidValue;
  PtrList<float> pl;
  for (int j = 0; j < k; ++j) pl.p[j] = v[j];
  const size_t n = (size_t)g.V * (SPINOR_NR / 2);
  k_multi_axpy_f32<<<dim3(batch_ctas(nf), nf), RED_TPB, 0, st>>>(pl, k, coef, sign, w, n, g.Vb, cstride);
  ++g_launches;
  return cudaGetLastError();
}
template <class R>
cudaError_t axpby(double a, const R* x, double b, R* y, size_t n, cudaStream_t st) {
  unsigned nb = nblk(n, 256);
  if (nb > 4096) nb = 4096;
  k_axpby<R><<<nb, 256, 0, st>>>((R)a, x, (R)b, y, n);
  ++g_launches;
  return cudaGetLastError();
}
template <class R>
cudaError_t scale_by_inv_norm_batched(const R* x, R* y, const double* s, size_t n, int nb, cudaStream_t st) {
  unsigned c = nblk(n, 256);
  const unsigned cap = 4096 / (nb > 0 ? nb : 1) > 0 ? 4096 / (nb > 0 ? nb : 1) : 1;
  if (c > cap) c = cap;
  k_scale_inv_norm<R><<<dim3(c, nb), 256, 0, st>>>(x, y, s, n);
  ++g_launches;
  return cudaGetLastError();
}
template <class R>
cudaError_t scale_by_inv_norm(const R* x, R* y, const double* s, size_t n, cudaStream_t st) {
  return scale_by_inv_norm_batched<R>(x, y, s, n, 1, st);
}

cudaError_t random_spinors(const Geom& g, uint64_t seed, int n, double* dev64, cudaStream_t st) {
  k_random_spinors<<<dim3(nblk(g.V, TPB), n), TPB, 0, st>>>(g, seed, n, dev64);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t index_maps(const Geom& g, int* parity, int* block, int* colour, cudaStream_t st) {
  k_index_maps<<<nblk(g.V, TPB), TPB, 0, st>>>(g, parity, block, colour);
  ++g_launches;
  return cudaGetLastError();
}

// explicit instantiations
template cudaError_t pack_spinor<float>(const Geom&, const double*, float*, int, cudaStream_t);
template cudaError_t pack_spinor<double>(const Geom&, const double*, double*, int, cudaStream_t);
template cudaError_t unpack_spinor<float>(const Geom&, const float*, double*, int, cudaStream_t);
template cudaError_t unpack_spinor<double>(const Geom&, const double*, double*, int, cudaStream_t);
template cudaError_t convert_field<float, double>(const double*, float*, size_t, cudaStream_t);
template cudaError_t convert_field<double, float>(const float*, double*, size_t, cudaStream_t);
template cudaError_t convert_field<double, double>(const double*, double*, size_t, cudaStream_t);
template cudaError_t convert_field<float, float>(const float*, float*, size_t, cudaStream_t);
template cudaError_t dslash<float>(const Geom&, int, const float*, const float*, float*, const float*,
                                   const float*, int, cudaStream_t);
template cudaError_t dslash<double>(const Geom&, int, const double*, const double*, double*,
                                    const double*, const double*, int, cudaStream_t);
template cudaError_t multi_dot<float>(const float* const*, int, const float*, size_t, double*, double*,
                                      cudaStream_t);
template cudaError_t multi_dot<double>(const double* const*, int, const double*, size_t, double*,
                                       double*, cudaStream_t);
template cudaError_t norm2<float>(const float*, size_t, double*, double*, cudaStream_t);
template cudaError_t norm2<double>(const double*, size_t, double*, double*, cudaStream_t);
template cudaError_t multi_axpy<float>(const float* const*, int, const double*, double, float*, size_t,
                                       cudaStream_t);
template cudaError_t multi_axpy<double>(const double* const*, int, const double*, double, double*,
                                        size_t, cudaStream_t);
template cudaError_t multi_axpy_norm<double>(const double* const*, int, const double*, double, double*,
                                             size_t, double*, double*, cudaStream_t);
template cudaError_t multi_dot_batched<double>(const double* const*, int, const double*, size_t, int, size_t,
                                               double*, double*, cudaStream_t);
template cudaError_t norm2_batched<double>(const double*, size_t, int, size_t, double*, double*, cudaStream_t);
template cudaError_t multi_axpy_batched<double>(const double* const*, int, const double*, int, double, double*,
                                                size_t, int, size_t, double*, double*, cudaStream_t);
template cudaError_t scale_by_inv_norm_batched<double>(const double*, double*, const double*, size_t, int,
                                                       cudaStream_t);
template cudaError_t axpby<float>(double, const float*, double, float*, size_t, cudaStream_t);
template cudaError_t axpby<double>(double, const double*, double, double*, size_t, cudaStream_t);
template cudaError_t scale_by_inv_norm<float>(const float*, float*, const double*, size_t, cudaStream_t);
template cudaError_t scale_by_inv_norm<double>(const double*, double*, const double*, size_t,
                                               cudaStream_t);

}  // namespace ddamg
