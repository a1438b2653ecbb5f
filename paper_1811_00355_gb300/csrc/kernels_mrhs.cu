// Restriction (Eq. 3) and prolongation (Eq. 4) of a batch of right-hand
// sides as complex matrix products on the tensor cores.
//
// For one aggregate X and chirality s the test vectors form a 6|X| x n
// complex matrix L (column i = lambda_i restricted to (X, s)).  With N
// right-hand sides B (6|X| x N) and coarse vectors C (n x N):
//   restriction   C = L^H B,        prolongation   B = L C.
// Complex products are taken as real ones on the interleaved (re, im) data:
// with k running over the real components of (X, s),
//   Re C = sum_k L[k] B[k],  Im C = sum_k L[k] B~[k],   B~ = (im, -re) pairs,
// so the restriction is one real product of the raw test-vector rows with
// the raw right-hand sides and their rotated copies; the prolongation is the
// real product of [L, L~] (L~ = (-im, re) pairs) with [Re C; Im C].  Every
// test vector is read once per batch (not once per right-hand side).
//
// Arithmetic: the 3xTF32 tensor-core products of mma_tf32.cuh (FP32
// accuracy).
#include "common.cuh"
#include "kernels.h"
#include "mma_tf32.cuh"

namespace ddamg {

namespace {

constexpr int MT_THREADS = 256;   // 8 warps
constexpr int MAXRQ = 64;         // sites per staged chunk
constexpr int RSTR = 4 * MAXRQ + 4;   // row stride (floats) of the restriction's staged rows
constexpr int PSTR = 4 * MAXRQ + 8;   // of the prolongation's
constexpr int OSTR = 4 * MAXRQ + 4;   // row stride of the prolongation's output tile
constexpr int CSTR = 24;              // row stride of its staged coarse coefficients

__device__ __forceinline__ void cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// chunk c of the (s, u, site range) sequence of an aggregate: units 3 s + u,
// sites [q0, q0 + rq); returns the float offset of its first value within a
// field (block X)
__device__ __forceinline__ size_t chunk_off(int X, int Vb, int s, int c, int rq) {
  const int per_u = Vb / rq;
  const int u = c / per_u, q0 = (c - u * per_u) * rq;
  return (((size_t)X * 6 + 3 * s + u) * Vb + q0) * 4;
}

// stage chunk c of `rows` fields (field j at base + j * fstride) into dst
// rows of `stride` floats: 16-byte asynchronous copies
__device__ __forceinline__ void stage_rows(float* dst, int stride, const float* base, size_t fstride, int rows,
                                           size_t off, int rq) {
  const int per_row = rq;   // float4 units per row
  for (int idx = threadIdx.x; idx < rows * per_row; idx += MT_THREADS) {
    const int j = idx / per_row, v = idx - j * per_row;
    cp16(dst + (size_t)j * stride + 4 * v, base + (size_t)j * fstride + off + 4 * v);
  }
}

// ---------------------------------------------------------------------------
// restriction: CTA per (aggregate, group of <= 16 right-hand sides)
//   acc[i][c] = sum_k lam_i[k] Bx[k][c],  Bx[.][c] = b_c (c < N) or b~_{c-N}
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(MT_THREADS) k_restrict_mma(Geom g, const float* __restrict__ lam, int n,
                                                             const float* __restrict__ b, int nrhs, int rq,
                                                             cpx<float>* __restrict__ bc) {
  extern __shared__ __align__(16) float msh[];
  const int X = blockIdx.x;
  const int r0 = blockIdx.y * 16;
  const int N = min(16, nrhs - r0);
  const size_t fstride = (size_t)g.V * SPINOR_NR;
  float* As[2] = {msh, msh + (size_t)n * RSTR};
  float* Bs[2] = {msh + (size_t)2 * n * RSTR, msh + (size_t)2 * n * RSTR + (size_t)N * RSTR};
  const float* bb = b + (size_t)r0 * fstride;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gq = lane >> 2, tq = lane & 3;
  const int MT = (n + 15) / 16, NT = (2 * N + 7) / 8;
  const int nchunk = 3 * (g.Vb / rq);
  const int ksteps = rq / 2;     // 8 reals per step

  for (int s = 0; s < 2; ++s) {
    float acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[a][c][e] = 0.f;
    // prologue: chunk 0
    stage_rows(As[0], RSTR, lam, fstride, n, chunk_off(X, g.Vb, s, 0, rq), rq);
    stage_rows(Bs[0], RSTR, bb, fstride, N, chunk_off(X, g.Vb, s, 0, rq), rq);
    cp_commit();
    for (int c = 0; c < nchunk; ++c) {
      const int cur = c & 1;
      if (c + 1 < nchunk) {
        const size_t off = chunk_off(X, g.Vb, s, c + 1, rq);
        stage_rows(As[cur ^ 1], RSTR, lam, fstride, n, off, rq);
        stage_rows(Bs[cur ^ 1], RSTR, bb, fstride, N, off, rq);
        cp_commit();
        cp_wait_one();
      } else {
        cp_wait_all();
      }
      __syncthreads();
      const float* A = As[cur];
      const float* B = Bs[cur];
      // the chunk's products go to fresh accumulators that are then added
      // to the running sums with ordinary FP32 additions: the tensor cores'
      // accumulation never runs over more than one chunk
      float part[2][4][4];
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c2 = 0; c2 < 4; ++c2)
#pragma unroll
          for (int e = 0; e < 4; ++e) part[a][c2][e] = 0.f;
      for (int ks = warp; ks < ksteps; ks += MT_THREADS / 32) {
        const int k0 = 8 * ks;
        Split<2> bs[4];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          const int col = nt * 8 + gq;
          const bool raw = col < N, live = col < 2 * N;
          const int r = raw ? col : (live ? col - N : 0);
          float bv[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int k = k0 + tq + 4 * h;
            const float v1 = B[r * RSTR + k], v2 = B[r * RSTR + (k ^ 1)];
            // b~ = (im, -re): at a real slot the imaginary part, at an imaginary slot minus the real part
            const float rot = (k & 1) ? -v2 : v2;
            bv[h] = live ? (raw ? v1 : rot) : 0.f;
          }
          bs[nt] = split_frag<2>(bv);
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          if (mt >= MT) break;
          const int r_lo = mt * 16 + gq, r_hi = r_lo + 8;
          float af[4];
          af[0] = r_lo < n ? A[r_lo * RSTR + k0 + tq] : 0.f;
          af[1] = r_hi < n ? A[r_hi * RSTR + k0 + tq] : 0.f;
          af[2] = r_lo < n ? A[r_lo * RSTR + k0 + tq + 4] : 0.f;
          af[3] = r_hi < n ? A[r_hi * RSTR + k0 + tq + 4] : 0.f;
          const Split<4> as = split_frag<4>(af);
#pragma unroll
          for (int nt = 0; nt < 4; ++nt)
            if (nt < NT) mma3(part[mt][nt], as, bs[nt]);
        }
      }
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c2 = 0; c2 < 4; ++c2)
#pragma unroll
          for (int e = 0; e < 4; ++e) acc[a][c2][e] += part[a][c2][e];
      __syncthreads();     // the buffer is refilled two chunks later
    }
    // sum the warps' partial products (the staging buffers are free now)
    float* red = msh;      // [warp][mt][nt][lane][4]
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) red[(((warp * 2 + mt) * 4 + nt) * 32 + lane) * 4 + e] = acc[mt][nt][e];
    __syncthreads();
    for (int idx = threadIdx.x; idx < 2 * 4 * 32 * 4; idx += MT_THREADS) {
      const int e = idx & 3, ln = (idx >> 2) & 31, nt = (idx >> 7) & 3, mt = idx >> 9;
      if (mt >= MT || nt >= NT) continue;
      float sum = 0.f;
      for (int w = 0; w < MT_THREADS / 32; ++w) sum += red[(((w * 2 + mt) * 4 + nt) * 32 + ln) * 4 + e];
      const int i = mt * 16 + (ln >> 2) + (e >= 2 ? 8 : 0);
      const int col = nt * 8 + 2 * (ln & 3) + (e & 1);
      if (i >= n || col >= 2 * N) continue;
      const int r = col < N ? col : col - N;
      float* dst = reinterpret_cast<float*>(bc + ((size_t)(r0 + r) * g.nb + X) * 2 * n + s * n + i);
      dst[col < N ? 0 : 1] = sum;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// prolongation: CTA per (aggregate, group of <= 16 right-hand sides)
//   x_r[k] = sum_j Lx[k][j] Cx[j][r],  Lx = [lam, lam~] (k rows), Cx = [Re; Im]
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(MT_THREADS) k_prolong_mma(Geom g, const float* __restrict__ lam, int n,
                                                            const cpx<float>* __restrict__ xc, int nrhs, int rq,
                                                            float* __restrict__ x) {
  extern __shared__ __align__(16) float msh[];
  const int X = blockIdx.x;
  const int r0 = blockIdx.y * 16;
  const int N = min(16, nrhs - r0);
  const size_t fstride = (size_t)g.V * SPINOR_NR;
  const int KG = ((2 * n + 7) / 8) * 8;        // inner dimension, padded to whole steps
  float* Ls[2] = {msh, msh + (size_t)n * PSTR};
  float* Cs = msh + (size_t)2 * n * PSTR;       // [KG][CSTR] (16 columns used)
  float* Os = Cs + (size_t)KG * CSTR;           // [16][OSTR] (output tile)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gq = lane >> 2, tq = lane & 3;
  const int NT = (N + 7) / 8;
  const int nchunk = 3 * (g.Vb / rq);
  const int mtiles = rq / 4;                    // 16 rows each, 4 rq rows per chunk
  float* xb = x + (size_t)r0 * fstride;

  for (int s = 0; s < 2; ++s) {
    for (int idx = threadIdx.x; idx < KG * 16; idx += MT_THREADS) {
      const int j = idx >> 4, r = idx & 15;
      float v = 0.f;
      if (r < N && j < 2 * n) {
        const cpx<float> c = xc[((size_t)(r0 + r) * g.nb + X) * 2 * n + s * n + (j < n ? j : j - n)];
        v = j < n ? c.re : c.im;
      }
      Cs[j * CSTR + r] = v;
    }
    stage_rows(Ls[0], PSTR, lam, fstride, n, chunk_off(X, g.Vb, s, 0, rq), rq);
    cp_commit();
    for (int c = 0; c < nchunk; ++c) {
      const int cur = c & 1;
      if (c + 1 < nchunk) {
        stage_rows(Ls[cur ^ 1], PSTR, lam, fstride, n, chunk_off(X, g.Vb, s, c + 1, rq), rq);
        cp_commit();
        cp_wait_one();
      } else {
        cp_wait_all();
      }
      __syncthreads();
      const float* Lm = Ls[cur];
      for (int mt = warp; mt < mtiles; mt += MT_THREADS / 32) {
        float acc[2][4];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int e = 0; e < 4; ++e) acc[nt][e] = 0.f;
        const int m_lo = mt * 16 + gq, m_hi = m_lo + 8;
        for (int k0 = 0; k0 < KG; k0 += 8) {
          float af[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int m = (e & 1) ? m_hi : m_lo;
            const int j = k0 + tq + ((e & 2) ? 4 : 0);
            // lam~ = (-im, re): at a real row minus the imaginary part, at an imaginary row the real part
            const bool raw = j < n, live = j < 2 * n;
            const int jj = raw ? j : (live ? j - n : 0);
            const float v1 = Lm[jj * PSTR + m], v2 = Lm[jj * PSTR + (m ^ 1)];
            af[e] = live ? (raw ? v1 : ((m & 1) ? v2 : -v2)) : 0.f;
          }
          const Split<4> as = split_frag<4>(af);
#pragma unroll
          for (int nt = 0; nt < 2; ++nt) {
            if (nt >= NT) break;
            const float bf[2] = {Cs[(k0 + tq) * CSTR + nt * 8 + gq], Cs[(k0 + tq + 4) * CSTR + nt * 8 + gq]};
            mma3(acc[nt], as, split_frag<2>(bf));
          }
        }
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          if (nt >= NT) break;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int m = (e >= 2) ? m_hi : m_lo;
            const int r = nt * 8 + 2 * tq + (e & 1);
            Os[r * OSTR + m] = acc[nt][e];
          }
        }
      }
      __syncthreads();
      // coalesced write of the chunk's output rows, one field per right-hand side
      const size_t off = chunk_off(X, g.Vb, s, c, rq);
      for (int idx = threadIdx.x; idx < N * rq; idx += MT_THREADS) {
        const int r = idx / rq, v = idx - r * rq;
        const float4 o = *reinterpret_cast<const float4*>(Os + r * OSTR + 4 * v);
        *reinterpret_cast<float4*>(xb + (size_t)r * fstride + off + 4 * v) = o;
      }
      __syncthreads();
    }
  }
}

// sites per chunk: the largest multiple of 4 up to 64 that divides the
// aggregate volume (a product of four even extents, so 4 always does)
int chunk_sites(int Vb) {
  int rq = MAXRQ;
  while (rq > 4 && Vb % rq) rq -= 4;
  return rq;
}

}  // namespace

bool mrhs_ok(const Geom& g, int n) { return n >= 1 && n <= 32 && g.Vb % 4 == 0; }

size_t restrict_mma_smem(int n, int N) {
  const size_t stage = (size_t)2 * (n + N) * RSTR * sizeof(float);
  const size_t red = (size_t)8 * 2 * 4 * 32 * 4 * sizeof(float);
  return stage > red ? stage : red;
}
size_t prolong_mma_smem(const Geom& g, int n) {
  const int rq = chunk_sites(g.Vb);
  const int KG = ((2 * n + 7) / 8) * 8;
  (void)rq;
  return ((size_t)2 * n * PSTR + (size_t)KG * CSTR + (size_t)16 * OSTR) * sizeof(float);
}

cudaError_t restrict_mrhs(const Geom& g, const float* lam, int n, const float* b, float* bc, int nrhs,
                          cudaStream_t st) {
  if (!mrhs_ok(g, n) || nrhs < 1) return cudaErrorInvalidValue;
  const int N = nrhs < 16 ? nrhs : 16;
  const size_t smem = restrict_mma_smem(n, N);
  cudaError_t e = raise_smem_limit((const void*)k_restrict_mma, smem);
  if (e != cudaSuccess) return e;
  k_restrict_mma<<<dim3(g.nb, (nrhs + 15) / 16), MT_THREADS, smem, st>>>(g, lam, n, b, nrhs, chunk_sites(g.Vb),
                                                                        reinterpret_cast<cpx<float>*>(bc));
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t prolong_mrhs(const Geom& g, const float* lam, int n, const float* xc, float* x, int nrhs,
                         cudaStream_t st) {
  if (!mrhs_ok(g, n) || nrhs < 1) return cudaErrorInvalidValue;
  const size_t smem = prolong_mma_smem(g, n);
  cudaError_t e = raise_smem_limit((const void*)k_prolong_mma, smem);
  if (e != cudaSuccess) return e;
  k_prolong_mma<<<dim3(g.nb, (nrhs + 15) / 16), MT_THREADS, smem, st>>>(
      g, lam, n, reinterpret_cast<const cpx<float>*>(xc), nrhs, chunk_sites(g.Vb), x);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace ddamg
