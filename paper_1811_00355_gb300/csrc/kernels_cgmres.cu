// Even-odd preconditioned restarted GMRES on the coarse operator, paper
// Sec. 2: the coarse solver works on the even-site Schur complement
//   S = A_ee - D_eo A_oo^-1 D_oe     (A = self blocks of D_c)
// with right-hand side b_e - D_eo A_oo^-1 b_o, stops when the Schur residual
// reaches tol * ||rhs|| (the method's 5e-2), and back-substitutes
// x_o = A_oo^-1 (b_o - D_oe x_e).
//
// One persistent cooperative kernel solves all right-hand sides, NR of them
// in lockstep (one Krylov space, Hessenberg matrix and stopping test each),
// so that the grid-wide barriers of an iteration are shared.  Every CTA owns
// `per` even and `per` odd coarse sites; its slice of the Krylov basis, of
// x_e and of the right-hand side stays in shared memory.  Only the vectors a
// neighbour reads (w and the odd-site temporaries) go through global memory,
// loaded with ld.cg.  Arnoldi orthogonalises with classical Gram-Schmidt:
// in FP64 with one re-orthogonalisation pass and an explicit norm (four grid
// barriers per iteration: odd hop, two passes, norm); in FP32 with a single
// pass whose reduction also carries ||w||^2, the new norm following from
// Pythagoras (three barriers: odd hop, dots, publication of w), with an
// explicit norm only when that difference cancels.  Reductions are
// deterministic (fixed trees).  Every barrier wait is bounded; on time-out
// the kernel records DDAMG_ETIMEOUT (6) and returns.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "mma_tf32.cuh"

namespace ddamg {

namespace {

constexpr int TPB = 512;
// partial-sum groups of mrhs_matvec (the plan's mvp buffer): more column
// chunks for few right-hand sides, fewer where the buffer grows with NR
__host__ __device__ constexpr int mvp_groups(int NR) { return NR >= 8 ? 9 : 18; }
// row stride (complex entries) of the staged vectors sv[r][d][.]: one more
// than n2, so that rows of different directions and right-hand sides read
// at the same column fall on different shared-memory banks
__host__ __device__ constexpr int sv_stride(int n2) { return n2 + 1; }
constexpr int NW = TPB / 32;
constexpr int MAXM = 64;
constexpr int NRMAX = 12;
// block ring: slots of one 2n x 2n block each through which the block
// operators of plans that do not keep them resident are streamed (FP32,
// blocks of at least RING_MIN_N2 rows, where the loads are worth hiding)
constexpr int RING = 4;
constexpr int RING_MIN_N2 = 32;

__device__ __forceinline__ cpx<float> ldc(const cpx<float>* p) {
  float2 t = __ldcg(reinterpret_cast<const float2*>(p));
  return mk(t.x, t.y);
}
__device__ __forceinline__ cpx<double> ldc(const cpx<double>* p) {
  double2 t = __ldcg(reinterpret_cast<const double2*>(p));
  return mk(t.x, t.y);
}

template <class T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Grid barrier on a counter that only grows during a launch (zeroed before
// it): at its e-th barrier every CTA adds 1 and waits until the counter
// reaches e * gridDim.x.  The arrival is a fence followed by a relaxed
// reduction (no reply awaited), the wait an acquire load, so a barrier costs
// about one L2 round trip after the last arrival.  The wait is bounded (about
// a second); on time-out the CTA records DDAMG_ETIMEOUT and leaves, and the
// CTAs still waiting for it then time out at this or their next barrier.
__device__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__shared__ unsigned bar_epoch;       // barriers passed by this CTA in this launch

// thread 0 zeroes the count at kernel entry (a __syncthreads must follow
// before the first barrier)
__device__ void grid_barrier_reset() {
  if (threadIdx.x == 0) bar_epoch = 0;
}

// Split form: grid_arrive publishes this CTA's writes and counts it in;
// grid_wait returns once every CTA has arrived.  Between the two a CTA may do
// work that touches only its own shared memory and registers.
__device__ void grid_arrive(unsigned* bar) {
  __syncthreads();
  if (threadIdx.x == 0) {
    ++bar_epoch;
    __threadfence();                 // the CTA's writes (ordered by the bar.sync above) first
    asm volatile("red.relaxed.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
  }
}

__device__ bool grid_wait(unsigned* bar, int* status, long long limit) {
  __shared__ int ok_s;
  if (threadIdx.x == 0) {
    const unsigned target = bar_epoch * gridDim.x;
    int ok = 1;
    long long spins = 0;
    while ((int)(ld_acquire_gpu(bar) - target) < 0) {
      if (++spins > limit) {
        atomicExch(status, 6);
        ok = 0;
        break;
      }
    }
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

__device__ bool grid_barrier(unsigned* bar, int* status, long long limit) {
  grid_arrive(bar);
  return grid_wait(bar, status, limit);
}

// L2 prefetch of `bytes` bytes at p (16-byte aligned, a multiple of 16) by
// the calling warp, in bulk prefetches of at most 32 KB per lane: the block
// operators of the next coarse site travel from HBM while this site's block
// product runs
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes) {
  constexpr size_t PIECE = 32768;
  for (size_t off = (size_t)(threadIdx.x & 31) * PIECE; off < bytes; off += 32 * PIECE) {
    const size_t n = bytes - off < PIECE ? bytes - off : PIECE;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(static_cast<const char*>(p) + off),
                 "r"((unsigned)n)
                 : "memory");
  }
}

// shared-memory plan, identical on host and device
struct Plan {
  size_t V, x, rl, w, sv, mvp, tmp;                                    // cpx offsets (bytes)
  size_t hc, h2, Rf, cs, sn, gv, yv, beta, bnorm, hn, scale;           // double offsets
  size_t act, kd, tot, conv;                                            // int offsets
  size_t nbo;          // [2][per][8] neighbour offsets of the CTA's odd and even sites
  size_t Mres;         // resident D_c blocks of the CTA's even site (0: none)
  size_t ring;         // block ring, RING blocks (0: none)
  size_t bytes;        // total shared memory
  size_t local_bytes;  // V + x + rl + w (moved to global when too large)
};

__host__ __device__ inline size_t al16(size_t v) { return (v + 15) / 16 * 16; }

__host__ __device__ inline Plan make_plan(int NR, int L, int n2, int m, int rs, bool local_in_smem,
                                          bool resident = false, bool ring = false) {
  Plan p;
  const size_t c = 2 * (size_t)rs;
  size_t o = 0;
  size_t lb = 0;
  auto put = [&](size_t bytes) { size_t r = o; o = al16(o + bytes); return r; };
  if (local_in_smem) {
    p.V = put((size_t)(m + 1) * NR * L * c);
    p.x = put((size_t)NR * L * c);
    p.rl = put((size_t)NR * L * c);
    p.w = put((size_t)NR * L * c);
    lb = o;
  } else {
    size_t g = 0;
    auto putg = [&](size_t bytes) { size_t r = g; g = al16(g + bytes); return r; };
    p.V = putg((size_t)(m + 1) * NR * L * c);
    p.x = putg((size_t)NR * L * c);
    p.rl = putg((size_t)NR * L * c);
    p.w = putg((size_t)NR * L * c);
    lb = g;
  }
  p.sv = put((size_t)NR * 9 * sv_stride(n2) * c);
  p.mvp = put((size_t)mvp_groups(NR) * NR * n2 * c);
  p.tmp = put((size_t)NR * n2 * c);
  p.hc = put((size_t)NR * 2 * (m + 1) * 8);
  p.h2 = put((size_t)NR * 2 * (m + 1) * 8);
  p.Rf = put((size_t)NR * m * (m + 1) * 8);
  p.cs = put((size_t)NR * m * 8);
  p.sn = put((size_t)NR * 2 * m * 8);
  p.gv = put((size_t)NR * 2 * (m + 1) * 8);
  p.yv = put((size_t)NR * 2 * m * 8);
  p.beta = put((size_t)NR * 8);
  p.bnorm = put((size_t)NR * 8);
  p.hn = put((size_t)NR * 8);
  p.scale = put((size_t)NR * 8);
  p.act = put((size_t)NR * 4);
  p.kd = put((size_t)NR * 4);
  p.tot = put((size_t)NR * 4);
  p.conv = put((size_t)NR * 4);
  p.nbo = put((size_t)2 * (L / n2) * 8 * 4);
  p.Mres = resident ? put((size_t)9 * n2 * n2 * c) : 0;
  p.ring = ring ? put((size_t)RING * n2 * n2 * c) : 0;
  p.bytes = o;
  p.local_bytes = lb;
  return p;
}

template <class R>
struct CGA {
  Geom g;
  const cpx<R>* Dc;
  const cpx<R>* Ainv;
  const cpx<R>* AD;    // [odd site][8] A_oo^-1 D_c blocks
  int n2;
  double tol;
  int m;
  int max_iter;
  const cpx<R>* b;
  cpx<R>* x;
  int nrhs;
  int NR;
  int NE;
  int per;
  int local_in_smem;
  int resident;      // the CTA keeps its even site's D_c blocks in shared memory
  int ring;          // block operators streamed through the shared-memory ring
  int tc;            // ring products of eight right-hand sides on the tensor cores
  cpx<R>* wg;        // [NR][NE][n2]
  cpx<R>* to;        // [NR][NE][n2]
  cpx<R>* xg;        // [NR][NE][n2]
  unsigned char* lglob;   // per-CTA local arrays when they do not fit in smem
  size_t lstride;         // bytes per CTA in lglob
  double* part;      // [(MAXM + 2) * NR][G][2]
  unsigned* bar;
  int* iters;
  int* iters_acc;
  int* status;
  long long spin_limit;   // polls of a barrier wait before it gives up
};

// Multi-right-hand-side block product on one coarse site, whole CTA:
//   out[r][row] = sum_{d in [d0, d1)} sum_c M_d[row][c] sv[r][d][c]
// (sv rows sv_stride(n2) entries apart)
// Blocks are column-major, so a thread streams RPU rows down the columns
// (16-byte loads, neighbouring threads on neighbouring rows) and applies each
// loaded entry to all NR vectors.  The column range is split into CC chunks
// when there are few directions.  Partials land in mvp[unit-group][r][row] and
// are summed in a fixed order.
// (M holds the blocks of directions d0 .. d1 - 1 from its start when
// m_from_d0 is set, else the blocks of directions 0 .. d1 - 1)
// (M in shared memory when SM: plain loads instead of the read-only path)
template <class R, int NR, bool SM = false>
__device__ __forceinline__ void mrhs_matvec(const cpx<R>* __restrict__ M, const cpx<R>* sv, int d0, int d1,
                                            int n2, cpx<R>* mvp, cpx<R>* out, int out_stride,
                                            bool m_from_d0 = false) {
  using T = typename U16<R>::T;
  constexpr int RPU = 16 / (2 * sizeof(R));
  // wide lockstep groups split their right-hand sides over RS units, so
  // that more threads share a site's work and each one's chain of
  // multiply-adds per column is shorter (the block entries are then read by
  // RS threads, the later ones from L1); the slices write disjoint rows of
  // the partial sums
  constexpr int RS = NR >= 8 ? 2 : 1;
  constexpr int NRS = NR / RS;
  static_assert(NR % RS == 0, "right-hand-side slices must divide the lockstep width");
  const int NP = n2 / RPU;
  const int ND = d1 - d0;
  // column chunks: enough units for every thread, at most mvp_groups(NR) groups
  int CC = (int)blockDim.x / (ND * NP * RS);
  if (CC * ND > mvp_groups(NR)) CC = mvp_groups(NR) / ND;
  if (CC < 1) CC = 1;
  if (CC > n2) CC = n2;
  const int CW = (n2 + CC - 1) / CC;
  const int units = ND * CC * NP * RS;
  for (int u = threadIdx.x; u < units; u += blockDim.x) {
    const int rs = u % RS, uu = u / RS;
    const int grp = uu / NP, j = uu - grp * NP;
    const int dd = grp / CC, cc = grp - dd * CC, d = d0 + dd;
    const int c0 = cc * CW, c1 = min(n2, c0 + CW);
    const T* col = reinterpret_cast<const T*>(M + (size_t)(m_from_d0 ? d - d0 : d) * n2 * n2) + j;
    const int svs = sv_stride(n2);
    const cpx<R>* svr = sv + (size_t)rs * NRS * 9 * svs;
    cpx<R> acc[NRS][RPU];
#pragma unroll
    for (int r = 0; r < NRS; ++r)
#pragma unroll
      for (int q = 0; q < RPU; ++q) acc[r][q] = mk(R(0), R(0));
#pragma unroll 8
    for (int c = c0; c < c1; ++c) {
      T mm;
      if constexpr (SM) mm = col[(size_t)c * NP];
      else mm = __ldg(col + (size_t)c * NP);
      cpx<R> e0, e1;
      if constexpr (RPU == 2) { e0 = mk((R)mm.x, (R)mm.y); e1 = mk((R)mm.z, (R)mm.w); }
      else { e0 = mk((R)mm.x, (R)mm.y); e1 = e0; }
#pragma unroll
      for (int r = 0; r < NRS; ++r) {
        cpx<R> v = svr[(r * 9 + d) * svs + c];
        fma(acc[r][0], e0, v);
        if constexpr (RPU == 2) fma(acc[r][1], e1, v);
      }
    }
#pragma unroll
    for (int r = 0; r < NRS; ++r)
#pragma unroll
      for (int q = 0; q < RPU; ++q)
        mvp[((size_t)grp * NR + rs * NRS + r) * n2 + RPU * j + q] = acc[r][q];
  }
  __syncthreads();
  const int ngrp = ND * CC;
  for (int idx = threadIdx.x; idx < NR * n2; idx += blockDim.x) {
    const int r = idx / n2, row = idx - r * n2;
    cpx<R> s = mk(R(0), R(0));
    for (int gq = 0; gq < ngrp; ++gq) s = s + mvp[((size_t)gq * NR + r) * n2 + row];
    out[(size_t)r * out_stride + row] = s;
  }
  __syncthreads();
}

template <class R, int NR>
__global__ void __launch_bounds__(TPB) k_cgmres(CGA<R> a) {
  extern __shared__ __align__(16) unsigned char sm[];
  // small dense state (Hessenberg column, Givens, least squares, norms) and
  // cross-CTA sums in the working precision: FP64 arithmetic is scarce on
  // GB300, FP32 is ample for a solve to a relative residual of 5e-2
  using A = R;
  const int n2 = a.n2, m = a.m, NE = a.NE;
  const int L = a.per * n2;
  const Plan P = make_plan(NR, L, n2, m, sizeof(R), a.local_in_smem != 0, a.resident != 0, a.ring != 0);
  cpx<R>* Mres = reinterpret_cast<cpx<R>*>(sm + P.Mres);   // [9][n2][n2] when resident
  unsigned char* lbase = a.local_in_smem ? sm : a.lglob + (size_t)blockIdx.x * a.lstride;
  cpx<R>* V = reinterpret_cast<cpx<R>*>(lbase + P.V);     // [m+1][NR][L]
  cpx<R>* xl = reinterpret_cast<cpx<R>*>(lbase + P.x);    // [NR][L]
  cpx<R>* rl = reinterpret_cast<cpx<R>*>(lbase + P.rl);   // [NR][L]
  cpx<R>* wl = reinterpret_cast<cpx<R>*>(lbase + P.w);    // [NR][L]
  cpx<R>* sv = reinterpret_cast<cpx<R>*>(sm + P.sv);      // [NR][9][n2]
  cpx<R>* mvp = reinterpret_cast<cpx<R>*>(sm + P.mvp);    // [9][NR][n2]
  cpx<R>* tmp = reinterpret_cast<cpx<R>*>(sm + P.tmp);    // [NR][n2]
  A* hc = reinterpret_cast<A*>(sm + P.hc);      // [NR][2(m+1)]
  A* h2 = reinterpret_cast<A*>(sm + P.h2);      // [NR][2(m+1)]
  A* Rf = reinterpret_cast<A*>(sm + P.Rf);      // [NR][m(m+1)] packed columns
  A* cs = reinterpret_cast<A*>(sm + P.cs);      // [NR][m]
  A* sn = reinterpret_cast<A*>(sm + P.sn);      // [NR][2m]
  A* gv = reinterpret_cast<A*>(sm + P.gv);      // [NR][2(m+1)]
  A* yv = reinterpret_cast<A*>(sm + P.yv);      // [NR][2m]
  A* beta = reinterpret_cast<A*>(sm + P.beta);
  A* bnorm = reinterpret_cast<A*>(sm + P.bnorm);
  A* hnv = reinterpret_cast<A*>(sm + P.hn);
  A* scl = reinterpret_cast<A*>(sm + P.scale);
  int* act = reinterpret_cast<int*>(sm + P.act);          // active in this cycle
  int* kd = reinterpret_cast<int*>(sm + P.kd);            // basis size of this cycle
  int* tot = reinterpret_cast<int*>(sm + P.tot);          // iterations so far
  int* conv = reinterpret_cast<int*>(sm + P.conv);        // converged (or gave up)
  __shared__ int any_s;
  __shared__ int any_act_s;
  __shared__ int exn[NR];      // explicit norm needed (FP32 path)

  const int G = gridDim.x;
  grid_barrier_reset();
  const int lo = min(NE, (int)blockIdx.x * a.per);
  const int hi = min(NE, lo + a.per);
  if (a.resident && lo < hi) {      // one even site per CTA: its nine blocks, once per launch
    using T = typename U16<R>::T;
    const T* src = reinterpret_cast<const T*>(a.Dc + (size_t)a.g.ceven[lo] * 9 * n2 * n2);
    T* dst = reinterpret_cast<T*>(Mres);
    const int units = 9 * n2 * n2 * (int)sizeof(cpx<R>) / 16;
    for (int i = threadIdx.x; i < units; i += blockDim.x) dst[i] = __ldg(src + i);
  }
  const int nown = hi - lo;
  const int Lo = nown * n2;          // owned local elements
  const size_t vstr = (size_t)NE * n2;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tx = threadIdx.x;
  const int TRI = m * (m + 1) / 2;
  const int svs = sv_stride(n2);
  // offsets (in the [NE][n2] vectors) of the eight neighbours of the CTA's
  // odd sites (nbo[kk][d - 1]) and even sites (nbo[per + kk][d - 1]), looked
  // up once per launch instead of two dependent loads per staging
  int* nbo = reinterpret_cast<int*>(sm + P.nbo);
  for (int i = tx; i < 2 * nown * 8; i += TPB) {
    const int par = i / (nown * 8), rem = i - par * nown * 8, kk = rem / 8, d = 1 + rem % 8;
    const int X = par ? a.g.ceven[lo + kk] : a.g.codd[lo + kk];
    nbo[(par * a.per + kk) * 8 + d - 1] = a.g.cpos[a.g.cnbr[d * a.g.nb + X]] * n2;
  }

  auto Vk = [&](int k, int r) { return V + ((size_t)k * NR + r) * L; };

  // stage neighbours of odd site X from global vectors src[r] (scaled), d >= 1
  // (one warp per row (r, d) of sv: the neighbour's position is looked up
  // once per row, and the lanes run along the row)
  auto stage_odd = [&](int kk, const cpx<R>* src) {
    for (int row = wid; row < NR * 9; row += NW) {
      const int r = row / 9, d = row - 9 * r;
      cpx<R>* dst = sv + (size_t)row * svs;
      if (d == 0) {
        for (int c = lane; c < n2; c += 32) dst[c] = mk(R(0), R(0));
        continue;
      }
      const cpx<R>* s = src + r * vstr + nbo[kk * 8 + d - 1];
      const R f = (R)scl[r];
      for (int c = lane; c < n2; c += 32) dst[c] = f * ldc(s + c);
    }
    __syncthreads();
  };
  // odd phase: to[r][ko] = sum_{d>=1} (A_oo^-1 Dc[X][d]) src[r][nbr]
  // block operators streamed from global memory (not resident): warp 0
  // prefetches the next site's into L2 while the CTA works on this one
  const size_t od_bytes = (size_t)8 * n2 * n2 * sizeof(cpx<R>), ev_bytes = (size_t)9 * n2 * n2 * sizeof(cpx<R>);
  auto prefetch_odd = [&](int ko) {
    if (ko < hi && tx < 32) prefetch_l2(a.AD + (size_t)ko * 8 * n2 * n2, od_bytes);
  };
  auto prefetch_even = [&](int ke) {
    if (!a.resident && ke < hi && tx < 32) prefetch_l2(a.Dc + (size_t)a.g.ceven[ke] * 9 * n2 * n2, ev_bytes);
  };
  // ---- block ring ------------------------------------------------------------
  // The blocks a phase multiplies (nd per site, for the CTA's sites in
  // order) are copied into RING shared-memory slots by bulk asynchronous
  // copies that thread 0 issues up to RING - 1 blocks ahead of the CTA's
  // use; slot s completes its copies on ring_full[s].  All threads wait for
  // block b's copy (bounded), then meet at a barrier: past it every thread
  // is done with block b - 1, so its slot may take block b + RING - 1.
  __shared__ __align__(8) uint64_t ring_full[RING];
  unsigned ring_used = 0;      // blocks consumed (the same in every thread)
  unsigned ring_issued = 0;    // blocks whose copy was issued (thread 0)
  if (a.ring && tx == 0) {
    for (int q = 0; q < RING; ++q) mbar_init(&ring_full[q], 1);
    mbar_fence_init();
  }
  // phase products out[si][r][row] = sum_t M_{b(si, t)}[row][c] sv[r][d0 + t][c]
  // for the CTA's sites si < nsites: blk(i) is the address of the phase's
  // block i (site i / nd, direction d0 + i % nd), stage(si) fills sv for
  // site si (ending with a barrier), emit(si, r, row, value) stores a
  // result.  False when a copy did not land in time (status DDAMG_ETIMEOUT
  // set, the copies in flight waited for).
  auto ring_phase = [&](int nsites, int nd, int d0, auto&& blk, auto&& stage, auto&& emit) -> bool {
    if constexpr (sizeof(R) != 4) {
      return false;        // FP32 only (the host never plans a ring otherwise)
    } else {
      using T = typename U16<R>::T;
      constexpr int RPU = 2;                       // complex rows per 16-byte unit
      constexpr int RS = NR >= 8 ? 2 : 1, NRS = NR / RS;
      const unsigned nn = (unsigned)(n2 * n2);
      const unsigned bytes = nn * (unsigned)sizeof(cpx<R>);
      cpx<R>* ringbuf = reinterpret_cast<cpx<R>*>(sm + P.ring);
      const unsigned base = ring_used, end = base + (unsigned)(nsites * nd);
      auto issue = [&](unsigned i) {
        const unsigned q = i % RING;
        mbar_expect_tx(&ring_full[q], bytes);
        bulk_g2s(ringbuf + (size_t)q * nn, blk(i - base), bytes, &ring_full[q]);
      };
      if (tx == 0)
        for (; ring_issued < end && ring_issued < base + RING; ++ring_issued) issue(ring_issued);
      // this thread's unit: row pair j, right-hand-side slice rs, column chunk cc
      const int NP = n2 / RPU;
      int CC = TPB / (NP * RS);
      if (CC > mvp_groups(NR)) CC = mvp_groups(NR);
      if (CC > n2) CC = n2;
      if (CC < 1) CC = 1;
      const int CW = (n2 + CC - 1) / CC;
      const int units = NP * RS * CC;
      const int j = tx % NP, rest = tx / NP, rs = rest % RS, cc = rest / RS;
      const int c0 = cc * CW, c1 = min(n2, c0 + CW);
      const cpx<R>* svr = sv + (size_t)rs * NRS * 9 * svs;
      // Eight right-hand sides on the tensor cores (3xTF32, FP32 accuracy):
      // per site C' (16 x n2) = A' (16 x 2K) B (2K x n2), with A' rows
      // m = r + 8 p the real (p = 0) and imaginary (p = 1) rows of the
      // staged vectors and B the raw blocks.  In a k-step of four complex
      // columns c0 .. c0 + 3, lane t's k = t and k = t + 4 stand for the real
      // and imaginary parts of column c0 + t, so for v = sv[r][d][c0 + t]
      //   A'[r][t] = v.re, A'[r][t + 4] = -v.im, A'[r + 8][t] = v.im, A'[r + 8][t + 4] = v.re
      // and (b0, b1) = M_d[n0 + g][c0 + t] (one 8-byte load).  Warp (kg, ng)
      // takes k-steps 2 kg, 2 kg + 1 of every block and n-tiles
      // ng TPW .. ng TPW + TPW - 1; each block's products go to fresh
      // accumulators added in FP32, the k-groups' partials meet in mvp.
      constexpr int TPWMAX = 4;
      const int NT = n2 / 8, KG = n2 / 8;      // n-tiles; k-groups of two k-steps (n2 / 4 k-steps a block)
      const int NGR = min(NT, NW / (KG > 0 ? KG : 1));
      const int TPW = NGR > 0 ? (NT + NGR - 1) / NGR : 0;
      const bool tc = a.tc && NR == 8 && n2 % 8 == 0 && NGR >= 1 && TPW <= TPWMAX;
      const int gq = lane >> 2, tq = lane & 3;
      const int kg = wid % (KG > 0 ? KG : 1), ng = wid / (KG > 0 ? KG : 1);
      const bool mw = tc && ng < NGR;
      float* mvpf = reinterpret_cast<float*>(mvp);
      for (int si = 0; si < nsites; ++si) {
        // a site's nd blocks are contiguous: the next site's go to L2 now
        if (si + 1 < nsites && tx < 32) prefetch_l2(blk((unsigned)((si + 1) * nd)), (size_t)nd * bytes);
        stage(si);
        cpx<R> acc[NRS][RPU];
#pragma unroll
        for (int r = 0; r < NRS; ++r)
#pragma unroll
          for (int q = 0; q < RPU; ++q) acc[r][q] = mk(R(0), R(0));
        float tacc[TPWMAX][4];
#pragma unroll
        for (int i = 0; i < TPWMAX; ++i)
#pragma unroll
          for (int e = 0; e < 4; ++e) tacc[i][e] = 0.f;
        for (int t = 0; t < nd; ++t) {
          const unsigned b = base + (unsigned)(si * nd + t);
          const bool ok = mbar_wait_bounded(&ring_full[b % RING], (b / RING) & 1u, a.spin_limit);
          if (__syncthreads_or(!ok)) {
            if (tx == 0) {
              atomicExch(a.status, 6);
              for (unsigned i = b; i < ring_issued; ++i)
                mbar_wait_bounded(&ring_full[i % RING], (i / RING) & 1u, MBAR_POLL_LIMIT);
            }
            return false;
          }
          if (tx == 0)
            for (; ring_issued < end && ring_issued < b + RING; ++ring_issued) issue(ring_issued);
          if (tc) {
            if (mw) {
              const float* slot = reinterpret_cast<const float*>(ringbuf + (size_t)(b % RING) * nn);
              const int d = d0 + t;
              float part[TPWMAX][4];
#pragma unroll
              for (int i = 0; i < TPWMAX; ++i)
#pragma unroll
                for (int e = 0; e < 4; ++e) part[i][e] = 0.f;
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const int c = 4 * (2 * kg + h) + tq;
                const cpx<R> v = sv[(size_t)(gq * 9 + d) * svs + c];
                const float af[4] = {v.re, v.im, -v.im, v.re};
                const Split<4> as = split_frag<4>(af);
#pragma unroll
                for (int i = 0; i < TPWMAX; ++i) {
                  const int nt = ng * TPW + i;
                  if (i < TPW && nt < NT) {
                    const float2 mv = *reinterpret_cast<const float2*>(slot + ((size_t)c * n2 + nt * 8 + gq) * 2);
                    const float bv[2] = {mv.x, mv.y};
                    mma3(part[i], as, split_frag<2>(bv));
                  }
                }
              }
#pragma unroll
              for (int i = 0; i < TPWMAX; ++i)
#pragma unroll
                for (int e = 0; e < 4; ++e) tacc[i][e] += part[i][e];
            }
          } else if (tx < units) {
            const T* col = reinterpret_cast<const T*>(ringbuf + (size_t)(b % RING) * nn) + j;
            const int d = d0 + t;
#pragma unroll 4
            for (int c = c0; c < c1; ++c) {
              const T mm = col[(size_t)c * NP];
              const cpx<R> e0 = mk(mm.x, mm.y), e1 = mk(mm.z, mm.w);
#pragma unroll
              for (int r = 0; r < NRS; ++r) {
                const cpx<R> v = svr[(r * 9 + d) * svs + c];
                fma(acc[r][0], e0, v);
                fma(acc[r][1], e1, v);
              }
            }
          }
        }
        if (tc) {
          if (mw)
#pragma unroll
            for (int i = 0; i < TPWMAX; ++i) {
              const int nt = ng * TPW + i;
              if (i < TPW && nt < NT)
#pragma unroll
                for (int e = 0; e < 4; ++e)
                  mvpf[((size_t)kg * 16 + gq + (e >= 2 ? 8 : 0)) * n2 + nt * 8 + 2 * tq + (e & 1)] = tacc[i][e];
            }
          __syncthreads();
          for (int idx = tx; idx < NR * n2; idx += TPB) {
            const int r = idx / n2, row = idx - r * n2;
            float re = 0.f, im = 0.f;
            for (int q = 0; q < KG; ++q) {
              re += mvpf[((size_t)q * 16 + r) * n2 + row];
              im += mvpf[((size_t)q * 16 + 8 + r) * n2 + row];
            }
            emit(si, r, row, mk(re, im));
          }
        } else {
          if (tx < units)
#pragma unroll
            for (int r = 0; r < NRS; ++r)
#pragma unroll
              for (int q = 0; q < RPU; ++q) mvp[((size_t)cc * NR + rs * NRS + r) * n2 + RPU * j + q] = acc[r][q];
          __syncthreads();
          for (int idx = tx; idx < NR * n2; idx += TPB) {
            const int r = idx / n2, row = idx - r * n2;
            cpx<R> sum = mk(R(0), R(0));
            for (int q = 0; q < CC; ++q) sum = sum + mvp[((size_t)q * NR + r) * n2 + row];
            emit(si, r, row, sum);
          }
        }
        __syncthreads();
      }
      ring_used = end;
      return true;
    }
  };

  // odd phase: to[r][ko] = sum_{d>=1} (A_oo^-1 Dc[X][d]) src[r][nbr]
  auto phase_odd = [&](const cpx<R>* src) -> bool {
    if (a.ring) {
      prefetch_even(lo);
      return ring_phase(
          hi - lo, 8, 1, [&](unsigned i) { return a.AD + ((size_t)lo * 8 + i) * n2 * n2; },
          [&](int si) { stage_odd(si, src); },
          [&](int si, int r, int row, cpx<R> v) { a.to[r * vstr + (size_t)(lo + si) * n2 + row] = v; });
    }
    for (int ko = lo; ko < hi; ++ko) {
      const int X = a.g.codd[ko];
      prefetch_odd(ko + 1);
      if (ko + 1 == hi) prefetch_even(lo);
      stage_odd(ko - lo, src);
      mrhs_matvec<R, NR>(a.AD + (size_t)ko * 8 * n2 * n2, sv, 1, 9, n2, mvp, a.to + (size_t)ko * n2, (int)vstr,
                         true);
    }
    return true;
  };
  // stage the vectors of even site ke: its own (self) and the odd neighbours' to
  auto stage_even = [&](int ke, const cpx<R>* vself, bool self) {
    const int kk = ke - lo;
    for (int row = wid; row < NR * 9; row += NW) {
      const int r = row / 9, d = row - 9 * r;
      cpx<R>* dst = sv + (size_t)row * svs;
      if (d == 0 && self) {
        const cpx<R>* s = vself + (size_t)r * L + kk * n2;
        for (int c = lane; c < n2; c += 32) dst[c] = s[c];
      } else if (d == 0) {
        for (int c = lane; c < n2; c += 32) dst[c] = mk(R(0), R(0));
      } else {
        const cpx<R>* s = a.to + r * vstr + nbo[(a.per + kk) * 8 + d - 1];
        for (int c = lane; c < n2; c += 32) dst[c] = -ldc(s + c);
      }
    }
    __syncthreads();
  };
  // even phase: out[r][kk] = (self ? A_ee v : 0) - sum_{d>=1} Dc[X][d] to[r][nbr] (+ bsrc)
  auto phase_even = [&](const cpx<R>* vself, bool self, cpx<R>* out, const cpx<R>* bsrc) -> bool {
    if (a.ring) {
      prefetch_odd(lo);
      const int nd = self ? 9 : 8, d0 = self ? 0 : 1;
      return ring_phase(
          hi - lo, nd, d0,
          [&](unsigned i) {
            return a.Dc + ((size_t)a.g.ceven[lo + (int)(i / (unsigned)nd)] * 9 + d0 + (int)(i % (unsigned)nd)) * n2 * n2;
          },
          [&](int si) { stage_even(lo + si, vself, self); },
          [&](int si, int r, int row, cpx<R> v) {
            if (bsrc) v = v + bsrc[(size_t)r * a.g.nb * n2 + (size_t)a.g.ceven[lo + si] * n2 + row];
            out[(size_t)r * L + si * n2 + row] = v;
          });
    }
    for (int ke = lo; ke < hi; ++ke) {
      const int X = a.g.ceven[ke], kk = ke - lo;
      prefetch_even(ke + 1);
      if (ke + 1 == hi) prefetch_odd(lo);
      stage_even(ke, vself, self);
      if (a.resident)
        mrhs_matvec<R, NR, true>(Mres, sv, self ? 0 : 1, 9, n2, mvp, out + kk * n2, L);
      else
        mrhs_matvec<R, NR>(a.Dc + (size_t)X * 9 * n2 * n2, sv, self ? 0 : 1, 9, n2, mvp, out + kk * n2, L);
      if (bsrc) {
        for (int idx = tx; idx < NR * n2; idx += TPB) {
          const int r = idx / n2, c = idx - r * n2;
          out[(size_t)r * L + kk * n2 + c] = out[(size_t)r * L + kk * n2 + c] + bsrc[(size_t)r * a.g.nb * n2 + (size_t)X * n2 + c];
        }
        __syncthreads();
      }
    }
    return true;
  };
  // partial dots (r, j < kcount) of V_j[r] with wl[r]; slot = j * NR + r
  auto partial = [&](int kcount, bool norm) {
    const int pairs = norm ? NR : kcount * NR;
    for (int pr = wid; pr < pairs; pr += NW) {
      const int j = norm ? 0 : pr / NR, r = norm ? pr : pr - (pr / NR) * NR;
      R re = 0, im = 0;
      if (act[r]) {
        const cpx<R>* vj = norm ? wl + (size_t)r * L : Vk(j, r);
        const cpx<R>* ww = wl + (size_t)r * L;
        for (int e = lane; e < Lo; e += 32) {
          cpx<R> p = vj[e], q = ww[e];
          re += p.re * q.re + p.im * q.im;
          im += p.re * q.im - p.im * q.re;
        }
      }
      re = wsum(re);
      im = wsum(im);
      if (lane == 0) {
        a.part[((size_t)pr * G + blockIdx.x) * 2] = (double)re;
        a.part[((size_t)pr * G + blockIdx.x) * 2 + 1] = (double)im;
      }
    }
  };
  // gather slot sums into dst[r][2 j] (norm: dst[r])
  auto gather = [&](int kcount, bool norm, A* dst, int dstride) {
    const int pairs = norm ? NR : kcount * NR;
    for (int pr = wid; pr < pairs; pr += NW) {
      A re = 0, im = 0;
      for (int c = lane; c < G; c += 32) {
        re += (A)__ldcg(a.part + ((size_t)pr * G + c) * 2);
        im += (A)__ldcg(a.part + ((size_t)pr * G + c) * 2 + 1);
      }
      re = wsum(re);
      im = wsum(im);
      if (lane == 0) {
        if (norm) {
          dst[(size_t)pr * dstride] = re;     // squared norm (real)
        } else {
          const int j = pr / NR, r = pr - j * NR;
          dst[(size_t)r * dstride + 2 * j] = re;
          dst[(size_t)r * dstride + 2 * j + 1] = im;
        }
      }
    }
    __syncthreads();
  };

  // gather(kcount, false, hc, dstride) and gather_norm_slot(kcount, hn) in
  // one pass: one round of L2 loads instead of two
  auto gather_dots_norm = [&](int kcount, A* dst, int dstride, A* hn) {
    const int pairs = (kcount + 1) * NR;
    for (int pr = wid; pr < pairs; pr += NW) {
      A re = 0, im = 0;
      for (int c = lane; c < G; c += 32) {
        re += (A)__ldcg(a.part + ((size_t)pr * G + c) * 2);
        im += (A)__ldcg(a.part + ((size_t)pr * G + c) * 2 + 1);
      }
      re = wsum(re);
      im = wsum(im);
      if (lane == 0) {
        const int j = pr / NR, r = pr - j * NR;
        if (j < kcount) {
          dst[(size_t)r * dstride + 2 * j] = re;
          dst[(size_t)r * dstride + 2 * j + 1] = im;
        } else {
          hn[r] = re;                  // squared norm (real)
        }
      }
    }
    __syncthreads();
  };

  // squared norms of wl[r] into the slots after the (kcount x NR) dot slots
  auto partial_norm_slot = [&](int kcount) {
    for (int r = wid; r < NR; r += NW) {
      R sq = 0;
      if (act[r]) {
        const cpx<R>* ww = wl + (size_t)r * L;
        for (int e = lane; e < Lo; e += 32) sq += norm2(ww[e]);
      }
      sq = wsum(sq);
      if (lane == 0) {
        const size_t pr = (size_t)kcount * NR + r;
        a.part[(pr * G + blockIdx.x) * 2] = (double)sq;
        a.part[(pr * G + blockIdx.x) * 2 + 1] = 0.0;
      }
    }
  };
  auto gather_norm_slot = [&](int kcount, A* dst) {
    for (int r = wid; r < NR; r += NW) {
      const size_t pr = (size_t)kcount * NR + r;
      A sq = 0;
      for (int c = lane; c < G; c += 32) sq += (A)__ldcg(a.part + (pr * G + c) * 2);
      sq = wsum(sq);
      if (lane == 0) dst[r] = sq;
    }
    __syncthreads();
  };

  for (int r0 = 0; r0 < a.nrhs; r0 += NR) {
    const int nr = min(NR, a.nrhs - r0);
    const cpx<R>* bb = a.b + (size_t)r0 * a.g.nb * n2;
    cpx<R>* xx = a.x + (size_t)r0 * a.g.nb * n2;
    if (tx < NR) {
      act[tx] = tx < nr ? 1 : 0;
      conv[tx] = tx < nr ? 0 : 1;
      tot[tx] = 0;
      scl[tx] = A(1);
    }
    __syncthreads();
    // to = A_oo^-1 b_o
    for (int ko = lo; ko < hi; ++ko) {
      const int X = a.g.codd[ko];
      for (int idx = tx; idx < NR * n2; idx += TPB) {
        const int r = idx / n2, c = idx - r * n2;
        sv[(r * 9) * svs + c] = r < nr ? bb[(size_t)r * a.g.nb * n2 + (size_t)X * n2 + c] : mk(R(0), R(0));
      }
      __syncthreads();
      mrhs_matvec<R, NR>(a.Ainv + (size_t)X * n2 * n2, sv, 0, 1, n2, mvp, a.to + (size_t)ko * n2, (int)vstr);
    }
    if (!grid_barrier(a.bar, a.status, a.spin_limit)) return;
    // rhs_e = b_e - D_eo to ; x_e = 0 ; w = rhs_e
    if (!phase_even(nullptr, false, rl, bb)) return;
    for (int idx = tx; idx < NR * L; idx += TPB) {
      const int r = idx / L, e = idx - r * L;
      cpx<R> v = (r < nr && e < Lo) ? rl[idx] : mk(R(0), R(0));
      rl[idx] = v;
      wl[idx] = v;
      xl[idx] = mk(R(0), R(0));
    }
    __syncthreads();
    partial(1, true);
    if (!grid_barrier(a.bar, a.status, a.spin_limit)) return;
    gather(1, true, bnorm, 1);
    if (tx < NR) {
      bnorm[tx] = sqrt(bnorm[tx]);
      beta[tx] = bnorm[tx];
      if (!(bnorm[tx] > A(0))) { conv[tx] = 1; act[tx] = 0; }
    }
    __syncthreads();

    while (true) {
      // start a cycle for every right-hand side that is not done
      if (tx < NR) {
        const bool go = !conv[tx] && tot[tx] < a.max_iter;
        act[tx] = go ? 1 : 0;
        if (!go) conv[tx] = 1;
        kd[tx] = 0;
        gv[tx * 2 * (m + 1)] = beta[tx];
        gv[tx * 2 * (m + 1) + 1] = A(0);
        scl[tx] = beta[tx] > A(0) ? A(1) / beta[tx] : A(0);
      }
      __syncthreads();
      if (tx == 0) {
        int any = 0;
        for (int r = 0; r < NR; ++r) any |= act[r];
        any_s = any;
      }
      __syncthreads();
      if (!any_s) break;
      // V_0 = w / beta (local) and the global copy of w for the neighbours
      for (int idx = tx; idx < NR * L; idx += TPB) {
        const int r = idx / L, e = idx - r * L;
        cpx<R> v = wl[idx];
        Vk(0, r)[e] = (R)scl[r] * v;
        if (e < Lo) a.wg[r * vstr + (size_t)lo * n2 + e] = v;
      }
      if (!grid_barrier(a.bar, a.status, a.spin_limit)) return;
      for (int k = 0; k < m; ++k) {
        // w = S V_k: odd phase from the neighbours' unnormalised w (scale 1/h)
        if (!phase_odd(a.wg)) return;
        if (!grid_barrier(a.bar, a.status, a.spin_limit)) return;
        if (!phase_even(V + (size_t)k * NR * L, true, wl, nullptr)) return;
        // Givens rotation of right-hand side r's new Hessenberg column (one
        // thread), new residual estimate, scale 1/h of V_{k+1}, convergence
        auto givens = [&](int r) {
          const A hn = sqrt(hnv[r]);
          A* col = hc + (size_t)r * 2 * (m + 1);   // this column of the Hessenberg matrix
          col[2 * (k + 1)] = hn;
          col[2 * (k + 1) + 1] = A(0);
          A* csr = cs + (size_t)r * m;
          A* snr = sn + (size_t)r * 2 * m;
          for (int j = 0; j < k; ++j) {
            A c = csr[j], sr = snr[2 * j], si = snr[2 * j + 1];
            A ar = col[2 * j], ai = col[2 * j + 1], br = col[2 * j + 2], bi = col[2 * j + 3];
            A tr = c * ar + (sr * br - si * bi), ti = c * ai + (sr * bi + si * br);
            A ur = -(sr * ar + si * ai) + c * br, ui = -(sr * ai - si * ar) + c * bi;
            col[2 * j] = tr; col[2 * j + 1] = ti; col[2 * j + 2] = ur; col[2 * j + 3] = ui;
          }
          A ar = col[2 * k], ai = col[2 * k + 1], br = col[2 * k + 2], bi = col[2 * k + 3];
          A a1 = sqrt(ar * ar + ai * ai), a2 = sqrt(br * br + bi * bi);
          A c, sr, si, rr, ri;
          if (a2 == A(0)) { c = A(1); sr = A(0); si = A(0); rr = ar; ri = ai; }
          else if (a1 == A(0)) { c = A(0); sr = br / a2; si = -bi / a2; rr = a2; ri = A(0); }
          else {
            A rho = hypot(a1, a2);
            A pr = ar / a1, pi = ai / a1;
            c = a1 / rho;
            sr = (pr * br + pi * bi) / rho;
            si = (pi * br - pr * bi) / rho;
            rr = pr * rho; ri = pi * rho;
          }
          csr[k] = c; snr[2 * k] = sr; snr[2 * k + 1] = si;
          col[2 * k] = rr; col[2 * k + 1] = ri;
          A* Rr = Rf + (size_t)r * 2 * TRI;
          const int base = k * (k + 1) / 2;          // packed column k: entries 0..k
          for (int j = 0; j <= k; ++j) { Rr[2 * (base + j)] = col[2 * j]; Rr[2 * (base + j) + 1] = col[2 * j + 1]; }
          A* g = gv + (size_t)r * 2 * (m + 1);
          A gr = g[2 * k], gi = g[2 * k + 1];
          g[2 * (k + 1)] = -(sr * gr + si * gi);
          g[2 * (k + 1) + 1] = -(sr * gi - si * gr);
          g[2 * k] = c * gr;
          g[2 * k + 1] = c * gi;
          A res = sqrt(g[2 * (k + 1)] * g[2 * (k + 1)] + g[2 * (k + 1) + 1] * g[2 * (k + 1) + 1]);
          kd[r] = k + 1;
          tot[r] += 1;
          scl[r] = hn > A(0) ? A(1) / hn : A(0);
          hnv[r] = hn;
          if (res <= (A)a.tol * bnorm[r] || hn == A(0) || tot[r] >= a.max_iter) act[r] = 0;
        };
        if constexpr (sizeof(R) == 4) {
          // FP32: one classical Gram-Schmidt pass whose reduction also carries
          // ||w||^2, so ||w_new||^2 = ||w||^2 - sum_j |h_j|^2 (Pythagoras); an
          // explicit norm is taken only if that difference has cancelled
          partial(k + 1, false);
          partial_norm_slot(k + 1);
          if (!grid_barrier(a.bar, a.status, a.spin_limit)) return;
          gather_dots_norm(k + 1, hc, 2 * (m + 1), hnv);
          if (tx < NR) {
            const A* hr = hc + (size_t)tx * 2 * (m + 1);
            A s2 = hnv[tx];
            for (int j = 0; j <= k; ++j) s2 -= hr[2 * j] * hr[2 * j] + hr[2 * j + 1] * hr[2 * j + 1];
            exn[tx] = (act[tx] && !(s2 > A(1e-3) * hnv[tx])) ? 1 : 0;
            hnv[tx] = s2 > A(0) ? s2 : A(0);
          }
          __syncthreads();
          if (tx == 0) {
            int any = 0;
            for (int r = 0; r < NR; ++r) any |= exn[r];
            any_s = any;
          }
          for (int idx = tx; idx < NR * Lo; idx += TPB) {
            const int r = idx / Lo, e = idx - r * Lo;
            if (!act[r]) continue;
            cpx<R> w0 = wl[(size_t)r * L + e];
            const A* hr = hc + (size_t)r * 2 * (m + 1);
            for (int j = 0; j <= k; ++j) {
              cpx<R> v = Vk(j, r)[e];
              cpx<R> c = mk((R)hr[2 * j], (R)hr[2 * j + 1]);
              w0 = w0 - c * v;
            }
            wl[(size_t)r * L + e] = w0;
            a.wg[r * vstr + (size_t)lo * n2 + e] = w0;
          }
          __syncthreads();
          if (any_s) {
            partial(1, true);
            if (!grid_barrier(a.bar, a.status, a.spin_limit)) return;
            gather(1, true, h2, 1);
            if (tx < NR && exn[tx]) hnv[tx] = h2[tx];
            __syncthreads();
            if (tx < NR && act[tx]) givens(tx);
            __syncthreads();
          } else {
            // publish w for the next odd phase; the Givens step and the new
            // basis vector are local work done while the other CTAs arrive
            grid_arrive(a.bar);
            if (tx < NR && act[tx]) givens(tx);
            __syncthreads();
          }
          for (int idx = tx; idx < NR * Lo; idx += TPB) {
            const int r = idx / Lo, e = idx - r * Lo;
            Vk(k + 1, r)[e] = (R)scl[r] * wl[(size_t)r * L + e];
          }
          if (tx == 0) {
            int any = 0;
            for (int r = 0; r < NR; ++r) any |= act[r];
            any_act_s = any;
          }
          if (!any_s) {
            if (!grid_wait(a.bar, a.status, a.spin_limit)) return;
          } else {
            __syncthreads();
          }
          if (!any_act_s) break;
        } else {
          // FP64: classical Gram-Schmidt with one re-orthogonalisation pass
          for (int pass = 0; pass < 2; ++pass) {
            partial(k + 1, false);
            if (!grid_barrier(a.bar, a.status, a.spin_limit)) return;
            A* hh = pass == 0 ? hc : h2;
            gather(k + 1, false, hh, 2 * (m + 1));
            for (int idx = tx; idx < NR * Lo; idx += TPB) {
              const int r = idx / Lo, e = idx - r * Lo;
              if (!act[r]) continue;
              cpx<R> w0 = wl[(size_t)r * L + e];
              const A* hr = hh + (size_t)r * 2 * (m + 1);
              for (int j = 0; j <= k; ++j) {
                cpx<R> v = Vk(j, r)[e];
                cpx<R> c = mk((R)hr[2 * j], (R)hr[2 * j + 1]);
                w0 = w0 - c * v;
              }
              wl[(size_t)r * L + e] = w0;
              if (pass == 1) a.wg[r * vstr + (size_t)lo * n2 + e] = w0;
            }
            if (pass == 1 && tx < NR)
              for (int j = 0; j <= k; ++j) {
                hc[(size_t)tx * 2 * (m + 1) + 2 * j] += h2[(size_t)tx * 2 * (m + 1) + 2 * j];
                hc[(size_t)tx * 2 * (m + 1) + 2 * j + 1] += h2[(size_t)tx * 2 * (m + 1) + 2 * j + 1];
              }
            __syncthreads();
          }
          // ||w||: this barrier also publishes the neighbours' w for the next odd phase
          partial(1, true);
          if (!grid_barrier(a.bar, a.status, a.spin_limit)) return;
          gather(1, true, hnv, 1);
          if (tx < NR && act[tx]) givens(tx);
          __syncthreads();
          for (int idx = tx; idx < NR * Lo; idx += TPB) {
            const int r = idx / Lo, e = idx - r * Lo;
            Vk(k + 1, r)[e] = (R)scl[r] * wl[(size_t)r * L + e];
          }
          if (tx == 0) {
            int any = 0;
            for (int r = 0; r < NR; ++r) any |= act[r];
            any_act_s = any;
          }
          __syncthreads();
          if (!any_act_s) break;
        }
      }
      // y = R^-1 g ; x_e += V y   (every right-hand side of this cycle)
      if (tx < NR && !conv[tx]) {
        const int r = tx, kk = kd[r];
        const A* Rr = Rf + (size_t)r * 2 * TRI;
        const A* g = gv + (size_t)r * 2 * (m + 1);
        A* y = yv + (size_t)r * 2 * m;
        for (int i = kk - 1; i >= 0; --i) {
          A accr = g[2 * i], acci = g[2 * i + 1];
          for (int j = i + 1; j < kk; ++j) {
            const int pj = j * (j + 1) / 2 + i;
            A rr = Rr[2 * pj], ri = Rr[2 * pj + 1];
            accr -= rr * y[2 * j] - ri * y[2 * j + 1];
            acci -= rr * y[2 * j + 1] + ri * y[2 * j];
          }
          const int pd = i * (i + 1) / 2 + i;
          A dr = Rr[2 * pd], di = Rr[2 * pd + 1];
          A dn = dr * dr + di * di;
          y[2 * i] = (accr * dr + acci * di) / dn;
          y[2 * i + 1] = (acci * dr - accr * di) / dn;
        }
      }
      __syncthreads();
      for (int idx = tx; idx < NR * Lo; idx += TPB) {
        const int r = idx / Lo, e = idx - r * Lo;
        if (conv[r]) continue;
        const A* y = yv + (size_t)r * 2 * m;
        cpx<R> s = xl[(size_t)r * L + e];
        for (int j = 0; j < kd[r]; ++j) s = s + mk((R)y[2 * j], (R)y[2 * j + 1]) * Vk(j, r)[e];
        xl[(size_t)r * L + e] = s;
        a.xg[r * vstr + (size_t)lo * n2 + e] = s;
      }
      if (tx < NR) scl[tx] = A(1);
      if (!grid_barrier(a.bar, a.status, a.spin_limit)) return;
      // true residual w = rhs_e - S x_e
      if (!phase_odd(a.xg)) return;
      if (!grid_barrier(a.bar, a.status, a.spin_limit)) return;
      if (!phase_even(xl, true, wl, nullptr)) return;
      for (int idx = tx; idx < NR * Lo; idx += TPB) {
        const int r = idx / Lo, e = idx - r * Lo;
        wl[(size_t)r * L + e] = rl[(size_t)r * L + e] - wl[(size_t)r * L + e];
      }
      if (tx < NR) act[tx] = conv[tx] ? 0 : 1;
      __syncthreads();
      partial(1, true);
      if (!grid_barrier(a.bar, a.status, a.spin_limit)) return;
      gather(1, true, beta, 1);
      if (tx < NR && !conv[tx]) {
        beta[tx] = sqrt(beta[tx]);
        if (beta[tx] <= (A)a.tol * bnorm[tx]) conv[tx] = 1;
      }
      __syncthreads();
    }
    // x_o = A_oo^-1 (b_o - D_oe x_e); write x
    for (int idx = tx; idx < NR * Lo; idx += TPB) {
      const int r = idx / Lo, e = idx - r * Lo;
      a.xg[r * vstr + (size_t)lo * n2 + e] = xl[(size_t)r * L + e];
    }
    if (tx < NR) scl[tx] = -A(1);
    if (!grid_barrier(a.bar, a.status, a.spin_limit)) return;
    for (int ko = lo; ko < hi; ++ko) {
      const int X = a.g.codd[ko];
      stage_odd(ko - lo, a.xg);
      mrhs_matvec<R, NR>(a.Dc + (size_t)X * 9 * n2 * n2, sv, 1, 9, n2, mvp, tmp, n2);
      for (int idx = tx; idx < NR * n2; idx += TPB) {
        const int r = idx / n2, c = idx - r * n2;
        sv[(r * 9) * svs + c] = tmp[idx] + (r < nr ? bb[(size_t)r * a.g.nb * n2 + (size_t)X * n2 + c] : mk(R(0), R(0)));
      }
      __syncthreads();
      mrhs_matvec<R, NR>(a.Ainv + (size_t)X * n2 * n2, sv, 0, 1, n2, mvp, tmp, n2);
      for (int idx = tx; idx < nr * n2; idx += TPB) {
        const int r = idx / n2, c = idx - r * n2;
        xx[(size_t)r * a.g.nb * n2 + (size_t)X * n2 + c] = tmp[idx];
      }
    }
    for (int idx = tx; idx < nr * Lo; idx += TPB) {
      const int r = idx / Lo, e = idx - r * Lo;
      const int ke = lo + e / n2, c = e - (e / n2) * n2;
      xx[(size_t)r * a.g.nb * n2 + (size_t)a.g.ceven[ke] * n2 + c] = xl[(size_t)r * L + e];
    }
    if (blockIdx.x == 0 && tx < nr) {
      if (a.iters) a.iters[r0 + tx] = tot[tx];
      if (a.iters_acc) atomicAdd(a.iters_acc, tot[tx]);
    }
    if (!grid_barrier(a.bar, a.status, a.spin_limit)) return;
  }
}

constexpr size_t SMEM_BUDGET = 200 * 1024;
constexpr size_t SMEM_RESIDENT_MAX = 224 * 1024;   // with resident blocks: one CTA per SM

template <class R>
const void* kernel_for(int NR) {
  switch (NR) {
    case 1: return (const void*)k_cgmres<R, 1>;
    case 2: return (const void*)k_cgmres<R, 2>;
    case 4: return (const void*)k_cgmres<R, 4>;
    case 8: return (const void*)k_cgmres<R, 8>;
    default: return (const void*)k_cgmres<R, 12>;
  }
}

struct Choice {
  int NR, G, per;
  bool local;
  Plan plan;
  bool resident;
  bool ring;
};

// Host state of the launch configurations: the dynamic shared-memory limit
// last set on each kernel instance per device (cudaFuncSetAttribute acts on
// the current device) and the cache of chosen configurations.  Several host
// threads may solve on different handles at once, so both are guarded by one
// mutex.
std::mutex g_cfg_mu;

constexpr int MAXDEV = 64;

// completion of the last cooperative coarse-GMRES launch per device
std::mutex g_coop_mu;
cudaEvent_t g_coop_done[MAXDEV] = {};

inline int nr_slot(int NR) { return NR == 1 ? 0 : NR == 2 ? 1 : NR == 4 ? 2 : NR == 8 ? 3 : 4; }

// caller holds g_cfg_mu
template <class R>
cudaError_t smem_attr_locked(int dev, int NR, size_t bytes) {
  static size_t current[MAXDEV][5] = {};
  if (dev < 0 || dev >= MAXDEV) return cudaErrorInvalidDevice;
  // the limit only grows: a thread that sized its launch for a plan and
  // released the lock must not find the limit lowered by another thread's
  // smaller plan when it launches
  size_t& c = current[dev][nr_slot(NR)];
  if (c >= bytes) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel_for<R>(NR), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) c = bytes;
  return e;
}

// widest lockstep group for nrhs right-hand sides (instances 1, 2, 4, 8, 12)
inline int first_nr(int nrhs) { return nrhs >= 12 ? 12 : nrhs >= 8 ? 8 : nrhs >= 4 ? 4 : nrhs >= 2 ? 2 : 1; }

template <class R>
Choice choose_uncached(int dev, const Geom& g, int n2, int m, int nrhs);

// launch configurations are cached: the occupancy queries behind them cost
// far more host time than a coarse solve's launch
template <class R>
Choice choose(const Geom& g, int n2, int m, int nrhs) {
  struct Entry {
    int dev, nb, n2, m, first;
    Choice c;
  };
  static Entry cache[16];
  static int used = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  const int first = first_nr(nrhs);
  std::lock_guard<std::mutex> lock(g_cfg_mu);
  for (int i = 0; i < used; ++i) {
    const Entry& e = cache[i];
    if (e.dev == dev && e.nb == g.nb && e.n2 == n2 && e.m == m && e.first == first) return e.c;
  }
  Choice c = choose_uncached<R>(dev, g, n2, m, nrhs);
  Entry e{dev, g.nb, n2, m, first, c};
  cache[used < 16 ? used++ : (dev + g.nb + first) % 16] = e;
  return c;
}

template <class R>
Choice choose_uncached(int dev, const Geom& g, int n2, int m, int nrhs) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int NE = g.nb / 2;
  Choice best{};
  for (int NR = first_nr(nrhs); NR >= 1; NR = NR == 12 ? 8 : NR / 2) {
    for (int pass = 0; pass < 2; ++pass) {
      const bool local = pass == 0;
      // grid: as many CTAs as fit (two per SM at most), each owning >= 1 site
      for (int per = 1; per <= NE; ++per) {
        int G = (NE + per - 1) / per;
        const void* fn = kernel_for<R>(NR);
        int occ = 0;
        if (per == 1 && local) {
          // one even site per CTA, its D_c blocks resident in shared memory
          Plan pr = make_plan(NR, n2, n2, m, sizeof(R), true, true);
          if (pr.bytes <= SMEM_RESIDENT_MAX && smem_attr_locked<R>(dev, NR, pr.bytes) == cudaSuccess &&
              cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, TPB, pr.bytes) == cudaSuccess &&
              occ >= 1 && G <= occ * sms)
            return Choice{NR, G, per, true, pr, true, false};
          cudaGetLastError();
        }
        if (sizeof(R) == 4 && n2 >= RING_MIN_N2 && n2 <= 256) {
          // the block operators streamed through a ring when it fits
          Plan pg = make_plan(NR, per * n2, n2, m, sizeof(R), local, false, true);
          int og = 0;
          if (pg.bytes <= SMEM_RESIDENT_MAX && smem_attr_locked<R>(dev, NR, pg.bytes) == cudaSuccess &&
              cudaOccupancyMaxActiveBlocksPerMultiprocessor(&og, fn, TPB, pg.bytes) == cudaSuccess &&
              og >= 1 && G <= og * sms)
            return Choice{NR, G, per, local, pg, false, true};
          cudaGetLastError();
        }
        Plan p = make_plan(NR, per * n2, n2, m, sizeof(R), local);
        if (p.bytes > SMEM_BUDGET) break;
        if (smem_attr_locked<R>(dev, NR, p.bytes) != cudaSuccess) break;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, TPB, p.bytes);
        if (occ < 1) break;
        if (G <= occ * sms) return Choice{NR, G, per, local, p, false, false};
      }
    }
  }
  return best;
}

}  // namespace

template <class R>
CoarsePlan coarse_gmres_plan(const Geom& g, int n, int restart, int nrhs) {
  CoarsePlan out{};
  if (restart > MAXM || restart < 1 || nrhs < 1) return out;
  Choice ch = choose<R>(g, 2 * n, restart, nrhs);
  if (ch.NR == 0) return out;
  out.NR = ch.NR;
  out.G = ch.G;
  out.per = ch.per;
  out.local_in_smem = ch.local ? 1 : 0;
  out.resident = ch.resident ? 1 : 0;
  out.ring = ch.ring ? 1 : 0;
  out.smem_bytes = ch.plan.bytes;
  // the layout of coarse_gmres() below
  const size_t NE = g.nb / 2, n2 = 2 * n;
  size_t bytes = al16(3 * (size_t)NRMAX * NE * n2 * sizeof(cpx<R>));
  bytes += al16((size_t)(MAXM + 2) * NRMAX * NE * 2 * sizeof(double));
  bytes += 256;
  if (!ch.local) bytes += (size_t)ch.G * al16(ch.plan.local_bytes);
  out.work_bytes = bytes;
  return out;
}
template CoarsePlan coarse_gmres_plan<float>(const Geom&, int, int, int);
template CoarsePlan coarse_gmres_plan<double>(const Geom&, int, int, int);

template <class R>
size_t coarse_gmres_exact_bytes(const Geom& g, int n, int restart, int nrhs) {
  return coarse_gmres_plan<R>(g, n, restart, nrhs).work_bytes;
}
template size_t coarse_gmres_exact_bytes<float>(const Geom&, int, int, int);
template size_t coarse_gmres_exact_bytes<double>(const Geom&, int, int, int);

size_t coarse_gmres_work_bytes(const Geom& g, int n, int restart, int real_size) {
  // vectors wg, to, xg for NRMAX right-hand sides, partial sums, barrier,
  // and room for per-CTA local arrays when they do not fit in shared memory
  const size_t NE = g.nb / 2, n2 = 2 * n;
  const size_t vec = NRMAX * NE * n2 * 2 * (size_t)real_size;
  size_t bytes = al16(3 * vec);
  bytes += al16((size_t)(MAXM + 2) * NRMAX * NE * 2 * sizeof(double));
  bytes += 256;
  bytes += al16((size_t)(restart + 4) * NRMAX * 2 * NE * n2 * 2 * real_size + 64 * NE);
  return bytes;
}

template <class R>
cudaError_t coarse_gmres(const Geom& g, const CoarseSolveArgs& ca, const R* b, R* x, int nrhs, void* work,
                         int* iters, int* iters_acc, int* status, cudaStream_t st, const CoarsePlan* sized) {
  if (ca.restart > MAXM || ca.restart < 1 || nrhs < 1) return cudaErrorInvalidValue;
  const int n2 = 2 * ca.n;
  Choice ch = choose<R>(g, n2, ca.restart, nrhs);
  if (ch.NR == 0) return cudaErrorInvalidConfiguration;
  // a caller that sized `work` for a plan must get exactly that plan
  if (sized && (sized->NR != ch.NR || sized->G != ch.G || sized->per != ch.per ||
                sized->local_in_smem != (ch.local ? 1 : 0) || sized->resident != (ch.resident ? 1 : 0) ||
                sized->ring != (ch.ring ? 1 : 0)))
    return cudaErrorInvalidValue;
  CGA<R> a;
  a.g = g;
  a.Dc = reinterpret_cast<const cpx<R>*>(ca.Dc);
  a.Ainv = reinterpret_cast<const cpx<R>*>(ca.Ainv);
  a.AD = reinterpret_cast<const cpx<R>*>(ca.AinvD);
  a.n2 = n2;
  a.tol = ca.tol;
  a.m = ca.restart;
  a.max_iter = ca.max_iter;
  a.b = reinterpret_cast<const cpx<R>*>(b);
  a.x = reinterpret_cast<cpx<R>*>(x);
  a.nrhs = nrhs;
  a.NR = ch.NR;
  a.NE = g.nb / 2;
  a.per = ch.per;
  a.local_in_smem = ch.local ? 1 : 0;
  a.resident = ch.resident ? 1 : 0;
  a.ring = ch.ring ? 1 : 0;
  a.tc = ca.tc;
  const size_t NE = a.NE;
  const size_t vec = (size_t)NRMAX * NE * n2;
  unsigned char* w8 = reinterpret_cast<unsigned char*>(work);
  a.wg = reinterpret_cast<cpx<R>*>(w8);
  a.to = a.wg + vec;
  a.xg = a.to + vec;
  size_t off = al16(3 * vec * sizeof(cpx<R>));
  a.part = reinterpret_cast<double*>(w8 + off);
  off += al16((size_t)(MAXM + 2) * NRMAX * NE * 2 * sizeof(double));
  a.bar = reinterpret_cast<unsigned*>(w8 + off);
  off += 256;
  a.lglob = w8 + off;
  a.lstride = al16(ch.plan.local_bytes);
  a.iters = iters;
  a.iters_acc = iters_acc;
  a.status = status;
  a.spin_limit = ca.wait_limit;
  cudaError_t e = cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  const void* fn = kernel_for<R>(ch.NR);
  {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(g_cfg_mu);
    e = smem_attr_locked<R>(dev, ch.NR, ch.plan.bytes);
  }
  if (e != cudaSuccess) return e;
  void* args[] = {&a};
  // Cooperative launches from different streams (several batches served at
  // once) must not overlap: each sizes its grid for the whole GPU and spins
  // on a grid barrier, so two of them sharing the SMs could wait on each
  // other's blocks.  Outside stream capture every launch waits for the
  // previous one of the process on this device.
  int dev = 0;
  cudaGetDevice(&dev);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess) return e;
  const bool order = cap == cudaStreamCaptureStatusNone && dev >= 0 && dev < MAXDEV;
  std::unique_lock<std::mutex> order_lock(g_coop_mu, std::defer_lock);
  if (order) {
    order_lock.lock();
    if (!g_coop_done[dev]) {
      e = cudaEventCreateWithFlags(&g_coop_done[dev], cudaEventDisableTiming);
      if (e != cudaSuccess) return e;
    } else {
      e = cudaStreamWaitEvent(st, g_coop_done[dev], 0);
      if (e != cudaSuccess) return e;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ch.G);
  cfg.blockDim = dim3(TPB);
  cfg.dynamicSmemBytes = ch.plan.bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;   // all CTAs co-resident (grid barrier)
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelExC(&cfg, fn, args);
  ++g_launches;
  if (e == cudaSuccess && order) e = cudaEventRecord(g_coop_done[dev], st);
  return e;
}

// A captured graph that holds a cooperative coarse-GMRES launch joins the
// order of the cooperative launches made outside graphs: it waits for the
// previous one of the process on this device, and the next one waits for it
cudaError_t launch_graph_ordered(cudaGraphExec_t g, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAXDEV) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_coop_mu);
  if (!g_coop_done[dev]) {
    e = cudaEventCreateWithFlags(&g_coop_done[dev], cudaEventDisableTiming);
  } else {
    e = cudaStreamWaitEvent(st, g_coop_done[dev], 0);
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphLaunch(g, st);
  if (e == cudaSuccess) e = cudaEventRecord(g_coop_done[dev], st);
  return e;
}

template cudaError_t coarse_gmres<float>(const Geom&, const CoarseSolveArgs&, const float*, float*, int, void*,
                                         int*, int*, int*, cudaStream_t, const CoarsePlan*);
template cudaError_t coarse_gmres<double>(const Geom&, const CoarseSolveArgs&, const double*, double*, int,
                                          void*, int*, int*, int*, cudaStream_t, const CoarsePlan*);

}  // namespace ddamg
