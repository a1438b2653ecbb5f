// Host-side launchers of the library's CUDA kernels (no torch types).  Every
// launcher enqueues on `st` and returns the cudaGetLastError() of its launch.
#pragma once

#include <cstddef>
#include <atomic>
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace ddamg {

// Geometry of the fine lattice as the kernels see it.
struct Geom {
  int L[4];        // lattice extents
  int b[4];        // Schwarz block (= aggregate) extents
  int grid[4];     // blocks per direction
  int V;           // sites
  int Vb;          // sites per block
  int nb;          // blocks (= coarse sites)
  const uint32_t* nbr;      // [8][V] neighbour device index | NEG_BIT, dir 2mu fwd, 2mu+1 bwd
  const int* lex_of_dev;    // [V]
  const int16_t* bnbr;      // [8][Vb] block-local neighbour (other parity half index) or -1
  const int16_t* face;      // [8][Vb] block-local sites whose hop in dir leaves the block
                            //   (first Vb / b[mu] entries of each row are used)
  const int* cnbr;          // [9][nb] coarse neighbour of each stencil direction
  const int* cparity;       // [nb] coarse parity
  const int* ceven;         // [nb/2] coarse sites of parity 0
  const int* codd;          // [nb/2] coarse sites of parity 1
  const int* cpos;          // [nb] position of a coarse site in its parity list
};

// Kernel launch counter: every launcher adds its launches to the process
// total (atomic, any host thread) and to a per-thread count, which lets a
// thread that captures a CUDA graph tell its own captured launches apart.
struct LaunchCount {
  std::atomic<uint64_t> all{0};
  static uint64_t& mine() {
    static thread_local uint64_t m = 0;
    return m;
  }
  void add(uint64_t n) {
    all.fetch_add(n, std::memory_order_relaxed);
    mine() += n;
  }
  // launches that were recorded into a graph, not run
  void remove_mine(uint64_t n) {
    all.fetch_sub(n, std::memory_order_relaxed);
    mine() -= n;
  }
  LaunchCount& operator++() {
    add(1);
    return *this;
  }
  LaunchCount& operator+=(uint64_t n) {
    add(n);
    return *this;
  }
  uint64_t total() const { return all.load(std::memory_order_relaxed); }
};
extern LaunchCount g_launches;

// ---- layout conversion ------------------------------------------------------
// host layout (FP64 lexicographic, interleaved complex) <-> device fields
template <class R>
cudaError_t pack_spinor(const Geom& g, const double* lex, R* dev, int nrhs, cudaStream_t st);
template <class R>
cudaError_t unpack_spinor(const Geom& g, const R* dev, double* lex, int nrhs, cudaStream_t st);
// flat element-wise conversion (same layout on both sides: coarse vectors)
template <class RD, class RS>
cudaError_t convert_field(const RS* src, RD* dst, size_t nreal, cudaStream_t st);
// spinor fields between the FP64 and FP32 device layouts (nf fields)
template <class RD, class RS>
cudaError_t convert_spinor(const Geom& g, const RS* src, RD* dst, int nf, cudaStream_t st);

// ---- gauge and clover -------------------------------------------------------
// compress lexicographic FP64 links into the two-row device layouts; the
// largest deviation from SU(3) (|U U^H - 1|, |det U - 1|) is max-reduced into
// *dev_dev (as ordered bits of a non-negative double)
cudaError_t import_gauge(const Geom& g, const double* lex, double* g64, float* g32,
                         unsigned long long* dev_dev, cudaStream_t st);
// A = (4 + m0) + C and A^-1, packed, in FP64 and FP32 device layouts
cudaError_t build_clover(const Geom& g, const double* lex_gauge, double m0, double csw,
                         double* A64, double* Ai64, float* A32, float* Ai32, cudaStream_t st);
// export packed blocks to [lex site][2][36] doubles
cudaError_t export_clover(const Geom& g, const double* dev, double* lex, cudaStream_t st);

// ---- fine operator ----------------------------------------------------------
enum DslashMode { DSLASH_D = 0, DSLASH_RES = 1, DSLASH_CLOVER = 2 };
// DSLASH_D: y = D x; DSLASH_RES: y = b - D x; DSLASH_CLOVER: y = A x
template <class R>
cudaError_t dslash(const Geom& g, int mode, const R* x, const R* b, R* y, const R* gauge,
                   const R* clover, int nrhs, cudaStream_t st);

// ---- half-precision storage (S = __half or __nv_bfloat16; half.cuh) ------------
// D in FP32 arithmetic with half links, clover blocks and spinors (each
// spinor field with its FP32 site norms xn / bn / yn, V per field)
template <class S>
cudaError_t dslash_h(const Geom& g, int mode, const void* x, const float* xn, const void* b, const float* bn,
                     void* y, float* yn, const void* gauge, const void* clover, int nrhs, cudaStream_t st);
// y = D x with four threads per site (one hop direction each), storage S =
// float (FP32 layout, xn / yn unused) or a half type (with site norms)
template <class S>
cudaError_t dslash4(const Geom& g, const void* x, const float* xn, void* y, float* yn, const void* gauge,
                    const void* clover, int nrhs, cudaStream_t st);
// nf FP32 spinor fields -> half fields with site norms, and back (dst = or +=)
template <class S>
cudaError_t spinor_to_half(const Geom& g, const float* src, void* dst, float* nrm, int nf, cudaStream_t st);
template <class S>
cudaError_t spinor_from_half(const Geom& g, const void* src, const float* nrm, float* dst, int nf, bool accumulate,
                             cudaStream_t st);
// an FP32 field of nr reals per site (links 48, clover 72) -> the half layout
template <class S>
cudaError_t to_half(const Geom& g, const float* src, void* dst, int nr, cudaStream_t st);

// ---- BLAS-1 on flat complex arrays (n complex numbers) -------------------------
// partial sums per CTA land in `scratch` (>= reduce_scratch_len(k) doubles)
size_t reduce_scratch_len(int k);
// out[j] = <v_j, w> for j < k (complex, FP64 accumulate); out in device memory
template <class R>
cudaError_t multi_dot(const R* const* v, int k, const R* w, size_t n, double* scratch,
                      double* out, cudaStream_t st);
// out[0] = ||w||^2
template <class R>
cudaError_t norm2(const R* w, size_t n, double* scratch, double* out, cudaStream_t st);
// w += sum_j coef[j] * v_j with coef = sign * (complex doubles in device memory)
template <class R>
cudaError_t multi_axpy(const R* const* v, int k, const double* coef, double sign, R* w,
                       size_t n, cudaStream_t st);
// multi_axpy, then out[0] = ||w||^2 of the updated w (scratch as multi_dot)
template <class R>
cudaError_t multi_axpy_norm(const R* const* v, int k, const double* coef, double sign, R* w, size_t n,
                            double* scratch, double* out, cudaStream_t st);
// nf FP64 spinor fields w_r += sum_j coef[r cstride + j] * v_j,r with FP32
// spinor fields v_j,r = v_j + r (each precision in its own device layout)
cudaError_t multi_axpy_f32_into_f64(const Geom& g, const float* const* v, int k, const double* coef, int cstride,
                                    double sign, double* w, int nf, cudaStream_t st);
// ---- batches of nb right-hand sides: vector j of right-hand side r is
// v[j] + r * rstride (complex numbers); results per r follow one another
// out[2 (r k + j)] = <v_j,r, w_r>
template <class R>
cudaError_t multi_dot_batched(const R* const* v, int k, const R* w, size_t n, int nb, size_t rstride,
                              double* scratch, double* out, cudaStream_t st);
// out[2 r] = ||w_r||^2
template <class R>
cudaError_t norm2_batched(const R* w, size_t n, int nb, size_t rstride, double* scratch, double* out,
                          cudaStream_t st);
// w_r += sign sum_j coef[r cstride + 2 j] v_j,r; with norms != nullptr also
// norms[2 r] = ||w_r||^2 after the update
template <class R>
cudaError_t multi_axpy_batched(const R* const* v, int k, const double* coef, int cstride, double sign, R* w,
                               size_t n, int nb, size_t rstride, double* scratch, double* norms, cudaStream_t st);
// y_r = x_r / sqrt(s[2 r]) for nb consecutive fields of n reals (0 if s = 0)
template <class R>
cudaError_t scale_by_inv_norm_batched(const R* x, R* y, const double* s, size_t n, int nb, cudaStream_t st);
// y = a x + b y (real scalars)
template <class R>
cudaError_t axpby(double a, const R* x, double b, R* y, size_t n, cudaStream_t st);
// y = x * (1/s[0]) with s a device scalar holding a squared norm (sqrt taken)
template <class R>
cudaError_t scale_by_inv_norm(const R* x, R* y, const double* s, size_t n, cudaStream_t st);

// ---- random initial vectors (Philox4x32-10 + Box-Muller) ----------------------
cudaError_t random_spinors(const Geom& g, uint64_t seed, int n, double* dev64, cudaStream_t st);

// ---- index maps for checking -------------------------------------------------
cudaError_t index_maps(const Geom& g, int* parity, int* block, int* colour, cudaStream_t st);

// ---- SAP smoother -------------------------------------------------------------
// one colour of a Schwarz sweep on all blocks of that colour:
//   r = b - D x (or r = b if x_is_zero), e = MR-even-odd block solve of r,
//   x += e (x is overwritten with e if x_is_zero)
// *status receives DDAMG_ETIMEOUT (6) if a bounded wait for staged data gives
// up after wait_limit polls (the CTA then leaves x untouched)
// (staged: the FP32 kernel with the block's links and clover blocks staged
// in shared memory where the block shape allows it, else the general one)
template <class R>
cudaError_t sap_sweep(const Geom& g, int colour, int mr_iters, bool x_is_zero, const R* b,
                      R* x, const R* gauge, const R* clover, const R* clover_inv, int nrhs,
                      int* status, long long wait_limit, cudaStream_t st, bool staged = true);
// the staged FP32 kernel applies to the block shape of g
bool sap_staged_ok(const Geom& g);
size_t sap_smem_bytes(const Geom& g, int real_size);
// one colour of a Schwarz sweep with half storage (FP32 arithmetic): links,
// clover blocks A and A^-1 and the spinors b, x (with their site norms) in
// the half type S; needs blocks whose half volume is a multiple of 32.
// widen: the staged block operators are widened to FP32 in shared memory
// (where the FP32 staging fits the block), else kept in the half type
template <class S>
cudaError_t sap_sweep_h(const Geom& g, int colour, int mr_iters, bool x_is_zero, const void* b, const float* bn,
                        void* x, float* xn, const void* gauge, const void* clover, const void* clover_inv, int nrhs,
                        int* status, long long wait_limit, cudaStream_t st, bool widen = true);
bool sap_half_ok(const Geom& g);

// ---- third level (kernels_level2.cu) ----------------------------------------------
// The coarse lattice of level 1 cut into blocks of coarse sites (the level-2
// Schwarz blocks and aggregates); device arrays
struct L2Geom {
  int NX;              // level-1 coarse sites
  int NXp;             // level-2 blocks (= aggregates = coarsest sites)
  int Vb;              // level-1 coarse sites per block
  const int* cnbr;     // [9][NX] neighbours of the level-1 coarse stencil
  const int* par;      // [NX] parity of the level-1 coarse sites
  const int* blk;      // [NX] block of each level-1 coarse site
  const int* loc;      // [NX] position of the site in its block's list
  const int* sites;    // [NXp][Vb] sites of each block, in increasing index
  const int* bcol;     // [2][NXp / 2] blocks of each colour
};
// one colour of the level-2 Schwarz sweep (blocks of that colour, nrhs
// coarse fields [X][2 n1]): x += the even-odd MR block solve of b - D_c x
// (x overwritten if x_is_zero); needs Vb * 2 n1 <= 1024
template <class R>
cudaError_t l2_sap_sweep(const L2Geom& d, const R* Dc, const R* Ainv, int n1, int colour, int mr_iters,
                         bool x_is_zero, const R* b, R* x, int nrhs, cudaStream_t st);
// b2 = R2 v ([r][X'][2 n2v]) and x (+)= P2 x2 with test vectors lam2 [n2v][X][2 n1]
template <class R>
cudaError_t l2_restrict(const L2Geom& d, const R* lam2, int n1, int n2v, const R* v, R* b2, int nrhs,
                        cudaStream_t st);
template <class R>
cudaError_t l2_prolong(const L2Geom& d, const R* lam2, int n1, int n2v, const R* x2, R* x, int nrhs, bool accumulate,
                       cudaStream_t st);
// classical Gram-Schmidt twice per (block, coarse chirality), FP64
cudaError_t l2_orthonormalise(const L2Geom& d, double* lam2, int n1, int n2v, cudaStream_t st);
// D_cc = P2^H D_c P2: [X'][9][2 n2v][2 n2v], column-major blocks
template <class R>
cudaError_t l2_assemble(const L2Geom& d, const R* Dc, const R* lam2, int n1, int n2v, R* Dcc, cudaStream_t st);
size_t l2_assemble_smem(int n1, int n2v, int real_size);

// ---- coarse grid ----------------------------------------------------------------
// classical Gram-Schmidt twice per (aggregate, chirality) on n FP64 or FP32
// fields
cudaError_t orthonormalise(const Geom& g, double* lam, int n, cudaStream_t st);
cudaError_t orthonormalise(const Geom& g, float* lam, int n, cudaStream_t st);
// b_c = R b  (coarse layout [rhs][X][2n] complex)
template <class R>
cudaError_t restrict_op(const Geom& g, const R* lam, int n, const R* b, R* bc, int nrhs,
                        cudaStream_t st);
// x (+)= P x_c
// the same with half test vectors (FP16, or BF16 if bf16; FP32 layout with
// 8-byte units), FP32 arithmetic
cudaError_t restrict_op_h(const Geom& g, int bf16, const void* lam16, int n, const float* b, float* bc, int nrhs,
                          cudaStream_t st);
cudaError_t prolong_op_h(const Geom& g, int bf16, const void* lam16, int n, const float* xc, float* x, int nrhs,
                         bool accumulate, cudaStream_t st);
// lam16 = half(lam32) and lam32 = FP32(lam16) (n reals, a multiple of 4)
cudaError_t round_vectors_half(int bf16, float* lam32, void* lam16, size_t n, cudaStream_t st);
template <class R>
cudaError_t prolong_op(const Geom& g, const R* lam, int n, const R* xc, R* x, int nrhs,
                       bool accumulate, cudaStream_t st);
// a batch of nrhs right-hand sides through R (Eq. 3) / P (Eq. 4) as complex
// matrix products per aggregate on the tensor cores (TF32 split into
// hi + lo parts: FP32 accuracy), each test vector read once per 16
// right-hand sides; FP32 fields and test vectors, n_v <= 32
bool mrhs_ok(const Geom& g, int n);
cudaError_t restrict_mrhs(const Geom& g, const float* lam, int n, const float* b, float* bc, int nrhs,
                          cudaStream_t st);
cudaError_t prolong_mrhs(const Geom& g, const float* lam, int n, const float* xc, float* x, int nrhs,
                         cudaStream_t st);
// D_c [X][9][2n][2n] from the test vectors; every 2n x 2n block is stored
// column-major on the device (entry (r, c) at c * 2n + r)
template <class R>
cudaError_t assemble_coarse(const Geom& g, const R* lam, int n, const R* gauge,
                            const R* clover, R* Dc, cudaStream_t st);
// inverses of the self blocks [X][2n][2n] (FP64 Gauss-Jordan, stored as R,
// column-major like D_c)
template <class R>
cudaError_t invert_self_blocks(const Geom& g, const R* Dc, int n, R* Ainv, int* singular,
                               cudaStream_t st);
// AD[ko][d - 1] = A_oo^-1(X) D_c[X][d] for the odd coarse sites X = codd[ko]
// and d = 1..8 (column-major, accumulated in R): the odd half of the
// even-odd Schur complement becomes one block product per site
template <class R>
cudaError_t premultiply_odd(const Geom& g, const R* Dc, const R* Ainv, int n, R* AD, cudaStream_t st);
// nblocks row-major complex doubles (host layout, device memory) -> column-major blocks
template <class R>
cudaError_t coarse_import(const double* src, int n, size_t nblocks, R* Dc, cudaStream_t st);
// nblocks column-major blocks -> row-major complex doubles (host layout)
template <class R>
cudaError_t coarse_export(const R* Dc, int n, size_t nblocks, double* out, cudaStream_t st);
// y = D_c x (all sites); g5: from the self and forward blocks only, the
// backward blocks taken as G5 (forward block of the neighbour)^H G5 (valid
// for a D_c assembled from a gamma5-hermitian D)
template <class R>
cudaError_t coarse_apply(const Geom& g, const R* Dc, int n, const R* x, R* y, int nrhs,
                         cudaStream_t st, bool g5 = false);
// coarse host layout <-> device coarse layout (same order, conversion only)
template <class R>
cudaError_t coarse_from_f64(const double* src, R* dst, size_t ncomplex, cudaStream_t st);
template <class R>
cudaError_t coarse_to_f64(const R* src, double* dst, size_t ncomplex, cudaStream_t st);

// even-odd preconditioned restarted GMRES on D_c: one persistent cooperative
// kernel solves all right-hand sides one after the other.  `work` must hold
// coarse_gmres_work_bytes() bytes; iters[rhs] receives the iteration counts,
// *status 0 (ok) or DDAMG_ETIMEOUT-style codes from the bounded grid barrier.
struct CoarseSolveArgs {
  const void* Dc;
  const void* Ainv;
  const void* AinvD;   // A_oo^-1 D_c[X][d], d = 1..8, per odd site (premultiply_odd)
  int n;            // test vectors (2n components per coarse site)
  double tol;
  int restart;      // <= 64
  int max_iter;
  long long wait_limit;   // polls of a grid-barrier wait before it gives up (DDAMG_ETIMEOUT)
  int tc = 0;             // eight right-hand sides through the block ring: products on the tensor cores
};
// launch configuration of the coarse GMRES for nrhs right-hand sides (all
// zero if none exists): NR right-hand sides in lockstep per launch pass, G
// CTAs owning `per` even and `per` odd coarse sites each, the Krylov slices
// in shared memory (local_in_smem) or in global scratch, the even site's D_c
// blocks resident in shared memory; dynamic shared memory per CTA and the
// bytes of `work` the launch touches
// Raise kernel fn's dynamic shared-memory limit on the current device to at
// least `bytes`.  The limit only grows (per device and kernel, under a lock):
// a launch sized by one host thread stays valid whatever a smaller launch of
// another thread sets in between.
cudaError_t raise_smem_limit(const void* fn, size_t bytes);
// launch a captured graph holding a cooperative coarse-GMRES kernel in the
// process-wide order of cooperative launches on the current device
cudaError_t launch_graph_ordered(cudaGraphExec_t g, cudaStream_t st);
struct CoarsePlan {
  int NR, G, per, local_in_smem, resident, ring;
  size_t smem_bytes, work_bytes;
};
template <class R>
CoarsePlan coarse_gmres_plan(const Geom& g, int n, int restart, int nrhs);
size_t coarse_gmres_work_bytes(const Geom& g, int n, int restart, int real_size);
// bytes of `work` that coarse_gmres() touches for nrhs right-hand sides (0 if
// no launch configuration exists)
template <class R>
size_t coarse_gmres_exact_bytes(const Geom& g, int n, int restart, int nrhs);
// (sized: the plan the caller sized `work` for; the launch refuses any other)
template <class R>
cudaError_t coarse_gmres(const Geom& g, const CoarseSolveArgs& a, const R* b, R* x, int nrhs,
                         void* work, int* iters, int* iters_acc, int* status, cudaStream_t st,
                         const CoarsePlan* sized = nullptr);

}  // namespace ddamg
