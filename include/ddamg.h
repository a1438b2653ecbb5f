/*
 * ddamg.h -- C ABI of the GB300 (sm_103a) 2-level DD-alpha-AMG solver for
 * Wilson-clover fermions (Ishikawa & Kanamori, "Porting DDalphaAMG solver to
 * K computer", arXiv 1811.00355).
 *
 * The method (paper Sec. 2): flexible GMRES preconditioned by the two-level
 * operator M = P D_c^-1 R + S (1 - D P D_c^-1 R)  (Eq. 5), with a
 * multiplicative Schwarz (SAP) smoother S whose block solver is site even-odd
 * preconditioned MR, a coarse operator D_c = <lambda_i(X,s)|D|lambda_j(Y,t)>
 * (Eq. 2) built from n test vectors projected on aggregates and chiralities
 * (Eq. 1), restriction R (Eq. 3) and prolongation P (Eq. 4), and an even-odd
 * preconditioned GMRES coarse solver stopped at a relative residual of 5e-2.
 * The test vectors come from the adaptive setup of Sec. 2.
 *
 * Conventions (the paper fixes none of them; these are the library's):
 *   D psi(x) = (4 + m0) psi(x) + C(x) psi(x)
 *              - 1/2 sum_mu [(1 - g_mu) U_mu(x) psi(x+mu)
 *                            + (1 + g_mu) U_mu(x-mu)^H psi(x-mu)],
 *   C(x) = -(csw/32) sum_{mu != nu} g_mu g_nu (x) (Q_munu(x) - Q_numu(x)),
 *   Q_munu the four-leaf clover of plaquettes at x.  Hermitian chiral gamma
 *   basis: g_k = [[0, -i sigma_k], [i sigma_k, 0]], g_t = [[0, 1], [1, 0]],
 *   g5 = diag(1, 1, -1, -1).  Periodic in x, y, z; antiperiodic in t (the
 *   library applies the sign to time hops that cross the lattice edge).
 *
 * Host exchange layouts (used by every call that takes or returns fields):
 *   site      = x + Lx*(y + Ly*(z + Lz*t))
 *   gauge     = double complex [site][mu=x,y,z,t][row 3][col 3], interleaved
 *               (re, im); U_mu(x) links x to x+mu; every link must be SU(3)
 *               (unitary, det 1): the library stores two rows and rebuilds
 *               the third, and rejects links that are off SU(3) by > 1e-9.
 *   spinor    = double complex [site][spin 4][colour 3]
 *   coarse    = double complex [X][s*n_v + i]: X the lexicographic index of
 *               the aggregate on the coarse lattice L/agg_block, s the
 *               chirality (0: spins 0,1; 1: spins 2,3), i the test vector.
 *   coarse op = double complex [X][d][2n_v][2n_v]: d = 0 self block,
 *               d = 1 + 2mu link to X+mu, d = 2 + 2mu link to X-mu.
 *   packed Hermitian 6x6 block = 36 doubles: the 6 real diagonal entries,
 *               then the 15 strictly-upper entries row-major as (re, im).
 *
 * Several right-hand sides (nrhs) are stored one after the other.
 *
 * Ownership and errors: the caller owns every buffer it passes; nothing is
 * retained after a call returns.  The handle owns all device state.  Every
 * call returns a status; no call aborts or throws.  The message of the last
 * failure is returned by ddamg_last_error().  Parameters are validated before
 * any allocation.  Calls with on_device = 1 take device pointers (same
 * layouts, FP64) and run on the handle's stream; every call synchronises that
 * stream before it returns.  A handle is not thread-safe.
 */
#ifndef DDAMG_H
#define DDAMG_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DDAMG_API __attribute__((visibility("default")))
#else
#define DDAMG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ddamg_ctx *ddamg_handle;

typedef enum {
  DDAMG_OK = 0,
  DDAMG_EINVAL = 1,   /* invalid parameter, size or layout                   */
  DDAMG_ENOMEM = 2,   /* device allocation failed or hbm_budget exceeded     */
  DDAMG_ECUDA = 3,    /* a CUDA runtime call or kernel launch failed         */
  DDAMG_ENOCONV = 4,  /* iteration cap reached; best x and residual returned */
  DDAMG_ENUMERIC = 5, /* NaN or Inf met in a norm                            */
  DDAMG_ETIMEOUT = 6, /* a bounded device-side wait gave up                  */
  DDAMG_ESTATE = 7    /* call needs state the handle does not have yet       */
} ddamg_status;

/* Arithmetic of the smoother, coarse grid and projections.  The outer
 * FGMRES, its residual r = b - D x and the test-vector orthonormalisation
 * are FP64 (the orthonormalisation FP32 on request, ortho_fp32).  DDAMG_BF16 and DDAMG_FP16 compute in FP32 like
 * DDAMG_FP32 but store in that half type: the smoother's links, clover
 * blocks (A and A^-1) and spinor fields (each spinor divided by its site
 * norm, the largest magnitude of its 24 reals, kept in FP32), and the test
 * vectors that R and P read (D_c is assembled from the same rounded
 * vectors); the coarse operator and the remaining fields stay FP32.  As a
 * step precision, BF16 / FP16 select the half-storage D (ddamg_apply_D),
 * SAP (ddamg_sap) and block solve (ddamg_block_solve). */
typedef enum { DDAMG_FP64 = 0, DDAMG_FP32 = 1, DDAMG_BF16 = 2, DDAMG_FP16 = 3 } ddamg_precision;

typedef struct {
  int L[4];            /* lattice extents x, y, z, t; each even             */
  int sap_block[4];    /* Schwarz block extents: even, divide L, and L/block
                          even in every direction (red/black block colours) */
  int agg_block[4];    /* aggregate extents; this library requires them to
                          equal sap_block (the paper's setting, Sec. 4)      */
  int n_v;             /* number of test vectors, >= 1                      */
  double m0, csw;      /* bare mass and clover coefficient                  */
  int setup_iters;     /* adaptive setup iterations (paper: 4)              */
  int n_sap;           /* SAP cycles per smoother application (paper: 4)    */
  int mr_iters;        /* MR iterations per block solve                     */
  double coarse_tol;   /* coarse GMRES relative residual (paper: 5e-2)      */
  int coarse_restart;  /* coarse GMRES restart length                       */
  int coarse_max_iter; /* coarse GMRES iteration cap                        */
  int precision;       /* ddamg_precision of the inner solver               */
  int outer_restart;   /* FGMRES restart length                             */
  int max_outer_iter;  /* FGMRES iteration cap per right-hand side          */
  uint64_t seed;       /* seed of the initial random test vectors           */
  size_t hbm_budget;   /* device-memory admission limit in bytes, 0 = none  */
  double outer_refine; /* FP32 inner precision only: if > 0, the FGMRES
                          operator products D z_k (z_k = M v_k, an FP32
                          result) are taken in FP32 and a cycle restarts from
                          the FP64 true residual r = b - D x once its
                          recurrence residual fell by this factor (iterative
                          refinement); the basis, Gram-Schmidt and r stay
                          FP64.  0 = D z_k in FP64, restart only at m.      */
  int half_vectors;    /* FP32 inner precision only: 1 = the test vectors
                          that R and P (Eq. 3, 4) read are stored in FP16
                          (FP32 arithmetic), and D_c is assembled from the
                          same rounded vectors; 0 = FP32 vectors (BF16 and
                          FP16 inner precisions always store them in half) */
  int ortho_fp32;      /* inner precision FP32, BF16 or FP16 only: 1 = the
                          test vectors are orthonormalised in FP32, the
                          precision R and P use them in (the FP64 copy takes
                          the FP32 result); 0 = in FP64 (default)            */
} ddamg_params;

typedef struct {
  int outer_iters;        /* FGMRES iterations (all restarts)                */
  int restarts;           /* FGMRES restart cycles                           */
  int coarse_iters;       /* coarse GMRES iterations summed over M calls     */
  int precond_calls;      /* applications of M                               */
  double true_residual;   /* ||b - D x|| / ||b|| in FP64                     */
  int converged;          /* 1 if true_residual <= tol                       */
  double seconds;         /* wall time of this right-hand side               */
} ddamg_solve_info;

typedef struct {
  uint64_t kernel_launches;   /* launches of the library's own kernels       */
  uint64_t dslash_launches;   /* launches of the site-parallel D kernel      */
  double dslash_ms;           /* their device time when timing is enabled    */
  uint64_t sap_launches;      /* launches of the SAP block kernel            */
  double sap_ms;
  uint64_t coarse_launches;   /* launches of the coarse GMRES kernel         */
  double coarse_ms;
  size_t device_bytes;        /* device memory held by the handle            */
  uint64_t coarse_apply_launches; /* launches of the coarse 9-point stencil  */
  double coarse_apply_ms;         /* (ddamg_apply_coarse) and their time     */
  uint64_t reorth_passes;         /* second Gram-Schmidt passes the outer
                                     FGMRES needed (refinement mode)         */
  double setup_flops;             /* theoretical flops of the adaptive setups */
  double solve_flops;             /* and of the solves (model of
                                     ddamg_get_history) since the last reset  */
  uint64_t restrict_launches;     /* launches of the restriction (Eq. 3)     */
  double restrict_ms;
  uint64_t prolong_launches;      /* launches of the prolongation (Eq. 4)    */
  double prolong_ms;
} ddamg_stats;

/* Fill *p with the library defaults (4^4 blocks, n_v 20, N_SAP 4, 4 MR,
 * coarse tol 5e-2, FP32 inner precision, restart 30, outer_refine 1e-5). */
DDAMG_API void ddamg_default_params(ddamg_params *p);

/* Name of a status code (static string). */
DDAMG_API const char *ddamg_status_string(ddamg_status s);

/* Create a handle: validate p, allocate, upload the gauge field (host or
 * device pointer, layout above), build the clover term and its inverse
 * (Sec. 3: two 6x6 Hermitian blocks per site, stored packed) in FP64 and in
 * the inner precision.  No test vectors yet.  cuda_stream is a cudaStream_t
 * (NULL = legacy default stream).  On failure *out is NULL. */
DDAMG_API ddamg_status ddamg_create(const ddamg_params *p, const double *gauge,
                          int gauge_on_device, void *cuda_stream,
                          ddamg_handle *out);

/* ddamg_create followed by the adaptive setup (Sec. 2) from random initial
 * vectors drawn on the device from p->seed (Philox4x32-10, Box-Muller). */
DDAMG_API ddamg_status ddamg_setup(const ddamg_params *p, const double *gauge,
                         int gauge_on_device, void *cuda_stream,
                         ddamg_handle *out);

/* Adaptive setup (Sec. 2) on an existing handle: the clover term and its
 * inverse are rebuilt from the resident links; initial vectors are
 * init_vectors (n_v spinor fields, host or device) or, if NULL, drawn from
 * p->seed; each is smoothed by SAP from a zero start; then setup_iters times
 * {orthonormalise per (X, s); assemble D_c; lambda_i <- M lambda_i}; finally
 * orthonormalise and assemble D_c once more. */
DDAMG_API ddamg_status ddamg_run_setup(ddamg_handle h, const double *init_vectors,
                             int on_device);

/* Replace the links of an existing handle (same lattice; host or device,
 * layout of ddamg_create; checked for SU(3) as there) and rebuild the clover
 * term.  The setup belongs to the old links: solves need ddamg_run_setup
 * first (DDAMG_ESTATE otherwise).  Reuses every device buffer, so a
 * sequence of gauge configurations costs no allocation.  After a
 * DDAMG_EINVAL (links not SU(3)) the handle holds no valid links until a
 * successful ddamg_set_gauge. */
DDAMG_API ddamg_status ddamg_set_gauge(ddamg_handle h, const double *gauge, int on_device);

/* Change m0 / csw keeping the test vectors (the paper's "new kappa", Sec. 4):
 * rebuild the clover term, its inverse and D_c. */
DDAMG_API ddamg_status ddamg_update_mass(ddamg_handle h, double m0, double csw);

/* Solve D x_k = rhs_k (k < nrhs) to ||b - D x|| <= tol ||b|| (checked on the
 * FP64 true residual) with FGMRES preconditioned by M (Sec. 2), one
 * right-hand side at a time, from a zero start.  The FGMRES basis, its
 * Gram-Schmidt and the residuals are FP64; with the FP32 inner precision and
 * outer_refine > 0 the operator products D z_k are FP32 and cycles restart
 * from the FP64 true residual (ddamg_params.outer_refine).  rhs and x are
 * nrhs spinor fields (host or device).  info (nullable) receives nrhs
 * records.  Returns DDAMG_ENOCONV if a right-hand side hit max_outer_iter
 * (its best x and residual are still written). */
DDAMG_API ddamg_status ddamg_solve(ddamg_handle h, int nrhs, const double *rhs,
                         double *x, int on_device, double tol,
                         ddamg_solve_info *info);

/* Solve the nrhs systems D x_k = rhs_k (nrhs <= 64) together.  Every right-
 * hand side has its own FGMRES -- basis, Hessenberg matrix, restarts and
 * convergence test, with the arithmetic of ddamg_solve -- but the iterations
 * of the batch advance in lockstep, so each application of M (Eq. 5), of D
 * and of the Gram-Schmidt reductions runs once for the whole batch, through
 * multi-right-hand-side kernels and the coarse GMRES with the right-hand
 * sides in lockstep.  The paper solves its 12 spin-colour sources one at a
 * time; batching them is this library's addition.  Arguments, layouts and
 * status codes as ddamg_solve; info[k].coarse_iters and precond_calls count
 * the whole batch, seconds is the batch's wall time.  Device memory grows by
 * about nrhs * (2 restart + 8) fine fields on first use. */
DDAMG_API ddamg_status ddamg_solve_batched(ddamg_handle h, int nrhs, const double *rhs,
                                 double *x, int on_device, double tol,
                                 ddamg_solve_info *info);

/* ---- the batch as a resumable run (continuous batching) ------------------
 * The lockstep batch of ddamg_solve_batched, advanced one FGMRES restart
 * cycle at a time, with right-hand sides entering and leaving between
 * cycles: a serving loop refills the slots of finished solves with waiting
 * requests instead of waiting for the whole batch.  Not in the paper.  Each
 * admitted right-hand side has its own tolerance and its own FGMRES (the
 * arithmetic of ddamg_solve_batched); a free slot holds zero fields, which
 * the batched kernels carry along.  Host or device buffers (on_device). */

/* Start a batch of `slots` free slots (1..64) on a handle with a setup;
 * replaces any batch in progress. */
DDAMG_API ddamg_status ddamg_batch_begin(ddamg_handle h, int slots);
/* Put one right-hand side (a spinor field) into a free slot, from a zero
 * start, to be solved to ||b - D x|| <= tol ||b||. */
DDAMG_API ddamg_status ddamg_batch_admit(ddamg_handle h, int slot, const double *rhs, int on_device,
                                         double tol);
/* One restart cycle of every running slot (Arnoldi steps in lockstep until
 * each slot's cycle ended, x += Z y, FP64 true residuals); *running
 * (nullable) receives the slots still running afterwards. */
DDAMG_API ddamg_status ddamg_batch_cycle(ddamg_handle h, int *running);
/* State of a slot: 0 free, 1 running, 2 finished (converged or capped). */
DDAMG_API ddamg_status ddamg_batch_slot(ddamg_handle h, int slot, int *state);
/* Copy a finished slot's solution to x (one spinor field) and its record to
 * info (nullable; coarse_iters counts the batch since ddamg_batch_begin) and
 * free the slot.  DDAMG_ENOCONV if it stopped at max_outer_iter (x holds
 * the best solution). */
DDAMG_API ddamg_status ddamg_batch_take(ddamg_handle h, int slot, double *x, int on_device,
                                        ddamg_solve_info *info);

/* ---- single steps of the method, for checking and benchmarking ---------- */

/* out = D in (Wilson-clover operator above) in the given precision. */
DDAMG_API ddamg_status ddamg_apply_D(ddamg_handle h, int precision, int nrhs,
                           const double *in, double *out, int on_device);

/* out = A in with A(x) = (4 + m0) + C(x) (inverse = 0) or A(x)^-1 in
 * (inverse = 1), site by site (Sec. 3: packed Hermitian blocks). */
DDAMG_API ddamg_status ddamg_apply_clover(ddamg_handle h, int precision, int inverse,
                                int nrhs, const double *in, double *out,
                                int on_device);

/* Export A (inverse = 0) or A^-1 (inverse = 1) as [site][chirality 2][36]
 * packed Hermitian doubles (host buffer of 72 V doubles). */
DDAMG_API ddamg_status ddamg_get_clover(ddamg_handle h, int inverse, double *out);

/* One colour of one Schwarz sweep from a zero start (Sec. 2): on every block
 * of colour `colour` (parity of the block coordinates) out = K_B in, K_B the
 * site even-odd MR block solve with mr_iters iterations; zero elsewhere. */
DDAMG_API ddamg_status ddamg_block_solve(ddamg_handle h, int precision, int colour,
                               int nrhs, const double *in, double *out,
                               int on_device);

/* The SAP smoother (Sec. 2): n_sap cycles of colour 0 then colour 1 blocks,
 * from a zero start, applied to in. */
DDAMG_API ddamg_status ddamg_sap(ddamg_handle h, int precision, int nrhs,
                       const double *in, double *out, int on_device);

/* Replace the test vectors by n_v spinor fields (as given, not
 * orthonormalised) / read the current ones (host buffer, n_v fields). */
DDAMG_API ddamg_status ddamg_set_test_vectors(ddamg_handle h, const double *vecs,
                                    int on_device);
DDAMG_API ddamg_status ddamg_get_test_vectors(ddamg_handle h, double *vecs);

/* Orthonormalise the test vectors inside every aggregate X and chirality s
 * (classical Gram-Schmidt applied twice, i = 1..n), so that the
 * projections of Eq. 1 satisfy P^H P = 1: in FP64, or in FP32 for a handle
 * created with ortho_fp32.  The setup orthonormalises the same way. */
DDAMG_API ddamg_status ddamg_orthonormalize(ddamg_handle h);

/* Assemble D_c (Eq. 2) from the current test vectors in the inner
 * precision, and invert its self blocks for the even-odd coarse solve. */
DDAMG_API ddamg_status ddamg_build_coarse(ddamg_handle h);

/* Release device memory the solves do not need once the setup is done: the
 * temporaries sized for the setup's batch of test vectors and the
 * host-exchange staging buffer (both reallocated when needed), and, for an
 * inner precision other than FP64, the FP64 copy of the test vectors (the
 * inner-precision copy that R, P and the D_c of Eq. 2 use is kept).
 * Afterwards calls that read the FP64 test vectors (ddamg_get_test_vectors,
 * ddamg_orthonormalize, FP64 R and P) return DDAMG_ESTATE; ddamg_run_setup
 * and ddamg_set_test_vectors allocate them again. */
DDAMG_API ddamg_status ddamg_trim(ddamg_handle h);

/* Outer FGMRES iterations (single and batched) through CUDA graphs captured
 * on first reuse (on: the default) or launched kernel by kernel (off).  A
 * graph capture on one host thread cannot overlap a synchronising call such
 * as cudaFree on another, so a program that drives several handles from
 * several host threads (the serving loop below does) turns graphs off. */
DDAMG_API ddamg_status ddamg_set_graphs(ddamg_handle h, int on);

/* Export D_c in the coarse-op layout (host buffer, NX*9*(2n)^2 complex). */
DDAMG_API ddamg_status ddamg_get_coarse_op(ddamg_handle h, double *out);

/* Install a coarse operator given in the coarse-op layout (host or device,
 * NX*9*(2n)^2 complex doubles), stored in the inner precision, and invert
 * its self blocks for the even-odd coarse solve (Sec. 2), as
 * ddamg_build_coarse does for the D_c of Eq. 2.  For running the coarse
 * stencil and solver on a given operator; the test vectors are left as they
 * are.  DDAMG_ENUMERIC if a self block is singular. */
DDAMG_API ddamg_status ddamg_set_coarse_op(ddamg_handle h, const double *dc, int on_device);

/* Launch configuration the coarse GMRES (Sec. 2) uses for nrhs right-hand
 * sides on this handle (chosen by the library from the coarse lattice, n_v,
 * the restart length and the device's shared memory and SM count). */
typedef struct {
  int rhs_per_pass;      /* right-hand sides solved in lockstep per pass     */
  int ctas;              /* CTAs of the cooperative launch                   */
  int sites_per_cta;     /* even (and odd) coarse sites owned by each CTA    */
  int krylov_in_shared;  /* 1: the CTA's Krylov-basis slices in shared memory,
                            0: in global scratch                             */
  int resident_blocks;   /* 1: the even site's nine D_c blocks stay in shared
                            memory for the launch                            */
  int block_ring;        /* 1: the blocks are streamed from global memory
                            through a ring of shared-memory slots filled by
                            bulk asynchronous copies ahead of their use      */
  size_t shared_bytes;   /* dynamic shared memory per CTA                    */
  size_t scratch_bytes;  /* global scratch the launch touches                */
} ddamg_coarse_plan;
DDAMG_API ddamg_status ddamg_get_coarse_plan(ddamg_handle h, int nrhs, ddamg_coarse_plan *out);

/* Measured choices of kernel variants (the library's autotuner): the first
 * time a kernel with variants runs for a problem (lattice, blocks,
 * precision, right-hand sides) outside a stream capture, each variant is
 * timed with CUDA events on the handle's stream and the fastest is used
 * from then on, process-wide.  Record i of ddamg_tuning_count(): kernel,
 * problem, the variants' mean times in microseconds and the choice.
 * Variants so far: the Wilson-clover D with one thread per site (0) or four
 * threads per site, one hop direction each (1), in FP32 and in BF16/FP16
 * storage; the coarse GMRES's block products for eight right-hand sides in
 * lockstep with the blocks streamed through shared memory, on the CUDA
 * cores (0) or the tensor cores (1, 3xTF32) ("coarse product"); the FP32
 * Schwarz sweep with the block's links and clover blocks staged in shared
 * memory (0) or read from global memory (1) ("SAP fp32"); the half-storage
 * Schwarz sweep with the staged block operators widened to FP32 in shared
 * memory (0) or kept in the half type (1) ("SAP bf16", "SAP fp16"); the
 * coarse stencil of an assembled D_c (ddamg_apply_coarse) from all nine
 * blocks (0) or from the self and forward blocks, the backward ones by
 * G5-hermiticity (1) ("coarse stencil"). */
typedef struct {
  char kernel[32];
  char problem[96];
  int variants;
  int best;
  float us[4];
} ddamg_tuning;
DDAMG_API int ddamg_tuning_count(void);
DDAMG_API ddamg_status ddamg_get_tuning(int i, ddamg_tuning *out);
/* Use `variant` of the named kernel ("D fp32", "D bf16", "D fp16", "coarse
 * product", "SAP fp32", "SAP bf16", "SAP fp16", "coarse stencil") for every
 * problem instead of the measured choice (variant < 0: measure again);
 * process-wide, for reproducible runs and for checking each variant. */
DDAMG_API ddamg_status ddamg_pin_variant(const char *kernel, int variant);

/* Polls of the device-side bounded waits before they give up and the call
 * returns DDAMG_ETIMEOUT: the SAP kernel's wait for its staged block and the
 * coarse GMRES grid barrier (default about a second each).  polls >= 0 sets
 * both (0: a wait gives up at its first unsuccessful poll, for exercising
 * the time-out path); polls < 0 restores the defaults.  A wait that gives up
 * leaves its outputs incomplete; the handle stays usable. */
DDAMG_API ddamg_status ddamg_set_wait_limit(ddamg_handle h, int64_t polls);

/* Eq. 3: out[X][s n + i] = <lambda_i(X,s)|in>; nrhs fine -> coarse. */
DDAMG_API ddamg_status ddamg_restrict(ddamg_handle h, int precision, int nrhs,
                            const double *in, double *out, int on_device);

/* Eq. 4: out = sum x_c(X,s,i) lambda_i(X,s); nrhs coarse -> fine. */
DDAMG_API ddamg_status ddamg_prolong(ddamg_handle h, int precision, int nrhs,
                           const double *in, double *out, int on_device);

/* out = D_c in (the 9-point coarse stencil); precision must be the inner
 * precision of the handle. */
DDAMG_API ddamg_status ddamg_apply_coarse(ddamg_handle h, int precision, int nrhs,
                                const double *in, double *out, int on_device);

/* Even-odd preconditioned coarse GMRES (Sec. 2) to relative residual tol of
 * the even-site Schur system, then odd-site back substitution.  iters
 * (nullable) receives nrhs iteration counts. */
DDAMG_API ddamg_status ddamg_coarse_solve(ddamg_handle h, int precision, int nrhs,
                                const double *in, double *out, int on_device,
                                double tol, int *iters);

/* The coarse solve of ddamg_coarse_solve without any device allocation, for
 * callers that cannot allocate device memory at solve time (a serving loop
 * that must avoid cudaMalloc's implicit synchronisation and allocator locks,
 * or a thread bound to a device-memory budget reserved in advance).  The
 * paper has no counterpart; it is a deployment variant of the same kernel.
 * in / out: DEVICE pointers, nrhs coarse vectors in the FP64 coarse layout;
 * tol as for ddamg_coarse_solve, in the handle's inner precision; iters
 * (nullable, host) receives nrhs iteration counts.  The kernel's scratch
 * (Krylov basis slices, vectors read by neighbouring coarse sites, partial
 * sums, the grid barrier) lives in one fixed 16 MiB array that every GPU
 * loading this library holds until the process exits; a request that needs
 * more is rejected with DDAMG_EINVAL and a message naming both sizes.  The
 * first call on a device looks up the array's device address, so make it
 * before any stream capture.  All calls share the array and leave their
 * contents in it (the barrier counters are cleared by every call): calls
 * that overlap on the GPU, on any stream or handle, race. */
DDAMG_API ddamg_status ddamg_coarse_solve_noalloc(ddamg_handle h, int nrhs,
                                                  const double *in, double *out,
                                                  double tol, int *iters);

/* out = M in (Eq. 5, post-smoothing only) in the inner precision. */
DDAMG_API ddamg_status ddamg_apply_M(ddamg_handle h, int precision, int nrhs,
                           const double *in, double *out, int on_device);

/* Index maps as the device stores them, per lexicographic fine site (host
 * int32 buffers of V entries, any may be NULL): site parity (x+y+z+t) mod 2,
 * Schwarz block index (lexicographic on the block grid), block colour,
 * aggregate index; coarse_parity has one entry per coarse site. */
DDAMG_API ddamg_status ddamg_get_index_maps(ddamg_handle h, int32_t *parity,
                                  int32_t *block, int32_t *colour,
                                  int32_t *aggregate, int32_t *coarse_parity);

/* Launch counters and (if enabled) device times of the main kernels. */
DDAMG_API ddamg_status ddamg_get_stats(ddamg_handle h, ddamg_stats *out);
DDAMG_API ddamg_status ddamg_reset_stats(ddamg_handle h);
/* Record CUDA events around the timed kernels (default off). */
DDAMG_API ddamg_status ddamg_enable_kernel_timing(ddamg_handle h, int enable);

/* Residual history of the last right-hand side of ddamg_solve (the axes of
 * the paper's Fig. 3): after every outer iteration the cumulative
 * theoretical cost in MFLOP per lattice site and the relative residual
 * (the recurrence estimate; at every restart the FP64 true residual).
 * Entry 0 is (0, 1).  *n receives the history length; at most cap entries
 * are written.  Cost model: real flops of the arithmetic (complex
 * multiply-add 8), per site 1320 for the Wilson hops, 552 for the two 6x6
 * clover blocks, 48 to combine; SAP, restriction / prolongation, coarse
 * GMRES (counted from its actual iterations) and Gram-Schmidt by their
 * operation counts. */
DDAMG_API ddamg_status ddamg_get_history(ddamg_handle h, int cap, double *mflop_per_site,
                               double *rel_residual, int *n);

/* Fill n_v * V spinor fields with the device generator's initial vectors
 * for seed (host buffer), for checking the generator. */
DDAMG_API ddamg_status ddamg_random_vectors(ddamg_handle h, uint64_t seed, int n,
                                  double *out);

DDAMG_API const char *ddamg_last_error(ddamg_handle h);
DDAMG_API void ddamg_destroy(ddamg_handle h);

/* ---- serving: continuous batching over resident gauge configurations ----
 * Not in the paper.  A server owns several gauge configurations ("configs"),
 * each with its own handle, setup and coarse operator kept resident in
 * device memory, and worker threads that run the solves.  Requests (a
 * config, nrhs right-hand sides, a tolerance) are submitted without blocking
 * and queue up.  A free worker takes the config of the oldest waiting
 * request that no other worker serves and runs that config's resumable
 * lockstep batch (ddamg_batch_*, max_batch slots): before every FGMRES
 * restart cycle it admits waiting requests of the config into free slots (in
 * arrival order, a request entering when all its right-hand sides fit),
 * and after it takes out every request whose right-hand sides have all
 * finished, each to its own tolerance.  It serves the config until no
 * request of it is running or waiting.  Workers serve different configs at
 * the same time, each config on its own CUDA stream, so their kernels
 * overlap on the device (the library orders the cooperative coarse-solver
 * launches of different streams one after the other).  A config is set up on
 * its first use; admission is by device-memory footprint: if setting up a
 * config would exceed hbm_budget, idle configs (served by no worker) are
 * released (least recently used first) and set up again on their next
 * request; a config that cannot fit fails its requests with DDAMG_ENOMEM.
 * Host buffers only; rhs and x of a request belong to the caller and must
 * stay valid until ddamg_server_wait returns for it. */
typedef struct ddamg_server *ddamg_server_handle;

typedef struct {
  ddamg_status status;    /* of this request's solves                         */
  int batch_rhs;          /* most slots in use during a cycle it took part in */
  int batch_requests;     /* most requests running together with it           */
  int setup_run;          /* 1 if the config had to be set up for it          */
  double queue_seconds;   /* submit -> admission into the batch               */
  double latency_seconds; /* submit -> results copied back                    */
} ddamg_request_info;

/* hbm_budget in bytes (0 = none), 1 <= max_batch <= 64 slots per config,
 * `workers` (1..16) configs served at the same time; cuda_stream: NULL = a
 * stream of its own for every config, else all configs on that stream
 * (then their kernels do not overlap). */
DDAMG_API ddamg_status ddamg_server_create2(size_t hbm_budget, int max_batch, int workers, void *cuda_stream,
                                            ddamg_server_handle *out);
/* ddamg_server_create2 with two workers. */
DDAMG_API ddamg_status ddamg_server_create(size_t hbm_budget, int max_batch, void *cuda_stream,
                                 ddamg_server_handle *out);
/* Register a gauge configuration (host FP64 links, layout of ddamg_create,
 * copied); its id is returned in *config_id.  No device work yet. */
DDAMG_API ddamg_status ddamg_server_add_config(ddamg_server_handle s, const ddamg_params *p,
                                     const double *gauge, int *config_id);
/* Queue a request of nrhs (1..max_batch) host right-hand sides; returns at
 * once with its id. */
DDAMG_API ddamg_status ddamg_server_submit(ddamg_server_handle s, int config_id, int nrhs,
                                 const double *rhs, double *x, double tol,
                                 ddamg_solve_info *info, uint64_t *request_id);
/* Block until the request has completed; its per-RHS records were written
 * to the info array given at submit, *rinfo (nullable) gets the request's
 * record.  Returns the request's status. */
DDAMG_API ddamg_status ddamg_server_wait(ddamg_server_handle s, uint64_t request_id,
                               ddamg_request_info *rinfo);
/* Device memory currently held by the server's resident configs. */
DDAMG_API ddamg_status ddamg_server_device_bytes(ddamg_server_handle s, size_t *bytes);
/* Message of the most recent failed library call made while serving (empty
 * when none failed).  The string belongs to the calling thread and stays
 * valid until its next call of this function. */
DDAMG_API const char *ddamg_server_last_error(ddamg_server_handle s);
/* Finish the queued requests, stop the worker, release everything. */
DDAMG_API void ddamg_server_destroy(ddamg_server_handle s);

/* ---- third level ------------------------------------------------------------
 * Paper Sec. 1 counts the recursion of the coarse-grid solve among the merits
 * of the method; Sec. 2 fixes two levels.  These calls build a third level:
 * the construction of Sec. 2 (Eq. 1-5) applied once more to D_c.  Level 2 is
 * the coarse lattice of the handle's aggregates with D_c as its 9-point
 * operator (2 n_v components per coarse site, coarse chirality G5 =
 * diag(1_n, -1_n)); its Schwarz blocks equal its aggregates, blocks of
 * coarse sites.  With three levels the coarse solve inside M (Eq. 5) is
 * flexible GMRES on D_c, right-preconditioned by M2 (Eq. 5 on level 2, with
 * the even-odd GMRES of the coarse solver on D_cc = P2^H D_c P2), stopped at
 * the handle's coarse_tol.  Arithmetic in the handle's inner precision
 * (FP32 for BF16/FP16), the level-2 test vectors kept and orthonormalised in
 * FP64.  Coarse fields are host arrays of complex doubles [nrhs][NX][2 n_v]
 * (NX = number of aggregates), level-2 test vectors [n_v2][NX][2 n_v],
 * D_cc [NX2][9][2 n_v2][2 n_v2] row-major (NX2 = number of level-2 blocks).
 * CUDA graphs are not used while three levels are on (the coarse FGMRES
 * reads its coefficients on the host). */
typedef struct {
  int block[4];          /* level-2 blocks (= aggregates) in coarse sites: each
                            even, dividing the coarse extents, with an even
                            number of blocks per direction; block volume x
                            2 n_v <= 1024                                   */
  int n_v;               /* level-2 test vectors, 1..32                      */
  int setup_iters;       /* adaptive setup iterations on D_c                 */
  int n_sap;             /* level-2 Schwarz cycles per smoother application  */
  int mr_iters;          /* MR iterations per level-2 block solve            */
  double coarsest_tol;   /* even-odd GMRES on D_cc: relative residual        */
  int coarsest_restart;  /* its restart length (<= 64)                       */
  int coarsest_max_iter; /* its iteration cap                                */
  int restart;           /* FGMRES on D_c: restart length (<= 63); its
                            iteration cap is the handle's coarse_max_iter    */
  uint64_t seed;         /* initial level-2 vectors when none are given      */
} ddamg_level2_params;
DDAMG_API ddamg_status ddamg_level2_default_params(ddamg_level2_params *p);
/* Lay out level 2 (geometry, buffers) on a handle whose D_c exists; any
 * earlier level 2 is released and the handle returns to two levels.
 * DDAMG_EINVAL for a block shape or size the kernels do not take. */
DDAMG_API ddamg_status ddamg_level2_init(ddamg_handle h, const ddamg_level2_params *p);
/* The adaptive setup on D_c from the given initial vectors (host,
 * [n_v2][NX][2 n_v], not orthonormalised) or, for NULL, Gaussian ones from
 * the seed: smoothed by the level-2 SAP, then setup_iters times
 * {orthonormalise per (block, coarse chirality); D_cc; lambda2 <- M2
 * lambda2}, then orthonormalised and D_cc once more. */
DDAMG_API ddamg_status ddamg_level2_setup(ddamg_handle h, const double *vecs);
/* Replace the level-2 test vectors (host, as above; orthonormalised here)
 * and build D_cc / read the current (orthonormal) ones. */
DDAMG_API ddamg_status ddamg_level2_set_vectors(ddamg_handle h, const double *vecs);
DDAMG_API ddamg_status ddamg_level2_get_vectors(ddamg_handle h, double *vecs);
/* D_cc as built (host, [NX2][9][2 n_v2][2 n_v2] row-major). */
DDAMG_API ddamg_status ddamg_level2_get_op(ddamg_handle h, double *out);
/* Level-2 Schwarz smoother from a zero start / M2 / the level-1 coarse
 * solve (FGMRES on D_c with M2, to tol) on nrhs host coarse fields; iters
 * (nullable, nrhs ints) receives the FGMRES iteration counts. */
DDAMG_API ddamg_status ddamg_level2_sap(ddamg_handle h, int nrhs, const double *in, double *out);
DDAMG_API ddamg_status ddamg_level2_apply_M2(ddamg_handle h, int nrhs, const double *in, double *out);
DDAMG_API ddamg_status ddamg_level2_coarse_solve(ddamg_handle h, int nrhs, const double *in, double *out,
                                                 double tol, int *iters);
/* Two levels (2) or three (3; needs ddamg_level2_setup or _set_vectors) for
 * the solves of the handle.  A new setup, mass or D_c keeps the level-2
 * test vectors and rebuilds D_cc from them. */
DDAMG_API ddamg_status ddamg_set_levels(ddamg_handle h, int levels);

#ifdef __cplusplus
}
#endif

#endif /* DDAMG_H */
