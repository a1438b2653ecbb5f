// Host driver and C ABI of the library (declared in include/ddamg.h).
//
// The handle owns every device buffer.  Fields live on the device in the
// block-major layout of common.cuh; the host exchange layout (lexicographic,
// FP64) is converted by kernels.  The outer flexible GMRES (paper Sec. 2) is
// driven from the host with one device-to-host read per iteration; the
// preconditioner M (Eq. 5), the SAP smoother and the coarse solve run as
// kernels without host synchronisation.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <complex>
#include <chrono>
#include <mutex>
#include <random>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "../../include/ddamg.h"
#include "kernels.h"

using namespace ddamg;
using cd = std::complex<double>;

namespace {

constexpr uint32_t NEG = 0x80000000u;
constexpr int NCLS = 6;               // kernel timing classes
// slot of h->dots / h->h_pinned that an outer iteration's graph copies to the
// host last: the host waits for it instead of synchronising the stream
constexpr int DONE_SLOT = 6 * 64 + 8;

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
};

// host state of a resumable lockstep batch (one entry per slot)
struct BatchRun {
  int nb = 0;
  std::vector<double> bnorm, beta, tol;
  std::vector<int> live, done, iters, restarts, calls;
  std::vector<std::chrono::steady_clock::time_point> t0;
  int cit0 = 0;
};

// polls before a device-side wait gives up (each poll about an L2 round
// trip): about a second for a staged SAP block and for a grid barrier
constexpr long long WAIT_SAP_DEFAULT = 1ll << 22;
constexpr long long WAIT_GRID_DEFAULT = 1ll << 21;

}  // namespace

struct ddamg_ctx {
  ddamg_params p{};
  cudaStream_t st = nullptr;
  std::string err;
  Geom g{};
  int n2 = 0;
  size_t V24 = 0;  // reals per spinor field

  // device memory bookkeeping
  std::vector<void*> allocs;
  size_t bytes = 0;

  // tables
  uint32_t* d_nbr = nullptr;
  int* d_lex = nullptr;
  int16_t* d_bnbr = nullptr;
  int16_t* d_face = nullptr;
  int* d_cnbr = nullptr;
  int* d_cpar = nullptr;
  int* d_ceven = nullptr;
  int* d_codd = nullptr;
  int* d_cpos = nullptr;

  // gauge and clover
  double* d_gauge_lex = nullptr;
  double* g64 = nullptr;
  float* g32 = nullptr;
  double *A64 = nullptr, *Ai64 = nullptr;
  float *A32 = nullptr, *Ai32 = nullptr;
  unsigned long long* d_dev = nullptr;

  // test vectors and coarse operator
  double* lam64 = nullptr;
  float* lam32 = nullptr;
  bool have_vectors = false;
  bool lam64_gone = false;       // FP64 test vectors released by ddamg_trim (lam32 holds them)
  bool have_coarse = false;
  bool dc_g5 = false;             // D_c assembled from D (G5-hermitian block by block), not given
  void* Dc = nullptr;
  void* Ainv = nullptr;
  void* AD = nullptr;             // A_oo^-1 D_c hop blocks of the odd coarse sites
  void* lam16 = nullptr;          // half test vectors of R and P (half_vectors, or a half inner precision)
  // half-precision copies of the FP32 links and clover blocks (index 0 FP16,
  // 1 BF16), made on first use and refreshed when the links or the clover
  // term change (op_gen counts those changes)
  void* gH[2] = {nullptr, nullptr};
  void* AH[2] = {nullptr, nullptr};
  void* AiH[2] = {nullptr, nullptr};
  uint64_t h_gen[2] = {0, 0};
  uint64_t op_gen = 1;
  // half spinor fields of the smoother (b, x) and of the half D (in, out),
  // each with its FP32 site norms
  void* hb = nullptr;
  void* hx = nullptr;
  float* hbn = nullptr;
  float* hxn = nullptr;
  size_t h_fields = 0;
  void* cwork = nullptr;
  int* d_iters = nullptr;        // per-rhs coarse iterations
  int* d_iters_acc = nullptr;    // running total
  int* d_status = nullptr;       // device status word

  // scratch
  double* red = nullptr;
  double* dots = nullptr;        // 3 x (restart + 1) complex
  double* lexbuf = nullptr;      // lexicographic staging
  size_t lexbuf_fields = 0;
  std::vector<void*> tmp;        // pool of nrhs-capable temporaries
  size_t tmp_fields = 0;
  int tmp_real = 0;

  // outer FGMRES
  double* fV = nullptr;          // (m+1) fields
  double* fZ = nullptr;          // m fields
  float* fZ32 = nullptr;         // m FP32 fields (iterative-refinement mode)
  // batched solve: blocks of bcap fields (one per right-hand side)
  int bcap = 0;
  size_t bbytes = 0;             // bytes of the one batch allocation
  unsigned char* bmem = nullptr;
  double* bV = nullptr;          // (m+1) blocks
  void* bZ = nullptr;            // m blocks (FP32 in refinement mode, else FP64)
  double *bx = nullptr, *bb = nullptr, *br = nullptr, *bw = nullptr;
  void *bin = nullptr, *bout = nullptr;   // inner-precision staging
  double* bsmall = nullptr;      // coefficients and norms of the batch
  double* h_bpinned = nullptr;
  BatchRun brun;                 // the lockstep batch in progress
  double *fx = nullptr, *fb = nullptr, *fr = nullptr, *fw = nullptr;
  void* fin = nullptr;           // inner-precision in/out for M
  void* fout = nullptr;
  double* d_coef = nullptr;

  // stats: per kernel class (0 D, 1 SAP sweep, 2 coarse solve) launch counts
  // and device time; timers recorded outside graphs wait in `pending`
  bool timing = false;
  uint64_t launches0 = 0;
  // timing classes: 0 fine D, 1 SAP sweep, 2 coarse GMRES, 3 coarse stencil,
  // 4 restriction, 5 prolongation
  uint64_t n_cls[NCLS] = {};
  double ms_cls[NCLS] = {};
  std::vector<std::pair<int, Timer>> pending;
  std::vector<Timer> pool;

  // CUDA graphs of the outer FGMRES iterations, one per Krylov index k
  struct GraphTimer {
    int cls;
    Timer t;
  };
  struct IterGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<GraphTimer> timers;
    uint64_t launches = 0;
    double flops = 0.0;                 // model flops of one replay
    uint64_t n_cls[NCLS] = {};
    int gen = -1;
    bool timing = false;
    int nb = 0;                         // batch width (batched iterations)
    int uses = 0;                       // eager runs since the last capture
  };
  std::vector<IterGraph> graphs;
  std::vector<IterGraph> bgraphs;       // batched outer iterations, per Krylov index
  bool graphs_on = true;                // outer iterations through CUDA graphs (ddamg_set_graphs)
  int gen = 0;                          // bumped whenever buffers move
  std::vector<GraphTimer>* capture_timers = nullptr;
  double* h_pinned = nullptr;           // device-to-host landing buffer
  uint64_t reorth = 0;                  // second Gram-Schmidt passes ordered by the host
  // theoretical flop counts (model below): [0] setup, [1] solves; fphase
  // selects the counter; a captured graph keeps its own share
  double flops[2] = {0.0, 0.0};
  int fphase = 1;
  int* d_cit = nullptr;                 // coarse iterations of each outer iteration
  std::vector<double> hist_flops, hist_res;   // last single-RHS solve
  cudaStream_t cap_st = nullptr;        // private stream used only to record graphs
  // polls of the device-side bounded waits before they give up
  // (ddamg_set_wait_limit): the SAP kernel's wait for its staged block and
  // the coarse GMRES grid barrier
  long long wait_sap = WAIT_SAP_DEFAULT;
  long long wait_grid = WAIT_GRID_DEFAULT;

  // third level (ddamg_level2_*): the coarse-grid solve of M as FGMRES on
  // D_c preconditioned by the two-level method built on D_c
  int levels = 2;
  struct Level2 {
    bool ready = false;                 // geometry and buffers exist
    bool have_ops = false;              // orthonormal test vectors and D_cc
    ddamg_level2_params p{};
    int NXp = 0, Vb = 0, n2v = 0;
    L2Geom d{};
    Geom g2{};                          // the coarsest lattice as the coarse kernels see it
    std::vector<std::pair<void*, size_t>> mem;
    double* lam64 = nullptr;            // [n2v][NX][2n] complex, FP64 master
    void* lam = nullptr;                // the inner-precision copy (lam64 itself in FP64)
    void* Dcc = nullptr;                // [NXp][9][2 n2v][2 n2v] column-major blocks
    void* Ainv2 = nullptr;
    void* AD2 = nullptr;
    void* work2 = nullptr;              // coarsest GMRES scratch
    void* V = nullptr;                  // level-1 FGMRES basis, restart + 1 coarse fields
    void* Z = nullptr;                  // its preconditioned directions, restart fields
    void* t[4] = {};                    // coarse temporaries
    void* c2[2] = {};                   // coarsest fields
    double* scr = nullptr;              // reduction scratch
    double* dres = nullptr;             // reduction results
    int* dit = nullptr;                 // [2] coarsest iterations of a call, and their sum
  } l2;
};

namespace {

ddamg_status fail(ddamg_ctx* h, ddamg_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  return s;
}

#define CK(...)                                                                           \
  do {                                                                                    \
    cudaError_t e_ = (__VA_ARGS__);                                                       \
    if (e_ != cudaSuccess)                                                                \
      return fail(h, DDAMG_ECUDA, "%s failed: %s (%s:%d)", #__VA_ARGS__,                  \
                  cudaGetErrorString(e_), __FILE__, __LINE__);                            \
  } while (0)

#define TRY(...)                                 \
  do {                                           \
    ddamg_status s_ = (__VA_ARGS__);             \
    if (s_ != DDAMG_OK) return s_;               \
  } while (0)

ddamg_status dalloc(ddamg_ctx* h, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (h->p.hbm_budget && h->bytes + bytes > h->p.hbm_budget)
    return fail(h, DDAMG_ENOMEM, "device memory budget exceeded: need %zu more bytes, %zu of %zu held",
                bytes, h->bytes, h->p.hbm_budget);
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, DDAMG_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
  }
  h->allocs.push_back(*p);
  h->bytes += bytes;
  return DDAMG_OK;
}
// release one allocation made by dalloc
void dfree(ddamg_ctx* h, void* p, size_t bytes) {
  if (!p) return;
  for (size_t i = 0; i < h->allocs.size(); ++i)
    if (h->allocs[i] == p) {
      h->allocs.erase(h->allocs.begin() + i);
      cudaFree(p);
      h->bytes -= bytes;
      return;
    }
}

template <class T>
ddamg_status dalloc_t(ddamg_ctx* h, T** p, size_t count) {
  void* v = nullptr;
  ddamg_status s = dalloc(h, &v, count * sizeof(T));
  *p = reinterpret_cast<T*>(v);
  return s;
}

bool is_prec(int p) { return p == DDAMG_FP64 || p == DDAMG_FP32 || p == DDAMG_BF16 || p == DDAMG_FP16; }
// half storage kind of a precision: 0 FP16, 1 BF16, -1 none
int half_kind(int p) { return p == DDAMG_FP16 ? 0 : p == DDAMG_BF16 ? 1 : -1; }
// FP32 arithmetic in the inner solver (FP32 or a half storage precision)
bool inner32(const ddamg_ctx* h) { return h->p.precision != DDAMG_FP64; }
// the test vectors of R and P are stored in half: FP16 with half_vectors, or
// the half type of a half inner precision
int lam_half_kind(const ddamg_ctx* h) {
  const int k = half_kind(h->p.precision);
  if (k >= 0) return k;
  return (inner32(h) && h->p.half_vectors) ? 0 : -1;
}

ddamg_status validate(const ddamg_params* p, std::string& why) {
  auto bad = [&](const char* m) {
    why = m;
    return DDAMG_EINVAL;
  };
  if (!p) return bad("params is NULL");
  for (int mu = 0; mu < 4; ++mu) {
    if (p->L[mu] < 2 || p->L[mu] % 2) return bad("every lattice extent must be even and >= 2");
    if (p->sap_block[mu] < 2 || p->sap_block[mu] % 2) return bad("Schwarz block extents must be even and >= 2");
    if (p->L[mu] % p->sap_block[mu]) return bad("Schwarz block extents must divide the lattice extents");
    if ((p->L[mu] / p->sap_block[mu]) % 2)
      return bad("the number of Schwarz blocks along every axis must be even (red/black colouring)");
    if (p->agg_block[mu] != p->sap_block[mu]) return bad("aggregates must equal the Schwarz blocks");
  }
  long long V = 1, Vb = 1;
  for (int mu = 0; mu < 4; ++mu) {
    V *= p->L[mu];
    Vb *= p->sap_block[mu];
  }
  if (V > (1ll << 30)) return bad("lattice too large (more than 2^30 sites)");
  if (Vb > 1024) return bad("Schwarz blocks larger than 1024 sites are not supported");
  if (p->n_v < 1 || p->n_v > 32) return bad("n_v must be in [1, 32]");
  if (p->setup_iters < 0 || p->n_sap < 1 || p->mr_iters < 0) return bad("setup_iters >= 0, n_sap >= 1, mr_iters >= 0");
  if (!(p->coarse_tol > 0.0) || p->coarse_restart < 1 || p->coarse_restart > 64 || p->coarse_max_iter < 1)
    return bad("coarse_tol > 0, coarse_restart in [1, 64], coarse_max_iter >= 1");
  if (!is_prec(p->precision)) return bad("precision must be DDAMG_FP64, DDAMG_FP32, DDAMG_BF16 or DDAMG_FP16");
  if (p->outer_restart < 1 || p->outer_restart > 62 || p->max_outer_iter < 1)
    return bad("outer_restart in [1, 62], max_outer_iter >= 1");
  if (!(p->outer_refine >= 0.0 && p->outer_refine < 1.0)) return bad("outer_refine in [0, 1)");
  if (p->half_vectors != 0 && (p->half_vectors != 1 || p->precision != DDAMG_FP32))
    return bad("half_vectors is 0, or 1 with the FP32 inner precision");
  if (p->ortho_fp32 != 0 && (p->ortho_fp32 != 1 || p->precision == DDAMG_FP64))
    return bad("ortho_fp32 is 0, or 1 with an FP32-arithmetic inner precision");
  if (!std::isfinite(p->m0) || !std::isfinite(p->csw)) return bad("m0 and csw must be finite");
  return DDAMG_OK;
}

// ---- geometry tables --------------------------------------------------------
ddamg_status build_tables(ddamg_ctx* h) {
  const ddamg_params& p = h->p;
  Geom& g = h->g;
  int V = 1, Vb = 1;
  for (int mu = 0; mu < 4; ++mu) {
    g.L[mu] = p.L[mu];
    g.b[mu] = p.sap_block[mu];
    g.grid[mu] = p.L[mu] / p.sap_block[mu];
    V *= p.L[mu];
    Vb *= p.sap_block[mu];
  }
  g.V = V;
  g.Vb = Vb;
  g.nb = V / Vb;
  const int* L = g.L;
  auto dev_of = [&](const int c[4]) {
    int bc[4], l[4];
    for (int mu = 0; mu < 4; ++mu) {
      bc[mu] = c[mu] / g.b[mu];
      l[mu] = c[mu] - bc[mu] * g.b[mu];
    }
    int B = bc[0] + g.grid[0] * (bc[1] + g.grid[1] * (bc[2] + g.grid[2] * bc[3]));
    int ll = l[0] + g.b[0] * (l[1] + g.b[1] * (l[2] + g.b[2] * l[3]));
    int par = (l[0] + l[1] + l[2] + l[3]) & 1;
    return B * Vb + par * (Vb / 2) + (ll >> 1);
  };
  std::vector<int> lex_of_dev(V), dev_of_lex(V);
  std::vector<uint32_t> nbr((size_t)8 * V);
  for (int s = 0; s < V; ++s) {
    int c[4], r = s;
    c[0] = r % L[0]; r /= L[0];
    c[1] = r % L[1]; r /= L[1];
    c[2] = r % L[2];
    c[3] = r / L[2];
    int d = dev_of(c);
    lex_of_dev[d] = s;
    dev_of_lex[s] = d;
  }
  for (int d = 0; d < V; ++d) {
    int s = lex_of_dev[d];
    int c[4], r = s;
    c[0] = r % L[0]; r /= L[0];
    c[1] = r % L[1]; r /= L[1];
    c[2] = r % L[2];
    c[3] = r / L[2];
    for (int mu = 0; mu < 4; ++mu) {
      for (int sg = 0; sg < 2; ++sg) {
        int cc[4] = {c[0], c[1], c[2], c[3]};
        bool wrap;
        if (sg == 0) { cc[mu] += 1; wrap = cc[mu] == L[mu]; if (wrap) cc[mu] = 0; }
        else { cc[mu] -= 1; wrap = cc[mu] < 0; if (wrap) cc[mu] = L[mu] - 1; }
        uint32_t e = (uint32_t)dev_of(cc);
        if (mu == 3 && wrap) e |= NEG;
        nbr[(size_t)(2 * mu + sg) * V + d] = e;
      }
    }
  }
  // block-local neighbours and faces (identical for every block)
  std::vector<int16_t> bnbr((size_t)8 * Vb, -1), face((size_t)8 * Vb, -1);
  std::vector<int> nface(8, 0);
  for (int ll = 0; ll < Vb; ++ll) {
    int l[4], r = ll;
    l[0] = r % g.b[0]; r /= g.b[0];
    l[1] = r % g.b[1]; r /= g.b[1];
    l[2] = r % g.b[2];
    l[3] = r / g.b[2];
    int par = (l[0] + l[1] + l[2] + l[3]) & 1;
    int q = par * (Vb / 2) + (ll >> 1);
    for (int mu = 0; mu < 4; ++mu)
      for (int sg = 0; sg < 2; ++sg) {
        int m[4] = {l[0], l[1], l[2], l[3]};
        m[mu] += sg == 0 ? 1 : -1;
        if (m[mu] < 0 || m[mu] >= g.b[mu]) {
          face[(size_t)(2 * mu + sg) * Vb + nface[2 * mu + sg]++] = (int16_t)q;
          continue;
        }
        int l2 = m[0] + g.b[0] * (m[1] + g.b[1] * (m[2] + g.b[2] * m[3]));
        int par2 = (m[0] + m[1] + m[2] + m[3]) & 1;
        bnbr[(size_t)(2 * mu + sg) * Vb + q] = (int16_t)(par2 * (Vb / 2) + (l2 >> 1));
      }
  }
  // coarse lattice
  const int nb = g.nb;
  std::vector<int> cnbr((size_t)9 * nb), cpar(nb), ceven, codd, cpos(nb);
  for (int X = 0; X < nb; ++X) {
    int c[4], r = X;
    c[0] = r % g.grid[0]; r /= g.grid[0];
    c[1] = r % g.grid[1]; r /= g.grid[1];
    c[2] = r % g.grid[2];
    c[3] = r / g.grid[2];
    cpar[X] = (c[0] + c[1] + c[2] + c[3]) & 1;
    cnbr[X] = X;
    for (int mu = 0; mu < 4; ++mu)
      for (int sg = 0; sg < 2; ++sg) {
        int cc[4] = {c[0], c[1], c[2], c[3]};
        cc[mu] = (cc[mu] + (sg == 0 ? 1 : -1) + g.grid[mu]) % g.grid[mu];
        cnbr[(size_t)(1 + 2 * mu + sg) * nb + X] =
            cc[0] + g.grid[0] * (cc[1] + g.grid[1] * (cc[2] + g.grid[2] * cc[3]));
      }
    if (cpar[X] == 0) { cpos[X] = (int)ceven.size(); ceven.push_back(X); }
    else { cpos[X] = (int)codd.size(); codd.push_back(X); }
  }
  TRY(dalloc_t(h, &h->d_nbr, nbr.size()));
  TRY(dalloc_t(h, &h->d_lex, (size_t)V));
  TRY(dalloc_t(h, &h->d_bnbr, bnbr.size()));
  TRY(dalloc_t(h, &h->d_face, face.size()));
  TRY(dalloc_t(h, &h->d_cnbr, cnbr.size()));
  TRY(dalloc_t(h, &h->d_cpar, (size_t)nb));
  TRY(dalloc_t(h, &h->d_ceven, ceven.size()));
  TRY(dalloc_t(h, &h->d_codd, codd.size()));
  TRY(dalloc_t(h, &h->d_cpos, (size_t)nb));
  CK(cudaMemcpy(h->d_nbr, nbr.data(), nbr.size() * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->d_lex, lex_of_dev.data(), (size_t)V * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->d_bnbr, bnbr.data(), bnbr.size() * 2, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->d_face, face.data(), face.size() * 2, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->d_cnbr, cnbr.data(), cnbr.size() * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->d_cpar, cpar.data(), (size_t)nb * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->d_ceven, ceven.data(), ceven.size() * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->d_codd, codd.data(), codd.size() * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->d_cpos, cpos.data(), (size_t)nb * 4, cudaMemcpyHostToDevice));
  g.nbr = h->d_nbr;
  g.lex_of_dev = h->d_lex;
  g.bnbr = h->d_bnbr;
  g.face = h->d_face;
  g.cnbr = h->d_cnbr;
  g.cparity = h->d_cpar;
  g.ceven = h->d_ceven;
  g.codd = h->d_codd;
  g.cpos = h->d_cpos;
  return DDAMG_OK;
}

// ---- temporaries --------------------------------------------------------------
// lexicographic FP64 staging for nf fields
ddamg_status need_lexbuf(ddamg_ctx* h, size_t nf) {
  if (h->lexbuf_fields >= nf) return DDAMG_OK;
  dfree(h, h->lexbuf, h->lexbuf_fields * h->V24 * sizeof(double));   // (cudaFree waits for its users)
  h->lexbuf = nullptr;
  h->lexbuf_fields = 0;
  void* p;
  TRY(dalloc(h, &p, nf * h->V24 * sizeof(double)));
  h->lexbuf = (double*)p;
  h->lexbuf_fields = nf;
  return DDAMG_OK;
}
// k temporaries of nf fields each, in doubles (big enough for either precision)
ddamg_status need_tmp(ddamg_ctx* h, size_t nf, int k) {
  if (h->tmp_fields >= nf && (int)h->tmp.size() >= k) return DDAMG_OK;
  size_t want = nf > h->tmp_fields ? nf : h->tmp_fields;
  for (void* p : h->tmp) dfree(h, p, h->tmp_fields * h->V24 * sizeof(double));
  h->tmp.clear();
  h->tmp_fields = 0;
  ++h->gen;   // captured graphs refer to the old temporaries
  for (int i = 0; i < (k > 6 ? k : 6); ++i) {
    void* p;
    TRY(dalloc(h, &p, want * h->V24 * sizeof(double)));
    h->tmp.push_back(p);
  }
  h->tmp_fields = want;
  return DDAMG_OK;
}

Timer next_timer(ddamg_ctx* h) {
  if (h->pool.empty()) {
    Timer t;
    cudaEventCreate(&t.a);
    cudaEventCreate(&t.b);
    return t;
  }
  Timer t = h->pool.back();
  h->pool.pop_back();
  return t;
}

template <class F>
cudaError_t timed(ddamg_ctx* h, int cls, F&& f) {
  ++h->n_cls[cls];
  if (!h->timing) return f();
  Timer t;
  if (h->capture_timers) {           // events owned by the graph being captured
    cudaEventCreate(&t.a);
    cudaEventCreate(&t.b);
  } else {
    t = next_timer(h);
  }
  // inside a capture the records must become event nodes of the graph
  const unsigned flags = h->capture_timers ? cudaEventRecordExternal : cudaEventRecordDefault;
  cudaEventRecordWithFlags(t.a, h->st, flags);
  cudaError_t e = f();
  cudaEventRecordWithFlags(t.b, h->st, flags);
  if (h->capture_timers) h->capture_timers->push_back({cls, t});
  else h->pending.push_back({cls, t});
  return e;
}

void collect_pending(ddamg_ctx* h) {
  for (auto& pt : h->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pt.second.a, pt.second.b) == cudaSuccess) h->ms_cls[pt.first] += ms;
    else cudaGetLastError();
    h->pool.push_back(pt.second);
  }
  h->pending.clear();
}

// ---- theoretical flop model -------------------------------------------------------
// Real flops of the method's arithmetic, counted per unit of work (complex
// multiply-add 8, complex add 2, real multiply-add 2), independent of how a
// kernel schedules it.  Per site: the Wilson hopping term 1320 (spin-projected
// form), the two 6x6 Hermitian clover blocks 552, combining 48 (24 more for a
// residual b - D x).
constexpr double F_HOP = 1320.0, F_CLOV = 552.0, F_D = F_HOP + F_CLOV + 48.0, F_RES = F_D + 24.0;

void addf(ddamg_ctx* h, double f) { h->flops[h->fphase] += f; }
// one SAP colour sweep of one right-hand side (sites of the colour: V/2)
double flops_sap_sweep(const ddamg_ctx* h, bool x_is_zero) {
  const double V = (double)h->g.V, q = V / 4.0;          // even (odd) sites of the colour
  double f = q * (F_CLOV + F_HOP + 24.0);               // u_o = A^-1 r_o, rhs_e
  f += h->p.mr_iters * q * ((F_HOP + 24.0 + F_CLOV) + (F_CLOV + F_HOP + 24.0 + 336.0));
  f += q * (F_HOP + 24.0 + F_CLOV);                     // e_o
  if (!x_is_zero) f += V / 2.0 * (F_RES + 24.0);        // residual, x += e
  return f;
}
// restriction or prolongation of one right-hand side
double flops_rp(const ddamg_ctx* h) { return (double)h->g.V * 12.0 * h->p.n_v * 8.0; }
// coarse GMRES: fixed part of one solve (odd elimination, right-hand side,
// back-substitution) and one iteration (Schur product, Gram-Schmidt with
// about 10 basis vectors, update), per right-hand side
double flops_coarse_fixed(const ddamg_ctx* h) {
  const double ne = h->g.nb / 2.0, n2 = 2.0 * h->p.n_v;
  return ne * (1.0 + 8.0 + 9.0) * n2 * n2 * 8.0;
}
double flops_coarse_iter(const ddamg_ctx* h) {
  const double ne = h->g.nb / 2.0, n2 = 2.0 * h->p.n_v;
  return ne * ((8.0 + 9.0) * n2 * n2 + 26.0 * n2) * 8.0;
}
// FP64 Gram-Schmidt pass over kv basis vectors (dots and update), one field
double flops_gs_pass(const ddamg_ctx* h, int kv) { return (double)h->g.V * 12.0 * kv * 16.0; }
// per-aggregate orthonormalisation (classical Gram-Schmidt twice, norms)
double flops_ortho(const ddamg_ctx* h) {
  const double n = h->p.n_v, V = h->g.V;
  return V * 6.0 * 2.0 * (n * (n - 1.0) * 16.0 + n * 8.0);
}
// D_c assembly (D applied to the 2 n chirality-projected test vectors and
// contracted with them), self-block inverses, premultiplied odd blocks
double flops_build(const ddamg_ctx* h) {
  const double n2 = 2.0 * h->p.n_v, V = h->g.V, nb = h->g.nb;
  return n2 * V * F_D + V * 12.0 * n2 * n2 * 8.0 + nb * n2 * n2 * n2 * 8.0 + nb / 2.0 * 8.0 * n2 * n2 * n2 * 8.0;
}

// ---- in/out of fields -----------------------------------------------------------
// host/device FP64 lexicographic -> device field of precision R (nf fields)
template <class R>
ddamg_status import_fields(ddamg_ctx* h, const double* src, int on_device, int nf, R* dst) {
  const double* lex = src;
  if (!on_device) {
    TRY(need_lexbuf(h, nf));
    CK(cudaMemcpyAsync(h->lexbuf, src, nf * h->V24 * sizeof(double), cudaMemcpyHostToDevice, h->st));
    lex = h->lexbuf;
  }
  CK(pack_spinor<R>(h->g, lex, dst, nf, h->st));
  return DDAMG_OK;
}
template <class R>
ddamg_status export_fields(ddamg_ctx* h, const R* src, int nf, double* dst, int on_device) {
  double* lex = dst;
  if (!on_device) {
    TRY(need_lexbuf(h, nf));
    lex = h->lexbuf;
  }
  CK(unpack_spinor<R>(h->g, src, lex, nf, h->st));
  if (!on_device)
    CK(cudaMemcpyAsync(dst, lex, nf * h->V24 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return DDAMG_OK;
}

template <class R> const R* gauge_of(ddamg_ctx* h);
template <> const float* gauge_of<float>(ddamg_ctx* h) { return h->g32; }
template <> const double* gauge_of<double>(ddamg_ctx* h) { return h->g64; }
template <class R> const R* clov_of(ddamg_ctx* h, bool inv);
template <> const float* clov_of<float>(ddamg_ctx* h, bool inv) { return inv ? h->Ai32 : h->A32; }
template <> const double* clov_of<double>(ddamg_ctx* h, bool inv) { return inv ? h->Ai64 : h->A64; }
template <class R> const R* lam_of(ddamg_ctx* h);
template <> const float* lam_of<float>(ddamg_ctx* h) { return h->lam32; }
template <> const double* lam_of<double>(ddamg_ctx* h) { return h->lam64; }

// batches of at least this many right-hand sides go through R and P as
// tensor-core matrix products (one read of the test vectors per 16)
constexpr int MRHS_MIN = 2;

// R and P of the inner solver (FP16 test vectors when half_vectors is set)
template <class R>
cudaError_t restrict_inner(ddamg_ctx* h, const R* in, R* bc, int nf) {
  return timed(h, 4, [&] {
    if constexpr (sizeof(R) == 4) {
      const int k = lam_half_kind(h);
      if (k >= 0) return restrict_op_h(h->g, k, h->lam16, h->p.n_v, in, bc, nf, h->st);
      // a batch: complex products over the right-hand sides on the tensor cores
      if (nf >= MRHS_MIN && mrhs_ok(h->g, h->p.n_v))
        return restrict_mrhs(h->g, h->lam32, h->p.n_v, in, bc, nf, h->st);
    }
    return restrict_op<R>(h->g, lam_of<R>(h), h->p.n_v, in, bc, nf, h->st);
  });
}
template <class R>
cudaError_t prolong_inner(ddamg_ctx* h, const R* xc, R* out, int nf) {
  return timed(h, 5, [&] {
    if constexpr (sizeof(R) == 4) {
      const int k = lam_half_kind(h);
      if (k >= 0) return prolong_op_h(h->g, k, h->lam16, h->p.n_v, xc, out, nf, false, h->st);
      if (nf >= MRHS_MIN && mrhs_ok(h->g, h->p.n_v))
        return prolong_mrhs(h->g, h->lam32, h->p.n_v, xc, out, nf, h->st);
    }
    return prolong_op<R>(h->g, lam_of<R>(h), h->p.n_v, xc, out, nf, false, h->st);
  });
}

// half storage: copies of the operators and the smoother's spinor buffers
ddamg_status half_operators(ddamg_ctx* h, int k);
ddamg_status need_half_fields(ddamg_ctx* h, size_t nf);
// f(S*) with S the half type of kind k (0 FP16, 1 BF16)
template <class F>
cudaError_t by_half(int k, F&& f) {
  if (k == 0) return f((__half*)nullptr);
  return f((__nv_bfloat16*)nullptr);
}

// ---- measured choice among kernel variants (autotuner) ----------------------------
// For a kernel and a problem (lattice, precision, right-hand sides) every
// variant runs once to warm up and then three times between CUDA events on
// the handle's stream; the fastest is kept for the process and used from
// then on, also inside captured graphs.  Inside a stream capture nothing can
// be timed: an undecided choice takes variant 0 there.  The variants compute
// the same result, so running them on the caller's data is harmless.
struct TuneEntry {
  std::string kernel, key;
  int best = 0;
  std::vector<float> us;
};
std::mutex g_tune_mu;
std::vector<TuneEntry> g_tune;
std::vector<std::pair<std::string, int>> g_pins;   // kernels whose variant the caller fixed

template <class F>
ddamg_status tuned(ddamg_ctx* h, const std::string& kernel, const std::string& key, int nvar, F&& run,
                   int* choice) {
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto& p : g_pins)
      if (p.first == kernel) {
        *choice = p.second < nvar ? p.second : 0;
        return DDAMG_OK;
      }
    for (const auto& e : g_tune)
      if (e.kernel == kernel && e.key == key) {
        *choice = e.best;
        return DDAMG_OK;
      }
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(h->st, &cap));
  if (cap != cudaStreamCaptureStatusNone) {
    *choice = 0;
    return DDAMG_OK;
  }
  TuneEntry e;
  e.kernel = kernel;
  e.key = key;
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  float best = 0.f;
  for (int v = 0; v < nvar; ++v) {
    CK(run(v));
    CK(cudaEventRecord(a, h->st));
    for (int k = 0; k < 3; ++k) CK(run(v));
    CK(cudaEventRecord(b, h->st));
    CK(cudaEventSynchronize(b));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, a, b));
    e.us.push_back(1e3f * ms / 3.f);
    if (v == 0 || e.us.back() < best) {
      best = e.us.back();
      e.best = v;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *choice = e.best;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.push_back(e);
  return DDAMG_OK;
}

std::string lattice_key(const ddamg_ctx* h, const char* prec, int nf) {
  char buf[96];
  snprintf(buf, sizeof buf, "%dx%dx%dx%d/%dx%dx%dx%d %s nrhs %d", h->g.L[0], h->g.L[1], h->g.L[2], h->g.L[3],
           h->g.b[0], h->g.b[1], h->g.b[2], h->g.b[3], prec, nf);
  return buf;
}

// ---- operators on device fields ---------------------------------------------------
// variant of the FP32 y = D x for nf fields: one thread per site (0) or
// four (1), measured on x and y the first time
ddamg_status dslash32_variant(ddamg_ctx* h, const float* x, float* y, int nf, int* v) {
  *v = 0;
  if (h->g.V % 8) return DDAMG_OK;
  auto run = [&](int var) -> cudaError_t {
    if (var == 1) return dslash4<float>(h->g, x, nullptr, y, nullptr, h->g32, h->A32, nf, h->st);
    return dslash<float>(h->g, DSLASH_D, x, nullptr, y, h->g32, h->A32, nf, h->st);
  };
  return tuned(h, "D fp32", lattice_key(h, "fp32", nf), 2, run, v);
}

template <class R>
ddamg_status op_dslash(ddamg_ctx* h, int mode, const R* x, const R* b, R* y, int nf) {
  addf(h, (double)nf * h->g.V * (mode == DSLASH_RES ? F_RES : mode == DSLASH_CLOVER ? F_CLOV : F_D));
  int v = 0;
  if constexpr (sizeof(R) == 4)
    if (mode == DSLASH_D) TRY(dslash32_variant(h, x, y, nf, &v));
  CK(timed(h, 0, [&] {
    if constexpr (sizeof(R) == 4)
      if (v == 1) return dslash4<float>(h->g, x, nullptr, y, nullptr, h->g32, h->A32, nf, h->st);
    return dslash<R>(h->g, mode, x, b, y, gauge_of<R>(h), clov_of<R>(h, false), nf, h->st);
  }));
  return DDAMG_OK;
}

// SAP from zero: x = S b
// FP32 Schwarz sweeps with blocks the staged kernel takes: staged (0) or
// general kernel (1), measured on the caller's fields the first time for a
// problem (the smoother starts from x = 0, so a trial run leaves nothing
// behind in x that the real run keeps)
ddamg_status sap32_staged(ddamg_ctx* h, const float* b, float* x, int nf, bool* staged) {
  *staged = true;
  if (!sap_staged_ok(h->g)) return DDAMG_OK;
  auto trial = [&](int var) -> cudaError_t {
    cudaError_t e = cudaMemsetAsync(x, 0, nf * h->V24 * sizeof(float), h->st);
    for (int cyc = 0; cyc < h->p.n_sap && e == cudaSuccess; ++cyc)
      for (int c = 0; c < 2 && e == cudaSuccess; ++c)
        e = sap_sweep<float>(h->g, c, h->p.mr_iters, cyc == 0 && c == 0, b, x, h->g32, h->A32, h->Ai32, nf,
                             h->d_status, h->wait_sap, h->st, var == 0);
    return e;
  };
  int v = 0;
  TRY(tuned(h, "SAP fp32", lattice_key(h, "fp32", nf), 2, trial, &v));
  *staged = v == 0;
  return DDAMG_OK;
}

// half-storage Schwarz sweeps: the staged block operators widened to FP32
// in shared memory (0) or kept in the half type (1), measured the first time
// for a problem on the half right-hand sides already in hb (the smoother
// starts from x = 0; the caller clears x afterwards)
ddamg_status sap_half_widen(ddamg_ctx* h, int kind, int nf, bool* widen) {
  *widen = true;
  if (!sap_staged_ok(h->g)) return DDAMG_OK;
  auto trial = [&](int var) -> cudaError_t {
    cudaError_t e = cudaMemsetAsync(h->hx, 0, nf * h->V24 * 2, h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->hxn, 0, nf * h->g.V * sizeof(float), h->st);
    for (int cyc = 0; cyc < h->p.n_sap && e == cudaSuccess; ++cyc)
      for (int c = 0; c < 2 && e == cudaSuccess; ++c)
        e = by_half(kind, [&](auto* tag) {
          using S = std::remove_pointer_t<decltype(tag)>;
          return sap_sweep_h<S>(h->g, c, h->p.mr_iters, cyc == 0 && c == 0, h->hb, h->hbn, h->hx, h->hxn,
                                h->gH[kind], h->AH[kind], h->AiH[kind], nf, h->d_status, h->wait_sap, h->st,
                                var == 0);
        });
    return e;
  };
  int v = 0;
  TRY(tuned(h, kind ? "SAP bf16" : "SAP fp16", lattice_key(h, kind ? "bf16" : "fp16", nf), 2, trial, &v));
  *widen = v == 0;
  return DDAMG_OK;
}

template <class R>
ddamg_status op_sap(ddamg_ctx* h, const R* b, R* x, int nf, int kind = -2) {
  if (kind == -2) kind = half_kind(h->p.precision);
  if constexpr (sizeof(R) == 4) {
    // half storage: links, clover blocks and the smoother's b and x in the
    // half type (FP32 arithmetic); b in and x out in FP32
    if (kind >= 0 && sap_half_ok(h->g)) {
      TRY(half_operators(h, kind));
      TRY(need_half_fields(h, nf));
      CK(by_half(kind, [&](auto* tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        return spinor_to_half<S>(h->g, b, h->hb, h->hbn, nf, h->st);
      }));
      bool widen = true;
      TRY(sap_half_widen(h, kind, nf, &widen));
      CK(cudaMemsetAsync(h->hx, 0, nf * h->V24 * 2, h->st));
      CK(cudaMemsetAsync(h->hxn, 0, nf * h->g.V * sizeof(float), h->st));
      for (int cyc = 0; cyc < h->p.n_sap; ++cyc)
        for (int c = 0; c < 2; ++c) {
          const bool zero = cyc == 0 && c == 0;
          addf(h, nf * flops_sap_sweep(h, zero));
          CK(timed(h, 1, [&] {
            return by_half(kind, [&](auto* tag) {
              using S = std::remove_pointer_t<decltype(tag)>;
              return sap_sweep_h<S>(h->g, c, h->p.mr_iters, zero, h->hb, h->hbn, h->hx, h->hxn, h->gH[kind],
                                    h->AH[kind], h->AiH[kind], nf, h->d_status, h->wait_sap, h->st, widen);
            });
          }));
        }
      CK(by_half(kind, [&](auto* tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        return spinor_from_half<S>(h->g, h->hx, h->hxn, x, nf, false, h->st);
      }));
      return DDAMG_OK;
    }
  }
  bool staged = true;
  if constexpr (sizeof(R) == 4) TRY(sap32_staged(h, b, x, nf, &staged));
  CK(cudaMemsetAsync(x, 0, nf * h->V24 * sizeof(R), h->st));
  for (int cyc = 0; cyc < h->p.n_sap; ++cyc)
    for (int c = 0; c < 2; ++c) {
      bool zero = cyc == 0 && c == 0;
      addf(h, nf * flops_sap_sweep(h, zero));
      CK(timed(h, 1, [&] {
        return sap_sweep<R>(h->g, c, h->p.mr_iters, zero, b, x, gauge_of<R>(h), clov_of<R>(h, false),
                            clov_of<R>(h, true), nf, h->d_status, h->wait_sap, h->st, staged);
      }));
    }
  return DDAMG_OK;
}

template <class R>
ddamg_status op_coarse_solve(ddamg_ctx* h, const R* bc, R* xc, int nf, double tol, int* iters_dev) {
  CoarseSolveArgs a;
  a.Dc = h->Dc;
  a.Ainv = h->Ainv;
  a.AinvD = h->AD;
  a.n = h->p.n_v;
  a.tol = tol;
  a.restart = h->p.coarse_restart;
  a.max_iter = h->p.coarse_max_iter;
  a.wait_limit = h->wait_grid;
  if (sizeof(R) == 4) {
    // eight right-hand sides through the block ring: the block products on
    // the CUDA cores (0) or the tensor cores (1), the faster one measured on
    // this call's data the first time (iteration counters left alone)
    const CoarsePlan pl = coarse_gmres_plan<R>(h->g, h->p.n_v, h->p.coarse_restart, nf);
    if (pl.ring && pl.NR == 8) {
      auto run = [&](int var) -> cudaError_t {
        CoarseSolveArgs t = a;
        t.tc = var;
        return coarse_gmres<R>(h->g, t, bc, xc, nf, h->cwork, nullptr, nullptr, h->d_status, h->st);
      };
      char key[96];
      snprintf(key, sizeof key, "coarse %d sites n_v %d fp32 nrhs %d", h->g.nb, h->p.n_v, nf);
      TRY(tuned(h, "coarse product", key, 2, run, &a.tc));
    }
  }
  addf(h, nf * flops_coarse_fixed(h));   // iterations are added when their counts are read
  CK(timed(h, 2, [&] {
    return coarse_gmres<R>(h->g, a, bc, xc, nf, h->cwork, iters_dev, h->d_iters_acc, h->d_status, h->st);
  }));
  return DDAMG_OK;
}

ddamg_status check_status(ddamg_ctx* h);

// ---- third level ----------------------------------------------------------------
// Paper Sec. 1 names the recursion of the coarse-grid solve as a merit of the
// method; Sec. 2 then fixes two levels.  The third level applies the
// construction of Sec. 2 (Eq. 1-5) once more, to D_c: a Schwarz smoother on
// blocks of coarse sites, aggregates of coarse sites with their own test
// vectors from the same adaptive setup run on D_c, D_cc = P2^H D_c P2, and
// M2 (Eq. 5 on level 2) with the even-odd GMRES of the coarse solver on D_cc.
// The level-1 coarse solve inside M becomes FGMRES on D_c right-preconditioned
// by M2, stopped at the same relative residual.

ddamg_status l2_alloc(ddamg_ctx* h, void** p, size_t bytes) {
  TRY(dalloc(h, p, bytes));
  h->l2.mem.emplace_back(*p, bytes);
  return DDAMG_OK;
}

void l2_release(ddamg_ctx* h) {
  for (auto& m : h->l2.mem) dfree(h, m.first, m.second);
  h->l2 = ddamg_ctx::Level2{};
  h->levels = 2;
}

// a coarse field of the inner precision: NX sites of 2n complex numbers
size_t l2_field_reals(const ddamg_ctx* h) { return (size_t)h->g.nb * h->n2 * 2; }

template <class R>
ddamg_status l2_init(ddamg_ctx* h, const ddamg_level2_params& p) {
  const int n1 = h->p.n_v, n2v = p.n_v, m2 = 2 * n2v;
  int Lc[4], Lcc[4], Vb = 1, NXp = 1;
  for (int mu = 0; mu < 4; ++mu) {
    Lc[mu] = h->g.grid[mu];
    if (p.block[mu] < 2 || p.block[mu] % 2 || Lc[mu] % p.block[mu] || (Lc[mu] / p.block[mu]) % 2)
      return fail(h, DDAMG_EINVAL,
                  "level-2 block extents must be even, divide the coarse lattice %dx%dx%dx%d and leave an even "
                  "number of blocks in every direction", Lc[0], Lc[1], Lc[2], Lc[3]);
    Lcc[mu] = Lc[mu] / p.block[mu];
    Vb *= p.block[mu];
    NXp *= Lcc[mu];
  }
  if (n2v < 1 || n2v > 32) return fail(h, DDAMG_EINVAL, "level-2 n_v must be in [1, 32]");
  if (Vb * 2 * n1 > 1024) return fail(h, DDAMG_EINVAL, "a level-2 block holds at most 1024 / (2 n_v) coarse sites");
  if (p.n_sap < 1 || p.mr_iters < 0 || p.setup_iters < 0)
    return fail(h, DDAMG_EINVAL, "level-2 n_sap >= 1, mr_iters >= 0, setup_iters >= 0");
  if (p.restart < 1 || p.restart > 63 || p.coarsest_restart < 1 || p.coarsest_restart > 64)
    return fail(h, DDAMG_EINVAL, "level-2 restart in [1, 63], coarsest_restart in [1, 64]");
  if (!(p.coarsest_tol > 0.0) || p.coarsest_max_iter < 1)
    return fail(h, DDAMG_EINVAL, "level-2 coarsest_tol > 0 and coarsest_max_iter >= 1");
  if (l2_assemble_smem(n1, n2v, sizeof(R)) > 200 * 1024)
    return fail(h, DDAMG_EINVAL, "the level-2 assembly needs more shared memory than a CTA has (lower n_v)");
  l2_release(h);
  auto& L = h->l2;
  const int NX = h->g.nb;
  // level-1 coarse sites in blocks of coarse sites (lexicographic block index,
  // colour = parity of the block coordinates, sites in increasing index)
  std::vector<int> blk(NX), loc(NX), sites((size_t)NXp * Vb), cnt(NXp, 0), bcol, bodd;
  for (int X = 0; X < NX; ++X) {
    int c[4], r = X;
    c[0] = r % Lc[0]; r /= Lc[0];
    c[1] = r % Lc[1]; r /= Lc[1];
    c[2] = r % Lc[2];
    c[3] = r / Lc[2];
    const int Xp = c[0] / p.block[0] + Lcc[0] * (c[1] / p.block[1] + Lcc[1] * (c[2] / p.block[2] + Lcc[2] * (c[3] / p.block[3])));
    blk[X] = Xp;
    loc[X] = cnt[Xp];
    sites[(size_t)Xp * Vb + cnt[Xp]++] = X;
  }
  // the coarsest lattice (the coarse kernels' tables, as for level 1)
  std::vector<int> cnbr((size_t)9 * NXp), cpar(NXp), ceven, codd, cpos(NXp);
  for (int X = 0; X < NXp; ++X) {
    int c[4], r = X;
    c[0] = r % Lcc[0]; r /= Lcc[0];
    c[1] = r % Lcc[1]; r /= Lcc[1];
    c[2] = r % Lcc[2];
    c[3] = r / Lcc[2];
    cpar[X] = (c[0] + c[1] + c[2] + c[3]) & 1;
    (cpar[X] ? bodd : bcol).push_back(X);
    cnbr[X] = X;
    for (int mu = 0; mu < 4; ++mu)
      for (int sg = 0; sg < 2; ++sg) {
        int cc[4] = {c[0], c[1], c[2], c[3]};
        cc[mu] = (cc[mu] + (sg == 0 ? 1 : -1) + Lcc[mu]) % Lcc[mu];
        cnbr[(size_t)(1 + 2 * mu + sg) * NXp + X] = cc[0] + Lcc[0] * (cc[1] + Lcc[1] * (cc[2] + Lcc[2] * cc[3]));
      }
    if (cpar[X] == 0) { cpos[X] = (int)ceven.size(); ceven.push_back(X); }
    else { cpos[X] = (int)codd.size(); codd.push_back(X); }
  }
  bcol.insert(bcol.end(), bodd.begin(), bodd.end());     // [colour 0 blocks][colour 1 blocks]
  std::vector<int> tab;
  auto put = [&](const std::vector<int>& v) { size_t o = tab.size(); tab.insert(tab.end(), v.begin(), v.end()); return o; };
  const size_t o_blk = put(blk), o_loc = put(loc), o_sites = put(sites), o_bcol = put(bcol), o_cnbr = put(cnbr),
               o_cpar = put(cpar), o_ceven = put(ceven), o_codd = put(codd), o_cpos = put(cpos);
  void* dt = nullptr;
  TRY(l2_alloc(h, &dt, tab.size() * sizeof(int)));
  CK(cudaMemcpy(dt, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice));
  const int* T = static_cast<const int*>(dt);
  L.d.NX = NX;
  L.d.NXp = NXp;
  L.d.Vb = Vb;
  L.d.cnbr = h->g.cnbr;
  L.d.par = h->g.cparity;
  L.d.blk = T + o_blk;
  L.d.loc = T + o_loc;
  L.d.sites = T + o_sites;
  L.d.bcol = T + o_bcol;
  L.g2 = h->g;
  for (int mu = 0; mu < 4; ++mu) L.g2.grid[mu] = Lcc[mu];
  L.g2.nb = NXp;
  L.g2.cnbr = T + o_cnbr;
  L.g2.cparity = T + o_cpar;
  L.g2.ceven = T + o_ceven;
  L.g2.codd = T + o_codd;
  L.g2.cpos = T + o_cpos;
  if (coarse_gmres_plan<R>(L.g2, n2v, p.coarsest_restart, 1).NR == 0) {
    l2_release(h);
    return fail(h, DDAMG_EINVAL, "no launch configuration of the coarsest GMRES for this level-2 lattice");
  }
  const size_t rs = sizeof(R), fr = l2_field_reals(h), NN2 = (size_t)m2 * m2;
  void* q = nullptr;
  TRY(l2_alloc(h, &q, (size_t)n2v * fr * sizeof(double)));
  L.lam64 = static_cast<double*>(q);
  TRY(l2_alloc(h, &L.lam, (size_t)n2v * fr * rs));
  TRY(l2_alloc(h, &L.t[3], (size_t)n2v * fr * rs));       // n2v fields: the setup's new vectors
  TRY(l2_alloc(h, &L.Dcc, (size_t)NXp * 9 * NN2 * 2 * rs));
  TRY(l2_alloc(h, &L.Ainv2, (size_t)NXp * NN2 * 2 * rs));
  TRY(l2_alloc(h, &L.AD2, (size_t)(NXp / 2) * 8 * NN2 * 2 * rs));
  TRY(l2_alloc(h, &L.work2, coarse_gmres_work_bytes(L.g2, n2v, p.coarsest_restart, (int)rs)));
  TRY(l2_alloc(h, &L.V, (size_t)(p.restart + 1) * fr * rs));
  TRY(l2_alloc(h, &L.Z, (size_t)p.restart * fr * rs));
  for (int k = 0; k < 3; ++k) TRY(l2_alloc(h, &L.t[k], fr * rs));
  for (int k = 0; k < 2; ++k) TRY(l2_alloc(h, &L.c2[k], (size_t)NXp * m2 * 2 * rs));
  TRY(l2_alloc(h, &q, (reduce_scratch_len(p.restart + 1) + 4 * (p.restart + 2) + 2) * sizeof(double)));
  L.scr = static_cast<double*>(q);
  L.dres = L.scr + reduce_scratch_len(p.restart + 1);
  TRY(l2_alloc(h, &q, 2 * sizeof(int)));
  L.dit = static_cast<int*>(q);
  CK(cudaMemsetAsync(L.dit, 0, 2 * sizeof(int), h->st));
  L.p = p;
  L.NXp = NXp;
  L.Vb = Vb;
  L.n2v = n2v;
  L.ready = true;
  return DDAMG_OK;
}

// orthonormalise the FP64 level-2 vectors (if ortho), copy them to the inner
// precision, assemble D_cc and invert its self blocks
template <class R>
ddamg_status l2_build(ddamg_ctx* h, bool ortho) {
  auto& L = h->l2;
  const int n1 = h->p.n_v;
  const size_t fr = l2_field_reals(h);
  if (ortho) CK(l2_orthonormalise(L.d, L.lam64, n1, L.n2v, h->st));
  if constexpr (sizeof(R) == 8)
    CK(cudaMemcpyAsync(L.lam, L.lam64, (size_t)L.n2v * fr * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  else
    CK(convert_field<float, double>(L.lam64, (float*)L.lam, (size_t)L.n2v * fr, h->st));
  CK(cudaMemsetAsync(h->d_status, 0, sizeof(int), h->st));
  CK(l2_assemble<R>(L.d, (const R*)h->Dc, (const R*)L.lam, n1, L.n2v, (R*)L.Dcc, h->st));
  CK(invert_self_blocks<R>(L.g2, (const R*)L.Dcc, L.n2v, (R*)L.Ainv2, h->d_status, h->st));
  CK(premultiply_odd<R>(L.g2, (const R*)L.Dcc, (const R*)L.Ainv2, L.n2v, (R*)L.AD2, h->st));
  int sing = 0;
  CK(cudaMemcpyAsync(&sing, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (sing) {
    cudaMemsetAsync(h->d_status, 0, sizeof(int), h->st);
    L.have_ops = false;
    return fail(h, DDAMG_ENUMERIC, "a self block of D_cc is singular");
  }
  L.have_ops = true;
  return DDAMG_OK;
}

// x = S2 b: n_sap level-2 Schwarz cycles from x = 0 on nf coarse fields
// (the first colour-0 sweep writes x on its blocks only: the other sites
// start from the zeros set here)
template <class R>
ddamg_status l2_smooth(ddamg_ctx* h, const R* b, R* x, int nf) {
  auto& L = h->l2;
  CK(cudaMemsetAsync(x, 0, (size_t)nf * l2_field_reals(h) * sizeof(R), h->st));
  for (int cyc = 0; cyc < L.p.n_sap; ++cyc)
    for (int c = 0; c < 2; ++c)
      CK(l2_sap_sweep<R>(L.d, (const R*)h->Dc, (const R*)h->Ainv, h->p.n_v, c, L.p.mr_iters, cyc == 0 && c == 0, b, x,
                         nf, h->st));
  return DDAMG_OK;
}

// out = M2 in (Eq. 5 on level 2), one coarse field:
// x1 = P2 D_cc^-1 R2 in; out = x1 + S2 (in - D_c x1); uses t[0], t[1], c2
template <class R>
ddamg_status l2_M2(ddamg_ctx* h, const R* in, R* out) {
  auto& L = h->l2;
  const int n1 = h->p.n_v;
  const size_t fr = l2_field_reals(h);
  R* t0 = (R*)L.t[0];
  R* t1 = (R*)L.t[1];
  CK(l2_restrict<R>(L.d, (const R*)L.lam, n1, L.n2v, in, (R*)L.c2[0], 1, h->st));
  CoarseSolveArgs a;
  a.Dc = L.Dcc;
  a.Ainv = L.Ainv2;
  a.AinvD = L.AD2;
  a.n = L.n2v;
  a.tol = L.p.coarsest_tol;
  a.restart = L.p.coarsest_restart;
  a.max_iter = L.p.coarsest_max_iter;
  a.wait_limit = h->wait_grid;
  CK(coarse_gmres<R>(L.g2, a, (const R*)L.c2[0], (R*)L.c2[1], 1, L.work2, L.dit, L.dit + 1, h->d_status, h->st));
  CK(l2_prolong<R>(L.d, (const R*)L.lam, n1, L.n2v, (const R*)L.c2[1], out, 1, false, h->st));
  CK(coarse_apply<R>(h->g, (const R*)h->Dc, n1, out, t0, 1, h->st));
  CK(axpby<R>(1.0, in, -1.0, t0, fr, h->st));
  TRY(l2_smooth<R>(h, t0, t1, 1));
  CK(axpby<R>(1.0, t1, 1.0, out, fr, h->st));
  return DDAMG_OK;
}

// the adaptive setup on D_c (level by level, after level 1's): the initial
// vectors (in lam64) through S2, then setup_iters times {orthonormalise,
// D_cc, lambda2 <- M2 lambda2}, then a last orthonormalisation and D_cc
template <class R>
ddamg_status l2_setup(ddamg_ctx* h) {
  auto& L = h->l2;
  const size_t fr = l2_field_reals(h), all = (size_t)L.n2v * fr;
  R* lam = (R*)L.lam;
  R* nw = (R*)L.t[3];
  auto to_master = [&]() -> cudaError_t {
    if constexpr (sizeof(R) == 8)
      return cudaMemcpyAsync(L.lam64, nw, all * sizeof(double), cudaMemcpyDeviceToDevice, h->st);
    else
      return convert_field<double, float>((const float*)nw, L.lam64, all, h->st);
  };
  if constexpr (sizeof(R) == 8)
    CK(cudaMemcpyAsync(lam, L.lam64, all * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  else
    CK(convert_field<float, double>(L.lam64, (float*)lam, all, h->st));
  TRY(l2_smooth<R>(h, lam, nw, L.n2v));
  CK(to_master());
  for (int it = 0; it < L.p.setup_iters; ++it) {
    TRY(l2_build<R>(h, true));
    for (int k = 0; k < L.n2v; ++k) TRY(l2_M2<R>(h, lam + (size_t)k * fr, nw + (size_t)k * fr));
    CK(to_master());
  }
  TRY(l2_build<R>(h, true));
  return check_status(h);
}

// FGMRES on D_c right-preconditioned by M2 (the level-1 coarse solve of the
// three-level method) for one coarse field, from x = 0, to ||b - D_c x|| <=
// tol ||b||: classical Gram-Schmidt twice, complex Givens rotations, the
// recurrence residual tested after every step and the true residual at
// every restart
template <class R>
ddamg_status l2_fgmres(ddamg_ctx* h, const R* b, R* x, double tol, int max_iter, int* iters) {
  using cd = std::complex<double>;
  auto& L = h->l2;
  const int m = L.p.restart;
  const size_t fr = l2_field_reals(h), nc = fr / 2;
  R* V = (R*)L.V;
  R* Z = (R*)L.Z;
  R* w = (R*)L.t[2];
  R* r = (R*)L.t[3];      // (the setup's vectors live there only between M2 calls of the setup)
  double* dres = L.dres;
  // the two Gram-Schmidt passes' coefficients and ||w||^2 land side by side
  // and come to the host in one copy per iteration
  double* d1 = dres;
  double* d2 = d1 + 2 * (m + 1);
  double* dn = d2 + 2 * (m + 1);
  std::vector<double> hh(4 * (m + 1) + 2);
  auto norm_host = [&](const R* v, double* out) -> ddamg_status {
    CK(norm2<R>(v, nc, L.scr, dres, h->st));
    CK(cudaMemcpyAsync(out, dres, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    return DDAMG_OK;
  };
  CK(cudaMemsetAsync(x, 0, fr * sizeof(R), h->st));
  double bn2 = 0.0;
  TRY(norm_host(b, &bn2));
  const double bnorm = std::sqrt(bn2);
  *iters = 0;
  if (bnorm == 0.0) return DDAMG_OK;
  CK(cudaMemcpyAsync(r, b, fr * sizeof(R), cudaMemcpyDeviceToDevice, h->st));
  int total = 0;
  for (;;) {
    double beta2 = 0.0;
    TRY(norm_host(r, &beta2));
    const double beta = std::sqrt(beta2);
    if (beta <= tol * bnorm || total >= max_iter) break;
    CK(scale_by_inv_norm<R>(r, V, dres, fr, h->st));      // dres[0] holds ||r||^2
    std::vector<std::vector<cd>> H(m + 1, std::vector<cd>(m, cd(0.0)));
    std::vector<double> cs(m, 0.0);
    std::vector<cd> sn(m, cd(0.0)), g(m + 1, cd(0.0));
    g[0] = cd(beta);
    int kd = 0;
    for (int k = 0; k < m; ++k) {
      TRY(l2_M2<R>(h, V + (size_t)k * fr, Z + (size_t)k * fr));
      CK(coarse_apply<R>(h->g, (const R*)h->Dc, h->p.n_v, Z + (size_t)k * fr, w, 1, h->st));
      std::vector<const R*> vl(k + 1);
      for (int j = 0; j <= k; ++j) vl[j] = V + (size_t)j * fr;
      for (double* dp : {d1, d2}) {
        CK(multi_dot<R>(vl.data(), k + 1, w, nc, L.scr, dp, h->st));
        CK(multi_axpy<R>(vl.data(), k + 1, dp, -1.0, w, nc, h->st));
      }
      CK(norm2<R>(w, nc, L.scr, dn, h->st));
      CK(cudaMemcpyAsync(hh.data(), dres, (4 * (m + 1) + 2) * sizeof(double), cudaMemcpyDeviceToHost, h->st));
      CK(cudaStreamSynchronize(h->st));
      std::vector<cd> hk(k + 1, cd(0.0));
      for (int j = 0; j <= k; ++j)
        hk[j] = cd(hh[2 * j], hh[2 * j + 1]) + cd(hh[2 * (m + 1) + 2 * j], hh[2 * (m + 1) + 2 * j + 1]);
      const double hn = std::sqrt(hh[4 * (m + 1)]);
      if (hn > 0.0) CK(scale_by_inv_norm<R>(w, V + (size_t)(k + 1) * fr, dn, fr, h->st));
      for (int j = 0; j <= k; ++j) H[j][k] = hk[j];
      H[k + 1][k] = cd(hn);
      for (int j = 0; j < k; ++j) {
        const cd t = cs[j] * H[j][k] + sn[j] * H[j + 1][k];
        H[j + 1][k] = -std::conj(sn[j]) * H[j][k] + cs[j] * H[j + 1][k];
        H[j][k] = t;
      }
      {  // rotation with [c, s; -conj(s), c] [h1; h2] = [rho; 0], c real
        const cd h1 = H[k][k], h2 = H[k + 1][k];
        const double a1 = std::abs(h1), a2 = std::abs(h2);
        if (a2 == 0.0) { cs[k] = 1.0; sn[k] = 0.0; }
        else if (a1 == 0.0) { cs[k] = 0.0; sn[k] = std::conj(h2) / a2; H[k][k] = cd(a2); }
        else {
          const double rho = std::hypot(a1, a2);
          const cd ph = h1 / a1;
          cs[k] = a1 / rho;
          sn[k] = ph * std::conj(h2) / rho;
          H[k][k] = ph * rho;
        }
      }
      H[k + 1][k] = cd(0.0);
      g[k + 1] = -std::conj(sn[k]) * g[k];
      g[k] = cs[k] * g[k];
      ++total;
      kd = k + 1;
      if (std::abs(g[k + 1]) <= tol * bnorm || total >= max_iter || hn == 0.0) break;
    }
    std::vector<cd> y(kd);
    for (int i = kd - 1; i >= 0; --i) {
      cd acc = g[i];
      for (int j = i + 1; j < kd; ++j) acc -= H[i][j] * y[j];
      y[i] = acc / H[i][i];
    }
    for (int i = 0; i < kd; ++i) { hh[2 * i] = y[i].real(); hh[2 * i + 1] = y[i].imag(); }
    CK(cudaMemcpyAsync(dres, hh.data(), 2 * kd * sizeof(double), cudaMemcpyHostToDevice, h->st));
    std::vector<const R*> zl(kd);
    for (int i = 0; i < kd; ++i) zl[i] = Z + (size_t)i * fr;
    CK(multi_axpy<R>(zl.data(), kd, dres, 1.0, x, nc, h->st));
    CK(coarse_apply<R>(h->g, (const R*)h->Dc, h->p.n_v, x, r, 1, h->st));
    CK(axpby<R>(1.0, b, -1.0, r, fr, h->st));
  }
  *iters = total;
  return check_status(h);
}

// the level-1 coarse solve of M with three levels: nf coarse fields one after
// the other; the total FGMRES iteration count goes to *cit_dev (if given)
// and joins the coarse-iteration total of the solve (d_iters_acc)
template <class R>
ddamg_status l2_coarse_solve(ddamg_ctx* h, const R* bc, R* xc, int nf, double tol, int* cit_dev) {
  const size_t fr = l2_field_reals(h);
  int total = 0;
  for (int k = 0; k < nf; ++k) {
    int it = 0;
    TRY(l2_fgmres<R>(h, bc + (size_t)k * fr, xc + (size_t)k * fr, tol, h->p.coarse_max_iter, &it));
    total += it;
  }
  int acc = 0;
  CK(cudaMemcpyAsync(&acc, h->d_iters_acc, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  acc += total;
  CK(cudaMemcpyAsync(h->d_iters_acc, &acc, sizeof(int), cudaMemcpyHostToDevice, h->st));
  if (cit_dev) CK(cudaMemcpyAsync(cit_dev, &total, sizeof(int), cudaMemcpyHostToDevice, h->st));
  CK(cudaStreamSynchronize(h->st));
  return DDAMG_OK;
}

// D_cc again after D_c changed (new setup, new mass, a given D_c)
ddamg_status l2_refresh(ddamg_ctx* h) {
  if (!h->l2.have_ops) return DDAMG_OK;
  if (inner32(h)) return l2_build<float>(h, false);
  return l2_build<double>(h, false);
}

// out = M in  (Eq. 5): x1 = P D_c^-1 R in; out = x1 + SAP(in - D x1)
// uses tmp[0..3]
template <class R>
ddamg_status op_M(ddamg_ctx* h, const R* in, R* out, int nf, int* cit_dev = nullptr) {
  TRY(need_tmp(h, nf, 6));
  R* r1 = (R*)h->tmp[0];
  R* e = (R*)h->tmp[1];
  R* bc = (R*)h->tmp[2];
  R* xc = (R*)h->tmp[3];
  addf(h, 2.0 * nf * flops_rp(h) + nf * 2.0 * h->V24);
  CK(restrict_inner<R>(h, in, bc, nf));
  if (h->levels == 3) TRY(l2_coarse_solve<R>(h, bc, xc, nf, h->p.coarse_tol, cit_dev));
  else TRY(op_coarse_solve<R>(h, bc, xc, nf, h->p.coarse_tol, cit_dev));
  CK(prolong_inner<R>(h, xc, out, nf));
  TRY(op_dslash<R>(h, DSLASH_RES, out, in, r1, nf));
  TRY(op_sap<R>(h, r1, e, nf));
  CK(axpby<R>(1.0, e, 1.0, out, nf * h->V24, h->st));
  return DDAMG_OK;
}

ddamg_status check_status(ddamg_ctx* h) {
  int st = 0;
  CK(cudaMemcpyAsync(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (st != 0) {
    cudaMemsetAsync(h->d_status, 0, sizeof(int), h->st);
    return fail(h, DDAMG_ETIMEOUT, "a bounded device-side wait (SAP staging or coarse grid barrier) gave up (status %d)",
                st);
  }
  return DDAMG_OK;
}

// ---- coarse operator ----------------------------------------------------------------
ddamg_status alloc_coarse(ddamg_ctx* h) {
  if (h->Dc) return DDAMG_OK;
  const int rs = inner32(h) ? 4 : 8;
  const size_t n2 = h->n2;
  TRY(dalloc(h, &h->Dc, (size_t)h->g.nb * 9 * n2 * n2 * 2 * rs));
  TRY(dalloc(h, &h->Ainv, (size_t)h->g.nb * n2 * n2 * 2 * rs));
  TRY(dalloc(h, &h->AD, (size_t)(h->g.nb / 2) * 8 * n2 * n2 * 2 * rs));
  TRY(dalloc(h, &h->cwork, coarse_gmres_work_bytes(h->g, h->p.n_v, h->p.coarse_restart, rs)));
  return DDAMG_OK;
}

// FP64 test vectors for a call that reads them (released by ddamg_trim)
ddamg_status need_lam64(ddamg_ctx* h) {
  if (!h->lam64_gone) return DDAMG_OK;
  return fail(h, DDAMG_ESTATE, "the FP64 test vectors were released by ddamg_trim");
}
// FP64 test vectors for a call that writes all of them
ddamg_status revive_lam64(ddamg_ctx* h) {
  if (!h->lam64_gone) return DDAMG_OK;
  TRY(dalloc_t(h, &h->lam64, (size_t)h->p.n_v * h->V24));
  h->lam64_gone = false;
  return DDAMG_OK;
}

ddamg_status sync_lam32(ddamg_ctx* h) {
  if (inner32(h)) {
    if (!h->lam32) TRY(dalloc_t(h, &h->lam32, (size_t)h->p.n_v * h->V24));
    // after ddamg_trim the FP32 copy is the only one (and current)
    if (!h->lam64_gone) CK(convert_spinor<float, double>(h->g, h->lam64, h->lam32, h->p.n_v, h->st));
    const int k = lam_half_kind(h);
    if (k >= 0) {
      if (!h->lam16) TRY(dalloc(h, &h->lam16, (size_t)h->p.n_v * h->V24 * 2));
      CK(round_vectors_half(k, h->lam32, h->lam16, (size_t)h->p.n_v * h->V24, h->st));
    }
  }
  return DDAMG_OK;
}

// half copies of the FP32 links and clover blocks for storage kind k
ddamg_status half_operators(ddamg_ctx* h, int k) {
  if (h->gH[k] && h->h_gen[k] == h->op_gen) return DDAMG_OK;
  const size_t V = h->g.V;
  if (!h->gH[k]) {
    TRY(dalloc(h, &h->gH[k], V * 48 * 2));
    TRY(dalloc(h, &h->AH[k], V * 72 * 2));
    TRY(dalloc(h, &h->AiH[k], V * 72 * 2));
  }
  if (k == 0) {
    CK(to_half<__half>(h->g, h->g32, h->gH[k], 48, h->st));
    CK(to_half<__half>(h->g, h->A32, h->AH[k], 72, h->st));
    CK(to_half<__half>(h->g, h->Ai32, h->AiH[k], 72, h->st));
  } else {
    CK(to_half<__nv_bfloat16>(h->g, h->g32, h->gH[k], 48, h->st));
    CK(to_half<__nv_bfloat16>(h->g, h->A32, h->AH[k], 72, h->st));
    CK(to_half<__nv_bfloat16>(h->g, h->Ai32, h->AiH[k], 72, h->st));
  }
  h->h_gen[k] = h->op_gen;
  return DDAMG_OK;
}

// the clover term A = (4 + m0) + C and its inverse from the resident links;
// half copies already in use are refreshed at once (captured graphs read
// them in place)
ddamg_status rebuild_clover(ddamg_ctx* h, double m0, double csw) {
  CK(build_clover(h->g, h->d_gauge_lex, m0, csw, h->A64, h->Ai64, h->A32, h->Ai32, h->st));
  ++h->op_gen;
  for (int k = 0; k < 2; ++k)
    if (h->gH[k]) TRY(half_operators(h, k));
  return DDAMG_OK;
}

// half spinor buffers b, x (with site norms) for nf fields
ddamg_status need_half_fields(ddamg_ctx* h, size_t nf) {
  if (h->h_fields >= nf) return DDAMG_OK;
  dfree(h, h->hb, h->h_fields * h->V24 * 2);
  dfree(h, h->hx, h->h_fields * h->V24 * 2);
  dfree(h, h->hbn, h->h_fields * h->g.V * sizeof(float));
  dfree(h, h->hxn, h->h_fields * h->g.V * sizeof(float));
  h->hb = h->hx = nullptr;
  h->hbn = h->hxn = nullptr;
  h->h_fields = 0;
  TRY(dalloc(h, &h->hb, nf * h->V24 * 2));
  TRY(dalloc(h, &h->hx, nf * h->V24 * 2));
  TRY(dalloc_t(h, &h->hbn, nf * h->g.V));
  TRY(dalloc_t(h, &h->hxn, nf * h->g.V));
  h->h_fields = nf;
  ++h->gen;                        // captured graphs refer to the old buffers
  return DDAMG_OK;
}





ddamg_status build_coarse_op(ddamg_ctx* h) {
  if (!h->have_vectors) return fail(h, DDAMG_ESTATE, "no test vectors");
  TRY(alloc_coarse(h));
  TRY(sync_lam32(h));
  CK(cudaMemsetAsync(h->d_status, 0, sizeof(int), h->st));
  addf(h, flops_build(h));
  if (inner32(h)) {
    CK(assemble_coarse<float>(h->g, h->lam32, h->p.n_v, h->g32, h->A32, (float*)h->Dc, h->st));
    CK(invert_self_blocks<float>(h->g, (float*)h->Dc, h->p.n_v, (float*)h->Ainv, h->d_status, h->st));
    CK(premultiply_odd<float>(h->g, (float*)h->Dc, (float*)h->Ainv, h->p.n_v, (float*)h->AD, h->st));
  } else {
    CK(assemble_coarse<double>(h->g, h->lam64, h->p.n_v, h->g64, h->A64, (double*)h->Dc, h->st));
    CK(invert_self_blocks<double>(h->g, (double*)h->Dc, h->p.n_v, (double*)h->Ainv, h->d_status, h->st));
    CK(premultiply_odd<double>(h->g, (double*)h->Dc, (double*)h->Ainv, h->p.n_v, (double*)h->AD, h->st));
  }
  int sing = 0;
  CK(cudaMemcpyAsync(&sing, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (sing) {
    cudaMemsetAsync(h->d_status, 0, sizeof(int), h->st);
    return fail(h, DDAMG_ENUMERIC, "a coarse self block is singular");
  }
  h->have_coarse = true;
  h->dc_g5 = true;
  return l2_refresh(h);
}

// ---- precision changes of spinor fields -----------------------------------------------
template <class R>
ddamg_status to_inner(ddamg_ctx* h, const double* src, R* dst, int nf) {
  if constexpr (sizeof(R) == 8)
    CK(cudaMemcpyAsync(dst, src, nf * h->V24 * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  else
    CK(convert_spinor<R, double>(h->g, src, dst, nf, h->st));
  return DDAMG_OK;
}
template <class R>
ddamg_status from_inner(ddamg_ctx* h, const R* src, double* dst, int nf) {
  if constexpr (sizeof(R) == 8)
    CK(cudaMemcpyAsync(dst, src, nf * h->V24 * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  else
    CK(convert_spinor<double, R>(h->g, src, dst, nf, h->st));
  return DDAMG_OK;
}

// ---- adaptive setup -----------------------------------------------------------------
// coarse GMRES iterations accumulated on the device since the last call
ddamg_status coarse_iters_since(ddamg_ctx* h, int* its) {
  int acc = 0;
  CK(cudaMemcpyAsync(&acc, h->d_iters_acc, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  CK(cudaMemsetAsync(h->d_iters_acc, 0, sizeof(int), h->st));
  *its = acc;
  return DDAMG_OK;
}

// the test vectors orthonormalised per (aggregate, chirality): FP64 in
// place, or (ortho_fp32, an FP32-arithmetic inner solver whose R and P use
// them in FP32) on the FP32 copy, which the FP64 copy then takes
ddamg_status ortho_inner(ddamg_ctx* h) {
  if (!inner32(h) || !h->p.ortho_fp32) {
    CK(orthonormalise(h->g, h->lam64, h->p.n_v, h->st));
    return DDAMG_OK;
  }
  if (!h->lam32) TRY(dalloc_t(h, &h->lam32, (size_t)h->p.n_v * h->V24));
  CK(convert_spinor<float, double>(h->g, h->lam64, h->lam32, h->p.n_v, h->st));
  CK(orthonormalise(h->g, h->lam32, h->p.n_v, h->st));
  CK(convert_spinor<double, float>(h->g, h->lam32, h->lam64, h->p.n_v, h->st));
  return DDAMG_OK;
}

template <class R>
ddamg_status setup_impl(ddamg_ctx* h) {
  const int n = h->p.n_v;
  // the vectors go through the smoother and M in chunks whose temporaries
  // (six FP64-sized fields each) fit in the device memory left once the
  // setup's other arrays (inner-precision test vectors, the coarse operator,
  // half-storage operators) are in place
  if (inner32(h) && !h->lam32) TRY(dalloc_t(h, &h->lam32, (size_t)n * h->V24));
  if (lam_half_kind(h) >= 0 && !h->lam16) TRY(dalloc(h, &h->lam16, (size_t)n * h->V24 * 2));
  TRY(alloc_coarse(h));
  if (half_kind(h->p.precision) >= 0 && sap_half_ok(h->g)) TRY(half_operators(h, half_kind(h->p.precision)));
  int ch = n;
  {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) {
      cudaGetLastError();
      const size_t per = 6 * h->V24 * sizeof(double) + 2 * h->V24 * 2 + 2 * h->g.V * sizeof(float);
      size_t avail = fr + h->tmp_fields * 6 * h->V24 * sizeof(double);
      if (h->p.hbm_budget) {
        const size_t left = h->p.hbm_budget > h->bytes ? h->p.hbm_budget - h->bytes : 0;
        avail = std::min(avail, left + h->tmp_fields * 6 * h->V24 * sizeof(double));
      }
      avail = avail / 10 * 8;            // headroom for the coarse scratch and the library's own
      const size_t fit = avail / per;
      ch = (int)std::max<size_t>(1, std::min<size_t>((size_t)n, fit));
    }
  }
  TRY(need_tmp(h, ch, 6));
  int its = 0;
  TRY(coarse_iters_since(h, &its));
  h->fphase = 0;
  struct Back { ddamg_ctx* h; ~Back() { h->fphase = 1; } } back{h};
  R* a = (R*)h->tmp[4];
  R* b = (R*)h->tmp[5];
  // lambda_i <- SAP(lambda_i)
  for (int c0 = 0; c0 < n; c0 += ch) {
    const int cn = std::min(ch, n - c0);
    double* lv = h->lam64 + (size_t)c0 * h->V24;
    TRY(to_inner<R>(h, lv, a, cn));
    TRY(op_sap<R>(h, a, b, cn));
    TRY(from_inner<R>(h, b, lv, cn));
  }
  for (int it = 0; it < h->p.setup_iters; ++it) {
    addf(h, flops_ortho(h));
    TRY(ortho_inner(h));
    TRY(build_coarse_op(h));
    // lambda_i <- M lambda_i
    for (int c0 = 0; c0 < n; c0 += ch) {
      const int cn = std::min(ch, n - c0);
      double* lv = h->lam64 + (size_t)c0 * h->V24;
      TRY(to_inner<R>(h, lv, a, cn));
      TRY(op_M<R>(h, a, b, cn));
      TRY(from_inner<R>(h, b, lv, cn));
    }
    TRY(check_status(h));
  }
  addf(h, flops_ortho(h));
  TRY(ortho_inner(h));
  TRY(build_coarse_op(h));
  TRY(coarse_iters_since(h, &its));
  addf(h, its * flops_coarse_iter(h));
  return check_status(h);
}

// ---- outer FGMRES (FP64) -----------------------------------------------------------
template <class R>
ddamg_status precond_to_f64(ddamg_ctx* h, const double* v, double* z, int* cit_dev) {
  if (sizeof(R) == 8) return op_M<double>(h, v, z, 1, cit_dev);
  float* fin = (float*)h->fin;
  float* fout = (float*)h->fout;
  TRY(to_inner<float>(h, v, fin, 1));
  TRY(op_M<float>(h, fin, fout, 1, cit_dev));
  return from_inner<float>(h, fout, z, 1);
}

// FGMRES as iterative refinement: FP32 operator products in the Arnoldi
// process, FP64 basis, Gram-Schmidt and true residuals
bool refine_mode(const ddamg_ctx* h) { return inner32(h) && h->p.outer_refine > 0.0; }

ddamg_status alloc_outer(ddamg_ctx* h) {
  if (h->fV) return DDAMG_OK;
  const int m = h->p.outer_restart;
  TRY(dalloc_t(h, &h->fV, (size_t)(m + 1) * h->V24));
  if (refine_mode(h)) TRY(dalloc_t(h, &h->fZ32, (size_t)m * h->V24));
  else TRY(dalloc_t(h, &h->fZ, (size_t)m * h->V24));
  TRY(dalloc_t(h, &h->fx, h->V24));
  TRY(dalloc_t(h, &h->fb, h->V24));
  TRY(dalloc_t(h, &h->fr, h->V24));
  TRY(dalloc_t(h, &h->fw, h->V24));
  TRY(dalloc(h, &h->fin, h->V24 * sizeof(double)));
  TRY(dalloc(h, &h->fout, h->V24 * sizeof(double)));
  TRY(dalloc_t(h, &h->d_coef, (size_t)2 * (m + 1)));
  TRY(dalloc_t(h, &h->d_cit, (size_t)m));
  if (!h->h_pinned) CK(cudaHostAlloc(&h->h_pinned, (6 * 64 + 16) * sizeof(double), cudaHostAllocDefault));
  h->graphs.resize(m);
  return DDAMG_OK;
}

// everything an outer iteration's graph touches must exist before capture
ddamg_status prepare_capture(ddamg_ctx* h) {
  TRY(alloc_outer(h));
  if (!h->cap_st) CK(cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking));
  TRY(need_tmp(h, 1, 6));
  const int k = half_kind(h->p.precision);
  if (k >= 0) {
    TRY(half_operators(h, k));
    TRY(need_half_fields(h, 1));
  }
  if (inner32(h)) coarse_gmres_exact_bytes<float>(h->g, h->p.n_v, h->p.coarse_restart, 1);
  else coarse_gmres_exact_bytes<double>(h->g, h->p.n_v, h->p.coarse_restart, 1);
  // the D of the captured iterations (FP32 inner precision) is chosen now:
  // nothing can be timed inside a capture
  if (refine_mode(h)) {
    int v = 0;
    TRY(dslash32_variant(h, (const float*)h->fin, (float*)h->fout, 1, &v));
  }
  // and the smoother's kernel (the FP32 fields as scratch)
  if (inner32(h) && k < 0) {
    bool staged = true;
    TRY(sap32_staged(h, (const float*)h->fin, (float*)h->fout, 1, &staged));
  }
  if (k >= 0 && sap_half_ok(h->g)) {
    CK(cudaMemsetAsync(h->fin, 0, h->V24 * sizeof(float), h->st));
    CK(by_half(k, [&](auto* tag) {
      using S = std::remove_pointer_t<decltype(tag)>;
      return spinor_to_half<S>(h->g, (const float*)h->fin, h->hb, h->hbn, 1, h->st);
    }));
    bool widen = true;
    TRY(sap_half_widen(h, k, 1, &widen));
  }
  return DDAMG_OK;
}

// The device work of one outer iteration k: z_k = M v_k, w = D z_k, two
// classical Gram-Schmidt passes (the preconditioned direction is nearly in
// the Krylov space, so the first pass always cancels most of w), ||w||^2,
// the coefficients to pinned host memory, v_{k+1} = w / ||w||.  In the
// iterative-refinement mode z_k stays FP32 (it is an FP32 result of M) and
// D z_k is taken in FP32 before w joins the FP64 basis.
template <class R>
ddamg_status enqueue_iteration(ddamg_ctx* h, int k, std::vector<const double*>& vlist, double* vk, double* zk,
                               double* vk1) {
  const int m = h->p.outer_restart;
  const size_t N = h->V24, NC = N / 2;
  if (refine_mode(h)) {
    float* z32 = h->fZ32 + (size_t)k * N;
    TRY(to_inner<float>(h, vk, (float*)h->fin, 1));
    TRY(op_M<float>(h, (float*)h->fin, z32, 1, h->d_cit + k));
    TRY(op_dslash<float>(h, DSLASH_D, z32, nullptr, (float*)h->fout, 1));
    TRY(from_inner<float>(h, (float*)h->fout, h->fw, 1));
  } else {
    TRY(precond_to_f64<R>(h, vk, zk, h->d_cit + k));
    TRY(op_dslash<double>(h, DSLASH_D, zk, nullptr, h->fw, 1));
  }
  double* c1 = h->dots;
  double* c2 = h->dots + 2 * (m + 2);
  double* nn = h->dots + 4 * (m + 2);
  addf(h, (refine_mode(h) ? 1 : 2) * flops_gs_pass(h, k + 1) + 2.0 * flops_gs_pass(h, 1));
  if (refine_mode(h)) {
    // one classical Gram-Schmidt pass; its reduction also carries ||w||^2
    // so that the host can order a second pass when the first cancelled
    // most of w (fgmres)
    const double* keep = vlist[k + 1];
    vlist[k + 1] = h->fw;
    CK(multi_dot<double>(vlist.data(), k + 2, h->fw, NC, h->red, c1, h->st));
    vlist[k + 1] = keep;
    CK(multi_axpy_norm<double>(vlist.data(), k + 1, c1, -1.0, h->fw, NC, h->red, nn, h->st));
  } else {
    CK(multi_dot<double>(vlist.data(), k + 1, h->fw, NC, h->red, c1, h->st));
    CK(multi_axpy<double>(vlist.data(), k + 1, c1, -1.0, h->fw, NC, h->st));
    CK(multi_dot<double>(vlist.data(), k + 1, h->fw, NC, h->red, c2, h->st));
    CK(multi_axpy_norm<double>(vlist.data(), k + 1, c2, -1.0, h->fw, NC, h->red, nn, h->st));
  }
  CK(cudaMemcpyAsync(h->h_pinned, h->dots, (4 * (m + 2) + 2) * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(h->h_pinned + DONE_SLOT, h->dots + DONE_SLOT, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(scale_by_inv_norm<double>(h->fw, vk1, nn, N, h->st));
  return DDAMG_OK;
}

// Wait until iteration k's coefficients have reached the host: poll the slot
// its graph copies last (stream order makes the coefficient copy complete
// first), so that the host works on the Givens step while the graph's last
// kernel still runs.  Falls back to a stream synchronisation after about a
// second, and when kernel timing needs the graph's events.
ddamg_status wait_coefficients(ddamg_ctx* h) {
  if (h->timing) {
    CK(cudaStreamSynchronize(h->st));
    return DDAMG_OK;
  }
  volatile double* flag = h->h_pinned + DONE_SLOT;
  const auto t0 = std::chrono::steady_clock::now();
  while (*flag != 1.0) {
    if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(1)) {
      CK(cudaStreamSynchronize(h->st));
      break;
    }
  }
  std::atomic_thread_fence(std::memory_order_acquire);
  return DDAMG_OK;
}

// In the refinement mode a second Gram-Schmidt pass is needed only when the
// first one cancelled most of w: below this ratio ||w_after||^2 / ||w||^2
// (orthogonality lost per pass is about eps ||w|| / ||w_after||; a cycle ends
// after a relative reduction of 1e-5 or m iterations, and restarts from the
// FP64 true residual)
constexpr double REORTH_RATIO = 1e-2;

// Launch iteration k from its CUDA graph (captured on first use, and again
// whenever buffers moved or kernel timing was switched).
template <class R>
ddamg_status run_iteration(ddamg_ctx* h, int k, std::vector<const double*>& vlist, double* vk, double* zk,
                           double* vk1) {
  // (three levels: the coarse FGMRES reads its coefficients on the host)
  if (!h->graphs_on || h->levels == 3) return enqueue_iteration<R>(h, k, vlist, vk, zk, vk1);
  auto& G = h->graphs[k];
  if (!G.exec || G.gen != h->gen || G.timing != h->timing) {
    if (G.exec) {
      cudaGraphExecDestroy(G.exec);
      G.exec = nullptr;
    }
    for (auto& gt : G.timers) {
      cudaEventDestroy(gt.t.a);
      cudaEventDestroy(gt.t.b);
    }
    G.timers.clear();
    const uint64_t l0 = LaunchCount::mine();
    const double f0 = h->flops[h->fphase];
    uint64_t c0[NCLS];
    for (int c = 0; c < NCLS; ++c) c0[c] = h->n_cls[c];
    // record on the handle's private stream (the caller's stream may be the
    // legacy default stream, which cannot be captured); replay on h->st
    cudaStream_t user = h->st;
    h->st = h->cap_st;
    cudaError_t e = cudaStreamBeginCapture(h->st, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
      h->st = user;
      CK(e);
    }
    h->capture_timers = &G.timers;
    ddamg_status s = enqueue_iteration<R>(h, k, vlist, vk, zk, vk1);
    h->capture_timers = nullptr;
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(h->st, &graph);
    h->st = user;
    G.launches = LaunchCount::mine() - l0;
    G.flops = h->flops[h->fphase] - f0;
    h->flops[h->fphase] = f0;
    for (int c = 0; c < NCLS; ++c) {
      G.n_cls[c] = h->n_cls[c] - c0[c];
      h->n_cls[c] = c0[c];
    }
    g_launches.remove_mine(G.launches);
    if (s != DDAMG_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    CK(e);
    e = cudaGraphInstantiate(&G.exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(e);
    G.gen = h->gen;
    G.timing = h->timing;
  }
  CK(launch_graph_ordered(G.exec, h->st));
  g_launches += G.launches;
  addf(h, G.flops);
  for (int c = 0; c < NCLS; ++c) h->n_cls[c] += G.n_cls[c];
  return DDAMG_OK;
}

// Run the work `enqueue` puts on the handle's stream through graph G: eagerly
// the first time (allocations and autotuning happen there), captured the
// second time and replayed from then on; captured anew when buffers moved or
// the batch width changed.  With kernel timing on every run is eager.
template <class F>
ddamg_status graph_run(ddamg_ctx* h, ddamg_ctx::IterGraph& G, int nb, F&& enqueue) {
  if (h->timing || !h->graphs_on || h->levels == 3) return enqueue();
  if (G.exec && (G.gen != h->gen || G.nb != nb)) {
    cudaGraphExecDestroy(G.exec);
    G.exec = nullptr;
    G.uses = 0;
  }
  if (!G.exec) {
    if (G.nb != nb) {
      G.nb = nb;
      G.uses = 0;
    }
    if (G.uses++ == 0) return enqueue();
    if (!h->cap_st) CK(cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking));
    const uint64_t l0 = LaunchCount::mine();
    const double f0 = h->flops[h->fphase];
    uint64_t c0[NCLS];
    for (int c = 0; c < NCLS; ++c) c0[c] = h->n_cls[c];
    cudaStream_t user = h->st;
    h->st = h->cap_st;
    cudaError_t e = cudaStreamBeginCapture(h->st, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
      h->st = user;
      CK(e);
    }
    ddamg_status s = enqueue();
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(h->st, &graph);
    h->st = user;
    G.launches = LaunchCount::mine() - l0;
    G.flops = h->flops[h->fphase] - f0;
    h->flops[h->fphase] = f0;
    for (int c = 0; c < NCLS; ++c) {
      G.n_cls[c] = h->n_cls[c] - c0[c];
      h->n_cls[c] = c0[c];
    }
    g_launches.remove_mine(G.launches);
    if (s != DDAMG_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    CK(e);
    e = cudaGraphInstantiate(&G.exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(e);
    G.gen = h->gen;
  }
  CK(launch_graph_ordered(G.exec, h->st));
  g_launches += G.launches;
  addf(h, G.flops);
  for (int c = 0; c < NCLS; ++c) h->n_cls[c] += G.n_cls[c];
  return DDAMG_OK;
}

// device time of the timed kernels of graph k's last replay (stream idle)
void collect_graph(ddamg_ctx* h, int k) {
  for (auto& gt : h->graphs[k].timers) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, gt.t.a, gt.t.b) == cudaSuccess) h->ms_cls[gt.cls] += ms;
    else cudaGetLastError();   // a failed query must not surface at the next launch
  }
}

template <class R>
ddamg_status fgmres(ddamg_ctx* h, double tol, ddamg_solve_info* info) {
  const int m = h->p.outer_restart;
  const size_t N = h->V24;          // reals
  const size_t NC = N / 2;          // complex
  double* V = h->fV;
  double* Z = h->fZ;
  const bool refine = refine_mode(h);
  auto Vk = [&](int k) { return V + (size_t)k * N; };
  auto Zk = [&](int k) { return refine ? nullptr : Z + (size_t)k * N; };
  std::vector<const double*> vlist(m + 1), zlist(m);
  std::vector<const float*> zlist32(m);
  for (int k = 0; k <= m; ++k) vlist[k] = Vk(k);
  for (int k = 0; k < m; ++k) {
    zlist[k] = Zk(k);
    zlist32[k] = refine ? h->fZ32 + (size_t)k * N : nullptr;
  }
  int iters = 0, restarts = 0, calls = 0;
  CK(cudaMemsetAsync(h->fx, 0, N * 8, h->st));
  CK(cudaMemsetAsync(h->d_iters_acc, 0, sizeof(int), h->st));
  // history of this solve: model flops (coarse iterations added per cycle,
  // from their counts) against the relative residual
  const double f_start = h->flops[h->fphase];
  double f_coarse = 0.0;
  h->hist_flops.assign(1, 0.0);
  h->hist_res.assign(1, 1.0);
  std::vector<double> f_iter(m);
  // ||b||
  double host[6 * 64 + 16];
  CK(norm2<double>(h->fb, NC, h->red, h->dots, h->st));
  CK(cudaMemcpyAsync(host, h->dots, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  const double bnorm = std::sqrt(host[0]);
  if (!std::isfinite(bnorm)) return fail(h, DDAMG_ENUMERIC, "right-hand side norm is not finite");
  CK(cudaMemcpyAsync(h->fr, h->fb, N * 8, cudaMemcpyDeviceToDevice, h->st));
  double beta = bnorm;
  bool converged = bnorm == 0.0;
  std::vector<cd> Hc((size_t)(m + 1) * m), g(m + 1), sn(m), y(m);
  std::vector<double> cs(m);
  while (!converged && iters < h->p.max_outer_iter) {
    // V0 = r / beta
    CK(axpby<double>(1.0 / beta, h->fr, 0.0, Vk(0), N, h->st));
    std::fill(g.begin(), g.end(), cd(0));
    g[0] = beta;
    int kdone = 0;
    // a refinement cycle ends once its recurrence residual fell by
    // outer_refine: beyond that the FP32 operator products, not the
    // iteration, limit the residual the recurrence can trust
    const double cycle_stop = std::max(tol * bnorm, refine ? h->p.outer_refine * beta : 0.0);
    for (int k = 0; k < m; ++k) {
      *(volatile double*)(h->h_pinned + DONE_SLOT) = 0.0;
      TRY(run_iteration<R>(h, k, vlist, Vk(k), Zk(k), Vk(k + 1)));
      ++calls;
      TRY(wait_coefficients(h));
      if (h->timing) collect_graph(h, k);
      const double* hp = h->h_pinned;
      std::vector<cd> col(k + 2);
      double n_after = hp[4 * (m + 2)];
      if (refine) {
        for (int j = 0; j <= k; ++j) col[j] = cd(hp[2 * j], hp[2 * j + 1]);
        const double n_before = hp[2 * (k + 1)];
        if (n_after < REORTH_RATIO * n_before) {
          double* c2 = h->dots + 2 * (m + 2);
          double* nn = h->dots + 4 * (m + 2);
          CK(multi_dot<double>(vlist.data(), k + 1, h->fw, NC, h->red, c2, h->st));
          CK(multi_axpy_norm<double>(vlist.data(), k + 1, c2, -1.0, h->fw, NC, h->red, nn, h->st));
          CK(cudaMemcpyAsync(host, c2, (2 * (m + 2) + 2) * sizeof(double), cudaMemcpyDeviceToHost, h->st));
          CK(scale_by_inv_norm<double>(h->fw, Vk(k + 1), nn, N, h->st));
          CK(cudaStreamSynchronize(h->st));
          for (int j = 0; j <= k; ++j) col[j] += cd(host[2 * j], host[2 * j + 1]);
          n_after = host[2 * (m + 2)];
          ++h->reorth;
          addf(h, flops_gs_pass(h, k + 1) + flops_gs_pass(h, 1));
        }
      } else {
        for (int j = 0; j <= k; ++j)
          col[j] = cd(hp[2 * j] + hp[2 * (m + 2) + 2 * j], hp[2 * j + 1] + hp[2 * (m + 2) + 2 * j + 1]);
      }
      const double hn = std::sqrt(n_after);
      if (!std::isfinite(hn)) return fail(h, DDAMG_ENUMERIC, "NaN or Inf in the FGMRES basis norm");
      col[k + 1] = hn;
      for (int j = 0; j < k; ++j) {
        cd t = cs[j] * col[j] + sn[j] * col[j + 1];
        col[j + 1] = -std::conj(sn[j]) * col[j] + cs[j] * col[j + 1];
        col[j] = t;
      }
      double a1 = std::abs(col[k]), a2 = std::abs(col[k + 1]);
      if (a2 == 0.0) { cs[k] = 1.0; sn[k] = 0.0; }
      else if (a1 == 0.0) { cs[k] = 0.0; sn[k] = std::conj(col[k + 1]) / a2; col[k] = a2; }
      else {
        double rho = std::hypot(a1, a2);
        cd ph = col[k] / a1;
        cs[k] = a1 / rho;
        sn[k] = ph * std::conj(col[k + 1]) / rho;
        col[k] = ph * rho;
      }
      for (int j = 0; j <= k; ++j) Hc[(size_t)j * m + k] = col[j];
      g[k + 1] = -std::conj(sn[k]) * g[k];
      g[k] = cs[k] * g[k];
      ++iters;
      kdone = k + 1;
      f_iter[k] = h->flops[h->fphase] - f_start;
      h->hist_res.push_back(std::abs(g[k + 1]) / (bnorm > 0 ? bnorm : 1.0));
      if (std::abs(g[k + 1]) <= cycle_stop || iters >= h->p.max_outer_iter || hn == 0.0) break;
    }
    {  // coarse iterations of this cycle's preconditioner calls -> history flops
      std::vector<int> cits(kdone);
      CK(cudaMemcpyAsync(cits.data(), h->d_cit, kdone * sizeof(int), cudaMemcpyDeviceToHost, h->st));
      CK(cudaStreamSynchronize(h->st));
      for (int j = 0; j < kdone; ++j) {
        f_coarse += cits[j] * flops_coarse_iter(h);
        h->hist_flops.push_back(f_iter[j] + f_coarse);
      }
    }
    for (int i = kdone - 1; i >= 0; --i) {
      cd acc = g[i];
      for (int j = i + 1; j < kdone; ++j) acc -= Hc[(size_t)i * m + j] * y[j];
      y[i] = acc / Hc[(size_t)i * m + i];
    }
    for (int j = 0; j < kdone; ++j) {
      host[2 * j] = y[j].real();
      host[2 * j + 1] = y[j].imag();
    }
    CK(cudaMemcpyAsync(h->d_coef, host, 2 * kdone * sizeof(double), cudaMemcpyHostToDevice, h->st));
    addf(h, (double)h->g.V * 12.0 * kdone * 8.0 + flops_gs_pass(h, 1));
    if (refine) CK(multi_axpy_f32_into_f64(h->g, zlist32.data(), kdone, h->d_coef, 0, 1.0, h->fx, 1, h->st));
    else CK(multi_axpy<double>(zlist.data(), kdone, h->d_coef, 1.0, h->fx, NC, h->st));
    // true residual
    TRY(op_dslash<double>(h, DSLASH_RES, h->fx, h->fb, h->fr, 1));
    CK(norm2<double>(h->fr, NC, h->red, h->dots, h->st));
    CK(cudaMemcpyAsync(host, h->dots, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    beta = std::sqrt(host[0]);
    ++restarts;
    if (!std::isfinite(beta)) return fail(h, DDAMG_ENUMERIC, "NaN or Inf in the true residual");
    converged = beta <= tol * bnorm;
    // the FP64 true residual replaces the recurrence estimate of the cycle's end
    h->hist_flops.push_back(h->flops[h->fphase] - f_start + f_coarse);
    h->hist_res.push_back(bnorm > 0 ? beta / bnorm : 0.0);
  }
  TRY(check_status(h));
  int cit = 0;
  CK(cudaMemcpy(&cit, h->d_iters_acc, sizeof(int), cudaMemcpyDeviceToHost));
  addf(h, cit * flops_coarse_iter(h));
  if (info) {
    info->outer_iters = iters;
    info->restarts = restarts;
    info->coarse_iters = cit;
    info->precond_calls = calls;
    info->true_residual = bnorm > 0 ? beta / bnorm : 0.0;
    info->converged = converged ? 1 : 0;
  }
  if (!converged) return fail(h, DDAMG_ENOCONV, "FGMRES reached max_outer_iter (residual %.3e)", beta / bnorm);
  return DDAMG_OK;
}

// ---- batched outer FGMRES -------------------------------------------------------
// Every right-hand side keeps its own FGMRES (basis, Hessenberg matrix,
// Givens rotations, restarts, convergence); the iterations of the batch run in
// lockstep so that M, D and the Gram-Schmidt reductions act on all of them in
// one launch each (multi-right-hand-side kernels, the coarse GMRES with the
// right-hand sides in lockstep).  A right-hand side that has converged keeps
// being carried (its results are no longer used) until the batch finishes.
constexpr int MAX_BATCH = 64;

size_t batch_small_len(int m, int nb) { return (size_t)nb * (4 * (m + 2) + 2 + 2 * (m + 1) + 2); }

ddamg_status alloc_batch(ddamg_ctx* h, int nb) {
  if (h->bcap >= nb) return DDAMG_OK;
  if (h->bmem) {
    dfree(h, h->bmem, h->bbytes);
    h->bmem = nullptr;
    h->bcap = 0;
    ++h->gen;                      // captured batched iterations referred to the old buffers
  }
  const int m = h->p.outer_restart;
  const size_t F = h->V24 * sizeof(double);            // one FP64 field
  const size_t zf = refine_mode(h) ? F / 2 : F;
  const size_t small = batch_small_len(m, nb) * sizeof(double);
  const size_t bytes = (size_t)nb * ((m + 1) * F + m * zf + 4 * F + 2 * F) + small + 256;
  void* p = nullptr;
  TRY(dalloc(h, &p, bytes));
  h->bmem = (unsigned char*)p;
  h->bbytes = bytes;
  unsigned char* q = h->bmem;
  auto take = [&](size_t b) { unsigned char* r = q; q += b; return r; };
  h->bV = (double*)take((size_t)nb * (m + 1) * F);
  h->bZ = take((size_t)nb * m * zf);
  h->bx = (double*)take(nb * F);
  h->bb = (double*)take(nb * F);
  h->br = (double*)take(nb * F);
  h->bw = (double*)take(nb * F);
  h->bin = take(nb * F);
  h->bout = take(nb * F);
  h->bsmall = (double*)take(small);
  if (h->h_bpinned) cudaFreeHost(h->h_bpinned);
  h->h_bpinned = nullptr;
  CK(cudaHostAlloc(&h->h_bpinned, small, cudaHostAllocDefault));
  h->bcap = nb;
  return DDAMG_OK;
}

// The lockstep batch as a resumable run: slots are admitted (a right-hand
// side with its own tolerance), advanced one restart cycle at a time, and
// taken out when finished, so that a serving loop can refill finished slots
// between cycles.  Slots without a right-hand side hold zero fields and are
// carried along by the batched kernels.
ddamg_status batch_begin(ddamg_ctx* h, int nb) {
  TRY(alloc_batch(h, nb));
  TRY(need_tmp(h, nb, 6));
  BatchRun& B = h->brun;
  B.nb = nb;
  B.bnorm.assign(nb, 0.0);
  B.beta.assign(nb, 0.0);
  B.tol.assign(nb, 0.0);
  B.live.assign(nb, 0);
  B.done.assign(nb, 1);
  B.iters.assign(nb, 0);
  B.restarts.assign(nb, 0);
  B.calls.assign(nb, 0);
  B.t0.assign(nb, std::chrono::steady_clock::now());
  B.cit0 = 0;
  const size_t bytes = (size_t)nb * h->V24 * sizeof(double);
  CK(cudaMemsetAsync(h->bb, 0, bytes, h->st));
  CK(cudaMemsetAsync(h->bx, 0, bytes, h->st));
  CK(cudaMemsetAsync(h->br, 0, bytes, h->st));
  const int m = h->p.outer_restart;
  double* norms = h->bsmall + (size_t)nb * (4 * (m + 2) + 2 + 2 * (m + 1));
  CK(cudaMemsetAsync(norms, 0, 2 * nb * sizeof(double), h->st));
  CK(cudaMemsetAsync(h->d_iters_acc, 0, sizeof(int), h->st));
  CK(cudaStreamSynchronize(h->st));
  return DDAMG_OK;
}

// right-hand side b (host or device, one spinor field) into a free slot
ddamg_status batch_admit(ddamg_ctx* h, int slot, const double* b, int on_device, double tol) {
  BatchRun& B = h->brun;
  const size_t N = h->V24, NC = N / 2;
  double* bs = h->bb + (size_t)slot * N;
  TRY(import_fields<double>(h, b, on_device, 1, bs));
  CK(cudaMemsetAsync(h->bx + (size_t)slot * N, 0, N * sizeof(double), h->st));
  CK(cudaMemcpyAsync(h->br + (size_t)slot * N, bs, N * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  const int m = h->p.outer_restart;
  const int nb = B.nb;
  double* norms = h->bsmall + (size_t)nb * (4 * (m + 2) + 2 + 2 * (m + 1));
  CK(norm2<double>(bs, NC, h->red, norms + 2 * slot, h->st));
  double nn[2];
  CK(cudaMemcpyAsync(nn, norms + 2 * slot, sizeof nn, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  const double bn = std::sqrt(nn[0]);
  if (!std::isfinite(bn)) {
    CK(cudaMemsetAsync(bs, 0, N * sizeof(double), h->st));
    CK(cudaMemsetAsync(h->br + (size_t)slot * N, 0, N * sizeof(double), h->st));
    CK(cudaMemsetAsync(norms + 2 * slot, 0, 2 * sizeof(double), h->st));
    CK(cudaStreamSynchronize(h->st));
    return fail(h, DDAMG_ENUMERIC, "right-hand side of slot %d: norm is not finite", slot);
  }
  B.bnorm[slot] = bn;
  B.beta[slot] = bn;
  B.tol[slot] = tol;
  B.live[slot] = 1;
  B.done[slot] = bn == 0.0;
  B.iters[slot] = 0;
  B.restarts[slot] = 0;
  B.calls[slot] = 0;
  B.t0[slot] = std::chrono::steady_clock::now();
  return DDAMG_OK;
}

// one restart cycle of every live slot that has not finished: Arnoldi steps
// in lockstep until each slot's cycle has ended (its recurrence residual
// reached its target, or m steps), then x += Z y and the FP64 true residual
template <class R>
ddamg_status batch_cycle(ddamg_ctx* h) {
  BatchRun& B = h->brun;
  const int nb = B.nb;
  const int m = h->p.outer_restart;
  const size_t N = h->V24, NC = N / 2;
  const bool refine = refine_mode(h);
  const size_t blk = (size_t)nb * N;                      // reals of one block of nb fields
  double* V = h->bV;
  auto Vk = [&](int k) { return V + (size_t)k * blk; };
  float* Z32 = (float*)h->bZ;
  double* Z64 = (double*)h->bZ;
  std::vector<const double*> vlist(m + 1), zlist(m);
  std::vector<const float*> zlist32(m);
  for (int k = 0; k <= m; ++k) vlist[k] = Vk(k);
  for (int k = 0; k < m; ++k) {
    zlist[k] = Z64 + (size_t)k * blk;
    zlist32[k] = Z32 + (size_t)k * blk;
  }
  // device small buffers: c1 | c2 (nb x 2(m+2) each) | nn (2 nb) | coef (nb x 2(m+1)) | norms (2 nb)
  double* c1 = h->bsmall;
  double* c2 = c1 + (size_t)nb * 2 * (m + 2);
  double* nn = c2 + (size_t)nb * 2 * (m + 2);
  double* coef = nn + 2 * nb;
  double* norms = coef + (size_t)nb * 2 * (m + 1);
  double* hp = h->h_bpinned;
  std::vector<double> cstop(nb), cs((size_t)nb * m);
  std::vector<cd> Hc((size_t)nb * (m + 1) * m), g((size_t)nb * (m + 1)), sn((size_t)nb * m), y(m);
  std::vector<int> kdone(nb, 0), open(nb, 0);
  auto& done = B.done;
  auto& iters = B.iters;
  auto& beta = B.beta;
  auto& bnorm = B.bnorm;

  // V_0 = r / beta for every right-hand side (norms holds beta^2)
  CK(scale_by_inv_norm_batched<double>(h->br, Vk(0), norms, N, nb, h->st));
  for (int r = 0; r < nb; ++r) {
    std::fill(g.begin() + (size_t)r * (m + 1), g.begin() + (size_t)(r + 1) * (m + 1), cd(0));
    g[(size_t)r * (m + 1)] = beta[r];
    kdone[r] = 0;
    open[r] = B.live[r] && !done[r];
    cstop[r] = std::max(B.tol[r] * bnorm[r], refine ? h->p.outer_refine * beta[r] : 0.0);
  }
  if ((int)h->bgraphs.size() < m) h->bgraphs.resize(m);
  for (int k = 0; k < m; ++k) {
    const int kk = k + 1;
    const int kd1 = refine ? kk + 1 : kk;     // first-pass dots (+ ||w||^2 in the refinement mode)
    // z_k = M v_k and w = D z_k for the whole batch, then the first
    // Gram-Schmidt pass (classical, per right-hand side; in the refinement
    // mode with ||w||^2, the update and the coefficients' copy to the host):
    // one CUDA graph per Krylov index and batch width
    auto front = [&]() -> ddamg_status {
      if (refine) {
        float* zk = Z32 + (size_t)k * blk;
        TRY(to_inner<float>(h, Vk(k), (float*)h->bin, nb));
        TRY(op_M<float>(h, (float*)h->bin, zk, nb));
        TRY(op_dslash<float>(h, DSLASH_D, zk, nullptr, (float*)h->bout, nb));
        TRY(from_inner<float>(h, (float*)h->bout, h->bw, nb));
      } else {
        double* zk = Z64 + (size_t)k * blk;
        if constexpr (sizeof(R) == 8) {
          TRY(op_M<double>(h, Vk(k), zk, nb));
        } else {
          TRY(to_inner<float>(h, Vk(k), (float*)h->bin, nb));
          TRY(op_M<float>(h, (float*)h->bin, (float*)h->bout, nb));
          TRY(from_inner<float>(h, (float*)h->bout, zk, nb));
        }
        TRY(op_dslash<double>(h, DSLASH_D, zk, nullptr, h->bw, nb));
      }
      const double* keep = vlist[k + 1];
      if (refine) vlist[k + 1] = h->bw;
      CK(multi_dot_batched<double>(vlist.data(), kd1, h->bw, NC, nb, NC, h->red, c1, h->st));
      vlist[k + 1] = keep;
      if (refine) {
        CK(multi_axpy_batched<double>(vlist.data(), kk, c1, 2 * kd1, -1.0, h->bw, NC, nb, NC, h->red, nn,
                                      h->st));
        CK(cudaMemcpyAsync(hp, c1, (size_t)nb * (4 * (m + 2) + 2) * sizeof(double), cudaMemcpyDeviceToHost,
                           h->st));
      } else {
        CK(multi_axpy_batched<double>(vlist.data(), kk, c1, 2 * kk, -1.0, h->bw, NC, nb, NC, nullptr, nullptr,
                                      h->st));
      }
      return DDAMG_OK;
    };
    TRY(graph_run(h, h->bgraphs[k], nb, front));
    for (int r = 0; r < nb; ++r)
      if (open[r]) ++B.calls[r];
    // second pass where needed (always without the refinement mode; in it
    // when the first pass cancelled most of some w -- as in fgmres), ||w||,
    // v_{k+1}
    bool second = !refine;
    if (refine) {
      CK(cudaStreamSynchronize(h->st));
      const double* hn2 = hp + (size_t)nb * 4 * (m + 2);
      for (int r = 0; r < nb; ++r)
        if (open[r] && hn2[2 * r] < REORTH_RATIO * hp[2 * (r * kd1 + kk)]) second = true;
      if (second) ++h->reorth;
    }
    if (second) {
      CK(multi_dot_batched<double>(vlist.data(), kk, h->bw, NC, nb, NC, h->red, c2, h->st));
      CK(multi_axpy_batched<double>(vlist.data(), kk, c2, 2 * kk, -1.0, h->bw, NC, nb, NC, h->red, nn, h->st));
    }
    addf(h, nb * ((second ? 2.0 : 1.0) * flops_gs_pass(h, kk) + 2.0 * flops_gs_pass(h, 1)));
    CK(scale_by_inv_norm_batched<double>(h->bw, Vk(k + 1), nn, N, nb, h->st));
    if (second) {
      CK(cudaMemcpyAsync(hp, c1, (size_t)nb * (4 * (m + 2) + 2) * sizeof(double), cudaMemcpyDeviceToHost,
                         h->st));
      CK(cudaStreamSynchronize(h->st));
    }
    const double* h1 = hp;
    const double* h2 = hp + (size_t)nb * 2 * (m + 2);
    const double* hn2 = h2 + (size_t)nb * 2 * (m + 2);
    bool any_open = false;
    for (int r = 0; r < nb; ++r) {
      if (!open[r]) continue;
      std::vector<cd> col(k + 2);
      for (int j = 0; j <= k; ++j) {
        col[j] = cd(h1[2 * (r * kd1 + j)], h1[2 * (r * kd1 + j) + 1]);
        if (second) col[j] += cd(h2[2 * (r * kk + j)], h2[2 * (r * kk + j) + 1]);
      }
      const double hn = std::sqrt(hn2[2 * r]);
      if (!std::isfinite(hn)) return fail(h, DDAMG_ENUMERIC, "right-hand side %d: NaN or Inf in the basis norm", r);
      col[k + 1] = hn;
      double* csr = cs.data() + (size_t)r * m;
      cd* snr = sn.data() + (size_t)r * m;
      cd* gr = g.data() + (size_t)r * (m + 1);
      for (int j = 0; j < k; ++j) {
        cd t = csr[j] * col[j] + snr[j] * col[j + 1];
        col[j + 1] = -std::conj(snr[j]) * col[j] + csr[j] * col[j + 1];
        col[j] = t;
      }
      double a1 = std::abs(col[k]), a2 = std::abs(col[k + 1]);
      if (a2 == 0.0) { csr[k] = 1.0; snr[k] = 0.0; }
      else if (a1 == 0.0) { csr[k] = 0.0; snr[k] = std::conj(col[k + 1]) / a2; col[k] = a2; }
      else {
        double rho = std::hypot(a1, a2);
        cd ph = col[k] / a1;
        csr[k] = a1 / rho;
        snr[k] = ph * std::conj(col[k + 1]) / rho;
        col[k] = ph * rho;
      }
      for (int j = 0; j <= k; ++j) Hc[((size_t)r * (m + 1) + j) * m + k] = col[j];
      gr[k + 1] = -std::conj(snr[k]) * gr[k];
      gr[k] = csr[k] * gr[k];
      ++iters[r];
      kdone[r] = k + 1;
      if (std::abs(gr[k + 1]) <= cstop[r] || iters[r] >= h->p.max_outer_iter || hn == 0.0) open[r] = 0;
      any_open |= open[r] != 0;
    }
    if (!any_open) break;
  }
  // x_r += Z_r y_r (zero coefficients beyond each right-hand side's kdone)
  int kmax = 0;
  std::vector<double> cf((size_t)nb * 2 * (m + 1), 0.0);
  for (int r = 0; r < nb; ++r) {
    if (done[r] || !B.live[r] || kdone[r] == 0) continue;
    const int kd = kdone[r];
    kmax = std::max(kmax, kd);
    const cd* gr = g.data() + (size_t)r * (m + 1);
    for (int i = kd - 1; i >= 0; --i) {
      cd acc = gr[i];
      for (int j = i + 1; j < kd; ++j) acc -= Hc[((size_t)r * (m + 1) + i) * m + j] * y[j];
      y[i] = acc / Hc[((size_t)r * (m + 1) + i) * m + i];
    }
    for (int j = 0; j < kd; ++j) {
      cf[(size_t)r * 2 * (m + 1) + 2 * j] = y[j].real();
      cf[(size_t)r * 2 * (m + 1) + 2 * j + 1] = y[j].imag();
    }
  }
  if (kmax > 0) {
    addf(h, nb * ((double)h->g.V * 12.0 * kmax * 8.0 + flops_gs_pass(h, 1)));
    CK(cudaMemcpyAsync(coef, cf.data(), cf.size() * sizeof(double), cudaMemcpyHostToDevice, h->st));
    if (refine)
      CK(multi_axpy_f32_into_f64(h->g, zlist32.data(), kmax, coef, 2 * (m + 1), 1.0, h->bx, nb, h->st));
    else
      CK(multi_axpy_batched<double>(zlist.data(), kmax, coef, 2 * (m + 1), 1.0, h->bx, NC, nb, NC, nullptr, nullptr,
                                    h->st));
  }
  // FP64 true residuals
  TRY(op_dslash<double>(h, DSLASH_RES, h->bx, h->bb, h->br, nb));
  CK(norm2_batched<double>(h->br, NC, nb, NC, h->red, norms, h->st));
  CK(cudaMemcpyAsync(hp, norms, 2 * nb * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  for (int r = 0; r < nb; ++r) {
    if (done[r] || !B.live[r]) continue;
    beta[r] = std::sqrt(hp[2 * r]);
    ++B.restarts[r];
    if (!std::isfinite(beta[r])) return fail(h, DDAMG_ENUMERIC, "right-hand side %d: NaN or Inf in the residual", r);
    if (beta[r] <= B.tol[r] * bnorm[r] || iters[r] >= h->p.max_outer_iter) done[r] = 1;
  }
  return check_status(h);
}

// finished slot -> x (host or device) and its record; the slot is freed
ddamg_status batch_take(ddamg_ctx* h, int slot, double* x, int on_device, ddamg_solve_info* info) {
  BatchRun& B = h->brun;
  const size_t N = h->V24;
  TRY(export_fields<double>(h, h->bx + (size_t)slot * N, 1, x, on_device));
  int cit = 0;
  CK(cudaMemcpy(&cit, h->d_iters_acc, sizeof(int), cudaMemcpyDeviceToHost));
  const double bn = B.bnorm[slot], be = B.beta[slot];
  const bool conv = bn == 0.0 || be <= B.tol[slot] * bn;
  if (info) {
    info->outer_iters = B.iters[slot];
    info->restarts = B.restarts[slot];
    info->coarse_iters = cit;
    info->precond_calls = B.calls[slot];
    info->true_residual = bn > 0 ? be / bn : 0.0;
    info->converged = conv ? 1 : 0;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - B.t0[slot]).count();
  }
  const int m = h->p.outer_restart;
  double* norms = h->bsmall + (size_t)B.nb * (4 * (m + 2) + 2 + 2 * (m + 1));
  CK(cudaMemsetAsync(h->bb + (size_t)slot * N, 0, N * sizeof(double), h->st));
  CK(cudaMemsetAsync(h->bx + (size_t)slot * N, 0, N * sizeof(double), h->st));
  CK(cudaMemsetAsync(h->br + (size_t)slot * N, 0, N * sizeof(double), h->st));
  CK(cudaMemsetAsync(norms + 2 * slot, 0, 2 * sizeof(double), h->st));
  CK(cudaStreamSynchronize(h->st));
  B.live[slot] = 0;
  B.done[slot] = 1;
  return conv ? DDAMG_OK : DDAMG_ENOCONV;
}

ddamg_status batch_cycle_any(ddamg_ctx* h) {
  return h->p.precision == DDAMG_FP64 ? batch_cycle<double>(h) : batch_cycle<float>(h);
}

bool is_prec_ok(ddamg_ctx* h, int prec) {
  if (!is_prec(prec)) {
    fail(h, DDAMG_EINVAL, "precision must be DDAMG_FP64, DDAMG_FP32, DDAMG_BF16 or DDAMG_FP16");
    return false;
  }
  return true;
}

template <class F>
ddamg_status dispatch(ddamg_ctx* h, int prec, F&& f) {
  if (!is_prec_ok(h, prec)) return DDAMG_EINVAL;
  if (prec == DDAMG_FP64) return f((double*)nullptr);
  return f((float*)nullptr);
}

// coarse vectors: host/device FP64 -> device R
template <class R>
ddamg_status coarse_in(ddamg_ctx* h, const double* src, int on_device, size_t nc, R* dst) {
  const double* s = src;
  if (!on_device) {
    TRY(need_lexbuf(h, (2 * nc + h->V24 - 1) / h->V24 + 1));
    CK(cudaMemcpyAsync(h->lexbuf, src, 2 * nc * sizeof(double), cudaMemcpyHostToDevice, h->st));
    s = h->lexbuf;
  }
  CK(coarse_from_f64<R>(s, dst, nc, h->st));
  return DDAMG_OK;
}
template <class R>
ddamg_status coarse_out(ddamg_ctx* h, const R* src, size_t nc, double* dst, int on_device) {
  double* d = dst;
  if (!on_device) {
    TRY(need_lexbuf(h, (2 * nc + h->V24 - 1) / h->V24 + 1));
    d = h->lexbuf;
  }
  CK(coarse_to_f64<R>(src, d, nc, h->st));
  if (!on_device) CK(cudaMemcpyAsync(dst, d, 2 * nc * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return DDAMG_OK;
}

// ---- coarse solve out of a fixed device array ------------------------------------
// Callers that cannot allocate device memory when they solve (a serving loop
// that must not take the allocator's implicit synchronisation or locks, or a
// host thread working inside a device-memory budget reserved up front) can
// run the coarse solve out of this array instead.  It is reserved in every
// GPU that loads the library and held until the process exits.
constexpr size_t NOALLOC_SCRATCH_BYTES = 16u << 20;   // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// The array's name is only a host-side stand-in: its device address comes
// from cudaGetSymbolAddress, looked up on every call with the caller's device
// current, so that it always belongs to the current context (a cached
// address would go stale after cudaDeviceReset or under another context).
// The first call on a device may load the library's device code (lazy
// loading), so it must come before any stream capture.
ddamg_status noalloc_scratch(ddamg_ctx* h, unsigned char** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    return fail(h, DDAMG_ECUDA, "cudaGetSymbolAddress of the fixed scratch array failed: %s", cudaGetErrorString(e));
  *out = reinterpret_cast<unsigned char*>(p);
  return DDAMG_OK;
}

template <class R>
ddamg_status coarse_solve_noalloc_impl(ddamg_ctx* h, int nrhs, const double* in, double* out, double tol,
                                       int* iters) {
  const size_t nc = (size_t)nrhs * h->g.nb * h->n2;
  const size_t vec = (nc * 2 * sizeof(R) + 255) / 256 * 256;
  const CoarsePlan plan = coarse_gmres_plan<R>(h->g, h->p.n_v, h->p.coarse_restart, nrhs);
  const size_t work = plan.work_bytes;
  if (work == 0) return fail(h, DDAMG_EINVAL, "no launch configuration for the coarse solve");
  const size_t need = 2 * vec + work;
  if (need > NOALLOC_SCRATCH_BYTES)
    return fail(h, DDAMG_EINVAL,
                "the coarse solve of %d right-hand sides needs %zu bytes of scratch; the fixed array holds %zu",
                nrhs, need, NOALLOC_SCRATCH_BYTES);
  unsigned char* base = nullptr;
  TRY(noalloc_scratch(h, &base));
  R* bin = reinterpret_cast<R*>(base);
  R* xout = reinterpret_cast<R*>(base + vec);
  void* wk = base + 2 * vec;
  CoarseSolveArgs a;
  a.Dc = h->Dc;
  a.Ainv = h->Ainv;
  a.AinvD = h->AD;
  a.n = h->p.n_v;
  a.tol = tol;
  a.restart = h->p.coarse_restart;
  a.max_iter = h->p.coarse_max_iter;
  a.wait_limit = h->wait_grid;
  CK(coarse_from_f64<R>(in, bin, nc, h->st));
  CK(coarse_gmres<R>(h->g, a, bin, xout, nrhs, wk, h->d_iters, nullptr, h->d_status, h->st, &plan));
  CK(coarse_to_f64<R>(xout, out, nc, h->st));
  TRY(check_status(h));
  if (iters) CK(cudaMemcpyAsync(iters, h->d_iters, nrhs * sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return DDAMG_OK;
}

}  // namespace

// =====================================================================================
// C ABI
// =====================================================================================
namespace {

// the level-2 calls on host coarse fields (op: 0 smoother, 1 M2, 2 coarse solve)
template <class R>
ddamg_status l2_call(ddamg_ctx* h, int op, int nrhs, const double* in, double* out, double tol, int* iters) {
  auto& L = h->l2;
  const size_t fr = l2_field_reals(h), nc = (size_t)nrhs * fr / 2;
  TRY(need_tmp(h, nrhs, 6));
  R* a = (R*)h->tmp[0];
  R* b = (R*)h->tmp[1];
  TRY(coarse_in<R>(h, in, 0, nc, a));
  if (op == 0) {
    TRY(l2_smooth<R>(h, a, b, nrhs));
    TRY(check_status(h));
  } else {
    for (int k = 0; k < nrhs; ++k) {
      if (op == 1) {
        TRY(l2_M2<R>(h, a + (size_t)k * fr, b + (size_t)k * fr));
        TRY(check_status(h));
      } else {
        int it = 0;
        TRY(l2_fgmres<R>(h, a + (size_t)k * fr, b + (size_t)k * fr, tol, h->p.coarse_max_iter, &it));
        if (iters) iters[k] = it;
      }
    }
  }
  (void)L;
  return coarse_out<R>(h, b, nc, out, 0);
}

ddamg_status l2_call_checked(ddamg_ctx* h, int op, int nrhs, const double* in, double* out, double tol, int* iters) {
  if (!h || nrhs < 1 || nrhs > 4096 || !in || !out) return DDAMG_EINVAL;
  if (!h->l2.have_ops) return fail(h, DDAMG_ESTATE, "no level 2: ddamg_level2_init, then set or set up its vectors");
  if (op == 2 && !(tol > 0.0)) return fail(h, DDAMG_EINVAL, "tolerance must be positive");
  if (inner32(h)) return l2_call<float>(h, op, nrhs, in, out, tol, iters);
  return l2_call<double>(h, op, nrhs, in, out, tol, iters);
}

}  // namespace

extern "C" {

void ddamg_default_params(ddamg_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  for (int mu = 0; mu < 4; ++mu) {
    p->L[mu] = 16;
    p->sap_block[mu] = 4;
    p->agg_block[mu] = 4;
  }
  p->n_v = 20;
  p->m0 = -0.3;
  p->csw = 1.2;
  p->setup_iters = 4;
  p->n_sap = 4;
  p->mr_iters = 4;
  p->coarse_tol = 5e-2;
  p->coarse_restart = 30;
  p->coarse_max_iter = 300;
  p->precision = DDAMG_FP32;
  p->outer_restart = 30;
  p->max_outer_iter = 1000;
  p->seed = 1;
  p->hbm_budget = 0;
  p->outer_refine = 1e-5;
  p->half_vectors = 0;
  p->ortho_fp32 = 0;
}

const char* ddamg_status_string(ddamg_status s) {
  switch (s) {
    case DDAMG_OK: return "DDAMG_OK";
    case DDAMG_EINVAL: return "DDAMG_EINVAL";
    case DDAMG_ENOMEM: return "DDAMG_ENOMEM";
    case DDAMG_ECUDA: return "DDAMG_ECUDA";
    case DDAMG_ENOCONV: return "DDAMG_ENOCONV";
    case DDAMG_ENUMERIC: return "DDAMG_ENUMERIC";
    case DDAMG_ETIMEOUT: return "DDAMG_ETIMEOUT";
    case DDAMG_ESTATE: return "DDAMG_ESTATE";
  }
  return "unknown status";
}

static thread_local std::string g_create_error;

ddamg_status ddamg_create(const ddamg_params* p, const double* gauge, int gauge_on_device, void* stream,
                          ddamg_handle* out) {
  if (!out) return DDAMG_EINVAL;
  *out = nullptr;
  std::string why;
  if (validate(p, why) != DDAMG_OK) {
    g_create_error = why;
    return DDAMG_EINVAL;
  }
  if (!gauge) {
    g_create_error = "gauge is NULL";
    return DDAMG_EINVAL;
  }
  ddamg_ctx* h = new ddamg_ctx();
  h->p = *p;
  h->st = (cudaStream_t)stream;
  h->n2 = 2 * p->n_v;
  ddamg_status s = [&]() -> ddamg_status {
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) return fail(h, DDAMG_ECUDA, "no CUDA device: %s", cudaGetErrorString(e));
    TRY(build_tables(h));
    h->V24 = (size_t)h->g.V * 24;
    const size_t V = h->g.V;
    TRY(dalloc_t(h, &h->d_gauge_lex, V * 72));
    TRY(dalloc_t(h, &h->g64, V * 48));
    TRY(dalloc_t(h, &h->g32, V * 48));
    TRY(dalloc_t(h, &h->A64, V * 72));
    TRY(dalloc_t(h, &h->Ai64, V * 72));
    TRY(dalloc_t(h, &h->A32, V * 72));
    TRY(dalloc_t(h, &h->Ai32, V * 72));
    TRY(dalloc_t(h, &h->d_dev, 1));
    TRY(dalloc_t(h, &h->d_iters, 4096));
    TRY(dalloc_t(h, &h->d_iters_acc, 1));
    TRY(dalloc_t(h, &h->d_status, 1));
    TRY(dalloc_t(h, &h->red, reduce_scratch_len(64)));
    TRY(dalloc_t(h, &h->dots, (size_t)6 * 64 + 16));
    {
      const double one = 1.0;
      CK(cudaMemcpyAsync(h->dots + DONE_SLOT, &one, sizeof one, cudaMemcpyHostToDevice, h->st));
      CK(cudaStreamSynchronize(h->st));
    }
    TRY(dalloc_t(h, &h->lam64, (size_t)p->n_v * h->V24));
    CK(cudaMemsetAsync(h->d_status, 0, sizeof(int), h->st));
    CK(cudaMemsetAsync(h->d_dev, 0, sizeof(unsigned long long), h->st));
    CK(cudaMemcpyAsync(h->d_gauge_lex, gauge, V * 72 * sizeof(double),
                       gauge_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
    CK(import_gauge(h->g, h->d_gauge_lex, h->g64, h->g32, h->d_dev, h->st));
    unsigned long long bits = 0;
    CK(cudaMemcpyAsync(&bits, h->d_dev, sizeof bits, cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    double dev;
    std::memcpy(&dev, &bits, sizeof dev);
    if (!(dev <= 1e-9))
      return fail(h, DDAMG_EINVAL, "gauge links are not SU(3): max deviation %.3e", dev);
    TRY(rebuild_clover(h, p->m0, p->csw));
    CK(cudaStreamSynchronize(h->st));
    return DDAMG_OK;
  }();
  if (s != DDAMG_OK) {
    g_create_error = h->err;
    ddamg_destroy(h);
    return s;
  }
  *out = h;
  return DDAMG_OK;
}

ddamg_status ddamg_set_gauge(ddamg_handle h, const double* gauge, int on_device) {
  if (!h || !gauge) return DDAMG_EINVAL;
  const size_t V = h->g.V;
  CK(cudaMemcpyAsync(h->d_gauge_lex, gauge, V * 72 * sizeof(double),
                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
  CK(cudaMemsetAsync(h->d_dev, 0, sizeof(unsigned long long), h->st));
  CK(import_gauge(h->g, h->d_gauge_lex, h->g64, h->g32, h->d_dev, h->st));
  unsigned long long bits = 0;
  CK(cudaMemcpyAsync(&bits, h->d_dev, sizeof bits, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  double dev;
  std::memcpy(&dev, &bits, sizeof dev);
  h->have_coarse = false;           // the clover term, test vectors and D_c belong to the old links
  if (!(dev <= 1e-9)) return fail(h, DDAMG_EINVAL, "gauge links are not SU(3): max deviation %.3e", dev);
  TRY(rebuild_clover(h, h->p.m0, h->p.csw));
  return DDAMG_OK;
}

ddamg_status ddamg_run_setup(ddamg_handle h, const double* init, int on_device) {
  if (!h) return DDAMG_EINVAL;
  const int n = h->p.n_v;
  // the clover term and its inverse are part of the setup (rebuilt from the
  // resident links, so a repeated setup redoes all of its work)
  TRY(rebuild_clover(h, h->p.m0, h->p.csw));
  TRY(revive_lam64(h));
  if (init) {
    TRY(import_fields<double>(h, init, on_device, n, h->lam64));
  } else {
    TRY(need_lexbuf(h, n));
    CK(random_spinors(h->g, h->p.seed, n, h->lexbuf, h->st));
    CK(pack_spinor<double>(h->g, h->lexbuf, h->lam64, n, h->st));
  }
  h->have_vectors = true;
  h->have_coarse = false;
  ddamg_status s = h->p.precision == DDAMG_FP64 ? setup_impl<double>(h) : setup_impl<float>(h);
  if (s != DDAMG_OK) return s;
  CK(cudaStreamSynchronize(h->st));
  return DDAMG_OK;
}

ddamg_status ddamg_setup(const ddamg_params* p, const double* gauge, int gauge_on_device, void* stream,
                         ddamg_handle* out) {
  ddamg_status s = ddamg_create(p, gauge, gauge_on_device, stream, out);
  if (s != DDAMG_OK) return s;
  s = ddamg_run_setup(*out, nullptr, 0);
  if (s != DDAMG_OK) {
    g_create_error = (*out)->err;
    ddamg_destroy(*out);
    *out = nullptr;
  }
  return s;
}

ddamg_status ddamg_update_mass(ddamg_handle h, double m0, double csw) {
  if (!h) return DDAMG_EINVAL;
  if (!std::isfinite(m0) || !std::isfinite(csw)) return fail(h, DDAMG_EINVAL, "m0 and csw must be finite");
  h->p.m0 = m0;
  h->p.csw = csw;
  TRY(rebuild_clover(h, m0, csw));
  if (h->have_coarse) TRY(build_coarse_op(h));
  CK(cudaStreamSynchronize(h->st));
  return DDAMG_OK;
}

ddamg_status ddamg_solve(ddamg_handle h, int nrhs, const double* rhs, double* x, int on_device, double tol,
                         ddamg_solve_info* info) {
  if (!h) return DDAMG_EINVAL;
  if (nrhs < 0 || (nrhs > 0 && (!rhs || !x))) return fail(h, DDAMG_EINVAL, "bad nrhs / buffers");
  if (!(tol > 0.0)) return fail(h, DDAMG_EINVAL, "tol must be > 0");
  if (!h->have_coarse) return fail(h, DDAMG_ESTATE, "run the setup first");
  TRY(prepare_capture(h));
  ddamg_status worst = DDAMG_OK;
  for (int k = 0; k < nrhs; ++k) {
    auto t0 = std::chrono::steady_clock::now();
    TRY(import_fields<double>(h, rhs + k * h->V24, on_device, 1, h->fb));
    ddamg_solve_info inf{};
    ddamg_status s = h->p.precision == DDAMG_FP64 ? fgmres<double>(h, tol, &inf) : fgmres<float>(h, tol, &inf);
    if (s != DDAMG_OK && s != DDAMG_ENOCONV) return s;
    if (s == DDAMG_ENOCONV) worst = s;
    TRY(export_fields<double>(h, h->fx, 1, x + k * h->V24, on_device));
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) info[k] = inf;
  }
  return worst;
}

ddamg_status ddamg_solve_batched(ddamg_handle h, int nrhs, const double* rhs, double* x, int on_device, double tol,
                                 ddamg_solve_info* info) {
  if (!h) return DDAMG_EINVAL;
  if (nrhs < 0 || nrhs > MAX_BATCH || (nrhs > 0 && (!rhs || !x)))
    return fail(h, DDAMG_EINVAL, "nrhs must be in [0, %d] with buffers", MAX_BATCH);
  if (!(tol > 0.0)) return fail(h, DDAMG_EINVAL, "tol must be > 0");
  if (!h->have_coarse) return fail(h, DDAMG_ESTATE, "run the setup first");
  if (nrhs == 0) return DDAMG_OK;
  auto t0 = std::chrono::steady_clock::now();
  TRY(batch_begin(h, nrhs));
  const size_t N = h->V24;
  for (int r = 0; r < nrhs; ++r) TRY(batch_admit(h, r, rhs + (size_t)r * N, on_device, tol));
  BatchRun& B = h->brun;
  for (;;) {
    bool running = false;
    for (int r = 0; r < nrhs; ++r) running |= B.live[r] && !B.done[r];
    if (!running) break;
    TRY(batch_cycle_any(h));
  }
  int cit = 0;
  CK(cudaMemcpy(&cit, h->d_iters_acc, sizeof(int), cudaMemcpyDeviceToHost));
  addf(h, cit * flops_coarse_iter(h));
  int calls = 0;
  for (int r = 0; r < nrhs; ++r) calls = std::max(calls, B.calls[r]);
  ddamg_status s = DDAMG_OK;
  for (int r = 0; r < nrhs; ++r) {
    ddamg_solve_info one{};
    const ddamg_status sr = batch_take(h, r, x + (size_t)r * N, on_device, &one);
    if (sr != DDAMG_OK && sr != DDAMG_ENOCONV) return sr;
    if (sr == DDAMG_ENOCONV) s = sr;
    one.precond_calls = calls;
    if (info) info[r] = one;
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info)
    for (int r = 0; r < nrhs; ++r) info[r].seconds = secs;
  if (s == DDAMG_ENOCONV) return fail(h, DDAMG_ENOCONV, "FGMRES reached max_outer_iter for part of the batch");
  return s;
}

ddamg_status ddamg_batch_begin(ddamg_handle h, int slots) {
  if (!h) return DDAMG_EINVAL;
  if (slots < 1 || slots > MAX_BATCH) return fail(h, DDAMG_EINVAL, "slots must be in [1, %d]", MAX_BATCH);
  if (!h->have_coarse) return fail(h, DDAMG_ESTATE, "run the setup first");
  return batch_begin(h, slots);
}

ddamg_status ddamg_batch_admit(ddamg_handle h, int slot, const double* rhs, int on_device, double tol) {
  if (!h) return DDAMG_EINVAL;
  BatchRun& B = h->brun;
  if (slot < 0 || slot >= B.nb || !rhs || !(tol > 0.0)) return fail(h, DDAMG_EINVAL, "bad slot, buffer or tolerance");
  if (B.live[slot]) return fail(h, DDAMG_ESTATE, "slot %d holds a right-hand side", slot);
  return batch_admit(h, slot, rhs, on_device, tol);
}

ddamg_status ddamg_batch_cycle(ddamg_handle h, int* running) {
  if (!h) return DDAMG_EINVAL;
  BatchRun& B = h->brun;
  if (B.nb == 0) return fail(h, DDAMG_ESTATE, "no batch begun");
  bool any = false;
  for (int r = 0; r < B.nb; ++r) any |= B.live[r] && !B.done[r];
  if (any) TRY(batch_cycle_any(h));
  if (running) {
    int n = 0;
    for (int r = 0; r < B.nb; ++r) n += B.live[r] && !B.done[r];
    *running = n;
  }
  return DDAMG_OK;
}

ddamg_status ddamg_batch_slot(ddamg_handle h, int slot, int* state) {
  if (!h || !state) return DDAMG_EINVAL;
  BatchRun& B = h->brun;
  if (slot < 0 || slot >= B.nb) return fail(h, DDAMG_EINVAL, "bad slot");
  *state = !B.live[slot] ? 0 : B.done[slot] ? 2 : 1;
  return DDAMG_OK;
}

ddamg_status ddamg_batch_take(ddamg_handle h, int slot, double* x, int on_device, ddamg_solve_info* info) {
  if (!h || !x) return DDAMG_EINVAL;
  BatchRun& B = h->brun;
  if (slot < 0 || slot >= B.nb) return fail(h, DDAMG_EINVAL, "bad slot");
  if (!B.live[slot] || !B.done[slot]) return fail(h, DDAMG_ESTATE, "slot %d has no finished solve", slot);
  const ddamg_status s = batch_take(h, slot, x, on_device, info);
  if (s == DDAMG_ENOCONV) return fail(h, DDAMG_ENOCONV, "slot %d reached max_outer_iter", slot);
  return s;
}

ddamg_status ddamg_apply_D(ddamg_handle h, int prec, int nrhs, const double* in, double* out, int on_device) {
  if (!h || nrhs < 1 || !in || !out) return DDAMG_EINVAL;
  const int k = half_kind(prec);
  if (k >= 0) {
    // half links, clover and spinors (FP32 arithmetic): in -> half, D, -> FP64
    TRY(need_tmp(h, nrhs, 6));
    TRY(half_operators(h, k));
    TRY(need_half_fields(h, nrhs));
    float* t0 = (float*)h->tmp[0];
    float* t1 = (float*)h->tmp[1];
    TRY(import_fields<float>(h, in, on_device, nrhs, t0));
    addf(h, (double)nrhs * h->g.V * F_D);
    CK(by_half(k, [&](auto* tag) {
      using S = std::remove_pointer_t<decltype(tag)>;
      return spinor_to_half<S>(h->g, t0, h->hb, h->hbn, nrhs, h->st);
    }));
    // one thread per site (0) or four (1), measured
    auto run = [&](int var) -> cudaError_t {
      return by_half(k, [&](auto* tag) {
        using S = std::remove_pointer_t<decltype(tag)>;
        if (var == 1 && h->g.V % 8 == 0)
          return dslash4<S>(h->g, h->hb, h->hbn, h->hx, h->hxn, h->gH[k], h->AH[k], nrhs, h->st);
        return dslash_h<S>(h->g, DSLASH_D, h->hb, h->hbn, nullptr, nullptr, h->hx, h->hxn, h->gH[k], h->AH[k],
                           nrhs, h->st);
      });
    };
    int v = 0;
    TRY(tuned(h, k ? "D bf16" : "D fp16", lattice_key(h, k ? "bf16" : "fp16", nrhs), h->g.V % 8 == 0 ? 2 : 1, run,
              &v));
    CK(timed(h, 0, [&] { return run(v); }));
    CK(by_half(k, [&](auto* tag) {
      using S = std::remove_pointer_t<decltype(tag)>;
      return spinor_from_half<S>(h->g, h->hx, h->hxn, t1, nrhs, false, h->st);
    }));
    return export_fields<float>(h, t1, nrhs, out, on_device);
  }
  return dispatch(h, prec, [&](auto* tag) -> ddamg_status {
    using R = std::remove_pointer_t<decltype(tag)>;
    TRY(need_tmp(h, nrhs, 6));
    TRY(import_fields<R>(h, in, on_device, nrhs, (R*)h->tmp[0]));
    TRY(op_dslash<R>(h, DSLASH_D, (R*)h->tmp[0], nullptr, (R*)h->tmp[1], nrhs));
    return export_fields<R>(h, (R*)h->tmp[1], nrhs, out, on_device);
  });
}

ddamg_status ddamg_apply_clover(ddamg_handle h, int prec, int inverse, int nrhs, const double* in, double* out,
                                int on_device) {
  if (!h || nrhs < 1 || !in || !out) return DDAMG_EINVAL;
  return dispatch(h, prec, [&](auto* tag) -> ddamg_status {
    using R = std::remove_pointer_t<decltype(tag)>;
    TRY(need_tmp(h, nrhs, 6));
    TRY(import_fields<R>(h, in, on_device, nrhs, (R*)h->tmp[0]));
    CK(dslash<R>(h->g, DSLASH_CLOVER, (R*)h->tmp[0], nullptr, (R*)h->tmp[1], gauge_of<R>(h),
                 clov_of<R>(h, inverse != 0), nrhs, h->st));
    return export_fields<R>(h, (R*)h->tmp[1], nrhs, out, on_device);
  });
}

ddamg_status ddamg_get_clover(ddamg_handle h, int inverse, double* out) {
  if (!h || !out) return DDAMG_EINVAL;
  size_t nd = (size_t)h->g.V * 72;
  if (h->lexbuf_fields * h->V24 < nd) TRY(need_lexbuf(h, (nd + h->V24 - 1) / h->V24));
  CK(export_clover(h->g, inverse ? h->Ai64 : h->A64, h->lexbuf, h->st));
  CK(cudaMemcpyAsync(out, h->lexbuf, nd * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return DDAMG_OK;
}

ddamg_status ddamg_block_solve(ddamg_handle h, int prec, int colour, int nrhs, const double* in, double* out,
                               int on_device) {
  if (!h || nrhs < 1 || !in || !out || (colour != 0 && colour != 1)) return DDAMG_EINVAL;
  const int k = half_kind(prec);
  if (k >= 0 && sap_half_ok(h->g)) {
    TRY(need_tmp(h, nrhs, 6));
    TRY(half_operators(h, k));
    TRY(need_half_fields(h, nrhs));
    float* t0 = (float*)h->tmp[0];
    TRY(import_fields<float>(h, in, on_device, nrhs, t0));
    CK(by_half(k, [&](auto* tag) {
      using S = std::remove_pointer_t<decltype(tag)>;
      return spinor_to_half<S>(h->g, t0, h->hb, h->hbn, nrhs, h->st);
    }));
    bool widen = true;
    TRY(sap_half_widen(h, k, nrhs, &widen));
    CK(cudaMemsetAsync(h->hx, 0, nrhs * h->V24 * 2, h->st));
    CK(cudaMemsetAsync(h->hxn, 0, nrhs * h->g.V * sizeof(float), h->st));
    ++h->n_cls[1];
    CK(by_half(k, [&](auto* tag) {
      using S = std::remove_pointer_t<decltype(tag)>;
      cudaError_t e = sap_sweep_h<S>(h->g, colour, h->p.mr_iters, true, h->hb, h->hbn, h->hx, h->hxn, h->gH[k],
                                     h->AH[k], h->AiH[k], nrhs, h->d_status, h->wait_sap, h->st, widen);
      if (e != cudaSuccess) return e;
      return spinor_from_half<S>(h->g, h->hx, h->hxn, t0, nrhs, false, h->st);
    }));
    TRY(check_status(h));
    return export_fields<float>(h, t0, nrhs, out, on_device);
  }
  return dispatch(h, prec, [&](auto* tag) -> ddamg_status {
    using R = std::remove_pointer_t<decltype(tag)>;
    TRY(need_tmp(h, nrhs, 6));
    R* b = (R*)h->tmp[0];
    R* x = (R*)h->tmp[1];
    TRY(import_fields<R>(h, in, on_device, nrhs, b));
    CK(cudaMemsetAsync(x, 0, nrhs * h->V24 * sizeof(R), h->st));
    ++h->n_cls[1];
    CK(sap_sweep<R>(h->g, colour, h->p.mr_iters, true, b, x, gauge_of<R>(h), clov_of<R>(h, false),
                    clov_of<R>(h, true), nrhs, h->d_status, h->wait_sap, h->st));
    TRY(check_status(h));
    return export_fields<R>(h, x, nrhs, out, on_device);
  });
}

ddamg_status ddamg_sap(ddamg_handle h, int prec, int nrhs, const double* in, double* out, int on_device) {
  if (!h || nrhs < 1 || !in || !out) return DDAMG_EINVAL;
  return dispatch(h, prec, [&](auto* tag) -> ddamg_status {
    using R = std::remove_pointer_t<decltype(tag)>;
    TRY(need_tmp(h, nrhs, 6));
    TRY(import_fields<R>(h, in, on_device, nrhs, (R*)h->tmp[4]));
    TRY(op_sap<R>(h, (R*)h->tmp[4], (R*)h->tmp[5], nrhs, half_kind(prec)));
    TRY(check_status(h));
    return export_fields<R>(h, (R*)h->tmp[5], nrhs, out, on_device);
  });
}

ddamg_status ddamg_set_test_vectors(ddamg_handle h, const double* vecs, int on_device) {
  if (!h || !vecs) return DDAMG_EINVAL;
  TRY(revive_lam64(h));
  TRY(import_fields<double>(h, vecs, on_device, h->p.n_v, h->lam64));
  CK(cudaStreamSynchronize(h->st));
  h->have_vectors = true;
  h->have_coarse = false;
  return sync_lam32(h);
}

ddamg_status ddamg_get_test_vectors(ddamg_handle h, double* vecs) {
  if (!h || !vecs) return DDAMG_EINVAL;
  if (!h->have_vectors) return fail(h, DDAMG_ESTATE, "no test vectors");
  TRY(need_lam64(h));
  return export_fields<double>(h, h->lam64, h->p.n_v, vecs, 0);
}

ddamg_status ddamg_orthonormalize(ddamg_handle h) {
  if (!h) return DDAMG_EINVAL;
  if (!h->have_vectors) return fail(h, DDAMG_ESTATE, "no test vectors");
  TRY(need_lam64(h));
  TRY(ortho_inner(h));
  TRY(sync_lam32(h));
  CK(cudaStreamSynchronize(h->st));
  h->have_coarse = false;
  return DDAMG_OK;
}

ddamg_status ddamg_level2_default_params(ddamg_level2_params* p) {
  if (!p) return DDAMG_EINVAL;
  *p = ddamg_level2_params{};
  for (int mu = 0; mu < 4; ++mu) p->block[mu] = 2;
  p->n_v = 8;
  p->setup_iters = 2;
  p->n_sap = 4;
  p->mr_iters = 4;
  p->coarsest_tol = 5e-2;
  p->coarsest_restart = 30;
  p->coarsest_max_iter = 300;
  p->restart = 30;
  p->seed = 4321;
  return DDAMG_OK;
}

ddamg_status ddamg_level2_init(ddamg_handle h, const ddamg_level2_params* p) {
  if (!h || !p) return DDAMG_EINVAL;
  if (!h->have_coarse) return fail(h, DDAMG_ESTATE, "level 2 is built on D_c: run the setup first");
  CK(cudaStreamSynchronize(h->st));
  if (inner32(h)) return l2_init<float>(h, *p);
  return l2_init<double>(h, *p);
}

ddamg_status ddamg_level2_setup(ddamg_handle h, const double* vecs) {
  if (!h) return DDAMG_EINVAL;
  auto& L = h->l2;
  if (!L.ready) return fail(h, DDAMG_ESTATE, "ddamg_level2_init first");
  if (!h->have_coarse) return fail(h, DDAMG_ESTATE, "no D_c");
  const size_t nreal = (size_t)L.n2v * l2_field_reals(h);
  if (vecs) {
    CK(cudaMemcpyAsync(L.lam64, vecs, nreal * sizeof(double), cudaMemcpyHostToDevice, h->st));
  } else {
    std::mt19937_64 gen(L.p.seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    std::vector<double> v(nreal);
    for (auto& e : v) e = nd(gen);
    CK(cudaMemcpyAsync(L.lam64, v.data(), nreal * sizeof(double), cudaMemcpyHostToDevice, h->st));
    CK(cudaStreamSynchronize(h->st));
  }
  if (inner32(h)) return l2_setup<float>(h);
  return l2_setup<double>(h);
}

ddamg_status ddamg_level2_set_vectors(ddamg_handle h, const double* vecs) {
  if (!h || !vecs) return DDAMG_EINVAL;
  auto& L = h->l2;
  if (!L.ready) return fail(h, DDAMG_ESTATE, "ddamg_level2_init first");
  if (!h->have_coarse) return fail(h, DDAMG_ESTATE, "no D_c");
  CK(cudaMemcpyAsync(L.lam64, vecs, (size_t)L.n2v * l2_field_reals(h) * sizeof(double), cudaMemcpyHostToDevice,
                     h->st));
  if (inner32(h)) return l2_build<float>(h, true);
  return l2_build<double>(h, true);
}

ddamg_status ddamg_level2_get_vectors(ddamg_handle h, double* vecs) {
  if (!h || !vecs) return DDAMG_EINVAL;
  auto& L = h->l2;
  if (!L.ready) return fail(h, DDAMG_ESTATE, "ddamg_level2_init first");
  CK(cudaMemcpyAsync(vecs, L.lam64, (size_t)L.n2v * l2_field_reals(h) * sizeof(double), cudaMemcpyDeviceToHost,
                     h->st));
  CK(cudaStreamSynchronize(h->st));
  return DDAMG_OK;
}

ddamg_status ddamg_level2_get_op(ddamg_handle h, double* out) {
  if (!h || !out) return DDAMG_EINVAL;
  auto& L = h->l2;
  if (!L.have_ops) return fail(h, DDAMG_ESTATE, "no D_cc: set or set up the level-2 test vectors first");
  const size_t m2 = 2 * (size_t)L.n2v, nd = (size_t)L.NXp * 9 * m2 * m2 * 2;
  TRY(need_lexbuf(h, (nd + h->V24 - 1) / h->V24 + 1));
  if (inner32(h)) CK(coarse_export<float>((const float*)L.Dcc, L.n2v, (size_t)L.NXp * 9, h->lexbuf, h->st));
  else CK(coarse_export<double>((const double*)L.Dcc, L.n2v, (size_t)L.NXp * 9, h->lexbuf, h->st));
  CK(cudaMemcpyAsync(out, h->lexbuf, nd * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return DDAMG_OK;
}

ddamg_status ddamg_level2_sap(ddamg_handle h, int nrhs, const double* in, double* out) {
  return l2_call_checked(h, 0, nrhs, in, out, 0.0, nullptr);
}

ddamg_status ddamg_level2_apply_M2(ddamg_handle h, int nrhs, const double* in, double* out) {
  return l2_call_checked(h, 1, nrhs, in, out, 0.0, nullptr);
}

ddamg_status ddamg_level2_coarse_solve(ddamg_handle h, int nrhs, const double* in, double* out, double tol,
                                       int* iters) {
  return l2_call_checked(h, 2, nrhs, in, out, tol, iters);
}

ddamg_status ddamg_set_levels(ddamg_handle h, int levels) {
  if (!h) return DDAMG_EINVAL;
  if (levels != 2 && levels != 3) return fail(h, DDAMG_EINVAL, "levels is 2 or 3");
  if (levels == 3 && !h->l2.have_ops) return fail(h, DDAMG_ESTATE, "level 2 is not set up");
  h->levels = levels;
  return DDAMG_OK;
}

ddamg_status ddamg_set_graphs(ddamg_handle h, int on) {
  if (!h) return DDAMG_EINVAL;
  h->graphs_on = on != 0;
  return DDAMG_OK;
}

ddamg_status ddamg_trim(ddamg_handle h) {
  if (!h) return DDAMG_EINVAL;
  CK(cudaStreamSynchronize(h->st));
  if (inner32(h) && h->have_vectors && h->lam32 && !h->lam64_gone) {
    dfree(h, h->lam64, (size_t)h->p.n_v * h->V24 * sizeof(double));
    h->lam64 = nullptr;
    h->lam64_gone = true;
  }
  for (void* q : h->tmp) dfree(h, q, h->tmp_fields * h->V24 * sizeof(double));
  h->tmp.clear();
  h->tmp_fields = 0;
  dfree(h, h->lexbuf, h->lexbuf_fields * h->V24 * sizeof(double));
  h->lexbuf = nullptr;
  h->lexbuf_fields = 0;
  ++h->gen;                        // captured graphs referred to the temporaries
  return DDAMG_OK;
}

ddamg_status ddamg_build_coarse(ddamg_handle h) {
  if (!h) return DDAMG_EINVAL;
  TRY(build_coarse_op(h));
  CK(cudaStreamSynchronize(h->st));
  return DDAMG_OK;
}

ddamg_status ddamg_get_coarse_op(ddamg_handle h, double* out) {
  if (!h || !out) return DDAMG_EINVAL;
  if (!h->have_coarse) return fail(h, DDAMG_ESTATE, "no coarse operator");
  size_t nc = (size_t)h->g.nb * 9 * h->n2 * h->n2;
  double* tmpd;
  TRY(dalloc_t(h, &tmpd, 2 * nc));
  if (inner32(h)) CK(coarse_export<float>((const float*)h->Dc, h->p.n_v, (size_t)h->g.nb * 9, tmpd, h->st));
  else CK(coarse_export<double>((const double*)h->Dc, h->p.n_v, (size_t)h->g.nb * 9, tmpd, h->st));
  CK(cudaMemcpyAsync(out, tmpd, 2 * nc * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  // release the export buffer
  cudaFree(tmpd);
  h->allocs.pop_back();
  h->bytes -= 2 * nc * sizeof(double);
  return DDAMG_OK;
}

ddamg_status ddamg_set_coarse_op(ddamg_handle h, const double* dc, int on_device) {
  if (!h || !dc) return DDAMG_EINVAL;
  TRY(alloc_coarse(h));
  const size_t nblk = (size_t)h->g.nb * 9;
  const size_t nc = nblk * h->n2 * h->n2;
  const double* src = dc;
  double* tmpd = nullptr;
  if (!on_device) {
    TRY(dalloc_t(h, &tmpd, 2 * nc));
    CK(cudaMemcpyAsync(tmpd, dc, 2 * nc * sizeof(double), cudaMemcpyHostToDevice, h->st));
    src = tmpd;
  }
  CK(cudaMemsetAsync(h->d_status, 0, sizeof(int), h->st));
  if (inner32(h)) {
    CK(coarse_import<float>(src, h->p.n_v, nblk, (float*)h->Dc, h->st));
    CK(invert_self_blocks<float>(h->g, (float*)h->Dc, h->p.n_v, (float*)h->Ainv, h->d_status, h->st));
    CK(premultiply_odd<float>(h->g, (float*)h->Dc, (float*)h->Ainv, h->p.n_v, (float*)h->AD, h->st));
  } else {
    CK(coarse_import<double>(src, h->p.n_v, nblk, (double*)h->Dc, h->st));
    CK(invert_self_blocks<double>(h->g, (double*)h->Dc, h->p.n_v, (double*)h->Ainv, h->d_status, h->st));
    CK(premultiply_odd<double>(h->g, (double*)h->Dc, (double*)h->Ainv, h->p.n_v, (double*)h->AD, h->st));
  }
  int sing = 0;
  CK(cudaMemcpyAsync(&sing, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (tmpd) {
    cudaFree(tmpd);
    h->allocs.pop_back();
    h->bytes -= 2 * nc * sizeof(double);
  }
  if (sing) {
    cudaMemsetAsync(h->d_status, 0, sizeof(int), h->st);
    h->have_coarse = false;
    return fail(h, DDAMG_ENUMERIC, "a coarse self block is singular");
  }
  h->have_coarse = true;
  h->dc_g5 = false;                  // a given stencil need not be G5-hermitian
  return l2_refresh(h);
}

ddamg_status ddamg_get_coarse_plan(ddamg_handle h, int nrhs, ddamg_coarse_plan* out) {
  if (!h || !out || nrhs < 1) return DDAMG_EINVAL;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  const CoarsePlan c = h->p.precision == DDAMG_FP64
                           ? coarse_gmres_plan<double>(h->g, h->p.n_v, h->p.coarse_restart, nrhs)
                           : coarse_gmres_plan<float>(h->g, h->p.n_v, h->p.coarse_restart, nrhs);
  if (c.NR == 0) return fail(h, DDAMG_EINVAL, "no launch configuration for the coarse solve");
  out->rhs_per_pass = c.NR;
  out->ctas = c.G;
  out->sites_per_cta = c.per;
  out->krylov_in_shared = c.local_in_smem;
  out->resident_blocks = c.resident;
  out->block_ring = c.ring;
  out->shared_bytes = c.smem_bytes;
  out->scratch_bytes = c.work_bytes;
  return DDAMG_OK;
}

ddamg_status ddamg_get_tuning(int i, ddamg_tuning* out) {
  if (!out) return DDAMG_EINVAL;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (i < 0 || i >= (int)g_tune.size()) return DDAMG_EINVAL;
  const TuneEntry& e = g_tune[i];
  std::memset(out, 0, sizeof *out);
  snprintf(out->kernel, sizeof out->kernel, "%s", e.kernel.c_str());
  snprintf(out->problem, sizeof out->problem, "%s", e.key.c_str());
  out->variants = (int)e.us.size();
  out->best = e.best;
  for (int v = 0; v < out->variants && v < 4; ++v) out->us[v] = e.us[v];
  return DDAMG_OK;
}

ddamg_status ddamg_pin_variant(const char* kernel, int variant) {
  if (!kernel) return DDAMG_EINVAL;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (auto it = g_pins.begin(); it != g_pins.end(); ++it)
    if (it->first == kernel) {
      g_pins.erase(it);
      break;
    }
  if (variant >= 0) g_pins.emplace_back(kernel, variant);
  return DDAMG_OK;
}

int ddamg_tuning_count(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return (int)g_tune.size();
}

ddamg_status ddamg_set_wait_limit(ddamg_handle h, int64_t polls) {
  if (!h) return DDAMG_EINVAL;
  if (polls < 0) {
    h->wait_sap = WAIT_SAP_DEFAULT;
    h->wait_grid = WAIT_GRID_DEFAULT;
  } else {
    h->wait_sap = polls;
    h->wait_grid = polls;
  }
  return DDAMG_OK;
}

ddamg_status ddamg_restrict(ddamg_handle h, int prec, int nrhs, const double* in, double* out, int on_device) {
  if (!h || nrhs < 1 || !in || !out) return DDAMG_EINVAL;
  if (!h->have_vectors) return fail(h, DDAMG_ESTATE, "no test vectors");
  return dispatch(h, prec, [&](auto* tag) -> ddamg_status {
    using R = std::remove_pointer_t<decltype(tag)>;
    if (sizeof(R) == 8 || !h->lam32) TRY(need_lam64(h));
    if (sizeof(R) == 4 && !h->lam32) TRY(dalloc_t(h, &h->lam32, (size_t)h->p.n_v * h->V24));
    if (sizeof(R) == 4 && !h->lam64_gone) CK(convert_spinor<float, double>(h->g, h->lam64, h->lam32, h->p.n_v, h->st));
    TRY(need_tmp(h, nrhs, 6));
    TRY(import_fields<R>(h, in, on_device, nrhs, (R*)h->tmp[0]));
    CK(restrict_inner<R>(h, (R*)h->tmp[0], (R*)h->tmp[1], nrhs));
    return coarse_out<R>(h, (R*)h->tmp[1], (size_t)nrhs * h->g.nb * h->n2, out, on_device);
  });
}

ddamg_status ddamg_prolong(ddamg_handle h, int prec, int nrhs, const double* in, double* out, int on_device) {
  if (!h || nrhs < 1 || !in || !out) return DDAMG_EINVAL;
  if (!h->have_vectors) return fail(h, DDAMG_ESTATE, "no test vectors");
  return dispatch(h, prec, [&](auto* tag) -> ddamg_status {
    using R = std::remove_pointer_t<decltype(tag)>;
    if (sizeof(R) == 8 || !h->lam32) TRY(need_lam64(h));
    if (sizeof(R) == 4 && !h->lam32) TRY(dalloc_t(h, &h->lam32, (size_t)h->p.n_v * h->V24));
    if (sizeof(R) == 4 && !h->lam64_gone) CK(convert_spinor<float, double>(h->g, h->lam64, h->lam32, h->p.n_v, h->st));
    TRY(need_tmp(h, nrhs, 6));
    TRY(coarse_in<R>(h, in, on_device, (size_t)nrhs * h->g.nb * h->n2, (R*)h->tmp[0]));
    CK(prolong_inner<R>(h, (R*)h->tmp[0], (R*)h->tmp[1], nrhs));
    return export_fields<R>(h, (R*)h->tmp[1], nrhs, out, on_device);
  });
}

ddamg_status ddamg_apply_coarse(ddamg_handle h, int prec, int nrhs, const double* in, double* out,
                                int on_device) {
  if (!h || nrhs < 1 || !in || !out) return DDAMG_EINVAL;
  if (!h->have_coarse) return fail(h, DDAMG_ESTATE, "no coarse operator");
  if (prec != h->p.precision) return fail(h, DDAMG_EINVAL, "the coarse operator is stored in the inner precision");
  return dispatch(h, prec, [&](auto* tag) -> ddamg_status {
    using R = std::remove_pointer_t<decltype(tag)>;
    TRY(need_tmp(h, nrhs, 6));
    size_t nc = (size_t)nrhs * h->g.nb * h->n2;
    TRY(coarse_in<R>(h, in, on_device, nc, (R*)h->tmp[0]));
    // an assembled D_c: all nine blocks (0) or the self and forward blocks
    // with the backward ones from G5-hermiticity (1), measured
    int v = 0;
    if (h->dc_g5) {
      char key[64];
      snprintf(key, sizeof key, "coarse %d sites n_v %d %s nrhs %d", h->g.nb, h->p.n_v,
               sizeof(R) == 4 ? "fp32" : "fp64", nrhs);
      TRY(tuned(h, "coarse stencil", key, 2, [&](int var) {
        return coarse_apply<R>(h->g, (const R*)h->Dc, h->p.n_v, (R*)h->tmp[0], (R*)h->tmp[1], nrhs, h->st,
                               var == 1);
      }, &v));
    }
    CK(timed(h, 3, [&] {
      return coarse_apply<R>(h->g, (const R*)h->Dc, h->p.n_v, (R*)h->tmp[0], (R*)h->tmp[1], nrhs, h->st, v == 1);
    }));
    return coarse_out<R>(h, (R*)h->tmp[1], nc, out, on_device);
  });
}

ddamg_status ddamg_coarse_solve(ddamg_handle h, int prec, int nrhs, const double* in, double* out, int on_device,
                                double tol, int* iters) {
  if (!h || nrhs < 1 || nrhs > 4096 || !in || !out || !(tol > 0.0)) return DDAMG_EINVAL;
  if (!h->have_coarse) return fail(h, DDAMG_ESTATE, "no coarse operator");
  if (prec != h->p.precision) return fail(h, DDAMG_EINVAL, "the coarse operator is stored in the inner precision");
  return dispatch(h, prec, [&](auto* tag) -> ddamg_status {
    using R = std::remove_pointer_t<decltype(tag)>;
    TRY(need_tmp(h, nrhs, 6));
    size_t nc = (size_t)nrhs * h->g.nb * h->n2;
    TRY(coarse_in<R>(h, in, on_device, nc, (R*)h->tmp[0]));
    TRY(op_coarse_solve<R>(h, (R*)h->tmp[0], (R*)h->tmp[1], nrhs, tol, h->d_iters));
    TRY(check_status(h));
    if (iters) CK(cudaMemcpy(iters, h->d_iters, nrhs * sizeof(int), cudaMemcpyDeviceToHost));
    return coarse_out<R>(h, (R*)h->tmp[1], nc, out, on_device);
  });
}

ddamg_status ddamg_coarse_solve_noalloc(ddamg_handle h, int nrhs, const double* in, double* out, double tol,
                                        int* iters) {
  if (!h) return DDAMG_EINVAL;
  if (nrhs < 1 || nrhs > 4096 || !in || !out || !(tol > 0.0))
    return fail(h, DDAMG_EINVAL, "bad nrhs, buffers or tolerance");
  if (!h->have_coarse) return fail(h, DDAMG_ESTATE, "no coarse operator");
  if (h->p.precision == DDAMG_FP64) return coarse_solve_noalloc_impl<double>(h, nrhs, in, out, tol, iters);
  return coarse_solve_noalloc_impl<float>(h, nrhs, in, out, tol, iters);
}

ddamg_status ddamg_apply_M(ddamg_handle h, int prec, int nrhs, const double* in, double* out, int on_device) {
  if (!h || nrhs < 1 || !in || !out) return DDAMG_EINVAL;
  if (!h->have_coarse) return fail(h, DDAMG_ESTATE, "no coarse operator");
  if (prec != h->p.precision) return fail(h, DDAMG_EINVAL, "M runs in the inner precision");
  return dispatch(h, prec, [&](auto* tag) -> ddamg_status {
    using R = std::remove_pointer_t<decltype(tag)>;
    TRY(need_tmp(h, nrhs, 6));
    TRY(import_fields<R>(h, in, on_device, nrhs, (R*)h->tmp[4]));
    TRY(op_M<R>(h, (R*)h->tmp[4], (R*)h->tmp[5], nrhs));
    TRY(check_status(h));
    return export_fields<R>(h, (R*)h->tmp[5], nrhs, out, on_device);
  });
}

ddamg_status ddamg_get_index_maps(ddamg_handle h, int32_t* parity, int32_t* block, int32_t* colour,
                                  int32_t* aggregate, int32_t* coarse_parity) {
  if (!h) return DDAMG_EINVAL;
  const size_t V = h->g.V;
  int* buf;
  TRY(dalloc_t(h, &buf, 3 * V));
  CK(index_maps(h->g, buf, buf + V, buf + 2 * V, h->st));
  std::vector<int> hb(3 * V);
  CK(cudaMemcpyAsync(hb.data(), buf, 3 * V * sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  cudaFree(buf);
  h->allocs.pop_back();
  h->bytes -= 3 * V * sizeof(int);
  if (parity) std::memcpy(parity, hb.data(), V * 4);
  if (block) std::memcpy(block, hb.data() + V, V * 4);
  if (colour) std::memcpy(colour, hb.data() + 2 * V, V * 4);
  if (aggregate) std::memcpy(aggregate, hb.data() + V, V * 4);   // aggregates = Schwarz blocks
  if (coarse_parity) CK(cudaMemcpy(coarse_parity, h->d_cpar, h->g.nb * sizeof(int), cudaMemcpyDeviceToHost));
  return DDAMG_OK;
}

ddamg_status ddamg_get_stats(ddamg_handle h, ddamg_stats* out) {
  if (!h || !out) return DDAMG_EINVAL;
  CK(cudaStreamSynchronize(h->st));
  collect_pending(h);
  out->kernel_launches = g_launches.total() - h->launches0;
  out->dslash_launches = h->n_cls[0];
  out->sap_launches = h->n_cls[1];
  out->coarse_launches = h->n_cls[2];
  out->dslash_ms = h->ms_cls[0];
  out->sap_ms = h->ms_cls[1];
  out->coarse_ms = h->ms_cls[2];
  out->device_bytes = h->bytes;
  out->coarse_apply_launches = h->n_cls[3];
  out->coarse_apply_ms = h->ms_cls[3];
  out->reorth_passes = h->reorth;
  out->restrict_launches = h->n_cls[4];
  out->restrict_ms = h->ms_cls[4];
  out->prolong_launches = h->n_cls[5];
  out->prolong_ms = h->ms_cls[5];
  out->setup_flops = h->flops[0];
  out->solve_flops = h->flops[1];
  return DDAMG_OK;
}

ddamg_status ddamg_get_history(ddamg_handle h, int cap, double* mflop_per_site, double* rel_residual, int* n) {
  if (!h || cap < 0 || !n || (cap > 0 && (!mflop_per_site || !rel_residual))) return DDAMG_EINVAL;
  const int len = (int)std::min(h->hist_flops.size(), h->hist_res.size());
  *n = len;
  for (int i = 0; i < std::min(cap, len); ++i) {
    mflop_per_site[i] = h->hist_flops[i] / h->g.V / 1e6;
    rel_residual[i] = h->hist_res[i];
  }
  return DDAMG_OK;
}

ddamg_status ddamg_reset_stats(ddamg_handle h) {
  if (!h) return DDAMG_EINVAL;
  CK(cudaStreamSynchronize(h->st));
  collect_pending(h);
  h->launches0 = g_launches.total();
  h->reorth = 0;
  h->flops[0] = h->flops[1] = 0.0;
  for (int c = 0; c < NCLS; ++c) {
    h->n_cls[c] = 0;
    h->ms_cls[c] = 0.0;
  }
  return DDAMG_OK;
}

ddamg_status ddamg_enable_kernel_timing(ddamg_handle h, int enable) {
  if (!h) return DDAMG_EINVAL;
  h->timing = enable != 0;
  return DDAMG_OK;
}

ddamg_status ddamg_random_vectors(ddamg_handle h, uint64_t seed, int n, double* out) {
  if (!h || n < 1 || !out) return DDAMG_EINVAL;
  TRY(need_lexbuf(h, n));
  CK(random_spinors(h->g, seed, n, h->lexbuf, h->st));
  CK(cudaMemcpyAsync(out, h->lexbuf, n * h->V24 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return DDAMG_OK;
}

const char* ddamg_last_error(ddamg_handle h) {
  if (!h) return g_create_error.c_str();
  return h->err.c_str();
}

void ddamg_destroy(ddamg_handle h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  else cudaDeviceSynchronize();
  for (void* p : h->allocs) cudaFree(p);
  collect_pending(h);
  for (auto& t : h->pool) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  for (auto& gph : h->bgraphs)
    if (gph.exec) cudaGraphExecDestroy(gph.exec);
  for (auto& gph : h->graphs) {
    if (gph.exec) cudaGraphExecDestroy(gph.exec);
    for (auto& gt : gph.timers) {
      cudaEventDestroy(gt.t.a);
      cudaEventDestroy(gt.t.b);
    }
  }
  if (h->h_pinned) cudaFreeHost(h->h_pinned);
  if (h->h_bpinned) cudaFreeHost(h->h_bpinned);
  if (h->cap_st) cudaStreamDestroy(h->cap_st);
  delete h;
}

}  // extern "C"
