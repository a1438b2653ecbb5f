// Serving loop of the library (declared in include/ddamg.h): propagator
// requests over several resident gauge configurations, solved by one worker
// thread in lockstep batches (continuous batching), with admission of
// configurations by device-memory footprint.  Host code only; every solve
// goes through ddamg_setup / ddamg_solve_batched of the same library.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/ddamg.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id = 0;
  int cfg = 0;
  int nrhs = 0;
  const double* rhs = nullptr;
  double* x = nullptr;
  double tol = 0.0;
  ddamg_solve_info* info = nullptr;
  Clock::time_point t_submit, t_start;
  ddamg_request_info rinfo{};
  bool done = false;
};

struct Config {
  ddamg_params p{};
  std::vector<double> gauge;     // host copy of the links
  size_t field_reals = 0;        // reals of one spinor field
  ddamg_handle h = nullptr;      // resident handle, nullptr when released
  size_t bytes = 0;              // device bytes last measured (0: never set up)
  uint64_t last_use = 0;
};

// Estimate of a configuration's device memory before its first setup (it
// only decides which idle configs to release; the handle's own budget
// enforces the limit):
// links and clover terms in both precisions, test vectors (FP64 + FP32),
// the temporaries of the setup (6 x n_v fields), the coarse operator with its
// inverses and premultiplied blocks, and the buffers of a full batch.
size_t estimate_bytes(const ddamg_params& p, int max_batch) {
  const size_t V = (size_t)p.L[0] * p.L[1] * p.L[2] * p.L[3];
  const size_t F = V * 24 * sizeof(double);               // one FP64 spinor field
  const size_t n = (size_t)p.n_v, m = (size_t)p.outer_restart;
  const size_t nb = V / ((size_t)p.sap_block[0] * p.sap_block[1] * p.sap_block[2] * p.sap_block[3]);
  size_t b = V * (4 * 12 + 2 * 72) * 12;                  // links + A, A^-1 in FP64 and FP32
  b += n * F * 3 / 2;                                     // test vectors
  b += 6 * n * F;                                         // temporaries
  b += nb * (9 + 1 + 4) * (2 * n) * (2 * n) * 16;         // D_c, A^-1, A^-1 D_c (FP64 bound)
  b += (size_t)max_batch * (m + 1 + m / 2 + 6) * F;       // batched FGMRES
  return b + ((size_t)16 << 20);
}

}  // namespace

struct ddamg_server {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> reqs;
  std::deque<Config> cfgs;       // stable references while configs are added
  std::thread worker;
  bool stop = false;
  size_t budget = 0;
  int max_batch = 12;
  int device = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  uint64_t next_id = 1, tick = 0;
  double* stage_rhs = nullptr;   // pinned staging of a batch
  double* stage_x = nullptr;
  size_t stage_reals = 0;
};

namespace {

// Configs are added by callers (under the lock) while the worker uses them:
// the worker changes a config's handle and byte count, and scans the list,
// only under the lock; the long calls (setup, solve) run outside it.
size_t resident_bytes(ddamg_server* s) {
  size_t u = 0;
  for (auto& c : s->cfgs)
    if (c.h) u += c.bytes;
  return u;
}

void release(ddamg_server* s, Config& c) {
  ddamg_handle h;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    h = c.h;
    c.h = nullptr;
  }
  if (h) ddamg_destroy(h);
}

void measure(ddamg_server* s, Config& c) {
  ddamg_stats st{};
  if (c.h && ddamg_get_stats(c.h, &st) == DDAMG_OK) {
    std::lock_guard<std::mutex> lk(s->mu);
    c.bytes = st.device_bytes;
  }
}

// make config ci resident (worker thread only); *setup_run = 1 if it was set up
ddamg_status ensure_resident(ddamg_server* s, int ci, int* setup_run) {
  Config* cp;
  size_t need, used;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    cp = &s->cfgs[ci];
    cp->last_use = ++s->tick;
  }
  Config& c = *cp;
  *setup_run = 0;
  if (c.h) return DDAMG_OK;
  need = c.bytes ? c.bytes : estimate_bytes(c.p, s->max_batch);
  for (;;) {
    Config* lru = nullptr;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      used = resident_bytes(s);
      if (!s->budget || used + need <= s->budget) break;
      for (auto& o : s->cfgs)
        if (o.h && &o != &c && (!lru || o.last_use < lru->last_use)) lru = &o;
    }
    if (!lru) break;                 // nothing left to release: try, the handle's budget decides
    release(s, *lru);
  }
  if (s->budget && used >= s->budget) return DDAMG_ENOMEM;
  ddamg_params p = c.p;
  p.hbm_budget = s->budget ? s->budget - used : 0;
  ddamg_handle h = nullptr;
  ddamg_status st = ddamg_setup(&p, c.gauge.data(), 0, s->st, &h);
  if (st != DDAMG_OK) {
    if (h) ddamg_destroy(h);
    return st;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    c.h = h;
  }
  measure(s, c);
  *setup_run = 1;
  return DDAMG_OK;
}

bool grow_stage(ddamg_server* s, size_t reals) {
  if (s->stage_reals >= reals) return true;
  if (s->stage_rhs) cudaFreeHost(s->stage_rhs);
  if (s->stage_x) cudaFreeHost(s->stage_x);
  s->stage_rhs = s->stage_x = nullptr;
  s->stage_reals = 0;
  if (cudaHostAlloc(&s->stage_rhs, reals * sizeof(double), cudaHostAllocDefault) != cudaSuccess ||
      cudaHostAlloc(&s->stage_x, reals * sizeof(double), cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  s->stage_reals = reals;
  return true;
}

// one batch: the config of the oldest request and every waiting request of
// that config, in arrival order, up to max_batch right-hand sides
void run_batch(ddamg_server* s, std::vector<Request*>& batch) {
  const int ci = batch[0]->cfg;
  int tot = 0;
  double tol = batch[0]->tol;
  for (Request* r : batch) {
    tot += r->nrhs;
    tol = std::min(tol, r->tol);
  }
  int setup_run = 0;
  ddamg_status st = ensure_resident(s, ci, &setup_run);
  Config* cp;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    cp = &s->cfgs[ci];
  }
  Config& c = *cp;
  std::vector<ddamg_solve_info> info(tot);
  if (st == DDAMG_OK && !grow_stage(s, (size_t)tot * c.field_reals)) st = DDAMG_ENOMEM;
  if (st == DDAMG_OK) {
    size_t off = 0;
    for (Request* r : batch) {
      std::memcpy(s->stage_rhs + off, r->rhs, (size_t)r->nrhs * c.field_reals * sizeof(double));
      off += (size_t)r->nrhs * c.field_reals;
    }
    st = ddamg_solve_batched(c.h, tot, s->stage_rhs, s->stage_x, 0, tol, info.data());
    measure(s, c);
    if (st == DDAMG_OK || st == DDAMG_ENOCONV) {
      off = 0;
      int k = 0;
      for (Request* r : batch) {
        std::memcpy(r->x, s->stage_x + off, (size_t)r->nrhs * c.field_reals * sizeof(double));
        off += (size_t)r->nrhs * c.field_reals;
        if (r->info) std::memcpy(r->info, info.data() + k, (size_t)r->nrhs * sizeof(ddamg_solve_info));
        k += r->nrhs;
      }
    } else {
      release(s, c);     // a handle that failed mid-solve is set up afresh next time
    }
  }
  const auto t_done = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  for (Request* r : batch) {
    r->rinfo.status = st;
    r->rinfo.batch_rhs = tot;
    r->rinfo.batch_requests = (int)batch.size();
    r->rinfo.setup_run = setup_run;
    r->rinfo.queue_seconds = std::chrono::duration<double>(r->t_start - r->t_submit).count();
    r->rinfo.latency_seconds = std::chrono::duration<double>(t_done - r->t_submit).count();
    r->done = true;
  }
  s->cv_done.notify_all();
}

void worker_loop(ddamg_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
    if (s->queue.empty()) break;          // stop requested and nothing left
    const int ci = s->queue.front()->cfg;
    std::vector<Request*> batch;
    int tot = 0;
    for (auto it = s->queue.begin(); it != s->queue.end();) {
      Request* r = *it;
      if (r->cfg == ci && tot + r->nrhs <= s->max_batch) {
        tot += r->nrhs;
        batch.push_back(r);
        it = s->queue.erase(it);
      } else {
        ++it;
      }
    }
    const auto t0 = Clock::now();
    for (Request* r : batch) r->t_start = t0;
    lk.unlock();
    run_batch(s, batch);
    lk.lock();
  }
}

}  // namespace

extern "C" {

DDAMG_API ddamg_status ddamg_server_create(size_t hbm_budget, int max_batch, void* cuda_stream,
                                           ddamg_server_handle* out) {
  if (!out) return DDAMG_EINVAL;
  *out = nullptr;
  if (max_batch < 1 || max_batch > 64) return DDAMG_EINVAL;
  auto* s = new ddamg_server();
  s->budget = hbm_budget;
  s->max_batch = max_batch;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return DDAMG_ECUDA;
  }
  if (cuda_stream) {
    s->st = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete s;
      return DDAMG_ECUDA;
    }
    s->own_stream = true;
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return DDAMG_OK;
}

DDAMG_API ddamg_status ddamg_server_add_config(ddamg_server_handle s, const ddamg_params* p, const double* gauge,
                                               int* config_id) {
  if (!s || !p || !gauge || !config_id) return DDAMG_EINVAL;
  for (int d = 0; d < 4; ++d)
    if (p->L[d] < 2) return DDAMG_EINVAL;
  Config c;
  c.p = *p;
  const size_t V = (size_t)p->L[0] * p->L[1] * p->L[2] * p->L[3];
  c.gauge.assign(gauge, gauge + V * 4 * 9 * 2);
  c.field_reals = V * 24;
  std::lock_guard<std::mutex> lk(s->mu);
  s->cfgs.push_back(std::move(c));
  *config_id = (int)s->cfgs.size() - 1;
  return DDAMG_OK;
}

DDAMG_API ddamg_status ddamg_server_submit(ddamg_server_handle s, int config_id, int nrhs, const double* rhs,
                                           double* x, double tol, ddamg_solve_info* info, uint64_t* request_id) {
  if (!s || !rhs || !x || !request_id || !(tol > 0.0)) return DDAMG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (config_id < 0 || config_id >= (int)s->cfgs.size()) return DDAMG_EINVAL;
  if (nrhs < 1 || nrhs > s->max_batch || s->stop) return DDAMG_EINVAL;
  auto* r = new Request();
  r->id = s->next_id++;
  r->cfg = config_id;
  r->nrhs = nrhs;
  r->rhs = rhs;
  r->x = x;
  r->tol = tol;
  r->info = info;
  r->t_submit = Clock::now();
  s->reqs[r->id] = r;
  s->queue.push_back(r);
  *request_id = r->id;
  s->cv_work.notify_one();
  return DDAMG_OK;
}

DDAMG_API ddamg_status ddamg_server_wait(ddamg_server_handle s, uint64_t request_id, ddamg_request_info* rinfo) {
  if (!s) return DDAMG_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(request_id);
  if (it == s->reqs.end()) return DDAMG_EINVAL;
  Request* r = it->second;
  s->cv_done.wait(lk, [&] { return r->done; });
  const ddamg_status st = r->rinfo.status;
  if (rinfo) *rinfo = r->rinfo;
  s->reqs.erase(it);
  delete r;
  return st;
}

DDAMG_API ddamg_status ddamg_server_device_bytes(ddamg_server_handle s, size_t* bytes) {
  if (!s || !bytes) return DDAMG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *bytes = resident_bytes(s);
  return DDAMG_OK;
}

DDAMG_API void ddamg_server_destroy(ddamg_server_handle s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto& c : s->cfgs) release(s, c);
  for (auto& kv : s->reqs) delete kv.second;
  if (s->stage_rhs) cudaFreeHost(s->stage_rhs);
  if (s->stage_x) cudaFreeHost(s->stage_x);
  if (s->own_stream) cudaStreamDestroy(s->st);
  delete s;
}

}  // extern "C"
