// Serving loop of the library (declared in include/ddamg.h): propagator
// requests over several resident gauge configurations with continuous
// batching.  A worker thread serves one configuration at a time through the
// resumable lockstep batch (ddamg_batch_*): between FGMRES restart cycles it
// takes finished solves out and admits waiting requests of that
// configuration into the freed slots.  Several workers serve different
// configurations at once, each on its own CUDA stream, so their kernels
// overlap on the device.  Configurations are admitted by device-memory
// footprint.  Host code only; every solve goes through the library's ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
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
  std::vector<int> slots;        // batch slots of its right-hand sides
  int taken = 0;                 // right-hand sides finished
  ddamg_status status = DDAMG_OK;
};

struct Config {
  ddamg_params p{};
  std::vector<double> gauge;     // host copy of the links
  size_t field_reals = 0;        // reals of one spinor field
  ddamg_handle h = nullptr;      // resident handle, nullptr when released
  size_t bytes = 0;              // device bytes last measured (0: never set up)
  size_t reserved = 0;           // bytes counted for a setup or batch allocation in progress
  size_t handle_budget = 0;      // the device-memory budget its handle was created with
  uint64_t last_use = 0;
  bool busy = false;             // a worker is serving it
  bool waiting = false;          // its worker waits for device memory
  cudaStream_t st = nullptr;     // its stream (created with its handle)
};

// Estimate of a configuration's device memory before its first setup (it
// only decides which idle configs to release; the handle's own budget
// enforces the limit):
// links and clover terms in both precisions, test vectors (FP64 + FP32),
// the temporaries of the setup (6 x n_v fields), the coarse operator with its
// inverses and premultiplied blocks, and the buffers of a full batch.
// the buffers of a batch of `slots` right-hand sides (FGMRES basis V, the
// preconditioned directions, six work fields per slot)
size_t batch_bytes(const ddamg_params& p, int slots) {
  const size_t V = (size_t)p.L[0] * p.L[1] * p.L[2] * p.L[3];
  const size_t F = V * 24 * sizeof(double);               // one FP64 spinor field
  const size_t m = (size_t)p.outer_restart;
  return (size_t)slots * (m + 1 + m / 2 + 6) * F;
}

size_t estimate_bytes(const ddamg_params& p, int max_batch) {
  const size_t V = (size_t)p.L[0] * p.L[1] * p.L[2] * p.L[3];
  const size_t F = V * 24 * sizeof(double);               // one FP64 spinor field
  const size_t n = (size_t)p.n_v;
  const size_t nb = V / ((size_t)p.sap_block[0] * p.sap_block[1] * p.sap_block[2] * p.sap_block[3]);
  size_t b = V * (4 * 12 + 2 * 72) * 12;                  // links + A, A^-1 in FP64 and FP32
  b += n * F * 3 / 2;                                     // test vectors
  b += 6 * n * F;                                         // temporaries
  b += nb * (9 + 1 + 4) * (2 * n) * (2 * n) * 16;         // D_c, A^-1, A^-1 D_c (FP64 bound)
  b += batch_bytes(p, max_batch);                         // batched FGMRES
  return b + ((size_t)16 << 20);
}

}  // namespace

struct ddamg_server {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::condition_variable cv_idle;   // a configuration stopped being served
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> reqs;
  std::deque<Config> cfgs;       // stable references while configs are added
  std::vector<std::thread> workers;
  bool stop = false;
  size_t budget = 0;
  int max_batch = 12;
  int device = 0;
  cudaStream_t st = nullptr;     // the caller's stream (nullptr: one stream per config)
  uint64_t next_id = 1, tick = 0;
  std::string last_error;        // message of the most recent failed library call
};

namespace {

// keep the message of a failed call on handle h (under the server's lock)
void note_error(ddamg_server* s, ddamg_handle h, ddamg_status st) {
  if (st == DDAMG_OK) return;
  std::lock_guard<std::mutex> lk(s->mu);
  s->last_error = ddamg_last_error(h);
}

// Configs are added by callers (under the lock) while the worker uses them:
// the worker changes a config's handle and byte count, and scans the list,
// only under the lock; the long calls (setup, solve) run outside it.  A
// configuration being set up, or allocating its batch, counts with the bytes
// reserved for it, so that no other worker admits itself into that memory
// before the allocations are done and measured.
size_t resident_bytes(ddamg_server* s) {
  size_t u = 0;
  for (auto& c : s->cfgs) u += std::max(c.h ? c.bytes : 0, c.reserved);
  return u;
}

void unreserve(ddamg_server* s, Config& c) {
  std::lock_guard<std::mutex> lk(s->mu);
  c.reserved = 0;
  s->cv_idle.notify_all();
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
      std::unique_lock<std::mutex> lk(s->mu);
      used = resident_bytes(s);
      if (!s->budget || used + need <= s->budget) {
        c.reserved = need;
        break;
      }
      bool other_busy = false;
      for (auto& o : s->cfgs) {
        if (o.h && &o != &c && !o.busy && (!lru || o.last_use < lru->last_use)) lru = &o;
        other_busy |= (o.h || o.reserved) && &o != &c && o.busy;    // served, or being set up
      }
      if (!lru && other_busy) {
        // the memory belongs to configurations being served: wait until one
        // of them is idle (and may be released), then look again
        c.waiting = true;
        s->cv_idle.wait(lk);
        c.waiting = false;
        continue;
      }
    }
    if (!lru) {                      // nothing left to release: try, the handle's budget decides
      std::lock_guard<std::mutex> lk(s->mu);
      c.reserved = need;
      break;
    }
    release(s, *lru);
  }
  if (s->budget && used >= s->budget) {
    std::lock_guard<std::mutex> lk(s->mu);
    c.reserved = 0;
    s->last_error = "device memory budget held by configurations being served";
    return DDAMG_ENOMEM;
  }
  ddamg_params p = c.p;
  p.hbm_budget = s->budget ? s->budget - used : 0;
  c.handle_budget = p.hbm_budget;
  if (!c.st) {
    if (s->st) {
      c.st = s->st;
    } else if (cudaStreamCreateWithFlags(&c.st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      c.st = nullptr;
      unreserve(s, c);
      return DDAMG_ECUDA;
    }
  }
  ddamg_handle h = nullptr;
  ddamg_status st = ddamg_setup(&p, c.gauge.data(), 0, c.st, &h);
  if (st != DDAMG_OK) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->last_error = ddamg_last_error(h);
    }
    if (h) ddamg_destroy(h);
    unreserve(s, c);
    return st;
  }
  ddamg_set_graphs(h, 0);          // the workers' threads share the device (no captures)
  {
    std::lock_guard<std::mutex> lk(s->mu);
    c.h = h;
  }
  measure(s, c);
  *setup_run = 1;
  return DDAMG_OK;
}

// the batch buffers of config c.  Device memory can still run short of the
// budget's arithmetic (other processes, the allocator's granularity): on
// DDAMG_ENOMEM idle configurations are released, least recently used first,
// and while other configurations are being served (and not waiting for
// memory themselves) the worker waits for one of them to end and tries
// again; with nothing left to wait for, or when the handle's own budget is
// what the batch exceeds, the error stands (the caller then sets the
// configuration up again).
ddamg_status begin_batch(ddamg_server* s, Config& c, int S) {
  for (;;) {
    const ddamg_status st = ddamg_batch_begin(c.h, S);
    if (st != DDAMG_ENOMEM) return st;
    {
      // the handle's own budget is the limit: waiting for memory cannot help
      ddamg_stats hs{};
      if (c.handle_budget && ddamg_get_stats(c.h, &hs) == DDAMG_OK &&
          hs.device_bytes + batch_bytes(c.p, S) > c.handle_budget)
        return st;
    }
    Config* lru = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      bool progress = false;
      for (auto& o : s->cfgs) {
        if (&o == &c) continue;
        if (o.h && !o.busy && (!lru || o.last_use < lru->last_use)) lru = &o;
        progress |= o.busy && !o.waiting;
      }
      if (!lru) {
        if (!progress) return st;
        c.waiting = true;
        s->cv_idle.wait_for(lk, std::chrono::milliseconds(200));
        c.waiting = false;
        continue;
      }
    }
    release(s, *lru);
  }
}

void finish(ddamg_server* s, Request* r, Clock::time_point t) {
  // caller holds s->mu
  r->rinfo.status = r->status;
  r->rinfo.queue_seconds = std::chrono::duration<double>(r->t_start - r->t_submit).count();
  r->rinfo.latency_seconds = std::chrono::duration<double>(t - r->t_submit).count();
  r->done = true;
  s->cv_done.notify_all();
}

// Serve configuration ci until it has neither running nor waiting requests:
// admit waiting requests (arrival order) into free slots, run a restart
// cycle, take out the requests whose right-hand sides have all finished.
void serve(ddamg_server* s, int ci) {
  int setup_run = 0;
  ddamg_status st = ensure_resident(s, ci, &setup_run);
  Config& c = s->cfgs[ci];
  const int S = s->max_batch;
  std::vector<Request*> slot_req(S, nullptr);
  std::vector<Request*> active;
  if (st == DDAMG_OK) {
    st = begin_batch(s, c, S);
    if (st == DDAMG_ENOMEM) {
      // the handle's own budget (what the server's budget left at its setup)
      // is too small for the batch: set the configuration up once more,
      // admitted with its full estimate, under what the budget leaves now
      note_error(s, c.h, st);
      release(s, c);
      {
        std::lock_guard<std::mutex> lk(s->mu);
        c.bytes = 0;
        c.reserved = 0;
      }
      st = ensure_resident(s, ci, &setup_run);
      if (st == DDAMG_OK) st = begin_batch(s, c, S);
    }
    if (c.h) note_error(s, c.h, st);     // (a failed setup kept its own message)
    // the footprint that later admissions count includes the batch buffers
    if (st == DDAMG_OK) measure(s, c);
    unreserve(s, c);
  }
  for (;;) {
    // admission (requests that fit into the free slots)
    std::vector<Request*> fresh;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      int free_slots = 0;
      for (int k = 0; k < S; ++k) free_slots += slot_req[k] == nullptr;
      for (auto it = s->queue.begin(); it != s->queue.end();) {
        Request* r = *it;
        if (r->cfg == ci && (st != DDAMG_OK || r->nrhs <= free_slots)) {
          if (st == DDAMG_OK) free_slots -= r->nrhs;
          fresh.push_back(r);
          it = s->queue.erase(it);
        } else {
          ++it;
        }
      }
    }
    const auto now = Clock::now();
    for (Request* r : fresh) {
      r->t_start = now;
      r->rinfo.setup_run = setup_run;
      if (st != DDAMG_OK) {          // the configuration could not be set up
        std::lock_guard<std::mutex> lk(s->mu);
        r->status = st;
        finish(s, r, now);
        continue;
      }
      for (int j = 0, k = 0; j < r->nrhs; ++j) {
        while (slot_req[k]) ++k;
        slot_req[k] = r;
        r->slots.push_back(k);
        const ddamg_status a = ddamg_batch_admit(c.h, k, r->rhs + (size_t)j * c.field_reals, 0, r->tol);
        note_error(s, c.h, a);
        if (a != DDAMG_OK && r->status == DDAMG_OK) r->status = a;
      }
      active.push_back(r);
    }
    setup_run = 0;
    if (active.empty()) {
      std::lock_guard<std::mutex> lk(s->mu);
      bool more = false;
      for (Request* r : s->queue) more |= r->cfg == ci;
      if (!more) break;
      continue;
    }
    int running = 0;
    for (Request* r : active) r->rinfo.batch_requests = std::max(r->rinfo.batch_requests, (int)active.size());
    int in_use = 0;
    for (int k = 0; k < S; ++k) in_use += slot_req[k] != nullptr;
    for (Request* r : active) r->rinfo.batch_rhs = std::max(r->rinfo.batch_rhs, in_use);
    const ddamg_status cy = ddamg_batch_cycle(c.h, &running);
    note_error(s, c.h, cy);
    // take out finished right-hand sides; complete requests
    std::vector<Request*> still;
    for (Request* r : active) {
      bool all = true;
      for (size_t j = 0; j < r->slots.size(); ++j) {
        const int k = r->slots[j];
        if (k < 0) continue;
        int state = 0;
        if (cy == DDAMG_OK) ddamg_batch_slot(c.h, k, &state);
        if (cy != DDAMG_OK || state == 2) {
          ddamg_solve_info inf{};
          ddamg_status t = cy;
          if (cy == DDAMG_OK) {
            t = ddamg_batch_take(c.h, k, r->x + j * c.field_reals, 0, &inf);
            if (t != DDAMG_ENOCONV) note_error(s, c.h, t);
          }
          if (r->info) r->info[j] = inf;
          if (t != DDAMG_OK && r->status == DDAMG_OK) r->status = t;
          slot_req[k] = nullptr;
          r->slots[j] = -1;
        } else {
          all = false;
        }
      }
      if (all) {
        std::lock_guard<std::mutex> lk(s->mu);
        finish(s, r, Clock::now());
      } else {
        still.push_back(r);
      }
    }
    active.swap(still);
    if (cy != DDAMG_OK) {
      release(s, c);                 // a handle that failed mid-solve is set up afresh next time
      st = cy;
    }
    measure(s, c);
  }
  std::lock_guard<std::mutex> lk(s->mu);
  c.busy = false;
  s->cv_idle.notify_all();
}

void worker_loop(ddamg_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    // the configuration of the oldest waiting request that no other worker serves
    int ci = -1;
    s->cv_work.wait(lk, [&] {
      ci = -1;
      for (Request* r : s->queue)
        if (!s->cfgs[r->cfg].busy) {
          ci = r->cfg;
          break;
        }
      return ci >= 0 || (s->stop && s->queue.empty());
    });
    if (ci < 0) break;                 // stop requested and nothing left
    s->cfgs[ci].busy = true;
    lk.unlock();
    serve(s, ci);
    lk.lock();
    s->cv_work.notify_all();         // another configuration may now be free to serve
  }
}

}  // namespace

extern "C" {

DDAMG_API ddamg_status ddamg_server_create(size_t hbm_budget, int max_batch, void* cuda_stream,
                                           ddamg_server_handle* out) {
  return ddamg_server_create2(hbm_budget, max_batch, 2, cuda_stream, out);
}

DDAMG_API ddamg_status ddamg_server_create2(size_t hbm_budget, int max_batch, int workers, void* cuda_stream,
                                            ddamg_server_handle* out) {
  if (!out) return DDAMG_EINVAL;
  *out = nullptr;
  if (max_batch < 1 || max_batch > 64 || workers < 1 || workers > 16) return DDAMG_EINVAL;
  auto* s = new ddamg_server();
  s->budget = hbm_budget;
  s->max_batch = max_batch;
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return DDAMG_ECUDA;
  }
  s->st = (cudaStream_t)cuda_stream;   // nullptr: every configuration gets a stream of its own
  for (int w = 0; w < workers; ++w) s->workers.emplace_back(worker_loop, s);
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
  s->cv_work.notify_all();
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

DDAMG_API const char* ddamg_server_last_error(ddamg_server_handle s) {
  static thread_local std::string copy;
  if (!s) return "";
  std::lock_guard<std::mutex> lk(s->mu);
  copy = s->last_error;
  return copy.c_str();
}

DDAMG_API void ddamg_server_destroy(ddamg_server_handle s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& w : s->workers)
    if (w.joinable()) w.join();
  for (auto& c : s->cfgs) {
    release(s, c);
    if (c.st && c.st != s->st) cudaStreamDestroy(c.st);
  }
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
}

}  // extern "C"
