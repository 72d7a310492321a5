// serve.cu -- the solve server of include/fmm.h: continuous batching of
// independent FMM requests over the batched tree of fmm_set_batch.
//
// Host runtime only (no kernels of its own): a FIFO queue of requests, an
// admission rule by a device-memory budget, and `lanes` worker threads.  Each
// lane owns a CUDA stream, device staging buffers and one resident handle per
// interpolation order, and loops: take the oldest queued request plus every
// later queued request of the same order that fits (particles, requests, the
// batch tree's leaf cells, the budget), copy their inputs into the staging
// buffers, fmm_set_batch + fmm_evaluate, copy each request's results out,
// release its budget.  While one lane computes, the others admit and run the
// requests that arrived in the meantime, so batches overlap on the device.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  int64_t id = 0, n = 0;
  int height = 0, order = 0;
  const double* xyz = nullptr;
  const double* q = nullptr;
  double* phi = nullptr;
  double* F = nullptr;
  int64_t bytes = 0, cells = 0;
  Clock::time_point t_submit, t_start, t_done;
  fmm_status status = FMM_OK;
  int batch_size = 0;
  bool done = false;
};

struct Lane {
  std::thread th;
  cudaStream_t stream = nullptr;
  std::map<int, fmm_handle> h;  // order -> resident handle
  double* in = nullptr;         // staging: xyz [cap][3] then q [cap]
  double* out = nullptr;        // staging: phi [cap] then F [cap][3]
  int64_t cap = 0;
  int64_t bytes = 0;            // staging bytes
  int64_t held = 0;             // device bytes of the handles + staging (as of the last update)
  int64_t floor = 0;            // what the handles hold with no tree (operators), as of the last full trim
  int64_t est = 0;              // memory estimate of the batch it runs (0 when idle)
  int last_order = 0;           // order of its last batch (its resident tree)
  bool busy = false;
  bool trimmed = true;          // nothing but operators held since the last full trim
  int64_t graph_fallbacks = 0;  // evaluations of its handles that ran without a graph (fmm_get_stats out[6])
};

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct fmm_server {
  fmm_server_config cfg{};
  int dev = 0;
  std::mutex mu;
  std::condition_variable cv_work;  // queue or budget changed
  std::condition_variable cv_done;  // a request finished
  std::deque<Req*> queue;
  std::unordered_map<int64_t, Req*> reqs;
  int64_t next_id = 1;
  int64_t inflight = 0, peak_inflight = 0;
  int busy = 0, peak_busy = 0;
  int64_t peak_held = 0;  // peak device bytes held by all lanes after a batch
  int64_t us_copy_in = 0, us_build = 0, us_eval = 0, trims = 0;  // lane time per phase (microseconds), trims
  int64_t n_done = 0, n_batches = 0, particles_done = 0, largest_batch = 0;
  bool stop = false;
  std::vector<Lane*> lanes;
  std::mutex err_mu;
  std::string err;
};

namespace {

fmm_status server_err(fmm_server* s, fmm_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (s) {
    std::lock_guard<std::mutex> lk(s->err_mu);
    s->err = buf;
  }
  return st;
}

int64_t leaf_cells(int height) { return (int64_t)1 << (3 * (height - 1)); }

// Device memory charged to a lane: the per-tree memory it holds (operators
// are a fixed cost and not charged), or the estimate of the batch it runs if
// that is larger.
int64_t tree_bytes(const Lane* M) { return std::max<int64_t>(0, M->held - M->floor); }
int64_t others_charge(fmm_server* s, const Lane* self) {
  int64_t c = 0;
  for (const Lane* M : s->lanes)
    if (M != self) c += M->busy ? std::max(tree_bytes(M), M->est) : tree_bytes(M);
  return c;
}

// Order affinity: a lane keeps taking requests of the order whose tree it
// holds (its handle's buffers are already sized, and it does not have to hold
// trees of two orders) unless the oldest request of another order has waited
// longer than this.
constexpr double AFFINITY_MS = 50.0;

// Requests lane L may take now (called with the lock held): the oldest queued
// request -- or, by affinity, the oldest of the lane's own order --, then
// later ones of the same order while they fit (particles, requests, leaf
// cells, and the memory rule: the other lanes' charge plus max(what L holds,
// the batch's estimate) within the budget).  Returns an empty list when the
// chosen head does not fit yet.
std::vector<Req*> pick(fmm_server* s, Lane* L) {
  std::vector<Req*> b;
  if (s->queue.empty()) return b;
  Req* head = s->queue.front();
  if (L->last_order != 0 && head->order != L->last_order &&
      ms_between(head->t_submit, Clock::now()) < AFFINITY_MS) {
    for (Req* r : s->queue)
      if (r->order == L->last_order) {
        head = r;
        break;
      }
  }
  const int64_t others = others_charge(s, L);
  if (others + std::max(tree_bytes(L), head->bytes) > s->cfg.hbm_budget_bytes) return b;
  int64_t parts = 0, bytes = 0, cells = 0;
  const int64_t max_cells = (int64_t)1 << (3 * FMM_MAX_FOREST_LEAF);
  bool seen_head = false;
  for (auto it = s->queue.begin(); it != s->queue.end();) {
    Req* r = *it;
    seen_head = seen_head || r == head;
    if (!seen_head || r->order != head->order) {
      ++it;
      continue;
    }
    const bool first = b.empty();
    if (!first && ((int)b.size() >= s->cfg.max_batch_requests || parts + r->n > s->cfg.max_batch_particles ||
                   cells + r->cells > max_cells ||
                   others + std::max(tree_bytes(L), bytes + r->bytes) > s->cfg.hbm_budget_bytes)) {
      ++it;
      continue;
    }
    b.push_back(r);
    parts += r->n;
    bytes += r->bytes;
    cells += r->cells;
    it = s->queue.erase(it);
  }
  L->est = bytes;
  L->last_order = head->order;
  s->inflight += bytes;
  s->peak_inflight = std::max(s->peak_inflight, others + std::max(tree_bytes(L), bytes));
  return b;
}

int64_t lane_held(Lane* L) {
  int64_t held = L->bytes;
  for (auto& kv : L->h) {
    int64_t st[8];
    if (fmm_get_stats(kv.second, st) == FMM_OK) held += st[3];
  }
  return held;
}

// Releases the lane's per-tree memory (its handles keep their operators):
// first the handles of orders other than `keep`, then, if `all`, every handle
// and the staging buffers.  Called with the lock held, by the lane itself.
void lane_trim(fmm_server* s, Lane* L, int keep, bool all) {
  s->trims++;
  for (auto& kv : L->h)
    if (all || kv.first != keep) fmm_trim(kv.second);
  if (all) {
    if (L->in) cudaFreeAsync(L->in, L->stream);
    if (L->out) cudaFreeAsync(L->out, L->stream);
    L->in = L->out = nullptr;
    L->cap = 0;
    L->bytes = 0;
  }
  L->held = lane_held(L);
  if (all) {
    L->floor = L->held;
    L->trimmed = true;
  }
}

fmm_status lane_handle(fmm_server* s, Lane* L, int order, fmm_handle* out) {
  auto it = L->h.find(order);
  if (it != L->h.end()) {
    *out = it->second;
    return FMM_OK;
  }
  fmm_handle h = nullptr;
  fmm_status st = fmm_create(3, order, &h);
  if (st != FMM_OK) return server_err(s, st, "lane handle for order %d: %s", order, fmm_last_error(nullptr));
  if ((st = fmm_set_precision(h, s->cfg.precision)) != FMM_OK || (st = fmm_set_stream(h, L->stream)) != FMM_OK) {
    fmm_destroy(h);
    return server_err(s, st, "lane handle for order %d: set-up failed", order);
  }
  L->h[order] = h;
  *out = h;
  return FMM_OK;
}

fmm_status stage_capacity(fmm_server* s, Lane* L, int64_t n) {
  if (n <= L->cap) return FMM_OK;
  if (L->in) cudaFreeAsync(L->in, L->stream);
  if (L->out) cudaFreeAsync(L->out, L->stream);
  L->in = L->out = nullptr;
  L->cap = 0;
  L->bytes = 0;
  const int64_t cap = n + n / 4 + 1024;
  if (fmm::pool_alloc(s->dev, L->stream, (void**)&L->in, 32 * (size_t)cap) != cudaSuccess ||
      fmm::pool_alloc(s->dev, L->stream, (void**)&L->out, 32 * (size_t)cap) != cudaSuccess) {
    cudaGetLastError();
    return server_err(s, FMM_ERR_OOM, "lane staging buffers for %lld particles", (long long)n);
  }
  L->cap = cap;
  L->bytes = 64 * cap;
  return FMM_OK;
}

fmm_status run_batch(fmm_server* s, Lane* L, const std::vector<Req*>& b, int64_t* us) {
  const Clock::time_point t0 = Clock::now();
  fmm_handle h = nullptr;
  FMM_TRY(lane_handle(s, L, b[0]->order, &h));
  int64_t n = 0;
  std::vector<int64_t> counts;
  std::vector<int32_t> heights;
  for (Req* r : b) {
    n += r->n;
    counts.push_back(r->n);
    heights.push_back(r->height);
  }
  FMM_TRY(stage_capacity(s, L, n));
  double* xyz = L->in;
  double* q = L->in + 3 * L->cap;
  double* phi = L->out;
  double* F = L->out + L->cap;
  int64_t off = 0;
  for (Req* r : b) {
    if (r->n > 0) {
      if (cudaMemcpyAsync(xyz + 3 * off, r->xyz, 24 * (size_t)r->n, cudaMemcpyDefault, L->stream) != cudaSuccess ||
          cudaMemcpyAsync(q + off, r->q, 8 * (size_t)r->n, cudaMemcpyDefault, L->stream) != cudaSuccess) {
        cudaGetLastError();
        return server_err(s, FMM_ERR_CUDA, "request %lld: input copy failed", (long long)r->id);
      }
    }
    off += r->n;
  }
  if (cudaStreamSynchronize(L->stream) != cudaSuccess) {
    cudaGetLastError();
    return server_err(s, FMM_ERR_CUDA, "batch of %zu requests: input copies failed", b.size());
  }
  const Clock::time_point t1 = Clock::now();
  fmm_status st = fmm_set_batch(h, (int32_t)b.size(), counts.data(), heights.data(), xyz, q);
  const Clock::time_point t2 = Clock::now();
  if (st == FMM_OK && n > 0) st = fmm_evaluate(h, phi, F);
  if (st != FMM_OK) return server_err(s, st, "batch of %zu requests: %s", b.size(), fmm_last_error(h));
  {
    int64_t sum = 0;
    for (auto& kv : L->h) {
      int64_t o[8];
      if (fmm_get_stats(kv.second, o) == FMM_OK) sum += o[6];
    }
    std::lock_guard<std::mutex> lk(s->mu);
    L->graph_fallbacks = sum;
  }
  off = 0;
  for (Req* r : b) {
    if (r->n > 0) {
      if (cudaMemcpyAsync(r->phi, phi + off, 8 * (size_t)r->n, cudaMemcpyDefault, L->stream) != cudaSuccess ||
          cudaMemcpyAsync(r->F, F + 3 * off, 24 * (size_t)r->n, cudaMemcpyDefault, L->stream) != cudaSuccess) {
        cudaGetLastError();
        return server_err(s, FMM_ERR_CUDA, "request %lld: output copy failed", (long long)r->id);
      }
    }
    off += r->n;
  }
  if (cudaStreamSynchronize(L->stream) != cudaSuccess) {
    cudaGetLastError();
    return server_err(s, FMM_ERR_CUDA, "batch of %zu requests: stream synchronisation failed", b.size());
  }
  const Clock::time_point t3 = Clock::now();
  us[0] = std::chrono::duration_cast<std::chrono::microseconds>(t1 - t0).count();
  us[1] = std::chrono::duration_cast<std::chrono::microseconds>(t2 - t1).count();
  us[2] = std::chrono::duration_cast<std::chrono::microseconds>(t3 - t2).count();
  return FMM_OK;
}

void lane_main(fmm_server* s, Lane* L) {
  cudaSetDevice(s->dev);
  for (;;) {
    std::vector<Req*> b;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] {
        if (s->stop) return true;
        if (s->queue.empty()) return false;
        b = pick(s, L);
        if (!b.empty()) return true;
        // the head does not fit: give back what this lane holds (handles of
        // other orders first) and wake the other idle lanes to do the same
        if (!L->trimmed) {
          lane_trim(s, L, s->queue.front()->order, false);
          b = pick(s, L);
          if (b.empty()) {
            lane_trim(s, L, 0, true);
            b = pick(s, L);
          }
          s->cv_work.notify_all();
        }
        return !b.empty();
      });
      if (s->stop && b.empty()) return;
      L->busy = true;
      L->trimmed = false;
      s->busy++;
      s->peak_busy = std::max(s->peak_busy, s->busy);
    }
    const Clock::time_point t0 = Clock::now();
    for (Req* r : b) r->t_start = t0;
    int64_t us[3] = {0, 0, 0};
    const fmm_status st = run_batch(s, L, b, us);
    const Clock::time_point t1 = Clock::now();
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->busy--;
      s->n_batches++;
      s->us_copy_in += us[0];
      s->us_build += us[1];
      s->us_eval += us[2];
      s->largest_batch = std::max<int64_t>(s->largest_batch, (int64_t)b.size());
      for (Req* r : b) {
        s->inflight -= r->bytes;
        r->status = st;
        r->t_done = t1;
        r->batch_size = (int)b.size();
        r->done = true;
        s->n_done++;
        if (st == FMM_OK) s->particles_done += r->n;
      }
      L->busy = false;
      L->est = 0;
      L->held = lane_held(L);
      // per-tree memory above the budget: this lane gives back what it holds
      int64_t total = tree_bytes(L) + others_charge(s, L);
      s->peak_held = std::max(s->peak_held, total);
      if (total > s->cfg.hbm_budget_bytes) lane_trim(s, L, b[0]->order, false);
      if (tree_bytes(L) + others_charge(s, L) > s->cfg.hbm_budget_bytes) lane_trim(s, L, 0, true);
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
  }
}

}  // namespace

extern "C" {

int64_t fmm_server_request_bytes(int64_t n, int height, int order) {
  if (n < 0 || height < 1 || height > 11 || order < 2 || order > FMM_MAX_ORDER) return -1;
  const int64_t cpad = ((int64_t)order * order * order + 1 + 31) / 32 * 32;
  const int64_t cells = (int64_t)(1.15 * (double)std::min<int64_t>(n, leaf_cells(height))) + 1;
  const int64_t per_cell = 28 * cpad + 4 * 189 * (order <= 5 ? 16 : 32) + 1024;
  return 256 * n + cells * per_cell;
}

fmm_status fmm_server_create(const fmm_server_config* cfg, fmm_server_handle* out) {
  if (!out || !cfg) return FMM_ERR_ARG;
  *out = nullptr;
  if (cfg->lanes < 1 || cfg->lanes > 16 || (cfg->precision != FMM_MIXED && cfg->precision != FMM_FP64) ||
      cfg->hbm_budget_bytes <= 0 || cfg->max_batch_particles < 1 || cfg->max_batch_requests < 1 ||
      cfg->max_batch_requests > FMM_MAX_BATCH)
    return FMM_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaFree(nullptr) != cudaSuccess) {
    cudaGetLastError();
    return FMM_ERR_CUDA;
  }
  fmm_server* s = new fmm_server();
  s->cfg = *cfg;
  s->dev = dev;
  for (int k = 0; k < cfg->lanes; ++k) {
    Lane* L = new Lane();
    if (cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete L;
      fmm_server_destroy(s);
      return FMM_ERR_CUDA;
    }
    s->lanes.push_back(L);
  }
  for (Lane* L : s->lanes) L->th = std::thread(lane_main, s, L);
  *out = s;
  return FMM_OK;
}

fmm_status fmm_server_warmup(fmm_server_handle s, int order) {
  if (!s || order < 2 || order > FMM_MAX_ORDER) return FMM_ERR_ARG;
  // the lanes' handles are only touched by their own threads while they run
  // a batch; warm-up takes the queue lock so that no batch starts meanwhile
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv_done.wait(lk, [&] { return s->busy == 0; });
  cudaSetDevice(s->dev);
  for (Lane* L : s->lanes) {
    fmm_handle h = nullptr;
    FMM_TRY(lane_handle(s, L, order, &h));
    int32_t ranks[16];
    const fmm_status st = fmm_get_svd_ranks(h, ranks);
    if (st != FMM_OK) return server_err(s, st, "warm-up of order %d: %s", order, fmm_last_error(h));
    if (L->trimmed) L->floor = L->held = lane_held(L);
  }
  return FMM_OK;
}

fmm_status fmm_server_submit(fmm_server_handle s, int64_t n, int height, int order, const double* xyz,
                             const double* q, double* phi, double* F, int64_t* ticket) {
  if (!s || !ticket) return FMM_ERR_ARG;
  *ticket = 0;
  if (n < 0 || n > ((int64_t)1 << 30) || height < 1 || height > FMM_MAX_FOREST_LEAF + 1 || order < 2 ||
      order > FMM_MAX_ORDER)
    return server_err(s, FMM_ERR_ARG, "fmm_server_submit: n %lld, height %d or order %d out of range",
                      (long long)n, height, order);
  if (n > 0 && (!xyz || !q || !phi || !F)) return server_err(s, FMM_ERR_ARG, "fmm_server_submit: NULL pointer");
  Req* r = new Req();
  r->n = n;
  r->height = height;
  r->order = order;
  r->xyz = xyz;
  r->q = q;
  r->phi = phi;
  r->F = F;
  r->bytes = fmm_server_request_bytes(n, height, order);
  r->cells = leaf_cells(height);
  if (r->bytes > s->cfg.hbm_budget_bytes) {
    delete r;
    return server_err(s, FMM_ERR_OOM, "fmm_server_submit: the request needs ~%lld bytes, the budget is %lld",
                      (long long)fmm_server_request_bytes(n, height, order), (long long)s->cfg.hbm_budget_bytes);
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      delete r;
      return server_err(s, FMM_ERR_STATE, "fmm_server_submit: server stopping");
    }
    r->id = s->next_id++;
    r->t_submit = Clock::now();
    s->reqs[r->id] = r;
    s->queue.push_back(r);
    *ticket = r->id;
  }
  s->cv_work.notify_all();
  return FMM_OK;
}

fmm_status fmm_server_wait(fmm_server_handle s, int64_t ticket, double timeout_s, double* times) {
  if (!s) return FMM_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return server_err(s, FMM_ERR_ARG, "fmm_server_wait: unknown ticket %lld", (long long)ticket);
  Req* r = it->second;
  auto ready = [&] { return r->done; };
  if (timeout_s < 0) {
    s->cv_done.wait(lk, ready);
  } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
    return FMM_ERR_TIMEOUT;
  }
  if (times) {
    times[0] = ms_between(r->t_submit, r->t_start);
    times[1] = ms_between(r->t_start, r->t_done);
    times[2] = ms_between(r->t_submit, r->t_done);
    times[3] = r->batch_size;
  }
  const fmm_status st = r->status;
  s->reqs.erase(it);
  delete r;
  return st;
}

fmm_status fmm_server_stats(fmm_server_handle s, int64_t* out) {
  if (!s || !out) return FMM_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  out[0] = s->n_done;
  out[1] = s->n_batches;
  out[2] = s->particles_done;
  out[3] = s->peak_inflight;
  out[4] = s->peak_busy;
  out[5] = s->largest_batch;
  out[6] = (int64_t)s->queue.size();
  int64_t held = 0;
  for (Lane* L : s->lanes) held += L->held;
  out[7] = held;
  out[8] = s->us_copy_in;
  out[9] = s->us_build;
  out[10] = s->us_eval;
  out[11] = s->trims;
  int64_t fb = 0;
  for (Lane* L : s->lanes) fb += L->graph_fallbacks;
  out[12] = fb;
  return FMM_OK;
}

fmm_status fmm_server_destroy(fmm_server_handle s) {
  if (!s) return FMM_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (Req* r : s->queue) {
      r->status = FMM_ERR_STATE;
      r->done = true;
    }
    s->queue.clear();
  }
  s->cv_work.notify_all();
  s->cv_done.notify_all();
  for (Lane* L : s->lanes)
    if (L->th.joinable()) L->th.join();
  cudaSetDevice(s->dev);
  for (Lane* L : s->lanes) {
    for (auto& kv : L->h) fmm_destroy(kv.second);
    if (L->in) cudaFreeAsync(L->in, L->stream);
    if (L->out) cudaFreeAsync(L->out, L->stream);
    if (L->stream) {
      cudaStreamSynchronize(L->stream);
      cudaStreamDestroy(L->stream);
    }
    delete L;
  }
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
  return FMM_OK;
}

const char* fmm_server_last_error(fmm_server_handle s) {
  if (!s) return "";
  static thread_local std::string copy;  // stays valid while lanes overwrite the server's message
  std::lock_guard<std::mutex> lk(s->err_mu);
  copy = s->err;
  return copy.c_str();
}

}  // extern "C"
