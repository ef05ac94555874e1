// Request server: continuous batching of MLMC level-pair sample requests on
// one context (include/mlmc.h, mlmc_server_*).
//
// A request is one level pair (level, seed, sample id, optional stimulus
// centre).  A scheduler thread owns all device work.  It admits queued
// requests as batches of one level whenever a slot (a pair of streams) is
// free and the device arena -- one allocation made at creation, carved by a
// first-fit allocator -- has room for the batch's workspace; a batch that
// does not fit is halved until it does.  Batches of different levels run
// concurrently on their slots.  When a batch's solves end, its differences
// Y_l are merged into the context's running estimates on one accumulation
// stream (so merges never race), its results are copied to pinned host
// memory, and the slot and its arena block are released for the next batch.
// The result of a request depends only on the request: every sample is
// solved by its own CTA or cluster with its own reductions, so a request
// gives the same bits alone and in any mix.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "ctx.cuh"

using namespace mlmc;

namespace {

// First-fit allocator over [0, size) in 256-byte units.
class Arena {
 public:
  void init(size_t size) {
    free_.clear();
    free_[0] = size;
    used_ = peak_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align256(bytes ? bytes : 1);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      size_t rest = it->second - bytes;
      size_t at = it->first + bytes;
      free_.erase(it);
      if (rest) free_[at] = rest;
      used_ += bytes;
      peak_ = std::max(peak_, used_);
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align256(bytes ? bytes : 1);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t peak() const { return peak_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0, peak_ = 0;
};

struct Pending {
  mlmc_request r;
  double t_submit;
};

struct Done {
  mlmc_result res;
  std::vector<double> y;     // Y_l on the coarsest grid
  std::vector<double> map;   // fine activation map (if kept)
};

struct Slot {
  cudaStream_t sf = nullptr, sc = nullptr;
  cudaEvent_t done = nullptr;
  bool busy = false;
  int level = 0, n = 0;
  size_t off = 0, bytes = 0;
  double t_admit = 0.0;
  std::vector<Pending> reqs;
  // pinned host staging: [ids n][seeds n][stim 3n] in, Y rows / info / maps out
  char* h_in = nullptr;
  double* h_y = nullptr;
  mlmc_sample_info* h_info = nullptr;
  double* h_map = nullptr;
};

}  // namespace

struct mlmc_server {
  mlmc_ctx* ctx = nullptr;
  mlmc_server_config cfg{};
  char* arena_base = nullptr;
  Arena arena;
  std::vector<Slot> slots;
  cudaStream_t acc = nullptr;
  std::mutex mu;                        // queue, results, counters, error
  std::condition_variable cv_work, cv_done;
  std::deque<Pending> queue[MLMC_MAX_LEVELS];
  std::deque<Done> done;
  std::mutex ctx_mu;                    // every use of ctx (scheduler vs estimate)
  std::thread th;
  std::atomic<bool> stop{false};
  mlmc_status err = MLMC_OK;
  std::string err_msg;
  int64_t submitted = 0, admitted = 0, completed = 0, batches = 0, max_queue = 0;
  int64_t inflight = 0;
  std::chrono::steady_clock::time_point t0;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

size_t in_bytes(int n) { return align256((size_t)n * 40); }

// Device bytes of a batch of n level-l requests: staging, Y and Y2, and the
// pair workspace (which holds the fine activation maps and the infos).
size_t batch_bytes(const mlmc_ctx* ctx, int level, int n) {
  const size_t n0 = (size_t)ctx->lv[0].nodes;
  return in_bytes(n) + 2 * align256((size_t)n * n0 * 8) + pair_ws(ctx, level, n).total;
}

void set_error(mlmc_server* s, mlmc_status st, const std::string& msg) {
  std::lock_guard<std::mutex> g(s->mu);
  if (s->err == MLMC_OK) {
    s->err = st;
    s->err_msg = msg;
  }
  s->cv_done.notify_all();
}

// Launches the batch held by slot k (requests already moved into it).
mlmc_status launch_batch(mlmc_server* s, Slot& sl) {
  mlmc_ctx* ctx = s->ctx;
  const int n = sl.n, l = sl.level;
  const size_t n0 = (size_t)ctx->lv[0].nodes;
  char* blk = s->arena_base + sl.off;
  uint64_t* hid = (uint64_t*)sl.h_in;
  uint64_t* hseed = hid + n;
  double* hstim = (double*)(hseed + n);
  bool any_stim = false;
  for (int i = 0; i < n; ++i) {
    const mlmc_request& r = sl.reqs[i].r;
    hid[i] = r.sample_id;
    hseed[i] = r.seed;
    const bool own = !isnan(r.stim_c[0]);
    any_stim = any_stim || own;
    for (int d = 0; d < 3; ++d) hstim[3 * i + d] = own ? r.stim_c[d] : ctx->cfg.stim_c[d];
  }
  uint64_t* d_ids = (uint64_t*)blk;
  uint64_t* d_seeds = d_ids + n;
  double* d_stim = (double*)(d_seeds + n);
  double* y = (double*)(blk + in_bytes(n));
  double* y2 = (double*)((char*)y + align256((size_t)n * n0 * 8));
  char* ws = (char*)y2 + align256((size_t)n * n0 * 8);
  PairWs w = pair_ws(ctx, l, n);
  std::lock_guard<std::mutex> g(s->ctx_mu);
  ctx->sync_used = 0;
  CK(ctx, cudaMemcpyAsync(blk, sl.h_in, (size_t)n * 40, cudaMemcpyHostToDevice, sl.sf));
  mlmc_status r = sample_level_into(ctx, l, 0, d_seeds, d_ids, any_stim ? d_stim : nullptr, n, y, y2,
                                    nullptr, nullptr, nullptr, ws, sl.sf, sl.sc);
  if (r != MLMC_OK) return r;
  if ((r = order_after(ctx, sl.sf, s->acc)) != MLMC_OK) return r;
  if ((r = mlmc_accumulate(ctx, l, y, y2, n, s->acc)) != MLMC_OK) return r;
  CK(ctx, cudaMemcpyAsync(sl.h_y, y, (size_t)n * n0 * 8, cudaMemcpyDeviceToHost, s->acc));
  CK(ctx, cudaMemcpyAsync(sl.h_info, ws + w.info, sizeof(mlmc_sample_info) * (size_t)(l > 0 ? 2 * n : n),
                          cudaMemcpyDeviceToHost, s->acc));
  if (s->cfg.keep_maps)
    CK(ctx, cudaMemcpyAsync(sl.h_map, ws + w.tf, (size_t)n * ctx->lv[l].nodes * 8,
                            cudaMemcpyDeviceToHost, s->acc));
  CK(ctx, cudaEventRecord(sl.done, s->acc));
  return MLMC_OK;
}

// Moves finished batches' results to the done queue; true if any finished.
bool harvest(mlmc_server* s) {
  bool any = false;
  for (Slot& sl : s->slots) {
    if (!sl.busy) continue;
    cudaError_t e = cudaEventQuery(sl.done);
    if (e == cudaErrorNotReady) continue;
    if (e != cudaSuccess) {
      set_error(s, MLMC_ERR_CUDA, std::string("server batch: ") + cudaGetErrorString(e));
      sl.busy = false;
      continue;
    }
    const double t = s->now();
    const int n = sl.n, l = sl.level;
    const size_t n0 = (size_t)s->ctx->lv[0].nodes, nl = (size_t)s->ctx->lv[l].nodes;
    std::vector<Done> out(n);
    for (int i = 0; i < n; ++i) {
      mlmc_result& r = out[i].res;
      const mlmc_sample_info& fi = sl.h_info[i];
      r.tag = sl.reqs[i].r.tag;
      r.level = l;
      r.status = fi.status;
      r.newton_iters = fi.newton_iters;
      r.cg_iters = fi.cg_iters;
      if (l > 0) {
        const mlmc_sample_info& ci = sl.h_info[n + i];
        if (r.status == MLMC_OK) r.status = ci.status;
        r.newton_iters += ci.newton_iters;
        r.cg_iters += ci.cg_iters;
      }
      r.t_submit = sl.reqs[i].t_submit;
      r.t_admit = sl.t_admit;
      r.t_done = t;
      out[i].y.assign(sl.h_y + i * n0, sl.h_y + (i + 1) * n0);
      if (s->cfg.keep_maps) out[i].map.assign(sl.h_map + i * nl, sl.h_map + (i + 1) * nl);
    }
    {
      std::lock_guard<std::mutex> g(s->mu);
      for (Done& d : out) s->done.push_back(std::move(d));
      s->completed += n;
      s->inflight -= n;
    }
    s->arena.release(sl.off, sl.bytes);
    sl.busy = false;
    sl.reqs.clear();
    any = true;
  }
  if (any) s->cv_done.notify_all();
  return any;
}

// Forms and launches at most one batch; true if one was launched.  Levels
// are tried oldest head request first; a partial batch is held back for up
// to max_wait_s while the device is busy anyway, so that batches fill.
bool admit(mlmc_server* s) {
  Slot* free_slot = nullptr;
  bool gpu_busy = false;
  for (Slot& sl : s->slots) {
    if (!sl.busy && !free_slot) free_slot = &sl;
    gpu_busy = gpu_busy || sl.busy;
  }
  if (!free_slot) return false;
  std::unique_lock<std::mutex> g(s->mu);
  if (s->err != MLMC_OK) return false;
  const int L = s->ctx->cfg.n_levels;
  int order[MLMC_MAX_LEVELS], k = 0;
  for (int l = 0; l < L; ++l)
    if (!s->queue[l].empty()) order[k++] = l;
  std::sort(order, order + k, [&](int a, int b) {
    return s->queue[a].front().t_submit < s->queue[b].front().t_submit;
  });
  const double t = s->now();
  int lev = -1, n = 0;
  size_t off = 0, bytes = 0;
  for (int q = 0; q < k && lev < 0; ++q) {
    const int l = order[q];
    int m = (int)std::min<size_t>(s->queue[l].size(), (size_t)s->cfg.max_batch);
    if (m < s->cfg.max_batch && gpu_busy && t - s->queue[l].front().t_submit < s->cfg.max_wait_s)
      continue;
    while (m > 0) {   // memory-based admission: halve until the batch fits
      bytes = batch_bytes(s->ctx, l, m);
      if (s->arena.alloc(bytes, &off)) break;
      m /= 2;
    }
    if (m > 0) { lev = l; n = m; }
  }
  if (lev < 0) return false;
  Slot& sl = *free_slot;
  sl.reqs.assign(s->queue[lev].begin(), s->queue[lev].begin() + n);
  s->queue[lev].erase(s->queue[lev].begin(), s->queue[lev].begin() + n);
  s->admitted += n;
  s->inflight += n;
  s->batches += 1;
  g.unlock();
  sl.level = lev;
  sl.n = n;
  sl.off = off;
  sl.bytes = bytes;
  sl.t_admit = t;
  sl.busy = true;
  mlmc_status r = launch_batch(s, sl);
  if (r != MLMC_OK) {
    std::string msg;
    {
      std::lock_guard<std::mutex> cg(s->ctx_mu);
      msg = s->ctx->err;
    }
    // nothing of the batch is in flight that its slot would still wait on:
    // wait for what was enqueued, then give the slot and its memory back
    cudaStreamSynchronize(sl.sf);
    cudaStreamSynchronize(sl.sc);
    cudaStreamSynchronize(s->acc);
    s->arena.release(sl.off, sl.bytes);
    sl.busy = false;
    sl.reqs.clear();
    {
      std::lock_guard<std::mutex> eg(s->mu);
      s->inflight -= n;
    }
    set_error(s, r, "server launch: " + msg);
  }
  return true;
}

void scheduler(mlmc_server* s) {
  cudaSetDevice(s->ctx->device);
  while (true) {
    bool worked = harvest(s);
    bool any_busy = false;
    for (Slot& sl : s->slots) any_busy = any_busy || sl.busy;
    if (s->stop.load() && !any_busy) break;
    if (!s->stop.load()) worked = admit(s) || worked;
    if (!worked) {
      std::unique_lock<std::mutex> g(s->mu);
      s->cv_work.wait_for(g, std::chrono::microseconds(any_busy ? 50 : 2000));
    }
  }
}

void destroy_server(mlmc_server* s) {
  for (Slot& sl : s->slots) {
    if (sl.sf) cudaStreamDestroy(sl.sf);
    if (sl.sc) cudaStreamDestroy(sl.sc);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.h_in) cudaFreeHost(sl.h_in);
    if (sl.h_y) cudaFreeHost(sl.h_y);
    if (sl.h_info) cudaFreeHost(sl.h_info);
    if (sl.h_map) cudaFreeHost(sl.h_map);
  }
  if (s->acc) cudaStreamDestroy(s->acc);
  if (s->arena_base) cudaFree(s->arena_base);
  delete s;
}

}  // namespace

extern "C" mlmc_status mlmc_server_create(mlmc_ctx* ctx, const mlmc_server_config* cfg,
                                          mlmc_server** out) {
  if (!ctx) return MLMC_ERR_ARG;
  if (!out || !cfg) return fail(ctx, MLMC_ERR_ARG, "mlmc_server_create: NULL argument");
  *out = nullptr;
  const mlmc_server_config& c = *cfg;
  if (c.max_batch < 1 || c.max_batch > 65535 || c.slots < 1 || c.slots > 16 || !(c.max_wait_s >= 0.0))
    return fail(ctx, MLMC_ERR_ARG, "mlmc_server_create: max_batch 1..65535, slots 1..16, max_wait_s >= 0");
  const int L = ctx->cfg.n_levels;
  size_t need1 = 0;
  for (int l = 0; l < L; ++l) need1 = std::max(need1, batch_bytes(ctx, l, 1));
  if (c.mem_budget < need1) {
    char b[160];
    snprintf(b, sizeof b, "mlmc_server_create: mem_budget %zu bytes holds no request of the finest level (%zu bytes)",
             c.mem_budget, need1);
    return fail(ctx, MLMC_ERR_WORKSPACE, b);
  }
  mlmc_server* s = new mlmc_server();
  s->ctx = ctx;
  s->cfg = c;
  s->t0 = std::chrono::steady_clock::now();
  auto bail = [&](cudaError_t e, const char* where) {
    destroy_server(s);
    return cuda_fail(ctx, e, where);
  };
  cudaError_t e;
  if ((e = cudaMalloc(&s->arena_base, c.mem_budget)) != cudaSuccess) return bail(e, "cudaMalloc(arena)");
  s->arena.init(c.mem_budget);
  if ((e = cudaStreamCreateWithFlags(&s->acc, cudaStreamNonBlocking)) != cudaSuccess) return bail(e, "cudaStreamCreate");
  const size_t n0 = (size_t)ctx->lv[0].nodes, nL = (size_t)ctx->lv[L - 1].nodes;
  const size_t nb = (size_t)c.max_batch;
  s->slots.resize(c.slots);
  for (Slot& sl : s->slots) {
    if ((e = cudaStreamCreateWithFlags(&sl.sf, cudaStreamNonBlocking)) != cudaSuccess) return bail(e, "cudaStreamCreate");
    if ((e = cudaStreamCreateWithFlags(&sl.sc, cudaStreamNonBlocking)) != cudaSuccess) return bail(e, "cudaStreamCreate");
    if ((e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming)) != cudaSuccess) return bail(e, "cudaEventCreate");
    if ((e = cudaMallocHost(&sl.h_in, nb * 40)) != cudaSuccess) return bail(e, "cudaMallocHost");
    if ((e = cudaMallocHost(&sl.h_y, nb * n0 * 8)) != cudaSuccess) return bail(e, "cudaMallocHost");
    if ((e = cudaMallocHost(&sl.h_info, nb * 2 * sizeof(mlmc_sample_info))) != cudaSuccess) return bail(e, "cudaMallocHost");
    if (c.keep_maps && (e = cudaMallocHost(&sl.h_map, nb * nL * 8)) != cudaSuccess) return bail(e, "cudaMallocHost");
  }
  s->th = std::thread(scheduler, s);
  *out = s;
  return MLMC_OK;
}

extern "C" mlmc_status mlmc_server_submit(mlmc_server* s, const mlmc_request* reqs, int n) {
  if (!s || n < 0 || (n > 0 && !reqs)) return MLMC_ERR_ARG;
  const int L = s->ctx->cfg.n_levels;
  for (int i = 0; i < n; ++i)
    if (reqs[i].level < 0 || reqs[i].level >= L) return MLMC_ERR_ARG;
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->err != MLMC_OK) return s->err;
    const double t = s->now();
    int64_t q = 0;
    for (int i = 0; i < n; ++i) s->queue[reqs[i].level].push_back(Pending{reqs[i], t});
    for (int l = 0; l < L; ++l) q += (int64_t)s->queue[l].size();
    s->submitted += n;
    s->max_queue = std::max(s->max_queue, q);
  }
  s->cv_work.notify_one();
  return MLMC_OK;
}

extern "C" mlmc_status mlmc_server_poll(mlmc_server* s, mlmc_result* out, int max, int* count,
                                        double* y, double* maps, int64_t map_stride,
                                        double timeout_s) {
  if (!s || !count || max < 0 || (max > 0 && !out)) return MLMC_ERR_ARG;
  *count = 0;
  const size_t n0 = (size_t)s->ctx->lv[0].nodes;
  std::unique_lock<std::mutex> g(s->mu);
  if (s->done.empty() && timeout_s > 0.0 && s->err == MLMC_OK)
    s->cv_done.wait_for(g, std::chrono::duration<double>(timeout_s),
                        [&] { return !s->done.empty() || s->err != MLMC_OK; });
  int k = 0;
  while (k < max && !s->done.empty()) {
    Done& d = s->done.front();
    out[k] = d.res;
    if (y) memcpy(y + (size_t)k * n0, d.y.data(), n0 * 8);
    if (maps && !d.map.empty())
      memcpy(maps + (size_t)k * (size_t)map_stride, d.map.data(),
             std::min(d.map.size(), (size_t)map_stride) * 8);
    s->done.pop_front();
    ++k;
  }
  *count = k;
  return k == 0 && s->err != MLMC_OK ? s->err : MLMC_OK;
}

extern "C" mlmc_status mlmc_server_drain(mlmc_server* s, double timeout_s) {
  if (!s) return MLMC_ERR_ARG;
  const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  std::unique_lock<std::mutex> g(s->mu);
  while (s->err == MLMC_OK && s->completed < s->submitted) {
    if (s->cv_done.wait_until(g, until) == std::cv_status::timeout && s->completed < s->submitted)
      return MLMC_ERR_TIMEOUT;
  }
  return s->err;
}

extern "C" mlmc_status mlmc_server_stats(mlmc_server* s, int64_t* stats) {
  if (!s || !stats) return MLMC_ERR_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  int64_t q = 0;
  for (int l = 0; l < s->ctx->cfg.n_levels; ++l) q += (int64_t)s->queue[l].size();
  stats[0] = s->submitted;
  stats[1] = q;
  stats[2] = s->inflight;
  stats[3] = s->completed;
  stats[4] = s->batches;
  stats[5] = s->max_queue;
  stats[6] = (int64_t)s->arena.peak();
  stats[7] = (int64_t)s->err;
  return MLMC_OK;
}

extern "C" mlmc_status mlmc_server_clock(mlmc_server* s, double* now) {
  if (!s || !now) return MLMC_ERR_ARG;
  *now = s->now();
  return MLMC_OK;
}

extern "C" mlmc_status mlmc_server_estimate(mlmc_server* s, double* mean, double* var, double* V_l,
                                            int64_t* N_l, double* rmse, double* bias) {
  if (!s) return MLMC_ERR_ARG;
  std::lock_guard<std::mutex> g(s->ctx_mu);
  return estimate_impl(s->ctx, mean, var, nullptr, nullptr, V_l, N_l, rmse, bias, s->acc);
}

extern "C" const char* mlmc_server_error(mlmc_server* s) {
  if (!s) return "NULL server";
  std::lock_guard<std::mutex> g(s->mu);
  return s->err_msg.c_str();
}

extern "C" void mlmc_server_destroy(mlmc_server* s) {
  if (!s) return;
  s->stop.store(true);
  s->cv_work.notify_all();
  if (s->th.joinable()) s->th.join();
  destroy_server(s);
}
