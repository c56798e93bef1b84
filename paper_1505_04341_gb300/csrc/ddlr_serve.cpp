// ddlr_serve.cpp -- solve service on one GPU: resident preconditioners,
// continuous batching, memory-based admission.
//
// Every registered model (a matrix with its DDLR setup) keeps its factors and
// low-rank data resident and owns a worker thread with its own CUDA stream.
// The worker runs a block PCG whose columns are slots: between chunks of a few
// iterations it retires the columns that have converged (their results go
// back to the waiting callers at once) and admits queued requests into the
// free slots, so a request never waits for a whole batch to finish.  When
// requests queue up and every slot is busy, the block is widened (up to
// max_batch columns) without disturbing the running columns.  At most
// max_concurrent models have a block on the GPU at once, so work of different
// models overlaps on the device; while another model waits for a place, a
// block admits nothing more and gives its place back once it drains.  A block is opened or widened only if its
// workspace fits in the device memory the server may use; otherwise it stays
// narrower, down to one column.  A column's iterates do not depend on when it
// was admitted or what shares its block, so a request's result is the same
// alone and in the mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "ddlr.h"
#include "ddlr_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  long long id = 0;
  int model = 0;
  std::vector<double> b, x;
  Clock::time_point t_submit, t_done;
  ddlr_solve_info info{};
  int batch = 0;
  bool done = false;
};

struct Model {
  ddlr_handle h = nullptr;
  cudaStream_t stream = nullptr;   // the model's own non-blocking stream
  int n = 0;
  long long nnz = 0;
  std::deque<std::shared_ptr<Request>> queue;
  std::thread worker;
  // the open block (worker thread; under the server mutex where shared)
  int width = 0;                                  // columns of the open block (0: none)
  int active = 0;                                 // occupied slots
  std::vector<std::shared_ptr<Request>> slot;     // request of each slot (null: free)
  long long reserved = 0;                         // workspace bytes counted for the block
};

}  // namespace

struct ddlr_server_ctx {
  ddlr_server_options opt{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_slot, cv_done;
  std::vector<std::unique_ptr<Model>> models;
  std::map<long long, std::shared_ptr<Request>> reqs;
  long long next_id = 1;
  int inflight = 0;
  int waiting = 0;          // models waiting for a place on the GPU
  bool stop = false;
  long long completed = 0;
  int max_batch_seen = 0, max_inflight_seen = 0;
  long long admitted_running = 0;   // admissions into a block with other requests running
  long long reserved = 0;   // workspace bytes admitted and not yet released
  std::string err;
};

namespace {

// device bytes of a block of R right-hand sides (FP64 PCG blocks, apply
// workspaces, FP32 copies), a conservative estimate
long long batch_bytes(int n, int R) { return (long long)n * R * (14 * 8 + 7 * 4) + (1 << 20); }

int pow2_at_least(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// widest block of at most `want` columns whose workspace fits the memory the
// server may still use (at least one column); S->mu held
int fit_width(ddlr_server_ctx *S, Model *M, int want) {
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  const long long budget = (long long)(S->opt.memory_fraction * double(fr)) - S->reserved + M->reserved;
  int R = std::max(1, std::min(want, S->opt.max_batch));
  while (R > 1 && batch_bytes(M->n, R) > budget) R /= 2;
  return R;
}

void fail_all(ddlr_server_ctx *S, Model *M, ddlr_status st) {
  const Clock::time_point t = Clock::now();
  for (auto &rq : M->slot) {
    if (!rq) continue;
    rq->info = ddlr_solve_info{0, 0.0, int(st)};
    rq->x.assign(size_t(M->n), 0.0);
    rq->t_done = t;
    rq->batch = M->width;
    rq->done = true;
    S->completed++;
    rq.reset();
  }
  M->active = 0;
}

void worker_loop(ddlr_server_ctx *S, Model *M) {
  cudaSetDevice(S->device);
  constexpr int kItersPerPoll = 4;
  std::vector<int> done;
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    S->cv_work.wait(lk, [&] { return S->stop || !M->queue.empty() || M->active > 0; });
    if (S->stop) break;
    int open_w = 0, resize_w = 0;
    std::vector<int> map;
    if (M->width == 0) {
      // a new block: needs one of the max_concurrent places on the GPU
      S->waiting++;
      S->cv_slot.wait(lk, [&] { return S->stop || S->inflight < S->opt.max_concurrent; });
      S->waiting--;
      if (S->stop) break;
      if (M->queue.empty()) continue;
      open_w = fit_width(S, M, pow2_at_least(int(M->queue.size())));
      S->inflight++;
      S->max_inflight_seen = std::max(S->max_inflight_seen, S->inflight);
      const long long bytes = batch_bytes(M->n, open_w);
      S->reserved += bytes - M->reserved;
      M->reserved = bytes;
      M->width = open_w;
      M->slot.assign(size_t(open_w), nullptr);
    } else if (!M->queue.empty() && M->active == M->width && M->width < S->opt.max_batch && S->waiting == 0) {
      // every slot busy and requests waiting: widen the block (the running
      // columns keep their slots)
      const int w = fit_width(S, M, pow2_at_least(M->active + int(M->queue.size())));
      if (w > M->width) {
        resize_w = w;
        map.assign(size_t(w), -1);
        for (int q = 0; q < M->width; q++) map[q] = q;
        M->slot.resize(size_t(w));
      }
    } else if ((M->queue.empty() || S->waiting > 0) && M->active > 0 && M->active * 4 <= M->width) {
      // few columns left in a wide block: narrow it to them (an iteration
      // costs in proportion to the width)
      const int w = pow2_at_least(M->active);
      resize_w = w;
      map.assign(size_t(w), -1);
      std::vector<std::shared_ptr<Request>> ns(static_cast<size_t>(w), nullptr);
      int j = 0;
      for (int q = 0; q < M->width; q++)
        if (M->slot[q]) { map[j] = q; ns[j] = M->slot[q]; j++; }
      M->slot.swap(ns);
    }
    if (resize_w) {
      const long long bytes = batch_bytes(M->n, resize_w);
      S->reserved += bytes - M->reserved;
      M->reserved = bytes;
      M->width = resize_w;
    }
    // admission into the free slots, first come first served; while other
    // models wait for a place on the GPU, an open block admits nothing more
    // and drains, so the places go round
    const int running = M->active;
    const bool drain = open_w == 0 && S->waiting > 0 && running > 0;
    std::vector<int> adm_slot;
    std::vector<const double *> adm_b;
    for (int q = 0; q < M->width && !M->queue.empty() && !drain; q++) {
      if (M->slot[q]) continue;
      M->slot[q] = M->queue.front();
      M->queue.pop_front();
      adm_slot.push_back(q);
      adm_b.push_back(M->slot[q]->b.data());
      M->active++;
    }
    S->max_batch_seen = std::max(S->max_batch_seen, M->active);
    if (running > 0) S->admitted_running += (long long)adm_slot.size();
    lk.unlock();
    ddlr_status st = DDLR_OK;
    if (open_w) st = slots_open(M->h, open_w, S->opt.tol, S->opt.maxit);
    if (st == DDLR_OK && resize_w) st = slots_resize(M->h, resize_w, map.data());
    if (st == DDLR_OK && !adm_slot.empty())
      st = slots_admit(M->h, int(adm_slot.size()), adm_slot.data(), adm_b.data());
    done.assign(size_t(M->width), 0);
    if (st == DDLR_OK) st = slots_run(M->h, kItersPerPoll, done.data());
    // results of the finished columns, copied out before taking the lock
    std::vector<std::pair<int, ddlr_solve_info>> fin;
    std::vector<std::vector<double>> xs;
    if (st == DDLR_OK) {
      for (int q = 0; q < M->width; q++) {
        if (!done[q] || !M->slot[q]) continue;
        ddlr_solve_info inf{};
        std::vector<double> x(size_t(M->n));
        st = slots_take(M->h, q, x.data(), &inf);
        if (st != DDLR_OK) break;
        fin.emplace_back(q, inf);
        xs.push_back(std::move(x));
      }
    }
    const Clock::time_point t = Clock::now();
    lk.lock();
    if (st != DDLR_OK) {
      S->err = ddlr_last_error(M->h);
      fail_all(S, M, st);
    } else {
      for (size_t i = 0; i < fin.size(); i++) {
        std::shared_ptr<Request> &rq = M->slot[fin[i].first];
        rq->x = std::move(xs[i]);
        rq->info = fin[i].second;
        rq->t_done = t;
        rq->batch = M->width;
        rq->done = true;
        S->completed++;
        rq.reset();
        M->active--;
      }
    }
    if (M->active == 0 && (M->queue.empty() || st != DDLR_OK || S->waiting > 0)) {
      // the block drains (or failed, or others wait): give its place back
      S->inflight--;
      S->reserved -= M->reserved;
      M->reserved = 0;
      M->width = 0;
      S->cv_slot.notify_all();
    }
    if (!fin.empty() || st != DDLR_OK) S->cv_done.notify_all();
  }
}

}  // namespace

extern "C" {

const char *ddlr_server_last_error(ddlr_server S) { return S ? S->err.c_str() : ""; }

ddlr_status ddlr_server_options_default(ddlr_server_options *o) {
  if (!o) return DDLR_ERR_INVALID;
  o->max_concurrent = 8;
  o->max_batch = 16;
  o->tol = 1e-8;
  o->maxit = 500;
  o->memory_fraction = 0.9;
  return DDLR_OK;
}

ddlr_status ddlr_server_create(const ddlr_server_options *opt, ddlr_server *out) {
  if (!out) return DDLR_ERR_INVALID;
  *out = nullptr;
  ddlr_server_ctx *S = new (std::nothrow) ddlr_server_ctx();
  if (!S) return DDLR_ERR_OOM;
  if (opt) S->opt = *opt; else ddlr_server_options_default(&S->opt);
  if (S->opt.max_concurrent < 1 || S->opt.max_batch < 1 || S->opt.max_batch > 64 ||
      !(S->opt.tol > 0) || !(S->opt.memory_fraction > 0) || S->opt.memory_fraction > 1) {
    delete S;
    return DDLR_ERR_INVALID;
  }
  if (S->opt.maxit <= 0) S->opt.maxit = 500;
  cudaGetDevice(&S->device);
  *out = S;
  return DDLR_OK;
}

ddlr_status ddlr_server_add_model(ddlr_server S, int n, const int *rowptr, const int *colind,
                                  const double *val, const int *part, int p,
                                  const ddlr_options *opt, int *model) {
  if (!S || !model) return DDLR_ERR_INVALID;
  // admission of the resident setup: a conservative footprint estimate
  const long long nnz = (n > 0 && rowptr) ? rowptr[n] : 0;
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  const long long need = (long long)n * 400 + nnz * 60;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (need > (long long)(S->opt.memory_fraction * double(fr)) - S->reserved) {
      S->err = "not enough device memory for the model";
      return DDLR_ERR_OOM;
    }
  }
  ddlr_handle h = nullptr;
  cudaStream_t stream = nullptr;
  if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
    S->err = "cudaStreamCreate failed";
    return DDLR_ERR_CUDA;
  }
  const ddlr_status st = ddlr_setup(n, rowptr, colind, val, part, p, opt, stream, &h);
  if (st != DDLR_OK) {
    S->err = ddlr_last_error(nullptr);
    cudaStreamDestroy(stream);
    return st;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  auto M = std::make_unique<Model>();
  M->h = h;
  M->stream = stream;
  M->n = n;
  M->nnz = nnz;
  const int mi = int(S->models.size());
  Model *mp = M.get();
  S->models.push_back(std::move(M));
  mp->worker = std::thread(worker_loop, S, mp);
  *model = mi;
  return DDLR_OK;
}

ddlr_status ddlr_server_submit(ddlr_server S, int model, const double *b, long long *request) {
  if (!S || !b || !request) return DDLR_ERR_INVALID;
  auto rq = std::make_shared<Request>();
  std::lock_guard<std::mutex> lk(S->mu);
  if (model < 0 || model >= int(S->models.size())) return DDLR_ERR_INVALID;
  Model *M = S->models[model].get();
  rq->id = S->next_id++;
  rq->model = model;
  rq->b.assign(b, b + M->n);
  rq->t_submit = Clock::now();
  S->reqs[rq->id] = rq;
  M->queue.push_back(rq);
  *request = rq->id;
  S->cv_work.notify_all();
  return DDLR_OK;
}

ddlr_status ddlr_server_wait(ddlr_server S, long long request, double timeout_s, double *x,
                             ddlr_solve_info *info, double *latency_s, int *batch) {
  if (!S) return DDLR_ERR_INVALID;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(request);
  if (it == S->reqs.end()) return DDLR_ERR_INVALID;
  std::shared_ptr<Request> rq = it->second;
  const auto pred = [&] { return rq->done; };
  if (timeout_s > 0) {
    if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) return DDLR_ERR_TIMEOUT;
  } else {
    S->cv_done.wait(lk, pred);
  }
  if (x) std::memcpy(x, rq->x.data(), sizeof(double) * rq->x.size());
  if (info) *info = rq->info;
  if (latency_s) *latency_s = std::chrono::duration<double>(rq->t_done - rq->t_submit).count();
  if (batch) *batch = rq->batch;
  S->reqs.erase(it);
  return rq->info.status == DDLR_OK ? DDLR_OK : (ddlr_status)rq->info.status;
}

ddlr_status ddlr_server_stats(ddlr_server S, long long *completed, int *max_batch_seen,
                              int *max_inflight_seen, int *nmodels, long long *admitted_running) {
  if (!S) return DDLR_ERR_INVALID;
  std::lock_guard<std::mutex> lk(S->mu);
  if (completed) *completed = S->completed;
  if (max_batch_seen) *max_batch_seen = S->max_batch_seen;
  if (max_inflight_seen) *max_inflight_seen = S->max_inflight_seen;
  if (admitted_running) *admitted_running = S->admitted_running;
  if (nmodels) *nmodels = int(S->models.size());
  return DDLR_OK;
}

ddlr_status ddlr_server_destroy(ddlr_server S) {
  if (!S) return DDLR_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  S->cv_slot.notify_all();
  for (auto &M : S->models)
    if (M->worker.joinable()) M->worker.join();
  for (auto &M : S->models) {
    ddlr_destroy(M->h);
    if (M->stream) cudaStreamDestroy(M->stream);
  }
  delete S;
  return DDLR_OK;
}

}  // extern "C"
