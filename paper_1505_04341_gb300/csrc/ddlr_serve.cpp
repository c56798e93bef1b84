// ddlr_serve.cpp -- solve service on one GPU: resident preconditioners,
// continuous batching, memory-based admission.
//
// Every registered model (a matrix with its DDLR setup) keeps its factors and
// low-rank data resident and owns a worker thread with its own CUDA streams.
// A worker takes every request of its model that is waiting when it becomes
// free (up to max_batch) and solves them together in one batched PCG; requests
// that arrive meanwhile wait for the next batch.  At most max_concurrent
// batches are on the GPU at once across models, so work of different models
// overlaps on the device.  A batch is admitted only if its workspace fits in
// the device memory the server may use; otherwise it is narrowed, down to one
// right-hand side.  The batched solve gives a column the same bits whatever
// else shares its batch, so a request's result does not depend on the mix.
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
  bool stop = false;
  long long completed = 0;
  int max_batch_seen = 0, max_inflight_seen = 0;
  long long reserved = 0;   // workspace bytes admitted and not yet released
  std::string err;
};

namespace {

// device bytes of a batch of R right-hand sides (FP64 PCG blocks, apply
// workspaces, FP32 copies), a conservative estimate
long long batch_bytes(int n, int R) { return (long long)n * R * (14 * 8 + 7 * 4) + (1 << 20); }

void worker_loop(ddlr_server_ctx *S, Model *M, int mi) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    S->cv_work.wait(lk, [&] { return S->stop || !M->queue.empty(); });
    if (S->stop) break;
    S->cv_slot.wait(lk, [&] { return S->stop || S->inflight < S->opt.max_concurrent; });
    if (S->stop) break;
    // admission: widest batch whose workspace fits the memory budget
    int R = std::min<int>((int)M->queue.size(), S->opt.max_batch);
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    const long long budget = (long long)(S->opt.memory_fraction * double(fr)) - S->reserved;
    while (R > 1 && batch_bytes(M->n, R) > budget) R /= 2;
    std::vector<std::shared_ptr<Request>> batch(M->queue.begin(), M->queue.begin() + R);
    M->queue.erase(M->queue.begin(), M->queue.begin() + R);
    const long long bytes = batch_bytes(M->n, R);
    S->reserved += bytes;
    S->inflight++;
    S->max_inflight_seen = std::max(S->max_inflight_seen, S->inflight);
    S->max_batch_seen = std::max(S->max_batch_seen, R);
    lk.unlock();
    const int n = M->n;
    std::vector<double> B(size_t(n) * R), X(size_t(n) * R);
    for (int q = 0; q < R; q++) std::memcpy(B.data() + size_t(q) * n, batch[q]->b.data(), sizeof(double) * n);
    std::vector<ddlr_solve_info> info(R);
    const ddlr_status st = pcg_batched_host(M->h, B.data(), X.data(), R, S->opt.tol, S->opt.maxit, info.data());
    const Clock::time_point t = Clock::now();
    lk.lock();
    S->reserved -= bytes;
    S->inflight--;
    for (int q = 0; q < R; q++) {
      Request &rq = *batch[q];
      rq.x.assign(X.begin() + size_t(q) * n, X.begin() + size_t(q + 1) * n);
      rq.info = info[q];
      if (st != DDLR_OK && st != DDLR_ERR_NOCONV && st != DDLR_ERR_NAN) rq.info.status = st;
      rq.t_done = t;
      rq.batch = R;
      rq.done = true;
      S->completed++;
    }
    (void)mi;
    S->cv_slot.notify_all();
    S->cv_done.notify_all();
  }
}

}  // namespace

extern "C" {

const char *ddlr_server_last_error(ddlr_server S) { return S ? S->err.c_str() : ""; }

ddlr_status ddlr_server_options_default(ddlr_server_options *o) {
  if (!o) return DDLR_ERR_INVALID;
  o->max_concurrent = 4;
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
  mp->worker = std::thread(worker_loop, S, mp, mi);
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
                              int *max_inflight_seen, int *nmodels) {
  if (!S) return DDLR_ERR_INVALID;
  std::lock_guard<std::mutex> lk(S->mu);
  if (completed) *completed = S->completed;
  if (max_batch_seen) *max_batch_seen = S->max_batch_seen;
  if (max_inflight_seen) *max_inflight_seen = S->max_inflight_seen;
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
