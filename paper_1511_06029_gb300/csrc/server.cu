// Solve server: continuous admission of qtt_solve requests onto one GPU.
//
// Requests (an operator pair K, P and nrhs host right-hand sides) enter a
// FIFO queue when submitted.  A request is admitted as soon as a slot is free
// and its device-memory estimate fits in what the budget has left (strict
// FIFO: the head waits rather than being overtaken, so large requests are
// not starved).  Each slot is a worker thread with its own CUDA stream; an
// admitted request's upload, solve (GMRES, refinement or direct, with its P
// in the server's precond_compute) and download run on that stream, so the
// kernels of all admitted requests overlap on the device while new requests
// keep arriving.  Finishing frees the slot and the memory, and the next
// requests are admitted at once.  Each request's arithmetic depends only on
// the request (deterministic reductions, private buffers), so its result is
// bitwise the same alone or in any mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "qtt_internal.h"

namespace qtt {
namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  int64_t id;
  const qtt_op *K, *P;
  const double *f_host;
  double *x_host;
  int64_t nrhs;
  size_t need;
  double t_submit = 0, t_admit = 0, t_finish = 0;
  bool done = false;
  qtt_status status = QTT_OK;
  std::string message;  // qtt_last_error() of the worker when status != QTT_OK
  std::vector<qtt_solve_info> info;
};

}  // namespace
}  // namespace qtt

struct qtt_server {
  qtt_solve_params prm;
  int slots = 1;
  size_t budget = 0, in_use = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<qtt::Request *> pending;     // submitted, not admitted (FIFO)
  std::deque<qtt::Request *> admitted;    // admitted, waiting for a worker
  std::map<int64_t, qtt::Request *> all;  // every request until retired
  std::vector<std::thread> workers;
  int running = 0;
  int64_t next_id = 0;
  bool stop = false;
  int device = 0;
  size_t peak_in_use = 0;
  int peak_running = 0;
};

namespace qtt {
namespace {

// Device bytes a request may hold at once: f and x, the solver's vectors,
// and the scratch of the two applies (the pool may keep both).
size_t request_bytes(const qtt_op *K, const qtt_op *P, int64_t nrhs, const qtt_solve_params &p) {
  const qtt_op *A = K ? K : P;
  const size_t N = (size_t)1 << A->d, R = (size_t)nrhs;
  size_t b = 2 * N * R * 8;  // f, x
  if (p.kind == QTT_SOLVE_GMRES) b += (size_t)(p.restart + 3 + (P ? p.restart : 0)) * N * R * 8;
  else b += 4 * N * R * 8;
  if (p.inner_iters > 0) b += 2 * N * R * 8;
  if (K) b += 2 * (size_t)K->rmax_inner * N * R * 8;
  if (K && p.inner_iters > 0) b += 2 * (size_t)K->rmax_inner * N * R * 4;
  if (P) {
    const size_t e = p.precond_compute == QTT_F64 ? 8 : (p.precond_compute == QTT_BF16 ? 2 : 4);
    b += 2 * (size_t)P->rmax_inner * N * R * e;
  }
  return b + (64u << 20);
}

// Move admissible requests from `pending` to `admitted` (caller holds mu).
void admit_locked(qtt_server *S) {
  while (!S->pending.empty()) {
    Request *r = S->pending.front();
    const int busy = S->running + (int)S->admitted.size();
    if (busy >= S->slots || S->in_use + r->need > S->budget) break;
    S->pending.pop_front();
    S->in_use += r->need;
    S->peak_in_use = std::max(S->peak_in_use, S->in_use);
    r->t_admit = now_s();
    S->admitted.push_back(r);
  }
  S->cv_work.notify_all();
}

void worker_main(qtt_server *S) {
  cudaSetDevice(S->device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (;;) {
    Request *r = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] { return S->stop || !S->admitted.empty(); });
      if (S->admitted.empty()) break;  // stop requested and nothing left
      r = S->admitted.front();
      S->admitted.pop_front();
      ++S->running;
      S->peak_running = std::max(S->peak_running, S->running);
    }
    const qtt_op *A = r->K ? r->K : r->P;
    const int64_t N = (int64_t)1 << A->d;
    const size_t bytes = (size_t)N * r->nrhs * sizeof(double);
    qtt_status s = QTT_OK;
    void *f = nullptr, *x = nullptr;
    s = scratch_alloc(&f, bytes, st);
    if (s == QTT_OK) s = scratch_alloc(&x, bytes, st);
    if (s == QTT_OK) {
      cudaError_t e = cudaMemcpyAsync(f, r->f_host, bytes, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) s = cuda_fail(e, "server: upload");
    }
    if (s == QTT_OK) {
      s = qtt_solve(r->K, r->P, static_cast<double *>(f), static_cast<double *>(x), r->nrhs, N,
                    &S->prm, r->info.data(), st);
      if (s == QTT_ERR_NOT_CONVERGED) s = QTT_OK;  // reported per right-hand side in info
    }
    if (s == QTT_OK) {
      cudaError_t e = cudaMemcpyAsync(r->x_host, x, bytes, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) s = cuda_fail(e, "server: download");
    }
    scratch_free(f, st);
    scratch_free(x, st);
    cudaStreamSynchronize(st);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      r->status = s;
      if (s != QTT_OK) r->message = qtt_last_error();
      r->t_finish = now_s();
      r->done = true;
      --S->running;
      S->in_use -= r->need;
      admit_locked(S);
    }
    S->cv_done.notify_all();
  }
  cudaStreamDestroy(st);
}

}  // namespace
}  // namespace qtt

using namespace qtt;

extern "C" {

qtt_status qtt_server_create(qtt_server **out, int slots, size_t mem_budget,
                             const qtt_solve_params *prm) {
  if (!out || !prm) return fail(QTT_ERR_INVALID_ARG, "qtt_server_create: NULL argument");
  *out = nullptr;
  if (slots < 1 || slots > 256) return fail(QTT_ERR_INVALID_ARG, "qtt_server_create: slots");
  if (prm->kind != QTT_SOLVE_DIRECT && prm->kind != QTT_SOLVE_GMRES &&
      prm->kind != QTT_SOLVE_REFINE)
    return fail(QTT_ERR_INVALID_ARG, "qtt_server_create: unknown solve kind");
  qtt_server *S = new (std::nothrow) qtt_server();
  if (!S) return fail(QTT_ERR_OOM, "qtt_server_create: host allocation");
  S->prm = *prm;
  S->slots = slots;
  cudaGetDevice(&S->device);
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  S->budget = mem_budget ? mem_budget : fr / 10 * 8;
  for (int i = 0; i < slots; ++i) S->workers.emplace_back(worker_main, S);
  *out = S;
  return QTT_OK;
}

qtt_status qtt_server_submit(qtt_server *S, const qtt_op *K, const qtt_op *P, const double *f_host,
                             double *x_host, int64_t nrhs, int64_t *request_id) {
  if (!S || !f_host || !x_host || !request_id)
    return fail(QTT_ERR_INVALID_ARG, "qtt_server_submit: NULL argument");
  if (nrhs < 1 || nrhs > 65535) return fail(QTT_ERR_INVALID_ARG, "qtt_server_submit: nrhs");
  if (S->prm.kind == QTT_SOLVE_DIRECT ? !P : !K)
    return fail(QTT_ERR_INVALID_ARG, "qtt_server_submit: missing operator for this solve kind");
  if (K && P && K->d != P->d) return fail(QTT_ERR_INVALID_ARG, "qtt_server_submit: d differs");
  for (const qtt_op *A : {K, P})
    if (A && A->device != S->device)
      return fail(QTT_ERR_INVALID_ARG, "qtt_server_submit: operator lives on another device");
  Request *r = new (std::nothrow) Request();
  if (!r) return fail(QTT_ERR_OOM, "qtt_server_submit: host allocation");
  r->K = K;
  r->P = P;
  r->f_host = f_host;
  r->x_host = x_host;
  r->nrhs = nrhs;
  r->need = request_bytes(K, P, nrhs, S->prm);
  r->info.resize(nrhs);
  if (r->need > S->budget) {
    delete r;
    return fail(QTT_ERR_OOM, "qtt_server_submit: request needs more device memory than the "
                             "server's whole budget");
  }
  std::lock_guard<std::mutex> lk(S->mu);
  r->id = S->next_id++;
  r->t_submit = now_s();
  S->all[r->id] = r;
  S->pending.push_back(r);
  admit_locked(S);
  *request_id = r->id;
  return QTT_OK;
}

qtt_status qtt_server_poll(qtt_server *S, int64_t id, int wait, int *done, qtt_solve_info *info,
                           double *t_submit, double *t_admit, double *t_finish) {
  if (!S || !done) return fail(QTT_ERR_INVALID_ARG, "qtt_server_poll: NULL argument");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->all.find(id);
  if (it == S->all.end()) return fail(QTT_ERR_INVALID_ARG, "qtt_server_poll: unknown request");
  Request *r = it->second;
  if (wait) S->cv_done.wait(lk, [&] { return r->done; });
  *done = r->done ? 1 : 0;
  if (!r->done) return QTT_OK;
  if (info) std::memcpy(info, r->info.data(), sizeof(qtt_solve_info) * r->nrhs);
  if (t_submit) *t_submit = r->t_submit;
  if (t_admit) *t_admit = r->t_admit;
  if (t_finish) *t_finish = r->t_finish;
  const qtt_status s = r->status;
  const std::string msg = r->message;
  S->all.erase(it);  // retired: the id is no longer known
  delete r;
  if (s != QTT_OK) return fail(s, "request failed: " + msg);
  return s;
}

qtt_status qtt_server_stats(qtt_server *S, int *pending, int *running, size_t *in_use,
                            size_t *peak_in_use, int *peak_running) {
  if (!S) return fail(QTT_ERR_INVALID_ARG, "qtt_server_stats: NULL server");
  std::lock_guard<std::mutex> lk(S->mu);
  if (pending) *pending = (int)S->pending.size();
  if (running) *running = S->running + (int)S->admitted.size();
  if (in_use) *in_use = S->in_use;
  if (peak_in_use) *peak_in_use = S->peak_in_use;
  if (peak_running) *peak_running = S->peak_running;
  return QTT_OK;
}

qtt_status qtt_server_destroy(qtt_server *S) {
  if (!S) return QTT_OK;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    // finish everything that was submitted
    S->cv_done.wait(lk, [&] { return S->pending.empty() && S->admitted.empty() && !S->running; });
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto &t : S->workers) t.join();
  for (auto &kv : S->all) delete kv.second;
  delete S;
  return QTT_OK;
}

}  // extern "C"
