// Solve-and-apply server with continuous batching on one GPU.
//
// Requests -- qtt_solve requests (operators K, P and host right-hand sides)
// and qtt_apply requests (an operator and host vectors) of any d and nrhs --
// enter a FIFO queue.  One scheduler thread runs the device in ticks.  At
// every tick boundary the queue head is admitted while a slot is free and
// its device-memory estimate fits what is left of the budget (strict FIFO:
// large requests are not starved), and finished requests leave.  One tick
// advances every active request by one step of its solve:
//   pre   per request, on the request's slot stream: the part of the step
//         before the forward apply -- upload, the preconditioner apply Z_j =
//         P v_j (in the server's precond_compute), the solution update
//   K     ONE grouped launch per core step for all requests that need a
//         forward apply this tick -- w = a z + K z of an Arnoldi step, the
//         residual f - (a x + K x) after a GMRES cycle or a correction, the
//         product of an apply request: launch L runs core step L of every
//         such request with d > L, each with its own sizes and buffers
//         (step_f64_grouped_kernel)
//   post  per request: Gram-Schmidt against its Krylov basis, norms, and the
//         copy of the few numbers the host needs into pinned memory
// then one synchronisation, after which the host applies the Givens
// rotations and decides each request's next step.  So requests that arrive
// while others run join at the next tick, their applies share launches, and
// their vector kernels overlap on the slot streams.
//
// A request's arithmetic is that of qtt_solve (qtt_apply): the same kernels
// in the same order on its own buffers -- the grouped launch runs, for each
// request, the same step body and form the single-operator launch would --
// so its result is bitwise the same alone, in any mix, and through
// qtt_solve.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "krylov.h"
#include "qtt_internal.h"
#include "solve_internal.h"

namespace qtt {
namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum Kind { KIND_SOLVE = 0, KIND_APPLY = 1 };
enum Phase { PH_START = 0, PH_ARNOLDI, PH_UPDATE, PH_CORRECT, PH_DONE };

struct Request {
  int64_t id = 0;
  int kind = KIND_SOLVE;
  const qtt_op *K = nullptr, *P = nullptr;
  qtt_dtype apply_compute = QTT_F64;
  const double *f_host = nullptr;  // f (solve) or x (apply)
  double *x_host = nullptr;        // x (solve) or y (apply)
  int64_t nrhs = 0;
  size_t need = 0;
  double t_submit = 0, t_admit = 0, t_finish = 0;
  bool done = false;
  qtt_status status = QTT_OK;
  std::string message;
  std::vector<qtt_solve_info> info;

  // ---- state while active (scheduler thread only)
  int slot = -1;
  int phase = PH_START;
  int j = 0, jl = 0, iters = 0;
  bool flex = false, new_cycle = false, has_k = false;
  std::vector<void *> blocks;
  double *f = nullptr, *x = nullptr, *w = nullptr, *z = nullptr, *V = nullptr, *Z = nullptr;
  double *t1 = nullptr, *t2 = nullptr, *partial = nullptr, *h1 = nullptr, *h2 = nullptr;
  double *ss = nullptr, *ss2 = nullptr, *ydev = nullptr, *kbuf[2] = {nullptr, nullptr};
  double *hv1 = nullptr, *hv2 = nullptr, *hs = nullptr, *hs2 = nullptr, *hy = nullptr;  // pinned
  std::vector<double> H, cs, sn, g, fn, rel;
  // the forward apply queued for this tick's grouped launches
  const qtt_op *kop = nullptr;
  const double *kin = nullptr;
  double *kout = nullptr;
  Epilogue kepi;
};

struct Slot {
  cudaStream_t st = nullptr;
  cudaEvent_t ev_pre = nullptr, ev_post = nullptr;
  double *pin = nullptr;  // pinned host block
  size_t pin_doubles = 0;
  bool busy = false;
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
  std::deque<qtt::Request *> admitted;    // admitted, not yet set up by the scheduler
  std::map<int64_t, qtt::Request *> all;  // every request until retired
  std::thread scheduler;
  int running = 0;  // admitted and not finished
  int64_t next_id = 0;
  bool stop = false;
  int device = 0;
  size_t peak_in_use = 0;
  int peak_running = 0;
  uint64_t ticks = 0, grouped_launches = 0;
  // scheduler-owned device resources
  std::vector<qtt::Slot> slot;
  cudaStream_t main = nullptr;
  cudaEvent_t ev_k = nullptr;
  qtt::GroupedStepF64 *gtab_host = nullptr, *gtab_dev = nullptr;
  size_t gtab_cap = 0;
};

namespace qtt {
namespace {

int gmres_m(const qtt_solve_params &p) { return p.kind == QTT_SOLVE_GMRES ? p.restart : 0; }

// Device bytes a request may hold at once: its own vectors and Krylov
// basis, the intermediates of its grouped forward apply, and the scratch of
// its preconditioner applies (the pool may keep them).
size_t request_bytes(int kind, const qtt_op *K, const qtt_op *P, int64_t nrhs,
                     const qtt_solve_params &p) {
  const qtt_op *A = K ? K : P;
  const size_t N = (size_t)1 << A->d, R = (size_t)nrhs;
  size_t b = 4 * N * R * 8;  // f, x, w, z
  if (kind == KIND_SOLVE) {
    const int m = gmres_m(p);
    if (p.kind == QTT_SOLVE_GMRES) b += (size_t)(2 * m + 1) * N * R * 8;
    if (p.inner_iters > 0) b += 2 * N * R * 8;
    b += (size_t)(m + 1) * std::min<size_t>(R, 65535) * (size_t)blocks_for((int64_t)N) * 8;
  }
  if (K) b += 2 * (size_t)K->rmax_inner * N * R * 8;
  if (K && kind == KIND_SOLVE && p.inner_iters > 0) b += 2 * (size_t)K->rmax_inner * N * R * 4;
  if (P && kind == KIND_SOLVE) {
    const size_t e = p.precond_compute == QTT_F64 ? 8 : (p.precond_compute == QTT_BF16 ? 2 : 4);
    b += 2 * (size_t)P->rmax_inner * N * R * e;
  }
  if (kind == KIND_APPLY && K) {
    const size_t e = p.precond_compute == QTT_F64 ? 8 : 4;
    b += 2 * (size_t)K->rmax_inner * N * R * e;
  }
  return b + (64u << 20);
}

// Move admissible requests from `pending` to `admitted` (caller holds mu).
void admit_locked(qtt_server *S) {
  while (!S->pending.empty()) {
    Request *r = S->pending.front();
    if (S->running >= S->slots || S->in_use + r->need > S->budget) break;
    S->pending.pop_front();
    S->in_use += r->need;
    S->peak_in_use = std::max(S->peak_in_use, S->in_use);
    ++S->running;
    S->peak_running = std::max(S->peak_running, S->running);
    r->t_admit = now_s();
    S->admitted.push_back(r);
  }
  S->cv_work.notify_all();
}

}  // namespace
}  // namespace qtt

namespace qtt {
namespace {

#define SRV_TRY(expr)                 \
  do {                                \
    const qtt_status s_ = (expr);     \
    if (s_ != QTT_OK) return s_;      \
  } while (0)
#define SRV_CUDA(expr, where)                               \
  do {                                                      \
    const cudaError_t e_ = (expr);                          \
    if (e_ != cudaSuccess) return cuda_fail(e_, where);     \
  } while (0)

int64_t req_N(const Request *r) {
  const qtt_op *A = r->K ? r->K : r->P;
  return (int64_t)1 << A->d;
}

SolveCtx ctx_of(const qtt_server *S, const Request *r) {
  return SolveCtx{r->K, r->P, S->prm.a, S->prm.precond_compute, req_N(r), r->nrhs,
                  S->slot[r->slot].st};
}

// Device buffers, pinned host slice and host state of a newly admitted
// request on slot `slot`.
qtt_status setup(qtt_server *S, Request *r, int slot) {
  Slot &sl = S->slot[slot];
  r->slot = slot;
  cudaStream_t st = sl.st;
  const int64_t N = req_N(r), nr = r->nrhs;
  const size_t v = (size_t)N * (size_t)nr;
  auto get = [&](double **p, size_t n) -> qtt_status {
    void *q = nullptr;
    const qtt_status s = scratch_alloc(&q, std::max<size_t>(n, 1) * sizeof(double), st);
    if (s != QTT_OK) return s;
    r->blocks.push_back(q);
    *p = static_cast<double *>(q);
    return QTT_OK;
  };
  SRV_TRY(get(&r->f, v));
  SRV_TRY(get(&r->x, v));
  SRV_TRY(get(&r->w, v));
  SRV_TRY(get(&r->z, v));
  if (r->K && r->K->d > 1) {
    SRV_TRY(get(&r->kbuf[0], (size_t)r->K->rmax_inner * v));
    SRV_TRY(get(&r->kbuf[1], (size_t)r->K->rmax_inner * v));
  }
  const int m = r->kind == KIND_SOLVE ? gmres_m(S->prm) : 0;
  if (r->kind == KIND_SOLVE) {
    const int inner = S->prm.inner_iters;
    if (S->prm.kind == QTT_SOLVE_GMRES) {
      SRV_TRY(get(&r->V, (size_t)(m + 1) * v));
      r->flex = r->P || inner > 0;
      if (r->flex) SRV_TRY(get(&r->Z, (size_t)m * v));
      SRV_TRY(get(&r->ydev, (size_t)m * nr));
    }
    if (inner > 0) {
      SRV_TRY(get(&r->t1, v));
      SRV_TRY(get(&r->t2, v));
    }
    SRV_TRY(get(&r->partial, (size_t)(m + 1) * std::min<int64_t>(nr, 65535) * blocks_for(N)));
    SRV_TRY(get(&r->h1, (size_t)(m + 1) * nr));
    SRV_TRY(get(&r->h2, (size_t)(m + 1) * nr));
    SRV_TRY(get(&r->ss, (size_t)nr));
    SRV_TRY(get(&r->ss2, (size_t)nr));
  }
  // pinned slice: hv1, hv2 ((m + 1) nr each), hs, hs2 (nr each), hy (m nr)
  const size_t pin = (size_t)(2 * (m + 1) + 2 + m) * (size_t)nr;
  if (sl.pin_doubles < pin) {
    if (sl.pin) cudaFreeHost(sl.pin);
    sl.pin = nullptr;
    sl.pin_doubles = 0;
    void *h = nullptr;
    SRV_CUDA(cudaMallocHost(&h, pin * sizeof(double)), "server: pinned host buffer");
    sl.pin = static_cast<double *>(h);
    sl.pin_doubles = pin;
  }
  r->hv1 = sl.pin;
  r->hv2 = r->hv1 + (size_t)(m + 1) * nr;
  r->hs = r->hv2 + (size_t)(m + 1) * nr;
  r->hs2 = r->hs + nr;
  r->hy = r->hs2 + nr;
  r->H.assign((size_t)nr * (m + 1) * std::max(m, 1), 0.0);
  r->cs.assign((size_t)nr * std::max(m, 1), 0.0);
  r->sn.assign((size_t)nr * std::max(m, 1), 0.0);
  r->g.assign((size_t)nr * (m + 1), 0.0);
  r->fn.assign((size_t)nr, 0.0);
  r->rel.assign((size_t)nr, 0.0);
  r->phase = PH_START;
  return QTT_OK;
}

void queue_k(Request *r, const qtt_op *A, const double *in, double *out, const Epilogue &e) {
  r->has_k = true;
  r->kop = A;
  r->kin = in;
  r->kout = out;
  r->kepi = e;
}

Epilogue residual_epi(const qtt_server *S, const Request *r) {
  // w = f - (a x + K x)
  Epilogue e;
  e.on = true;
  e.v = r->f;
  e.s_v = 1.0;
  e.u = r->x;
  e.s_u = -S->prm.a;
  e.s_acc = -1.0;
  return e;
}

// The part of this tick's step before the forward apply (slot stream).
qtt_status pre_work(qtt_server *S, Request *r) {
  r->has_k = false;
  const SolveCtx c = ctx_of(S, r);
  const int64_t N = c.N, nr = c.nrhs;
  const size_t bytes = (size_t)N * nr * sizeof(double);
  const int m = gmres_m(S->prm), inner = S->prm.inner_iters;
  const int64_t vstride = N * nr;
  if (r->phase == PH_START) {
    SRV_CUDA(cudaMemcpyAsync(r->f, r->f_host, bytes, cudaMemcpyHostToDevice, c.st), "upload");
    if (r->kind == KIND_APPLY) {
      if (r->apply_compute == QTT_F64) {
        queue_k(r, r->K, r->f, r->x, Epilogue());
      } else {
        SRV_TRY(apply_lp(r->K, r->apply_compute, r->f, QTT_F64, r->x, QTT_F64, nr, N, c.st,
                         LpEpilogue()));
      }
      return QTT_OK;
    }
    switch (S->prm.kind) {
      case QTT_SOLVE_GMRES:
        SRV_CUDA(cudaMemsetAsync(r->x, 0, bytes, c.st), "zero x");
        SRV_CUDA(vec_copy(vecs(r->w, N), vecs(r->f, N), N, nr, c.st), "copy");
        break;
      case QTT_SOLVE_REFINE:
        if (inner > 0) {
          SRV_TRY(solve_apply_M(c, inner, r->f, r->z, r->t1, r->t2));
          SRV_CUDA(vec_copy(vecs(r->x, N), vecs(r->z, N), N, nr, c.st), "copy");
        } else {
          SRV_TRY(solve_apply_P(c, r->f, r->x, false));
        }
        queue_k(r, r->K, r->x, r->w, residual_epi(S, r));
        break;
      default:  // DIRECT
        SRV_TRY(solve_apply_P(c, r->f, r->x, false));
        if (r->K) queue_k(r, r->K, r->x, r->w, residual_epi(S, r));
        break;
    }
    return QTT_OK;
  }
  if (r->phase == PH_ARNOLDI) {
    if (r->new_cycle) {
      SRV_CUDA(vec_normalize(vecs(r->V, N), vecs(r->w, N), r->ss, N, nr, c.st), "normalize");
      r->new_cycle = false;
    }
    double *Vj = r->V + (int64_t)r->j * vstride;
    double *Zj = r->flex ? r->Z + (int64_t)r->j * vstride : Vj;
    if (r->flex) SRV_TRY(solve_apply_M(c, inner, Vj, Zj, r->t1, r->t2));
    Epilogue e;  // w = a z + K z
    e.on = true;
    e.u = Zj;
    e.s_u = S->prm.a;
    e.s_acc = 1.0;
    queue_k(r, r->K, Zj, r->w, e);
    return QTT_OK;
  }
  if (r->phase == PH_UPDATE) {
    SRV_CUDA(cudaMemcpyAsync(r->ydev, r->hy, sizeof(double) * r->jl * nr, cudaMemcpyHostToDevice,
                             c.st),
             "upload y");
    SRV_CUDA(vec_combine(vecs(r->z, N), vecs(r->flex ? r->Z : r->V, N, vstride), r->jl, r->ydev, N,
                         nr, c.st),
             "combine");
    SRV_CUDA(vec_axpy(vecs(r->x, N), vecs(r->z, N), 1.0, N, nr, c.st), "axpy");
    queue_k(r, r->K, r->x, r->w, residual_epi(S, r));
    (void)m;
    return QTT_OK;
  }
  if (r->phase == PH_CORRECT) {
    if (inner > 0) {
      SRV_TRY(solve_apply_M(c, inner, r->w, r->z, r->t1, r->t2));
      SRV_CUDA(vec_axpy(vecs(r->x, N), vecs(r->z, N), 1.0, N, nr, c.st), "axpy");
    } else {
      SRV_TRY(solve_apply_P(c, r->w, r->x, true));
    }
    queue_k(r, r->K, r->x, r->w, residual_epi(S, r));
    return QTT_OK;
  }
  return QTT_OK;
}

}  // namespace
}  // namespace qtt

namespace qtt {
namespace {

// The part of this tick's step after the forward apply (slot stream): the
// Gram-Schmidt and norms, and the copies the host reads after the tick.
qtt_status post_work(qtt_server *S, Request *r) {
  if (r->kind == KIND_APPLY) return QTT_OK;
  const SolveCtx c = ctx_of(S, r);
  const int64_t N = c.N, nr = c.nrhs;
  const int64_t vstride = N * nr;
  auto read = [&](double *dst, const double *src, size_t n) -> qtt_status {
    SRV_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost, c.st), "read");
    return QTT_OK;
  };
  if (r->phase == PH_START) {
    if (S->prm.kind == QTT_SOLVE_GMRES) {
      // ||f||, also the first residual's norm (x = 0): one sum of squares of w = f
      SRV_CUDA(vec_dots(vecs(r->w, N), 1, vecs(r->w, N), N, nr, r->partial, r->ss, nullptr, c.st),
               "dots");
      return read(r->hs, r->ss, nr);
    }
    SRV_CUDA(vec_dots(vecs(r->f, N), 1, vecs(r->f, N), N, nr, r->partial, r->ss2, nullptr, c.st),
             "dots");
    SRV_TRY(read(r->hs2, r->ss2, nr));
    if (r->has_k) {
      SRV_CUDA(vec_dots(vecs(r->w, N), 1, vecs(r->w, N), N, nr, r->partial, r->ss, nullptr, c.st),
               "dots");
      SRV_TRY(read(r->hs, r->ss, nr));
    }
    return QTT_OK;
  }
  if (r->phase == PH_ARNOLDI) {
    const int j = r->j, nv = j + 1;
    const VecSet V = vecs(r->V, N, vstride), W = vecs(r->w, N);
    SRV_CUDA(vec_dots(V, nv, W, N, nr, r->partial, r->h1, nullptr, c.st), "dots");
    SRV_CUDA(vec_gs_update(W, V, nv, r->h1, N, nr, c.st), "gs");
    SRV_CUDA(vec_dots(V, nv, W, N, nr, r->partial, r->h2, nullptr, c.st), "dots");
    SRV_CUDA(vec_gs_update(W, V, nv, r->h2, N, nr, c.st), "gs");
    SRV_CUDA(vec_dots(W, 1, W, N, nr, r->partial, r->ss, nullptr, c.st), "dots");
    SRV_CUDA(vec_normalize(vecs(r->V + (int64_t)(j + 1) * vstride, N), W, r->ss, N, nr, c.st),
             "normalize");
    SRV_TRY(read(r->hv1, r->h1, (size_t)nv * nr));
    SRV_TRY(read(r->hv2, r->h2, (size_t)nv * nr));
    return read(r->hs, r->ss, nr);
  }
  // PH_UPDATE, PH_CORRECT: the residual's sum of squares
  SRV_CUDA(vec_dots(vecs(r->w, N), 1, vecs(r->w, N), N, nr, r->partial, r->ss, nullptr, c.st),
           "dots");
  return read(r->hs, r->ss, nr);
}

// This tick's forward applies, all requests together: launch L runs core
// step L of every queued apply with d > L (each with its own buffers and,
// on its last step, its epilogue).
qtt_status grouped_forward(qtt_server *S, const std::vector<Request *> &act) {
  std::vector<Request *> ks;
  for (Request *r : act)
    if (r->has_k) ks.push_back(r);
  if (ks.empty()) return QTT_OK;
  int maxd = 0;
  for (Request *r : ks) {
    SRV_CUDA(cudaStreamWaitEvent(S->main, S->slot[r->slot].ev_pre, 0), "wait pre");
    maxd = std::max(maxd, r->kop->d);
  }
  std::vector<GroupedStepF64> tab;
  std::vector<size_t> first(maxd + 1, 0);
  std::vector<int64_t> total(maxd, 0);
  for (int L = 0; L < maxd; ++L) {
    first[L] = tab.size();
    int64_t cta = 0;
    for (Request *r : ks) {
      const qtt_op *A = r->kop;
      if (A->d <= L) continue;
      const int64_t N = (int64_t)1 << A->d;
      GroupedStepF64 g;
      std::memset(&g, 0, sizeof(g));
      StepF64 &p = g.s;
      p.k = L;
      p.rin = A->ranks[L];
      p.rout = A->ranks[L + 1];
      p.N = N;
      p.nrhs = r->nrhs;
      p.M = A->m64 + A->off[L];
      if (L == 0) {
        p.in = r->kin;
        p.in_rhs_stride = N;
      } else {
        p.in = r->kbuf[(L - 1) & 1];
        p.in_rhs_stride = (int64_t)p.rin * N;
      }
      if (L == A->d - 1) {
        p.out = r->kout;
        p.out_rhs_stride = N;
        if (r->kepi.on) {
          p.epi = 1;
          p.u = r->kepi.u;
          p.v = r->kepi.v;
          p.uv_rhs_stride = N;
          p.s_acc = r->kepi.s_acc;
          p.s_u = r->kepi.s_u;
          p.s_v = r->kepi.s_v;
        }
      } else {
        p.out = r->kbuf[L & 1];
        p.out_rhs_stride = (int64_t)p.rout * N;
      }
      g.small = f64_step_small(N, p.rout) ? 1 : 0;
      g.ctas_per_rhs = f64_step_ctas_per_rhs(p, g.small != 0);
      g.cta0 = cta;
      cta += g.ctas_per_rhs * r->nrhs;
      tab.push_back(g);
    }
    total[L] = cta;
  }
  first[maxd] = tab.size();
  if (tab.size() > S->gtab_cap) {
    // grow the staging tables (the previous tick has finished with them)
    if (S->gtab_host) cudaFreeHost(S->gtab_host);
    S->gtab_host = nullptr;
    release_after({S->gtab_dev}, {});
    S->gtab_dev = nullptr;
    S->gtab_cap = 0;
    const size_t cap = tab.size() * 2;
    void *h = nullptr;
    SRV_CUDA(cudaMallocHost(&h, cap * sizeof(GroupedStepF64)), "server: pinned step table");
    S->gtab_host = static_cast<GroupedStepF64 *>(h);
    SRV_TRY(persistent_alloc(reinterpret_cast<void **>(&S->gtab_dev),
                             cap * sizeof(GroupedStepF64), S->main));
    S->gtab_cap = cap;
  }
  std::memcpy(S->gtab_host, tab.data(), tab.size() * sizeof(GroupedStepF64));
  SRV_CUDA(cudaMemcpyAsync(S->gtab_dev, S->gtab_host, tab.size() * sizeof(GroupedStepF64),
                           cudaMemcpyHostToDevice, S->main),
           "upload step table");
  for (int L = 0; L < maxd; ++L) {
    SRV_CUDA(launch_step_f64_grouped(S->gtab_dev + first[L], (int)(first[L + 1] - first[L]),
                                     total[L], S->main),
             "grouped step");
    ++S->grouped_launches;
  }
  for (Request *r : ks) note_use(r->kop, S->main);
  SRV_CUDA(cudaEventRecord(S->ev_k, S->main), "record");
  for (Request *r : ks)
    SRV_CUDA(cudaStreamWaitEvent(S->slot[r->slot].st, S->ev_k, 0), "wait forward apply");
  return QTT_OK;
}

void fill_info(qtt_server *S, Request *r) {
  for (int64_t k = 0; k < r->nrhs; ++k) {
    qtt_solve_info &in = r->info[k];
    if (r->kind == KIND_APPLY) {
      in.iters = 1;
      in.rel_residual = -1.0;
      in.status = QTT_OK;
    } else {
      in.iters = r->iters;
      in.rel_residual = r->rel[k];
      in.status = S->prm.kind == QTT_SOLVE_DIRECT || r->rel[k] <= S->prm.tol
                      ? QTT_OK : QTT_ERR_NOT_CONVERGED;
    }
  }
}

// After the tick's synchronisation: decide each request's next step.
void host_step(qtt_server *S, Request *r) {
  const int64_t nr = r->nrhs;
  const qtt_solve_params &p = S->prm;
  const int m = gmres_m(p);
  auto converged = [&]() {
    bool all = true;
    for (int64_t k = 0; k < nr; ++k) {
      r->rel[k] = r->fn[k] > 0.0 ? std::sqrt(r->hs[k]) / r->fn[k] : 0.0;
      if (r->fn[k] > 0.0 && r->rel[k] > p.tol) all = false;
    }
    return all;
  };
  auto new_cycle = [&]() {
    std::fill(r->H.begin(), r->H.end(), 0.0);
    std::fill(r->g.begin(), r->g.end(), 0.0);
    for (int64_t k = 0; k < nr; ++k) r->g[(size_t)k * (m + 1)] = std::sqrt(r->hs[k]);
    r->j = 0;
    r->phase = PH_ARNOLDI;
    r->new_cycle = true;
  };
  if (r->kind == KIND_APPLY) {
    r->phase = PH_DONE;
    return;
  }
  if (r->phase == PH_START) {
    if (p.kind == QTT_SOLVE_GMRES) {
      for (int64_t k = 0; k < nr; ++k) r->fn[k] = std::sqrt(r->hs[k]);
      if (converged() || r->iters >= p.max_iter) r->phase = PH_DONE;
      else new_cycle();
      return;
    }
    for (int64_t k = 0; k < nr; ++k) r->fn[k] = std::sqrt(r->hs2[k]);
    r->iters = 1;
    if (p.kind == QTT_SOLVE_DIRECT) {
      for (int64_t k = 0; k < nr; ++k)
        r->rel[k] = !r->K ? -1.0 : (r->fn[k] > 0.0 ? std::sqrt(r->hs[k]) / r->fn[k] : 0.0);
      r->phase = PH_DONE;
      return;
    }
    r->phase = converged() || r->iters >= p.max_iter ? PH_DONE : PH_CORRECT;
    return;
  }
  if (r->phase == PH_ARNOLDI) {
    const bool done = gmres_host_step(nr, m, r->j, r->hv1, r->hv2, r->hs, r->fn, p.tol, r->H,
                                      r->cs, r->sn, r->g);
    ++r->iters;
    r->jl = r->j + 1;
    if (done || r->j + 1 >= m || r->iters >= p.max_iter) {
      gmres_back_solve(nr, m, r->jl, r->H, r->g, r->hy);
      r->phase = PH_UPDATE;
    } else {
      ++r->j;
    }
    return;
  }
  if (r->phase == PH_UPDATE) {
    if (converged() || r->iters >= p.max_iter) r->phase = PH_DONE;
    else new_cycle();
    return;
  }
  if (r->phase == PH_CORRECT) {
    ++r->iters;
    if (converged() || r->iters >= p.max_iter) r->phase = PH_DONE;
  }
}

}  // namespace
}  // namespace qtt

namespace qtt {
namespace {

// Download the result, return the request's buffers and slot, and publish
// it (scheduler thread).
void finish(qtt_server *S, Request *r) {
  if (r->slot >= 0) {
    Slot &sl = S->slot[r->slot];
    if (r->status == QTT_OK) {
      const size_t bytes = (size_t)req_N(r) * r->nrhs * sizeof(double);
      cudaError_t e = cudaMemcpyAsync(r->x_host, r->x, bytes, cudaMemcpyDeviceToHost, sl.st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(sl.st);
      if (e != cudaSuccess) {
        r->status = cuda_fail(e, "server: download");
        r->message = qtt_last_error();
      }
    }
    for (void *q : r->blocks) scratch_free(q, sl.st);
    r->blocks.clear();
    cudaStreamSynchronize(sl.st);
    sl.busy = false;
  }
  fill_info(S, r);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    r->t_finish = now_s();
    r->done = true;
    --S->running;
    S->in_use -= r->need;
    admit_locked(S);
  }
  S->cv_done.notify_all();
}

void fail_request(Request *r, qtt_status s) {
  r->status = s;
  r->message = qtt_last_error();
  r->phase = PH_DONE;
}

// One tick over the active requests.
void tick(qtt_server *S, std::vector<Request *> &act) {
  for (Request *r : act) {
    const qtt_status s = pre_work(S, r);
    if (s != QTT_OK) fail_request(r, s);
    cudaEventRecord(S->slot[r->slot].ev_pre, S->slot[r->slot].st);
  }
  std::vector<Request *> live;
  for (Request *r : act)
    if (r->status == QTT_OK) live.push_back(r);
  const qtt_status gs = grouped_forward(S, live);
  if (gs != QTT_OK)
    for (Request *r : live)
      if (r->has_k) fail_request(r, gs);
  for (Request *r : act) {
    if (r->status == QTT_OK) {
      const qtt_status s = post_work(S, r);
      if (s != QTT_OK) fail_request(r, s);
    }
    cudaEventRecord(S->slot[r->slot].ev_post, S->slot[r->slot].st);
  }
  for (Request *r : act) {
    const cudaError_t e = cudaEventSynchronize(S->slot[r->slot].ev_post);
    if (e != cudaSuccess && r->status == QTT_OK) fail_request(r, cuda_fail(e, "server: tick"));
  }
  for (Request *r : act)
    if (r->status == QTT_OK && r->phase != PH_DONE) host_step(S, r);
  ++S->ticks;
}

void scheduler_main(qtt_server *S) {
  cudaSetDevice(S->device);
  std::vector<Request *> active;
  for (;;) {
    std::vector<Request *> fresh;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] { return S->stop || !S->admitted.empty() || !active.empty(); });
      if (S->stop && S->admitted.empty() && active.empty()) break;
      while (!S->admitted.empty()) {
        fresh.push_back(S->admitted.front());
        S->admitted.pop_front();
      }
    }
    for (Request *r : fresh) {
      int slot = -1;
      for (int i = 0; i < S->slots; ++i)
        if (!S->slot[i].busy) {
          slot = i;
          break;
        }
      // admission never exceeds the slot count, so a slot is free
      S->slot[slot].busy = true;
      const qtt_status s = setup(S, r, slot);
      if (s != QTT_OK) {
        fail_request(r, s);
        finish(S, r);
      } else {
        active.push_back(r);
      }
    }
    if (active.empty()) continue;
    tick(S, active);
    std::vector<Request *> still;
    for (Request *r : active) {
      if (r->phase == PH_DONE || r->status != QTT_OK) finish(S, r);
      else still.push_back(r);
    }
    active.swap(still);
  }
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
  if (prm->kind == QTT_SOLVE_GMRES && (prm->restart < 1 || prm->restart > 1000))
    return fail(QTT_ERR_INVALID_ARG, "qtt_server_create: restart must be in [1, 1000]");
  if (prm->max_iter < 1 || !(prm->tol >= 0.0) || prm->inner_iters < 0 || prm->inner_iters > 1000)
    return fail(QTT_ERR_INVALID_ARG, "qtt_server_create: bad tol, max_iter or inner_iters");
  qtt_server *S = new (std::nothrow) qtt_server();
  if (!S) return fail(QTT_ERR_OOM, "qtt_server_create: host allocation");
  S->prm = *prm;
  S->slots = slots;
  cudaGetDevice(&S->device);
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  S->budget = mem_budget ? mem_budget : fr / 10 * 8;
  S->slot.resize(slots);
  cudaError_t e = cudaStreamCreateWithFlags(&S->main, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ev_k, cudaEventDisableTiming);
  for (int i = 0; i < slots && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&S->slot[i].st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->slot[i].ev_pre, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->slot[i].ev_post, cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    qtt_server_destroy(S);
    return cuda_fail(e, "qtt_server_create: streams");
  }
  S->scheduler = std::thread(scheduler_main, S);
  *out = S;
  return QTT_OK;
}

static qtt_status submit(qtt_server *S, Request *r, int64_t *request_id) {
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
  const qtt_dtype pc = S->prm.precond_compute;
  auto packed = [&](const qtt_op *A) {
    return pc == QTT_F64 || (pc == QTT_F32 ? A->m32 != nullptr
                             : pc == QTT_TF32 ? A->mtf32 != nullptr : A->mbf16 != nullptr);
  };
  if (P && !packed(P))
    return fail(QTT_ERR_INVALID_ARG, "qtt_server_submit: P lacks the packed copy for precond_compute");
  if (K && S->prm.inner_iters > 0 && S->prm.kind != QTT_SOLVE_DIRECT && !packed(K))
    return fail(QTT_ERR_INVALID_ARG, "qtt_server_submit: inner iterations need K packed");
  Request *r = new (std::nothrow) Request();
  if (!r) return fail(QTT_ERR_OOM, "qtt_server_submit: host allocation");
  r->kind = KIND_SOLVE;
  r->K = K;
  r->P = P;
  r->f_host = f_host;
  r->x_host = x_host;
  r->nrhs = nrhs;
  r->need = request_bytes(KIND_SOLVE, K, P, nrhs, S->prm);
  r->info.resize(nrhs);
  return submit(S, r, request_id);
}

qtt_status qtt_server_submit_apply(qtt_server *S, const qtt_op *A, const double *x_host,
                                   double *y_host, int64_t nrhs, qtt_dtype compute,
                                   int64_t *request_id) {
  if (!S || !A || !x_host || !y_host || !request_id)
    return fail(QTT_ERR_INVALID_ARG, "qtt_server_submit_apply: NULL argument");
  if (nrhs < 1 || nrhs > 65535) return fail(QTT_ERR_INVALID_ARG, "qtt_server_submit_apply: nrhs");
  if (A->device != S->device)
    return fail(QTT_ERR_INVALID_ARG, "qtt_server_submit_apply: operator lives on another device");
  if (compute != QTT_F64 && compute != QTT_F32 && compute != QTT_TF32 && compute != QTT_BF16)
    return fail(QTT_ERR_INVALID_ARG, "qtt_server_submit_apply: unknown compute");
  if ((compute == QTT_F32 && !A->m32) || (compute == QTT_TF32 && !A->mtf32) ||
      (compute == QTT_BF16 && !A->mbf16))
    return fail(QTT_ERR_INVALID_ARG, "qtt_server_submit_apply: operator lacks the packed copy");
  Request *r = new (std::nothrow) Request();
  if (!r) return fail(QTT_ERR_OOM, "qtt_server_submit_apply: host allocation");
  r->kind = KIND_APPLY;
  r->K = A;
  r->apply_compute = compute;
  r->f_host = x_host;
  r->x_host = y_host;
  r->nrhs = nrhs;
  qtt_solve_params p = S->prm;
  p.precond_compute = compute;
  r->need = request_bytes(KIND_APPLY, A, nullptr, nrhs, p);
  r->info.resize(nrhs);
  return submit(S, r, request_id);
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
  if (running) *running = S->running;
  if (in_use) *in_use = S->in_use;
  if (peak_in_use) *peak_in_use = S->peak_in_use;
  if (peak_running) *peak_running = S->peak_running;
  return QTT_OK;
}

qtt_status qtt_server_ticks(qtt_server *S, uint64_t *ticks, uint64_t *grouped_launches) {
  if (!S) return fail(QTT_ERR_INVALID_ARG, "qtt_server_ticks: NULL server");
  std::lock_guard<std::mutex> lk(S->mu);
  if (ticks) *ticks = S->ticks;
  if (grouped_launches) *grouped_launches = S->grouped_launches;
  return QTT_OK;
}

qtt_status qtt_server_destroy(qtt_server *S) {
  if (!S) return QTT_OK;
  if (S->scheduler.joinable()) {
    {
      std::unique_lock<std::mutex> lk(S->mu);
      // finish everything that was submitted
      S->cv_done.wait(lk, [&] { return S->pending.empty() && S->admitted.empty() && !S->running; });
      S->stop = true;
    }
    S->cv_work.notify_all();
    S->scheduler.join();
  }
  for (auto &kv : S->all) delete kv.second;
  for (Slot &sl : S->slot) {
    if (sl.st) cudaStreamSynchronize(sl.st);
    if (sl.pin) cudaFreeHost(sl.pin);
    if (sl.ev_pre) cudaEventDestroy(sl.ev_pre);
    if (sl.ev_post) cudaEventDestroy(sl.ev_post);
    if (sl.st) cudaStreamDestroy(sl.st);
  }
  if (S->main) cudaStreamSynchronize(S->main);
  if (S->gtab_host) cudaFreeHost(S->gtab_host);
  if (S->gtab_dev) release_after({S->gtab_dev}, {});
  if (S->ev_k) cudaEventDestroy(S->ev_k);
  if (S->main) cudaStreamDestroy(S->main);
  delete S;
  return QTT_OK;
}

}  // extern "C"
