// Internal declarations shared by the CUDA translation units of libqtt.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/qtt.h"

namespace qtt {

// Record a message for qtt_last_error() and return the status.
qtt_status fail(qtt_status s, const std::string &msg);
qtt_status cuda_fail(cudaError_t e, const char *where);

#define QTT_CUDA_TRY(call)                                   \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return ::qtt::cuda_fail(e_, #call); \
  } while (0)

// Count of kernel launches issued by the library (all threads).
void count_launches(uint64_t n);

// Stream-ordered scratch from the library's pool (one pool per device, keeps
// freed blocks cached).  Returns QTT_ERR_OOM if `bytes` cannot be had.
qtt_status scratch_alloc(void **ptr, size_t bytes, cudaStream_t stream);
void scratch_free(void *ptr, cudaStream_t stream);
// Bytes the pool could hand out right now without growing past free memory
// (and below the cap set by QTT_SCRATCH_CAP_BYTES, when that is set).
size_t scratch_available();
// The same, but answered from the pool's own cached bytes (no query of the
// device's free memory) when those already cover `bytes`.
size_t scratch_available_at_least(size_t bytes);

// Long-lived device buffers (operator cores, batch tables) come from the same
// pool, so that releasing them is stream-ordered and never synchronises the
// device.  persistent_alloc returns once the buffer is usable on any stream.
qtt_status persistent_alloc(void **ptr, size_t bytes, cudaStream_t stream);
// Release `ptrs` once every event in `after` has completed, without blocking
// the host or any other stream: a per-device release stream waits on the
// events and frees the buffers.
void release_after(const std::vector<void *> &ptrs, const std::vector<cudaEvent_t> &after);

}  // namespace qtt

struct qtt_op;
namespace qtt {
// How an apply in a given arithmetic runs (the fusion plan).  Chosen per
// operator and arithmetic by qtt_apply_autotune (or set by the caller);
// the defaults are the rules the library uses untuned.
struct ApplyPlan {
  bool fusion = true;   // merge steps: head/tail kernels (2-3 steps) and fused pairs (2 steps)
  int pairs = 2;        // fused-pair kernel family: 2 tcgen05, 1 mma.sync, 0 none
  int groups_cap = 0;   // tcgen05 pairs: 0 = as many epilogue groups as fit, 2 = two
  bool staged = true;   // FP32/TF32 single steps on the staged (shared-memory) kernel
};
// plan code = fusion + 2 pairs + 8 (groups_cap == 2) + 16 staged
inline int encode_plan(const ApplyPlan &p) {
  return (p.fusion ? 1 : 0) + 2 * p.pairs + (p.groups_cap == 2 ? 8 : 0) + (p.staged ? 16 : 0);
}
inline bool decode_plan(int code, ApplyPlan *p) {
  if (code < 0 || code > 31 || ((code >> 1) & 3) == 3) return false;
  p->fusion = (code & 1) != 0;
  p->pairs = (code >> 1) & 3;
  p->groups_cap = (code & 8) ? 2 : 0;
  p->staged = (code & 16) != 0;
  return true;
}
// Record that work just queued on `stream` reads A (one event per stream,
// re-recorded at each use; nothing is recorded while the stream is being
// captured into a graph).  qtt_destroy releases A after these events.
void note_use(const qtt_op *A, cudaStream_t stream);
// QTT_ERR_INVALID_ARG unless the current device is the one A lives on.
qtt_status check_device(const qtt_op *A, const char *where);

// Two streams per device for host <-> device copies that overlap the work
// on the caller's stream (qtt_apply_host, qtt_batch_run_host): created on
// first use, kept until the process ends.
struct CopyStreams {
  cudaStream_t in = nullptr, out = nullptr;
};
qtt_status copy_streams(CopyStreams *cs);
// Commit the static array of qtt_apply_noalloc on the current device (loads
// its module); done by qtt_create, which allocates anyway.
qtt_status noalloc_prepare();
}  // namespace qtt

// One QTT matrix resident on the device.  Core k is packed as the matrix
// M_k of Algorithm 2 (rows (alpha_{k+1}, i_k), columns (alpha_k, j_k)) in
// the order each kernel reads it:
//   m64 / m32 / mbf16 : [alpha_{k+1}][alpha_k][j_k][i_k], i.e. for each output
//                       rank b a run of 2 r_k pairs (i = 0, i = 1).
struct qtt_op {
  int d = 0;
  int device = 0;
  std::vector<int> ranks;       // d + 1
  std::vector<int64_t> off;     // element offset of core k in the packed arrays
  int64_t nparams = 0;          // sum_k 4 r_k r_{k+1}
  int rmax_inner = 1;           // max_{0<k<d} r_k (intermediate width)
  double flops_per_rhs = 0.0;   // 4 N sum_k r_k r_{k+1}
  unsigned packs = 0;           // QTT_PACK_* built
  double *m64 = nullptr;
  float *m32 = nullptr;         // FP32 copy (QTT_PACK_F32)
  float *mtf32 = nullptr;       // FP32 storage of TF32-rounded values
  __nv_bfloat16 *mbf16 = nullptr;
  // BF16 tensor-core copy: core k as [Mp][Kp] (rows 2b+i, columns 2a+j,
  // zero padded to multiples of 16) at element offset moff[k]; only for
  // cores whose ranks are <= 64 (mp[k] = 0 otherwise).
  __nv_bfloat16 *mma_bf16 = nullptr;
  std::vector<int64_t> moff;
  std::vector<int> mp, kp;
  // TF32 tensor-core copies for the tcgen05 pair kernel, TF32-rounded: core k
  // as the first step of a pair, [128][2 r_k rounded up to 8] (rows 2b+i,
  // zero past 2 r_{k+1}; columns 2a+j) at element offset toff[k], and as the
  // second, [80][2 r'] with r' = r_k rounded up to 4 (rows 2b+i, zero past
  // 2 r_{k+1}; columns j r' + a) at t2off[k]; only for 8 <= r_k <= 40 and
  // r_{k+1} <= 40 (-1 otherwise).
  float *mma_tf32 = nullptr;
  std::vector<int64_t> toff, t2off;
  // Reduced-precision packing [a][j][b padded to rpad[k+1]][i]:
  std::vector<int> rpad;        // padded output rank per core (index k+1)
  std::vector<int64_t> offlp;   // element offset of core k
  int64_t nlp = 0;              // total packed elements
  // Host copies of cores 0..2 for the head kernel, per reduced precision
  // (F32, TF32, BF16), [k][2a + j][b][i] with 16 x 8 x 2 floats per core;
  // empty when the first ranks are too large.
  std::vector<float> head[3];
  // The same for the last three cores (d-3, d-2, d-1 as slots 0, 1, 2), for
  // the tail kernel.
  std::vector<float> tail[3];
  // Fusion plan per arithmetic (index = qtt_dtype).
  qtt::ApplyPlan plan[4];
  // Streams that have queued work reading the operator, each with an event
  // recorded after its latest use (see qtt::note_use).
  mutable std::mutex use_mu;
  mutable std::vector<std::pair<cudaStream_t, cudaEvent_t>> uses;
};

// One recorded apply (qtt_plan_*): the instantiated graph and how many of
// the library's kernels one replay launches.
struct qtt_plan {
  const qtt_op *op = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t launches = 0;
};

namespace qtt {

// FP64 core step (Algorithm 2, one k).  in/out rhs strides in elements.
struct StepF64 {
  const double *in;
  int64_t in_rhs_stride;
  double *out;
  int64_t out_rhs_stride;
  const double *M;  // packed core k
  int k, rin, rout;
  int64_t N;
  int64_t nrhs;
  // Epilogue of the last step (rout == 1), when `epi` is set:
  //   out = s_v v + s_u u + s_acc acc      (u, v may be NULL)
  // residual f - a x - K x: v = f, u = x, s_v = 1, s_u = -a, s_acc = -1;
  // operator a z + K z: u = z, s_u = a; accumulate y += K z: u = out.
  int epi;
  const double *u;
  const double *v;
  int64_t uv_rhs_stride;
  double s_acc, s_u, s_v;
};
cudaError_t launch_step_f64(const StepF64 &s, cudaStream_t stream);

// Grouped FP64 steps (the serving loop): one launch runs one step each of
// several operators.  A descriptor holds the step, whether it takes the
// split-sum form (f64_step_small, the same choice launch_step_f64 makes),
// its first CTA and its CTAs per right-hand side; descriptors are ordered by
// cta0 and the table lives in device memory.
struct GroupedStepF64 {
  StepF64 s;
  int small;
  int64_t cta0, ctas_per_rhs;
};
bool f64_step_small(int64_t N, int rout);
int64_t f64_step_ctas_per_rhs(const StepF64 &s, bool small);
cudaError_t launch_step_f64_grouped(const GroupedStepF64 *dev_table, int n, int64_t total_ctas,
                                    cudaStream_t stream);

// Epilogue request for a whole apply (applies to its last step).
struct Epilogue {
  bool on = false;
  const double *u = nullptr;
  const double *v = nullptr;
  double s_acc = 1.0, s_u = 0.0, s_v = 0.0;
};

// Reduced-precision apply (compute = QTT_F32 / QTT_TF32 / QTT_BF16); x of
// type xt, y of type yt; epilogue on the last step: y = s_acc acc + s_u u.
struct LpEpilogue {
  bool on = false;
  const void *u = nullptr;
  const void *v = nullptr;
  double s_acc = 1.0, s_u = 0.0, s_v = 0.0;
};
qtt_status apply_lp(const qtt_op *A, qtt_dtype compute, const void *x, qtt_dtype xt, void *y,
                    qtt_dtype yt, int64_t nrhs, int64_t ld, cudaStream_t st,
                    const LpEpilogue &epi);
#ifdef QTT_CHECKED
cudaError_t launch_check_selftest(cudaStream_t st);
#endif

// Number of step pairs a TF32 apply of A runs on the tcgen05 tensor cores
// under its current plan (0 when none: no TF32 tensor-core copy, fusion or
// pairs off, or no eligible pair).
int tf32_tc_pairs(const qtt_op *A);

// FP64 apply of A to nrhs vectors (ld = leading dimension of x and y) with
// an optional epilogue; scratch from the pool.  Host-side, asynchronous.
qtt_status apply_f64(const qtt_op *A, const double *x, double *y, int64_t nrhs, int64_t ld,
                     cudaStream_t st, const Epilogue &epi);

}  // namespace qtt
