// qtt_apply_host: y = A x with x and y in host memory.
//
// The copies are part of the product here: a caller whose vectors live on
// the host pays for moving them, so the right-hand sides go through the
// device in chunks and the copy of chunk i+1 in, the apply of chunk i and
// the copy of chunk i-1 out overlap.  Two staging slots (x and y of one
// chunk each, compact leading dimension N) come from the library's
// stream-ordered pool; the applies run on the caller's stream, the copies
// on two streams the library keeps per device, and events order the three:
//
//   copy-in  of chunk i  waits for the apply  of chunk i-2 (its x slot),
//   apply    of chunk i  waits for copy-in  i and copy-out i-2 (its y slot),
//   copy-out of chunk i  waits for the apply  of chunk i.
//
// Each right-hand side's apply is independent of the others, and qtt_apply
// gives a right-hand side the same bits whatever its neighbours, so the
// result is bitwise qtt_apply's on the same vectors.
#include <cuda_runtime.h>

#include <mutex>

#include "qtt_internal.h"

namespace qtt {
namespace {

constexpr int kMaxDevices = 64;
constexpr size_t kStagingBudget = (size_t)1 << 30;  // both slots, x and y

}  // namespace

// The copy streams of the current device, created on first use and kept
// until the process ends.
qtt_status copy_streams(CopyStreams *cs) {
  static std::mutex mu;
  static CopyStreams per_device[kMaxDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "host copy streams: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices)
    return fail(QTT_ERR_UNSUPPORTED, "host copy streams: device index above 63");
  std::lock_guard<std::mutex> lock(mu);
  CopyStreams &c = per_device[dev];
  if (!c.in) {
    e = cudaStreamCreateWithFlags(&c.in, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "host copy streams: cudaStreamCreate");
    e = cudaStreamCreateWithFlags(&c.out, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      cudaStreamDestroy(c.in);
      c.in = nullptr;
      return cuda_fail(e, "host copy streams: cudaStreamCreate");
    }
  }
  *cs = c;
  return QTT_OK;
}

namespace {

size_t io_size(qtt_dtype t) { return t == QTT_F64 ? 8 : (t == QTT_BF16 ? 2 : 4); }

// Rows r0 .. r0 + n - 1 (right-hand sides) between a host array of leading
// dimension ld and a compact device array (leading dimension N).
cudaError_t copy_rows(void *dst, size_t dpitch, const void *src, size_t spitch, size_t width,
                      int64_t n, cudaMemcpyKind kind, cudaStream_t st) {
  return cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, (size_t)n, kind, st);
}

}  // namespace
}  // namespace qtt

using namespace qtt;

extern "C" qtt_status qtt_apply_host(const qtt_op *A, const void *x_host, void *y_host,
                                     int64_t nrhs, int64_t ld, qtt_dtype io_dtype,
                                     qtt_dtype compute, int64_t chunk, void *stream) {
  if (!A) return fail(QTT_ERR_INVALID_ARG, "qtt_apply_host: NULL operator");
  if (nrhs < 0) return fail(QTT_ERR_INVALID_ARG, "qtt_apply_host: nrhs < 0");
  if (chunk < 0) return fail(QTT_ERR_INVALID_ARG, "qtt_apply_host: chunk < 0");
  if (io_dtype != QTT_F64 && io_dtype != QTT_F32 && io_dtype != QTT_BF16)
    return fail(QTT_ERR_INVALID_ARG, "qtt_apply_host: io_dtype must be F64, F32 or BF16");
  if (nrhs == 0) return QTT_OK;
  const int64_t N = (int64_t)1 << qtt_op_d(A);
  if (ld < N) return fail(QTT_ERR_INVALID_ARG, "qtt_apply_host: ld < N");
  if (!x_host || !y_host) return fail(QTT_ERR_INVALID_ARG, "qtt_apply_host: NULL vector");
  const size_t esz = io_size(io_dtype);
  {
    const char *xb = static_cast<const char *>(x_host);
    const char *yb = static_cast<const char *>(y_host);
    const size_t span = ((size_t)(nrhs - 1) * (size_t)ld + (size_t)N) * esz;
    if (xb < yb + span && yb < xb + span)
      return fail(QTT_ERR_INVALID_ARG, "qtt_apply_host: x and y overlap");
  }
  if (qtt_status ds = check_device(A, "qtt_apply_host")) return ds;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t row = (size_t)N * esz;  // one right-hand side, compact
  const size_t hpitch = (size_t)ld * esz;

  // chunk: given, else a quarter of the right-hand sides within the budget
  int64_t per = chunk;
  if (per == 0) per = nrhs >= 4 ? (nrhs + 3) / 4 : nrhs;
  const int64_t fit = (int64_t)(kStagingBudget / (4 * row));
  if (per > fit) per = fit < 1 ? 1 : fit;
  if (per > nrhs) per = nrhs;
  const int64_t nchunks = (nrhs + per - 1) / per;
  const int slots = nchunks > 1 ? 2 : 1;

  void *stage = nullptr;
  qtt_status s = scratch_alloc(&stage, (size_t)slots * 2 * (size_t)per * row, st);
  if (s != QTT_OK) return s;
  auto xslot = [&](int64_t i) {
    return static_cast<char *>(stage) + (size_t)(i % slots) * 2 * (size_t)per * row;
  };
  auto yslot = [&](int64_t i) { return xslot(i) + (size_t)per * row; };
  const char *xh = static_cast<const char *>(x_host);
  char *yh = static_cast<char *>(y_host);

  if (nchunks == 1) {
    // everything on the caller's stream
    cudaError_t e = copy_rows(xslot(0), row, xh, hpitch, row, nrhs, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      scratch_free(stage, st);
      return cuda_fail(e, "qtt_apply_host: copy in");
    }
    s = qtt_apply(A, xslot(0), yslot(0), nrhs, N, io_dtype, compute, st);
    if (s == QTT_OK) {
      e = copy_rows(yh, hpitch, yslot(0), row, row, nrhs, cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) s = cuda_fail(e, "qtt_apply_host: copy out");
    }
    scratch_free(stage, st);
    return s;
  }

  CopyStreams cs;
  s = copy_streams(&cs);
  if (s != QTT_OK) {
    scratch_free(stage, st);
    return s;
  }
  // events per slot: copied in, applied, copied out; plus the start
  cudaEvent_t ev_in[2] = {}, ev_app[2] = {}, ev_out[2] = {}, ev_start = nullptr;
  cudaError_t e = cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = cudaEventCreateWithFlags(&ev_in[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_app[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_out[k], cudaEventDisableTiming);
  }
  // the staging memory is the caller's stream's from here on
  if (e == cudaSuccess) e = cudaEventRecord(ev_start, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs.in, ev_start, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs.out, ev_start, 0);
  for (int64_t i = 0; i < nchunks && e == cudaSuccess && s == QTT_OK; ++i) {
    const int k = (int)(i % 2);
    const int64_t r0 = i * per;
    const int64_t n = nrhs - r0 < per ? nrhs - r0 : per;
    // copy in (the slot's previous apply must be done with its x)
    if (i >= 2) e = cudaStreamWaitEvent(cs.in, ev_app[k], 0);
    if (e == cudaSuccess)
      e = copy_rows(xslot(i), row, xh + (size_t)r0 * hpitch, hpitch, row, n,
                    cudaMemcpyHostToDevice, cs.in);
    if (e == cudaSuccess) e = cudaEventRecord(ev_in[k], cs.in);
    // apply (the slot's previous copy-out must be done with its y)
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev_in[k], 0);
    if (e == cudaSuccess && i >= 2) e = cudaStreamWaitEvent(st, ev_out[k], 0);
    if (e != cudaSuccess) break;
    s = qtt_apply(A, xslot(i), yslot(i), n, N, io_dtype, compute, st);
    if (s != QTT_OK) break;
    e = cudaEventRecord(ev_app[k], st);
    // copy out
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs.out, ev_app[k], 0);
    if (e == cudaSuccess)
      e = copy_rows(yh + (size_t)r0 * hpitch, hpitch, yslot(i), row, row, n,
                    cudaMemcpyDeviceToHost, cs.out);
    if (e == cudaSuccess) e = cudaEventRecord(ev_out[k], cs.out);
  }
  // the caller's stream ends after every copy (also on an error: nothing
  // may still use the staging memory when it returns to the pool)
  cudaEvent_t tail_in = nullptr, tail_out = nullptr;
  cudaError_t e2 = cudaEventCreateWithFlags(&tail_in, cudaEventDisableTiming);
  if (e2 == cudaSuccess) e2 = cudaEventCreateWithFlags(&tail_out, cudaEventDisableTiming);
  if (e2 == cudaSuccess) e2 = cudaEventRecord(tail_in, cs.in);
  if (e2 == cudaSuccess) e2 = cudaEventRecord(tail_out, cs.out);
  if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(st, tail_in, 0);
  if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(st, tail_out, 0);
  if (e2 != cudaSuccess) {
    // the ordering could not be expressed: wait for the copies on the host
    cudaStreamSynchronize(cs.in);
    cudaStreamSynchronize(cs.out);
  }
  scratch_free(stage, st);
  for (cudaEvent_t ev : {ev_start, ev_in[0], ev_in[1], ev_app[0], ev_app[1], ev_out[0], ev_out[1],
                         tail_in, tail_out})
    if (ev) cudaEventDestroy(ev);  // released once their work completes
  if (s != QTT_OK) return s;
  if (e != cudaSuccess) return cuda_fail(e, "qtt_apply_host: pipelined copy");
  if (e2 != cudaSuccess) return cuda_fail(e2, "qtt_apply_host: final ordering");
  return QTT_OK;
}
