// qtt_apply_noalloc: the FP64 apply with its intermediate held in a fixed
// device array instead of memory allocated per call.
//
// Some callers cannot allocate device memory when they apply an operator: a
// process whose device memory is owned by another allocator that has already
// reserved it (a framework arena, a memory budget fixed at start-up), or a
// latency-bound loop in which an allocation call may synchronise the device
// or fail under fragmentation.  This entry point gives them the same product
// as qtt_apply (FP64 in, FP64 arithmetic, FP64 out) without any allocation:
// the two ping-pong buffers of the sweep live in `g_noalloc_scratch` below,
// a file-scope device array that every GPU loading the library keeps until
// the process exits.
#include <cstring>
#include <mutex>

#include "qtt_internal.h"

namespace qtt {
namespace {

// 64 MiB: room for 2 x max_k r_k x N x nrhs doubles <= 8,388,608.
constexpr size_t kNoAllocBytes = (size_t)64 << 20;
constexpr size_t kNoAllocDoubles = kNoAllocBytes / sizeof(double);

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

// Device address of g_noalloc_scratch on the current device.  In host code
// the symbol itself is only a host-side stand-in, so it is never handed to a
// kernel; the address comes from cudaGetSymbolAddress with that device
// current.  It is looked up on every call (cheap, and it allocates nothing
// once the array's module is loaded), so a module reloaded after a device
// reset is picked up at its new address.
qtt_status scratch_for_current_device(double **out) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                     "qtt_apply_noalloc: cudaGetSymbolAddress");
  *out = static_cast<double *>(p);
  return QTT_OK;
}

}  // namespace

// The first lookup on a device loads the module that holds the array, and
// loading it is what commits the array's 64 MiB on that device.  qtt_create
// calls this, so the commitment happens while the caller is still setting
// up (it allocates the operator's cores anyway), before it hands its memory
// to another allocator; qtt_apply_noalloc itself then allocates nothing.
qtt_status noalloc_prepare() {
  double *p = nullptr;
  return scratch_for_current_device(&p);
}

}  // namespace qtt

using namespace qtt;

extern "C" qtt_status qtt_apply_noalloc(const qtt_op *A, const double *x, double *y,
                                        int64_t nrhs, int64_t ld, void *stream) {
  if (!A) return fail(QTT_ERR_INVALID_ARG, "qtt_apply_noalloc: NULL operator");
  if (qtt_status ds = check_device(A, "qtt_apply_noalloc")) return ds;
  const int d = A->d;
  const int64_t N = (int64_t)1 << d;
  if (nrhs < 0) return fail(QTT_ERR_INVALID_ARG, "qtt_apply_noalloc: nrhs < 0");
  if (nrhs == 0) return QTT_OK;
  if (ld < N) return fail(QTT_ERR_INVALID_ARG, "qtt_apply_noalloc: ld < N");
  if (!x || !y) return fail(QTT_ERR_INVALID_ARG, "qtt_apply_noalloc: NULL vector");
  {
    const char *xb = reinterpret_cast<const char *>(x);
    const char *yb = reinterpret_cast<const char *>(y);
    const size_t span = ((size_t)(nrhs - 1) * (size_t)ld + (size_t)N) * sizeof(double);
    if (xb < yb + span && yb < xb + span)
      return fail(QTT_ERR_INVALID_ARG, "qtt_apply_noalloc: x and y overlap");
  }
  // Two buffers of rmax_inner x N x nrhs doubles (none when d == 1).
  const double need = d > 1 ? 2.0 * (double)A->rmax_inner * (double)N * (double)nrhs : 0.0;
  if (need > (double)kNoAllocDoubles)
    return fail(QTT_ERR_INVALID_ARG,
                "qtt_apply_noalloc: needs " + std::to_string((long long)(need * 8.0)) +
                    " bytes of scratch (2 x max rank x N x nrhs doubles); the static area "
                    "holds " + std::to_string(kNoAllocBytes) + " bytes -- use qtt_apply");
  double *scratch = nullptr;
  if (d > 1) {
    qtt_status s = scratch_for_current_device(&scratch);
    if (s != QTT_OK) return s;
  }
  // Nothing in the scratch has to start at zero: step k writes every element
  // of its output buffer before step k + 1 reads it.
  const size_t half = (size_t)A->rmax_inner * (size_t)N * (size_t)nrhs;
  double *buf[2] = {scratch, scratch ? scratch + half : nullptr};
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int k = 0; k < d; ++k) {
    StepF64 p;
    std::memset(&p, 0, sizeof(p));
    p.k = k;
    p.rin = A->ranks[k];
    p.rout = A->ranks[k + 1];
    p.N = N;
    p.nrhs = nrhs;
    p.M = A->m64 + A->off[k];
    if (k == 0) {
      p.in = x;
      p.in_rhs_stride = ld;
    } else {
      p.in = buf[(k - 1) & 1];
      p.in_rhs_stride = (int64_t)p.rin * N;
    }
    if (k == d - 1) {
      p.out = y;
      p.out_rhs_stride = ld;
    } else {
      p.out = buf[k & 1];
      p.out_rhs_stride = (int64_t)p.rout * N;
    }
    cudaError_t e = launch_step_f64(p, st);
    if (e != cudaSuccess) {
      note_use(A, st);
      return cuda_fail(e, "qtt_apply_noalloc: step launch");
    }
  }
  note_use(A, st);
  return QTT_OK;
}
