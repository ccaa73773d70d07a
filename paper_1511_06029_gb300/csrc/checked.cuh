// The checked build (compiled with -DQTT_CHECKED; a second library,
// libqtt_checked.so, next to the normal one).  compute-sanitizer is not
// available where the library runs, so the kernels check their own derived
// indices instead: QTT_CK(i, n, site) is i when 0 <= i < n; otherwise it
// records `site` in this file's device status word and yields 0, a valid
// index, so the access that follows stays in bounds and no control flow
// changes (no thread leaves a barrier, nothing faults).  qtt_sync_status
// reads and clears every file's word and returns QTT_ERR_CHECK with the
// first site.  In the normal build QTT_CK(i, n, site) is just i.
//
// Sites: 1xx FP64 steps, 2xx reduced-precision steps (lp, staged, head,
// tail), 3xx tensor-core pairs, 4xx batch, 5xx self-test.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace qtt {
// Registers a reader of one translation unit's status word (host side; the
// library's qtt_sync_status calls every registered reader).
bool register_check_word(cudaError_t (*take)(int *site));
}  // namespace qtt

#ifdef QTT_CHECKED
namespace {
__device__ int g_qtt_check_word = 0;  // one per translation unit
__device__ __forceinline__ int64_t qtt_ck(int64_t i, int64_t n, int site) {
  if (i >= 0 && i < n) return i;
  atomicCAS(&g_qtt_check_word, 0, site);
  return 0;
}
cudaError_t qtt_check_take(int *site) {
  int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(site, g_qtt_check_word, sizeof(int));
  if (e == cudaSuccess && *site != 0) e = cudaMemcpyToSymbol(g_qtt_check_word, &zero, sizeof(int));
  return e;
}
const bool g_qtt_check_registered = qtt::register_check_word(&qtt_check_take);
}  // namespace
#define QTT_CK(i, n, site) qtt_ck((int64_t)(i), (int64_t)(n), (site))
#else
#define QTT_CK(i, n, site) (i)
#endif
