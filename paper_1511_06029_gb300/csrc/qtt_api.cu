// C-ABI of libqtt: operator lifetime, argument validation, scratch pool and
// dispatch of the apply to the kernels.
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "checked.cuh"
#include "qtt_internal.h"
#include "step_lp.h"
#include "step_mma.h"

namespace qtt {

static thread_local std::string g_last_error;

// Readers of the translation units' index-check words (the checked build;
// empty otherwise).  Filled by static initialisers, so constructed on first
// use.
static std::vector<cudaError_t (*)(int *)> &check_words() {
  static std::vector<cudaError_t (*)(int *)> w;
  return w;
}
bool register_check_word(cudaError_t (*take)(int *site)) {
  check_words().push_back(take);
  return true;
}

#ifdef QTT_CHECKED
// The self-test of the checked build: one index derived past its range on
// purpose (site 501); QTT_CK clamps it, so the store lands in bounds.
__device__ int g_check_selftest_cell[4];
__global__ void check_selftest_kernel(int over) {
  const int64_t i = QTT_CK(3 + over, 4, 501);
  g_check_selftest_cell[i] = 1;
}
cudaError_t launch_check_selftest(cudaStream_t st) {
  check_selftest_kernel<<<1, 1, 0, st>>>(1);
  count_launches(1);
  return cudaGetLastError();
}
#endif
static std::atomic<uint64_t> g_launches{0};

static thread_local uint64_t t_launches = 0;  // this thread's launches (plan recording)
void count_launches(uint64_t n) {
  g_launches.fetch_add(n, std::memory_order_relaxed);
  t_launches += n;
}

qtt_status fail(qtt_status s, const std::string &msg) {
  g_last_error = msg;
  return s;
}

qtt_status cuda_fail(cudaError_t e, const char *where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();  // allocation failures are not sticky; clear them
    return fail(QTT_ERR_OOM, m);
  }
  return fail(QTT_ERR_CUDA, m);
}

// ------------------------------------------------------------ scratch pool
namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64] = {};

cudaMemPool_t pool_for_current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
    uint64_t keep = UINT64_MAX;  // keep freed blocks for the next call
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pool[dev] = p;
  }
  return g_pool[dev];
}
}  // namespace

// Bytes the pool holds already reserved but unused (no driver query of free
// memory: cheap enough for every small apply).
static size_t scratch_cached() {
  cudaMemPool_t p = pool_for_current_device();
  if (!p) return 0;
  uint64_t reserved = 0, used = 0;
  cudaMemPoolGetAttribute(p, cudaMemPoolAttrReservedMemCurrent, &reserved);
  cudaMemPoolGetAttribute(p, cudaMemPoolAttrUsedMemCurrent, &used);
  return reserved > used ? (size_t)(reserved - used) : 0;
}

// Scratch accounting for the cap of qtt_set_scratch_limit: bytes of scratch
// handed out and not yet given back (all devices), and each block's size.
static std::mutex g_scratch_mu;
static std::unordered_map<void *, size_t> g_scratch_live;
static size_t g_scratch_in_use = 0;
static std::atomic<size_t> g_scratch_cap{0};  // 0 = no cap

// What the cap leaves (SIZE_MAX without a cap).
static size_t scratch_cap_room() {
  const size_t cap = g_scratch_cap.load(std::memory_order_relaxed);
  if (!cap) return SIZE_MAX;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  return cap > g_scratch_in_use ? cap - g_scratch_in_use : 0;
}

size_t scratch_available() {
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return 0;
  const size_t cached = scratch_cached();
  // Leave a margin for the driver and other allocators in the process.
  const size_t margin = (size_t)512 << 20;
  const size_t avail = free_b > margin ? free_b - margin + cached : cached;
  return std::min(avail, scratch_cap_room());
}

size_t scratch_available_at_least(size_t bytes) {
  const size_t cached = std::min(scratch_cached(), scratch_cap_room());
  return cached >= bytes ? cached : scratch_available();
}

qtt_status scratch_alloc(void **ptr, size_t bytes, cudaStream_t stream) {
  *ptr = nullptr;
  if (bytes == 0) return QTT_OK;
  cudaMemPool_t p = pool_for_current_device();
  if (!p) return fail(QTT_ERR_CUDA, "cannot create the scratch memory pool");
  if (bytes > scratch_available_at_least(bytes))
    return fail(QTT_ERR_OOM, "scratch of " + std::to_string(bytes) +
                                 " bytes exceeds free device memory (or the scratch limit)");
  cudaError_t e = cudaMallocFromPoolAsync(ptr, bytes, p, stream);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    return cuda_fail(e, "cudaMallocFromPoolAsync");
  }
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  g_scratch_live[*ptr] = bytes;
  g_scratch_in_use += bytes;
  return QTT_OK;
}

void scratch_free(void *ptr, cudaStream_t stream) {
  if (!ptr) return;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    auto it = g_scratch_live.find(ptr);
    if (it != g_scratch_live.end()) {
      g_scratch_in_use -= it->second;
      g_scratch_live.erase(it);
    }
  }
  cudaFreeAsync(ptr, stream);
}

// ----------------------------------------------------- long-lived buffers
qtt_status persistent_alloc(void **ptr, size_t bytes, cudaStream_t stream) {
  *ptr = nullptr;
  if (bytes == 0) return QTT_OK;
  cudaMemPool_t p = pool_for_current_device();
  if (!p) return fail(QTT_ERR_CUDA, "cannot create the device memory pool");
  cudaError_t e = cudaMallocFromPoolAsync(ptr, bytes, p, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    if (*ptr) cudaFreeAsync(*ptr, stream);
    *ptr = nullptr;
    return cuda_fail(e, "persistent allocation");
  }
  return QTT_OK;
}

namespace {
std::mutex g_release_mu;
cudaStream_t g_release[64] = {};

cudaStream_t release_stream_for_current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_release_mu);
  if (!g_release[dev]) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    g_release[dev] = s;
  }
  return g_release[dev];
}
}  // namespace

void release_after(const std::vector<void *> &ptrs, const std::vector<cudaEvent_t> &after) {
  cudaStream_t rs = release_stream_for_current_device();
  bool ordered = rs != nullptr;
  for (cudaEvent_t ev : after)
    if (ordered && cudaStreamWaitEvent(rs, ev, 0) != cudaSuccess) ordered = false;
  if (!ordered) {
    // no release stream: wait on the host for the recorded uses instead
    for (cudaEvent_t ev : after) cudaEventSynchronize(ev);
    if (!rs) cudaDeviceSynchronize();
  }
  for (void *p : ptrs)
    if (p) cudaFreeAsync(p, rs);
}

void note_use(const qtt_op *A, cudaStream_t stream) {
  if (!A) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return;
  }
  std::lock_guard<std::mutex> lk(A->use_mu);
  cudaEvent_t ev = nullptr;
  for (auto &u : A->uses)
    if (u.first == stream) ev = u.second;
  if (!ev) {
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    A->uses.emplace_back(stream, ev);
  }
  cudaEventRecord(ev, stream);
}

qtt_status check_device(const qtt_op *A, const char *where) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, where);
  if (dev != A->device)
    return fail(QTT_ERR_INVALID_ARG, std::string(where) + ": the operator lives on device " +
                                         std::to_string(A->device) + " but device " +
                                         std::to_string(dev) + " is current");
  return QTT_OK;
}

// Host copy of the device TF32 rounding: round to nearest even at 13 dropped
// mantissa bits (finite values).
static float host_tf32_rne(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) {
    u += 0x0fffu + ((u >> 13) & 1u);
    u &= 0xffffe000u;
  }
  std::memcpy(&x, &u, 4);
  return x;
}

// Records, on every exit of an apply, that the work it queued on `st` reads A.
struct UseGuard {
  const qtt_op *A;
  cudaStream_t st;
  ~UseGuard() { note_use(A, st); }
};

// ------------------------------------------------------------ validation
static bool valid_dtype(qtt_dtype t) {
  return t == QTT_F64 || t == QTT_F32 || t == QTT_TF32 || t == QTT_BF16;
}

// Apply of an FP64 operator, optionally with an epilogue on the last step.
qtt_status apply_f64(const qtt_op *A, const double *x, double *y, int64_t nrhs,
                     int64_t ld, cudaStream_t st, const Epilogue &epi) {
  const UseGuard use{A, st};
  const int d = A->d;
  const int64_t N = (int64_t)1 << d;
  // Scratch: two ping-pong buffers of rmax_inner x N per right-hand side.
  const size_t per_rhs = d > 1 ? (size_t)2 * A->rmax_inner * (size_t)N * sizeof(double) : 0;
  int64_t chunk = nrhs;
  if (per_rhs) {
    const size_t avail = scratch_available_at_least(per_rhs * (size_t)nrhs);
    const int64_t fit = (int64_t)(avail / per_rhs);
    if (fit < 1)
      return fail(QTT_ERR_OOM, "apply scratch for one right-hand side (" +
                                   std::to_string(per_rhs) + " bytes) does not fit");
    chunk = std::min<int64_t>(nrhs, fit);
  }
  void *scratch = nullptr;
  qtt_status s = scratch_alloc(&scratch, per_rhs * (size_t)chunk, st);
  if (s != QTT_OK) return s;
  double *buf[2] = {nullptr, nullptr};
  if (per_rhs) {
    buf[0] = static_cast<double *>(scratch);
    buf[1] = buf[0] + (size_t)A->rmax_inner * (size_t)N * (size_t)chunk;
  }
  for (int64_t c0 = 0; c0 < nrhs; c0 += chunk) {
    const int64_t nc = std::min<int64_t>(chunk, nrhs - c0);
    for (int k = 0; k < d; ++k) {
      StepF64 p;
      std::memset(&p, 0, sizeof(p));
      p.k = k;
      p.rin = A->ranks[k];
      p.rout = A->ranks[k + 1];
      p.N = N;
      p.nrhs = nc;
      p.M = A->m64 + A->off[k];
      if (k == 0) {
        p.in = x + c0 * ld;
        p.in_rhs_stride = ld;
      } else {
        p.in = buf[(k - 1) & 1];
        p.in_rhs_stride = (int64_t)p.rin * N;
      }
      if (k == d - 1) {
        p.out = y + c0 * ld;
        p.out_rhs_stride = ld;
        if (epi.on) {
          p.epi = 1;
          p.u = epi.u ? epi.u + c0 * ld : nullptr;
          p.v = epi.v ? epi.v + c0 * ld : nullptr;
          p.uv_rhs_stride = ld;
          p.s_acc = epi.s_acc;
          p.s_u = epi.s_u;
          p.s_v = epi.s_v;
        }
      } else {
        p.out = buf[k & 1];
        p.out_rhs_stride = (int64_t)p.rout * N;
      }
      cudaError_t e = launch_step_f64(p, st);
      if (e != cudaSuccess) {
        scratch_free(scratch, st);
        return cuda_fail(e, "step_f64 launch");
      }
    }
  }
  scratch_free(scratch, st);
  return QTT_OK;
}

// BF16 steps go to the tensor cores unless QTT_NO_TENSOR_CORES is set (kept
// for A/B measurements of the CUDA-core kernel).
static bool use_tensor_cores() {
  static const bool on = [] {
    const char *v = std::getenv("QTT_NO_TENSOR_CORES");
    return !(v && *v && *v != '0');
  }();
  return on;
}

// FP32/TF32 intermediate steps use the staged kernel unless
// QTT_NO_STAGED_F32 is set (kept for A/B measurements).
static bool use_staged_f32() {
  static const bool on = [] {
    const char *v = std::getenv("QTT_NO_STAGED_F32");
    return !(v && *v && *v != '0');
  }();
  return on;
}

// Several steps per launch -- the head kernel for the first steps, pairs of
// tensor-core steps (QTT_NO_FUSION=1 keeps one launch per step, for
// comparison).
static bool use_fusion() {
  static const bool on = [] {
    const char *v = std::getenv("QTT_NO_FUSION");
    return !(v && *v && *v != '0');
  }();
  return on;
}

// Fused pairs run on the tcgen05 tensor cores (QTT_NO_TCGEN05=1 selects the
// mma.sync pair kernel instead, for comparison).
static bool use_tcgen05() {
  static const bool on = [] {
    const char *v = std::getenv("QTT_NO_TCGEN05");
    return !(v && *v && *v != '0');
  }();
  return on;
}

// Steps k and k+1 of a TF32 apply run as one tcgen05 pair (the middle
// steps k0 .. kend-1 are the ones outside the head and tail kernels).
static bool tf32_pair_at(const qtt_op *A, int k, int kend, int64_t N) {
  const int d = A->d;
  return A->mma_tf32 && use_tensor_cores() && use_tcgen05() && k >= 1 && k + 2 < d &&
         k + 1 < kend && A->toff[k] >= 0 && A->t2off[k + 1] >= 0 &&
         tc2f_steps_eligible(k, A->ranks[k], A->ranks[k + 1], A->ranks[k + 2], N);
}

static size_t dtype_size(qtt_dtype t) {
  return t == QTT_F64 ? 8 : (t == QTT_BF16 ? 2 : 4);
}

int tf32_tc_pairs(const qtt_op *A) {
  const ApplyPlan &pl = A->plan[QTT_TF32];
  if (!A->mtf32 || !A->mma_tf32 || !use_fusion() || !pl.fusion || pl.pairs != 2) return 0;
  const int d = A->d;
  const int64_t N = (int64_t)1 << d;
  const int hm = !A->head[1].empty() ? head_steps(A->ranks.data(), d) : 0;
  const int tm = !A->tail[1].empty() ? tail_steps(A->ranks.data(), d, hm) : 0;
  const int kend = d - tm;
  int n = 0;
  for (int k = hm; k < kend; ++k)
    if (tf32_pair_at(A, k, kend, N)) {
      ++n;
      ++k;
    }
  return n;
}

qtt_status apply_lp(const qtt_op *A, qtt_dtype compute, const void *x, qtt_dtype xt, void *y,
                    qtt_dtype yt, int64_t nrhs, int64_t ld, cudaStream_t st,
                    const LpEpilogue &epi) {
  const UseGuard use{A, st};
  int mode;
  const void *cores;
  switch (compute) {
    case QTT_F32: mode = LP_F32; cores = A->m32; break;
    case QTT_TF32: mode = LP_TF32; cores = A->mtf32; break;
    case QTT_BF16: mode = LP_BF16; cores = A->mbf16; break;
    default: return fail(QTT_ERR_INVALID_ARG, "apply_lp: compute must be F32, TF32 or BF16");
  }
  if (!cores)
    return fail(QTT_ERR_INVALID_ARG,
                "apply: operator was created without the packed copy for this precision "
                "(QTT_PACK_* bit missing)");
  const qtt_dtype mid = compute == QTT_BF16 ? QTT_BF16 : QTT_F32;
  const size_t esz = dtype_size(mid);
  const size_t core_esz = compute == QTT_BF16 ? 2 : 4;
  const int d = A->d;
  const int64_t N = (int64_t)1 << d;
  const size_t per_rhs = d > 1 ? (size_t)2 * A->rmax_inner * (size_t)N * esz : 0;
  int64_t chunk = nrhs;
  if (per_rhs) {
    const int64_t fit = (int64_t)(scratch_available_at_least(per_rhs * (size_t)nrhs) / per_rhs);
    if (fit < 1)
      return fail(QTT_ERR_OOM, "apply scratch for one right-hand side does not fit");
    chunk = std::min<int64_t>(nrhs, fit);
  }
  void *scratch = nullptr;
  qtt_status s = scratch_alloc(&scratch, per_rhs * (size_t)chunk, st);
  if (s != QTT_OK) return s;
  char *buf[2] = {nullptr, nullptr};
  if (per_rhs) {
    buf[0] = static_cast<char *>(scratch);
    buf[1] = buf[0] + (size_t)A->rmax_inner * (size_t)N * (size_t)chunk * esz;
  }
  const size_t xsz = dtype_size(xt), ysz = dtype_size(yt);
  const ApplyPlan &pl = A->plan[compute];
  const bool fuse = use_fusion() && pl.fusion;
  const bool tc = compute == QTT_BF16 && use_tensor_cores() && A->mma_bf16;
  for (int64_t c0 = 0; c0 < nrhs; c0 += chunk) {
    const int64_t nc = std::min<int64_t>(chunk, nrhs - c0);
    int src = 0;  // scratch half holding the current intermediate (k >= 1)
    int k0 = 0;
    const int mi = mode == LP_F32 ? 0 : mode == LP_TF32 ? 1 : 2;
    const std::vector<float> &hcores = A->head[mi];
    const int hm = fuse && !hcores.empty() ? head_steps(A->ranks.data(), d) : 0;
    const int tm = fuse && !A->tail[mi].empty() ? tail_steps(A->ranks.data(), d, hm) : 0;
    const int kend = d - tm;  // steps k0 .. kend-1 here, kend .. d-1 in the tail kernel
    if (hm) {
      // steps 0 .. hm-1 in one launch; y_hm lands in scratch half 0
      StepHead h;
      std::memset(&h, 0, sizeof(h));
      h.in = static_cast<const char *>(x) + (size_t)c0 * ld * xsz;
      h.in_rhs_stride = ld;
      h.out = buf[0];
      h.out_rhs_stride = (int64_t)A->ranks[hm] * N;
      std::memcpy(h.G, hcores.data(), sizeof(h.G));
      for (int k = 0; k <= hm; ++k) h.r[k] = A->ranks[k];
      h.N = N;
      h.nrhs = nc;
      h.m = hm;
      h.mode = mode;
      h.in_type = xt;
      const cudaError_t e = launch_step_head(h, st);
      if (e != cudaSuccess) {
        scratch_free(scratch, st);
        return cuda_fail(e, "head step launch");
      }
      k0 = hm;
    }
    for (int k = k0; k < kend; ++k) {
      // TF32: steps k and k+1 on the tcgen05 tensor cores (kind::tf32)
      if (compute == QTT_TF32 && fuse && pl.pairs == 2 && tf32_pair_at(A, k, kend, N)) {
        StepTF2 t;
        t.in = reinterpret_cast<const float *>(buf[src]);
        t.in_rhs_stride = (int64_t)A->ranks[k] * N;
        t.out = reinterpret_cast<float *>(buf[src ^ 1]);
        t.out_rhs_stride = (int64_t)A->ranks[k + 2] * N;
        t.A1 = A->mma_tf32 + A->toff[k];
        t.A2 = A->mma_tf32 + A->t2off[k + 1];
        t.k = k;
        t.r0 = A->ranks[k];
        t.r1 = A->ranks[k + 1];
        t.r2 = A->ranks[k + 2];
        t.N = N;
        t.nrhs = nc;
        const cudaError_t e = launch_step_tc2_tf32(t, st);
        if (e == cudaSuccess) {
          src ^= 1;
          ++k;
          continue;
        }
        if (e != cudaErrorNotSupported) {
          scratch_free(scratch, st);
          return cuda_fail(e, "TF32 tensor-core step launch");
        }
        cudaGetLastError();  // nothing was launched: the steps run one by one
      }
      const bool pair = tc && fuse && pl.pairs > 0 && k + 2 < d && k + 1 < kend && A->mp[k] &&
                        A->mp[k + 1];
      const bool tc5 = pair && use_tcgen05() && pl.pairs == 2 &&
                       tc2_steps_eligible(k, A->ranks[k], A->ranks[k + 1], A->ranks[k + 2], N);
      const bool mma2 =
          pair && mma2_steps_eligible(k, A->ranks[k], A->ranks[k + 1], A->ranks[k + 2], N);
      if (tc5 || mma2) {
        // steps k and k+1 in one launch; y_{k+2} lands in the other half
        StepMMA2 m;
        m.in = reinterpret_cast<const __nv_bfloat16 *>(buf[src]);
        m.in_rhs_stride = (int64_t)A->ranks[k] * N;
        m.out = reinterpret_cast<__nv_bfloat16 *>(buf[src ^ 1]);
        m.out_rhs_stride = (int64_t)A->ranks[k + 2] * N;
        m.A1 = A->mma_bf16 + A->moff[k];
        m.A2 = A->mma_bf16 + A->moff[k + 1];
        m.k = k;
        m.r0 = A->ranks[k];
        m.r1 = A->ranks[k + 1];
        m.r2 = A->ranks[k + 2];
        m.Mp1 = A->mp[k];
        m.Kp1 = A->kp[k];
        m.Mp2 = A->mp[k + 1];
        m.N = N;
        m.nrhs = nc;
        m.groups_cap = pl.groups_cap;
        cudaError_t e = cudaErrorNotSupported;
        if (tc5) e = launch_step_tc2_bf16(m, st);
        if (e == cudaErrorNotSupported && mma2) e = launch_step_mma2_bf16(m, st);
        if (e == cudaErrorNotSupported) {
          cudaGetLastError();  // nothing was launched: run the two steps one by one
          goto single_step;
        }
        if (e != cudaSuccess) {
          scratch_free(scratch, st);
          return cuda_fail(e, "fused tensor-core step launch");
        }
        src ^= 1;
        ++k;
        continue;
      }
    single_step:
      StepLP p;
      std::memset(&p, 0, sizeof(p));
      p.k = k;
      p.rin = A->ranks[k];
      p.rout = A->ranks[k + 1];
      p.rout_pad = A->rpad[k + 1];
      p.N = N;
      p.nrhs = nc;
      p.mode = mode;
      p.M = static_cast<const char *>(cores) + (size_t)A->offlp[k] * core_esz;
      if (k == 0) {
        p.in = static_cast<const char *>(x) + (size_t)c0 * ld * xsz;
        p.in_rhs_stride = ld;
        p.in_type = xt;
      } else {
        p.in = buf[src];
        p.in_rhs_stride = (int64_t)p.rin * N;
        p.in_type = mid;
      }
      if (k == d - 1) {
        p.out = static_cast<char *>(y) + (size_t)c0 * ld * ysz;
        p.out_rhs_stride = ld;
        p.out_type = yt;
        if (epi.on) {
          p.epi = 1;
          p.u = epi.u ? static_cast<const char *>(epi.u) + (size_t)c0 * ld * ysz : nullptr;
          p.v = epi.v ? static_cast<const char *>(epi.v) + (size_t)c0 * ld * ysz : nullptr;
          p.u_rhs_stride = ld;
          p.s_acc = epi.s_acc;
          p.s_u = epi.s_u;
          p.s_v = epi.s_v;
        }
      } else {
        p.out = buf[k == 0 ? 0 : src ^ 1];
        p.out_rhs_stride = (int64_t)p.rout * N;
        p.out_type = mid;
        p.round_tf32_out = mode == LP_TF32;
      }
      cudaError_t e;
      if (tc && A->mp[k] &&
          p.in_type == QTT_BF16 && p.out_type == QTT_BF16 && !p.epi &&
          mma_step_eligible(k, p.rin, p.rout, N)) {
        StepMMA m;
        m.in = static_cast<const __nv_bfloat16 *>(p.in);
        m.in_rhs_stride = p.in_rhs_stride;
        m.out = static_cast<__nv_bfloat16 *>(p.out);
        m.out_rhs_stride = p.out_rhs_stride;
        m.A = A->mma_bf16 + A->moff[k];
        m.k = k;
        m.rin = p.rin;
        m.rout = p.rout;
        m.Mp = A->mp[k];
        m.Kp = A->kp[k];
        m.N = N;
        m.nrhs = nc;
        e = launch_step_mma_bf16(m, st);
      } else if (use_staged_f32() && pl.staged && f32s_step_eligible(p)) {
        e = launch_step_f32s(p, st);
      } else {
        e = launch_step_lp(p, st);
      }
      if (e != cudaSuccess) {
        scratch_free(scratch, st);
        return cuda_fail(e, "step_lp launch");
      }
      if (k > 0) src ^= 1;
    }
    if (tm) {
      // steps kend .. d-1 in one launch: y_kend -> y (with the epilogue)
      StepTail t;
      std::memset(&t, 0, sizeof(t));
      t.in = buf[src];
      t.in_rhs_stride = (int64_t)A->ranks[kend] * N;
      t.out = static_cast<char *>(y) + (size_t)c0 * ld * ysz;
      t.out_rhs_stride = ld;
      for (int s2 = 0; s2 <= tm; ++s2) t.r[s2] = A->ranks[kend + s2];
      t.N = N;
      t.nrhs = nc;
      t.k0 = kend;
      t.m = tm;
      t.mode = mode;
      t.out_type = yt;
      if (epi.on) {
        t.epi = 1;
        t.u = epi.u ? static_cast<const char *>(epi.u) + (size_t)c0 * ld * ysz : nullptr;
        t.v = epi.v ? static_cast<const char *>(epi.v) + (size_t)c0 * ld * ysz : nullptr;
        t.u_rhs_stride = ld;
        t.s_acc = epi.s_acc;
        t.s_u = epi.s_u;
        t.s_v = epi.s_v;
      }
      // cores kend .. d-1 are slots 3 - tm .. 2 of the tail copy
      std::memcpy(t.G, A->tail[mi].data() + (size_t)(3 - tm) * 16 * 8 * 2,
                  sizeof(float) * (size_t)tm * 16 * 8 * 2);
      const cudaError_t e = launch_step_tail(t, st);
      if (e != cudaSuccess) {
        scratch_free(scratch, st);
        return cuda_fail(e, "tail step launch");
      }
    }
  }
  scratch_free(scratch, st);
  return QTT_OK;
}

}  // namespace qtt

using namespace qtt;

// ================================================================== C-ABI
extern "C" {

const char *qtt_status_string(qtt_status s) {
  switch (s) {
    case QTT_OK: return "ok";
    case QTT_ERR_INVALID_ARG: return "invalid argument";
    case QTT_ERR_OOM: return "out of device memory";
    case QTT_ERR_CUDA: return "CUDA error";
    case QTT_ERR_NOT_CONVERGED: return "not converged";
    case QTT_ERR_TIMEOUT: return "device wait timed out";
    case QTT_ERR_UNSUPPORTED: return "unsupported combination";
    case QTT_ERR_CHECK: return "checked build: a kernel met an out-of-range index";
  }
  return "unknown status";
}

const char *qtt_last_error(void) { return g_last_error.c_str(); }

uint64_t qtt_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

qtt_status qtt_create(qtt_op **out, int d, const int *ranks, const double *const *cores,
                      unsigned precision_mask, void *stream) {
  if (!out) return fail(QTT_ERR_INVALID_ARG, "qtt_create: out is NULL");
  *out = nullptr;
  if (d < 1 || d > 30) return fail(QTT_ERR_INVALID_ARG, "qtt_create: d must be in [1, 30]");
  if (!ranks || !cores) return fail(QTT_ERR_INVALID_ARG, "qtt_create: NULL ranks or cores");
  for (int k = 0; k <= d; ++k)
    if (ranks[k] < 1 || ranks[k] > 4096)
      return fail(QTT_ERR_INVALID_ARG, "qtt_create: ranks must be in [1, 4096]");
  std::vector<double> flat;
  for (int k = 0; k < d; ++k) {
    if (!cores[k]) return fail(QTT_ERR_INVALID_ARG, "qtt_create: NULL core pointer");
    const size_t n = (size_t)4 * ranks[k] * ranks[k + 1];
    flat.insert(flat.end(), cores[k], cores[k] + n);
  }
  return qtt_create_flat(out, d, ranks, flat.data(), precision_mask, stream);
}

qtt_status qtt_create_flat(qtt_op **out, int d, const int *ranks, const double *cores,
                           unsigned precision_mask, void *stream) {
  if (!out) return fail(QTT_ERR_INVALID_ARG, "qtt_create: out is NULL");
  *out = nullptr;
  if (d < 1 || d > 30) return fail(QTT_ERR_INVALID_ARG, "qtt_create: d must be in [1, 30]");
  if (!ranks || !cores) return fail(QTT_ERR_INVALID_ARG, "qtt_create: NULL ranks or cores");
  if (ranks[0] != 1 || ranks[d] != 1)
    return fail(QTT_ERR_INVALID_ARG, "qtt_create: ranks[0] and ranks[d] must be 1");
  for (int k = 0; k <= d; ++k)
    if (ranks[k] < 1 || ranks[k] > 4096)
      return fail(QTT_ERR_INVALID_ARG, "qtt_create: ranks must be in [1, 4096]");
  if (precision_mask & ~(unsigned)(QTT_PACK_F32 | QTT_PACK_TF32 | QTT_PACK_BF16))
    return fail(QTT_ERR_INVALID_ARG, "qtt_create: unknown precision_mask bits");

  qtt_op *A = new (std::nothrow) qtt_op();
  if (!A) return fail(QTT_ERR_OOM, "qtt_create: host allocation failed");
  A->d = d;
  cudaGetDevice(&A->device);
  A->ranks.assign(ranks, ranks + d + 1);
  A->off.resize(d + 1);
  int64_t off = 0;
  double sig = 0.0;
  for (int k = 0; k < d; ++k) {
    A->off[k] = off;
    off += (int64_t)4 * ranks[k] * ranks[k + 1];
    sig += (double)ranks[k] * ranks[k + 1];
  }
  A->off[d] = off;
  A->nparams = off;
  A->flops_per_rhs = 4.0 * std::ldexp(1.0, d) * sig;
  A->rmax_inner = 1;
  for (int k = 1; k < d; ++k) A->rmax_inner = std::max(A->rmax_inner, ranks[k]);
  A->packs = precision_mask;

  // Permute each core G_k[a][i][j][b] into M_k packed as [b][a][j][i].
  std::vector<double> packed((size_t)off);
  for (int k = 0; k < d; ++k) {
    const int ra = ranks[k], rb = ranks[k + 1];
    const double *G = cores + A->off[k];
    double *M = packed.data() + A->off[k];
    for (int a = 0; a < ra; ++a)
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
          for (int b = 0; b < rb; ++b)
            M[(((size_t)b * ra + a) * 2 + j) * 2 + i] = G[(((size_t)a * 2 + i) * 2 + j) * rb + b];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // qtt_apply_noalloc's static array is committed here, by an entry point
  // that allocates anyway, so that a later qtt_apply_noalloc allocates nothing
  {
    const qtt_status ps = noalloc_prepare();
    if (ps != QTT_OK) {
      delete A;
      return ps;
    }
  }
  const size_t bytes = (size_t)off * sizeof(double);
  {
    const qtt_status as = persistent_alloc(reinterpret_cast<void **>(&A->m64), bytes, st);
    if (as != QTT_OK) {
      delete A;
      return as;
    }
  }
  cudaError_t e = cudaMemcpyAsync(A->m64, packed.data(), bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    qtt_destroy(A);
    return cuda_fail(e, "qtt_create: upload");
  }
  // Reduced-precision copies: [a][j][b padded][i] per core.
  if (precision_mask) {
    A->rpad.assign(d + 1, 1);
    A->offlp.assign(d + 1, 0);
    int64_t o = 0;
    for (int k = 0; k < d; ++k) {
      A->rpad[k + 1] = lp_rank_pad(ranks[k + 1]);
      A->offlp[k] = o;
      o += (int64_t)4 * ranks[k] * A->rpad[k + 1];
    }
    A->offlp[d] = o;
    A->nlp = o;
    std::vector<double> lpd((size_t)o, 0.0);
    for (int k = 0; k < d; ++k) {
      const int ra = ranks[k], rb = ranks[k + 1], rp = A->rpad[k + 1];
      const double *G = cores + A->off[k];
      double *L = lpd.data() + A->offlp[k];
      for (int a = 0; a < ra; ++a)
        for (int i = 0; i < 2; ++i)
          for (int j = 0; j < 2; ++j)
            for (int b = 0; b < rb; ++b)
              L[(((size_t)a * 2 + j) * rp + b) * 2 + i] = G[(((size_t)a * 2 + i) * 2 + j) * rb + b];
    }
    std::vector<float> lp(lpd.begin(), lpd.end());
    // head- and tail-kernel copies of cores 0..2 and d-3..d-1 (the same values
    // as the packed copies); a core with a rank above 8 stays zero (the
    // kernels never take it)
    auto small_copy = [&](int kfirst, auto value_of) {
      std::vector<float> hc(3 * 16 * 8 * 2, 0.0f);
      for (int slot = 0; slot < 3; ++slot) {
        const int k = kfirst + slot;
        if (k < 0 || k >= d || ranks[k] > kHeadMaxRank || ranks[k + 1] > kHeadMaxRank) continue;
        const int rp = A->rpad[k + 1];
        for (int a = 0; a < ranks[k]; ++a)
          for (int j = 0; j < 2; ++j)
            for (int b = 0; b < ranks[k + 1]; ++b)
              for (int i = 0; i < 2; ++i)
                hc[(((size_t)slot * 16 + 2 * a + j) * 8 + b) * 2 + i] =
                    value_of(A->offlp[k] + (((int64_t)a * 2 + j) * rp + b) * 2 + i);
      }
      return hc;
    };
    auto v32 = [&](int64_t q) { return lp[q]; };
    auto vtf = [&](int64_t q) { return host_tf32_rne(lp[q]); };
    auto vbf = [&](int64_t q) { return __bfloat162float(__double2bfloat16(lpd[q])); };
    if (precision_mask & QTT_PACK_F32) {
      A->head[0] = small_copy(0, v32);
      A->tail[0] = small_copy(d - 3, v32);
    }
    if (precision_mask & QTT_PACK_TF32) {
      A->head[1] = small_copy(0, vtf);
      A->tail[1] = small_copy(d - 3, vtf);
    }
    if (precision_mask & QTT_PACK_BF16) {
      A->head[2] = small_copy(0, vbf);
      A->tail[2] = small_copy(d - 3, vbf);
    }
    auto upload = [&](void **dst, const void *src, size_t bytes) -> cudaError_t {
      if (persistent_alloc(dst, bytes, st) != QTT_OK) return cudaErrorMemoryAllocation;
      cudaError_t e2 = cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, st);
      if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
      return e2;
    };
    cudaError_t e2 = cudaSuccess;
    if (precision_mask & QTT_PACK_F32)
      e2 = upload(reinterpret_cast<void **>(&A->m32), lp.data(), lp.size() * sizeof(float));
    if (e2 == cudaSuccess && (precision_mask & QTT_PACK_TF32)) {
      std::vector<float> t(lp);
      for (float &v : t) v = host_tf32_rne(v);
      e2 = upload(reinterpret_cast<void **>(&A->mtf32), t.data(), t.size() * sizeof(float));
      // tensor-core layout [128][2 r_k], rows 2b+i, columns 2a+j (the same
      // TF32 values as the packed copy)
      A->toff.assign(d, -1);
      A->t2off.assign(d, -1);
      int64_t to = 0;
      // first-step copy [128][K1], K1 = 2 r_k rounded up to 8, columns 2a + j;
      // second-step copy [80][K2], K2 = 2 r_k rounded up to 4 per half,
      // columns j (r_k rounded up to 4) + a; padding zero
      for (int k = 0; k < d; ++k) {
        if (ranks[k] < 8 || ranks[k] > 40 || ranks[k + 1] > 40) continue;
        const int k1 = (2 * ranks[k] + 7) / 8 * 8, k2 = 2 * ((ranks[k] + 3) / 4 * 4);
        A->toff[k] = to;
        to += (int64_t)128 * k1;
        A->t2off[k] = to;
        to += (int64_t)80 * k2;
      }
      if (e2 == cudaSuccess && to > 0) {
        std::vector<float> m((size_t)to, 0.0f);
        for (int k = 0; k < d; ++k) {
          if (A->toff[k] < 0) continue;
          const int ra = ranks[k], rb = ranks[k + 1];
          const int k1 = (2 * ra + 7) / 8 * 8, rap = (ra + 3) / 4 * 4, k2 = 2 * rap;
          const double *G = cores + A->off[k];
          float *M = m.data() + A->toff[k];
          float *M2 = m.data() + A->t2off[k];
          for (int a = 0; a < ra; ++a)
            for (int i = 0; i < 2; ++i)
              for (int j = 0; j < 2; ++j)
                for (int b = 0; b < rb; ++b) {
                  const float v =
                      host_tf32_rne((float)G[(((size_t)a * 2 + i) * 2 + j) * rb + b]);
                  M[(size_t)(2 * b + i) * k1 + 2 * a + j] = v;
                  M2[(size_t)(2 * b + i) * k2 + j * rap + a] = v;
                }
        }
        e2 = upload(reinterpret_cast<void **>(&A->mma_tf32), m.data(), m.size() * sizeof(float));
      }
    }
    if (e2 == cudaSuccess && (precision_mask & QTT_PACK_BF16)) {
      std::vector<__nv_bfloat16> h(lp.size());
      for (size_t q = 0; q < lp.size(); ++q) h[q] = __double2bfloat16(lpd[q]);
      e2 = upload(reinterpret_cast<void **>(&A->mbf16), h.data(), h.size() * 2);
      // tensor-core layout [Mp][Kp], rows 2b+i, columns 2a+j
      A->moff.assign(d + 1, 0);
      A->mp.assign(d, 0);
      A->kp.assign(d, 0);
      int64_t mo = 0;
      for (int k = 0; k < d; ++k) {
        if (ranks[k] > kMmaMaxRank || ranks[k + 1] > kMmaMaxRank) continue;
        A->mp[k] = (2 * ranks[k + 1] + 15) / 16 * 16;
        A->kp[k] = (2 * ranks[k] + 15) / 16 * 16;
        A->moff[k] = mo;
        mo += (int64_t)A->mp[k] * A->kp[k];
      }
      A->moff[d] = mo;
      if (e2 == cudaSuccess && mo > 0) {
        std::vector<__nv_bfloat16> m((size_t)mo, __float2bfloat16(0.0f));
        for (int k = 0; k < d; ++k) {
          if (!A->mp[k]) continue;
          const int ra = ranks[k], rb = ranks[k + 1], K = A->kp[k];
          const double *G = cores + A->off[k];
          __nv_bfloat16 *M = m.data() + A->moff[k];
          for (int a = 0; a < ra; ++a)
            for (int i = 0; i < 2; ++i)
              for (int j = 0; j < 2; ++j)
                for (int b = 0; b < rb; ++b)
                  M[(size_t)(2 * b + i) * K + 2 * a + j] =
                      __double2bfloat16(G[(((size_t)a * 2 + i) * 2 + j) * rb + b]);
        }
        e2 = upload(reinterpret_cast<void **>(&A->mma_bf16), m.data(), m.size() * 2);
      }
    }
    if (e2 != cudaSuccess) {
      qtt_destroy(A);
      return cuda_fail(e2, "qtt_create: reduced-precision upload");
    }
  }
  *out = A;
  return QTT_OK;
}

qtt_status qtt_destroy(qtt_op *A) {
  if (!A) return QTT_OK;
  // The buffers go back to the pool once the work recorded by note_use has
  // finished: other streams and the host are not held up (no device-wide
  // synchronisation).
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != A->device) cudaSetDevice(A->device);
  std::vector<cudaEvent_t> evs;
  {
    std::lock_guard<std::mutex> lk(A->use_mu);
    for (auto &u : A->uses) evs.push_back(u.second);
    A->uses.clear();
  }
  release_after({A->m64, A->m32, A->mtf32, A->mbf16, A->mma_bf16, A->mma_tf32}, evs);
  for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
  if (cur >= 0 && cur != A->device) cudaSetDevice(cur);
  delete A;
  return QTT_OK;
}

int qtt_op_d(const qtt_op *A) { return A ? A->d : -1; }

int qtt_op_rank(const qtt_op *A, int k) {
  if (!A || k < 0 || k > A->d) return -1;
  return A->ranks[k];
}

double qtt_op_flops(const qtt_op *A) { return A ? A->flops_per_rhs : 0.0; }

qtt_status qtt_apply(const qtt_op *A, const void *x, void *y, int64_t nrhs, int64_t ld,
                     qtt_dtype io_dtype, qtt_dtype compute, void *stream) {
  if (!A) return fail(QTT_ERR_INVALID_ARG, "qtt_apply: NULL operator");
  if (qtt_status ds = check_device(A, "qtt_apply")) return ds;
  if (!valid_dtype(io_dtype) || !valid_dtype(compute))
    return fail(QTT_ERR_INVALID_ARG, "qtt_apply: unknown dtype");
  const int64_t N = (int64_t)1 << A->d;
  if (nrhs < 0) return fail(QTT_ERR_INVALID_ARG, "qtt_apply: nrhs < 0");
  if (nrhs == 0) return QTT_OK;
  if (ld < N) return fail(QTT_ERR_INVALID_ARG, "qtt_apply: ld < N");
  if (!x || !y) return fail(QTT_ERR_INVALID_ARG, "qtt_apply: NULL vector");
  const size_t esz = io_dtype == QTT_F64 ? 8 : (io_dtype == QTT_BF16 ? 2 : 4);
  {
    const char *xb = static_cast<const char *>(x), *yb = static_cast<const char *>(y);
    const size_t span = ((size_t)(nrhs - 1) * (size_t)ld + (size_t)N) * esz;
    if (xb < yb + span && yb < xb + span)
      return fail(QTT_ERR_INVALID_ARG, "qtt_apply: x and y overlap");
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (compute == QTT_F64) {
    if (io_dtype != QTT_F64)
      return fail(QTT_ERR_UNSUPPORTED, "qtt_apply: FP64 compute needs FP64 vectors");
    return apply_f64(A, static_cast<const double *>(x), static_cast<double *>(y), nrhs, ld,
                     st, Epilogue());
  }
  if (io_dtype == QTT_TF32)
    return fail(QTT_ERR_INVALID_ARG, "qtt_apply: TF32 is not a storage type (use F32)");
  return apply_lp(A, compute, x, io_dtype, y, io_dtype, nrhs, ld, st, LpEpilogue());
}

qtt_status qtt_plan_create(qtt_plan **out, const qtt_op *A, const void *x, void *y,
                           int64_t nrhs, int64_t ld, qtt_dtype io_dtype, qtt_dtype compute) {
  if (!out) return fail(QTT_ERR_INVALID_ARG, "qtt_plan_create: out is NULL");
  *out = nullptr;
  qtt_plan *P = new (std::nothrow) qtt_plan();
  if (!P) return fail(QTT_ERR_OOM, "qtt_plan_create: host allocation failed");
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete P;
    return cuda_fail(e, "qtt_plan_create: stream");
  }
  // record the apply (relaxed mode: the first call of a kernel family sets
  // its attributes, which is not a stream operation)
  const uint64_t before = t_launches;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  qtt_status s = QTT_OK;
  if (e == cudaSuccess) s = qtt_apply(A, x, y, nrhs, ld, io_dtype, compute, cs);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess || e2 != cudaSuccess || s != QTT_OK) {
    if (g) cudaGraphDestroy(g);
    delete P;
    if (s != QTT_OK) return s;
    return cuda_fail(e != cudaSuccess ? e : e2, "qtt_plan_create: stream capture");
  }
  P->op = A;
  P->launches = t_launches - before;
  g_launches.fetch_sub(P->launches, std::memory_order_relaxed);  // recorded, not run
  t_launches = before;
  P->graph = g;
  e = cudaGraphInstantiate(&P->exec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    delete P;
    return cuda_fail(e, "qtt_plan_create: instantiate");
  }
  *out = P;
  return QTT_OK;
}

qtt_status qtt_plan_run(qtt_plan *P, void *stream) {
  if (!P || !P->exec) return fail(QTT_ERR_INVALID_ARG, "qtt_plan_run: no plan");
  const cudaError_t e = cudaGraphLaunch(P->exec, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "qtt_plan_run: graph launch");
  note_use(P->op, static_cast<cudaStream_t>(stream));
  count_launches(P->launches);
  return QTT_OK;
}

qtt_status qtt_plan_destroy(qtt_plan *P) {
  if (!P) return QTT_OK;
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  delete P;
  return QTT_OK;
}

qtt_status qtt_residual(const qtt_op *K, double a, const double *f, const double *x,
                        double *r, int64_t nrhs, int64_t ld, void *stream) {
  if (!K) return fail(QTT_ERR_INVALID_ARG, "qtt_residual: NULL operator");
  if (qtt_status ds = check_device(K, "qtt_residual")) return ds;
  const int64_t N = (int64_t)1 << K->d;
  if (nrhs < 0 || (nrhs > 0 && ld < N))
    return fail(QTT_ERR_INVALID_ARG, "qtt_residual: bad nrhs or ld");
  if (nrhs == 0) return QTT_OK;
  if (!f || !x || !r) return fail(QTT_ERR_INVALID_ARG, "qtt_residual: NULL vector");
  const size_t span = ((size_t)(nrhs - 1) * (size_t)ld + (size_t)N) * sizeof(double);
  const char *rb = reinterpret_cast<const char *>(r);
  for (const double *v : {f, x}) {
    const char *vb = reinterpret_cast<const char *>(v);
    if (vb < rb + span && rb < vb + span)
      return fail(QTT_ERR_INVALID_ARG, "qtt_residual: r overlaps f or x");
  }
  Epilogue e;
  e.on = true;
  e.v = f;
  e.s_v = 1.0;
  e.u = x;
  e.s_u = -a;
  e.s_acc = -1.0;
  return apply_f64(K, x, r, nrhs, ld, static_cast<cudaStream_t>(stream), e);
}

qtt_status qtt_apply_set_plan(qtt_op *A, qtt_dtype compute, int plan) {
  if (!A || !valid_dtype(compute)) return fail(QTT_ERR_INVALID_ARG, "qtt_apply_set_plan: bad operator or compute");
  ApplyPlan p;
  if (!decode_plan(plan, &p)) return fail(QTT_ERR_INVALID_ARG, "qtt_apply_set_plan: unknown plan code");
  A->plan[compute] = p;
  return QTT_OK;
}

qtt_status qtt_apply_get_plan(const qtt_op *A, qtt_dtype compute, int *plan) {
  if (!A || !plan || !valid_dtype(compute))
    return fail(QTT_ERR_INVALID_ARG, "qtt_apply_get_plan: bad argument");
  *plan = encode_plan(A->plan[compute]);
  return QTT_OK;
}

qtt_status qtt_apply_autotune(qtt_op *A, int64_t nrhs, qtt_dtype compute, int reps, void *stream,
                              int *plan, double *seconds) {
  if (!A || nrhs < 1 || !valid_dtype(compute))
    return fail(QTT_ERR_INVALID_ARG, "qtt_apply_autotune: bad operator, nrhs or compute");
  if (qtt_status ds = check_device(A, "qtt_apply_autotune")) return ds;
  if (reps < 1) reps = 1;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // candidate plans for this arithmetic (the default first)
  std::vector<ApplyPlan> cands;
  ApplyPlan p0;
  cands.push_back(p0);
  if (compute == QTT_BF16) {
    ApplyPlan p = p0;
    p.groups_cap = 2;
    cands.push_back(p);          // tcgen05 pairs, two epilogue groups
    p = p0;
    p.pairs = 1;
    cands.push_back(p);          // mma.sync pairs
    p = p0;
    p.pairs = 0;
    cands.push_back(p);          // head/tail merged, single middle steps
    p = p0;
    p.fusion = false;
    cands.push_back(p);          // one launch per step
  } else if (compute == QTT_F32 || compute == QTT_TF32) {
    ApplyPlan p = p0;
    if (compute == QTT_TF32) {
      p.pairs = 0;
      cands.push_back(p);        // no tcgen05 pairs: every middle step on the FP32 pipe
      p = p0;
    }
    p.staged = false;
    cands.push_back(p);
    p = p0;
    p.fusion = false;
    cands.push_back(p);
    p.staged = false;
    cands.push_back(p);
  }
  const qtt_dtype io = compute == QTT_F64 ? QTT_F64 : compute == QTT_BF16 ? QTT_BF16 : QTT_F32;
  const int64_t N = (int64_t)1 << A->d;
  const size_t bytes = (size_t)N * (size_t)nrhs * dtype_size(io);
  void *x = nullptr, *y = nullptr;
  qtt_status s = scratch_alloc(&x, bytes, st);
  if (s == QTT_OK) s = scratch_alloc(&y, bytes, st);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (s == QTT_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    s = fail(QTT_ERR_CUDA, "qtt_apply_autotune: events");
  if (s == QTT_OK && cudaMemsetAsync(x, 0, bytes, st) != cudaSuccess)
    s = fail(QTT_ERR_CUDA, "qtt_apply_autotune: clear x");
  const ApplyPlan keep = A->plan[compute];
  double best_t = 1e300;
  ApplyPlan best = keep;
  for (size_t c = 0; c < cands.size() && s == QTT_OK; ++c) {
    A->plan[compute] = cands[c];
    // timing does not depend on the values (the arithmetic is data-independent)
    qtt_status t = qtt_apply(A, x, y, nrhs, N, io, compute, st);  // warm-up
    if (t != QTT_OK) continue;
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps && t == QTT_OK; ++r) t = qtt_apply(A, x, y, nrhs, N, io, compute, st);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      s = cuda_fail(cudaGetLastError(), "qtt_apply_autotune: sync");
      break;
    }
    if (t != QTT_OK) continue;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double sec = ms / 1e3 / reps;
    if (sec < best_t) {
      best_t = sec;
      best = cands[c];
    }
  }
  A->plan[compute] = s == QTT_OK ? best : keep;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  scratch_free(x, st);
  scratch_free(y, st);
  if (s != QTT_OK) return s;
  if (plan) *plan = encode_plan(best);
  if (seconds) *seconds = best_t;
  return QTT_OK;
}

qtt_status qtt_set_scratch_limit(size_t bytes) {
  g_scratch_cap.store(bytes, std::memory_order_relaxed);
  return QTT_OK;
}

qtt_status qtt_scratch_stats(size_t *in_use, size_t *pool_reserved, size_t *pool_used) {
  if (in_use) {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    *in_use = g_scratch_in_use;
  }
  cudaMemPool_t p = pool_for_current_device();
  uint64_t reserved = 0, used = 0;
  if (p) {
    cudaMemPoolGetAttribute(p, cudaMemPoolAttrReservedMemCurrent, &reserved);
    cudaMemPoolGetAttribute(p, cudaMemPoolAttrUsedMemCurrent, &used);
  }
  if (pool_reserved) *pool_reserved = (size_t)reserved;
  if (pool_used) *pool_used = (size_t)used;
  return p ? QTT_OK : fail(QTT_ERR_CUDA, "qtt_scratch_stats: no memory pool");
}

qtt_status qtt_selftest_wait(double seconds, void *stream) {
  if (!(seconds > 0.0 && seconds <= 10.0))
    return fail(QTT_ERR_INVALID_ARG, "qtt_selftest_wait: seconds must be in (0, 10]");
  const cudaError_t e = wait_selftest(seconds, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "qtt_selftest_wait");
  return QTT_OK;
}

int qtt_checked_build(void) {
#ifdef QTT_CHECKED
  return 1;
#else
  return 0;
#endif
}

qtt_status qtt_check_selftest(void *stream) {
#ifdef QTT_CHECKED
  const cudaError_t e = launch_check_selftest(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "qtt_check_selftest");
  return QTT_OK;
#else
  (void)stream;
  return fail(QTT_ERR_UNSUPPORTED, "qtt_check_selftest: not the checked build");
#endif
}

qtt_status qtt_sync_status(void *stream) {
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "qtt_sync_status");
  {
    // checked build: every translation unit's index-check word
    int first = 0;
    for (auto take : check_words()) {
      int site = 0;
      e = take(&site);
      if (e != cudaSuccess) return cuda_fail(e, "qtt_sync_status: check word");
      if (site != 0 && first == 0) first = site;
    }
    if (first != 0)
      return fail(QTT_ERR_CHECK, "checked build: out-of-range index at site " +
                                     std::to_string(first));
  }
  int h = 0;
  e = tc_status_take(&h);
  int hf = 0, ht = 0;
  if (e == cudaSuccess) e = tcf_status_take(&hf);
  if (e == cudaSuccess) e = tail_status_take(&ht);
  if (e != cudaSuccess) return cuda_fail(e, "qtt_sync_status: device status word");
  if (h != 0 || hf != 0)
    return fail(QTT_ERR_TIMEOUT, "tensor-core kernel: an mbarrier wait ran out of its budget");
  if (ht != 0)
    return fail(QTT_ERR_TIMEOUT, "staged tail kernel: an mbarrier wait ran out of its budget");
  return QTT_OK;
}

}  // extern "C"
