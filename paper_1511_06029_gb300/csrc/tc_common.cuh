// Device helpers shared by the tcgen05 step kernels (BF16 and TF32 pairs):
// shared-memory addresses, cp.async, mbarriers with bounded waits, the
// tcgen05 fences, commit and TMEM load, TMA tile copies, shared-memory
// matrix descriptors and the K-major 128-byte-swizzled operand layout.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace qtt {
namespace tcx {

constexpr long long kWaitBudget = 4000000000LL;  // clock64 ticks (about 2 s)

__device__ __forceinline__ unsigned su32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cpa16(unsigned dst, const void *src, int n) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(n));
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cpa_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_init(unsigned a, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count) : "memory");
}
// One test of phase `parity` of the mbarrier at `a`.
__device__ __forceinline__ bool mbar_try(unsigned a, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}

// Shared-memory matrix descriptor: start address, leading and stride byte
// offsets, version 1 (bits 46-47), layout (bits 61-63: 0 none, 2 128-byte
// swizzle).  No swizzle: LBO = distance between core matrices adjacent in K,
// SBO = adjacent in M/N.  128-byte swizzle, MN-major: LBO = distance between
// 64-element MN blocks, SBO = between 8-row K groups (1024 bytes).
__device__ __forceinline__ uint64_t smem_desc(unsigned addr, unsigned lbo, unsigned sbo,
                                              unsigned layout = 0) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46) |
         ((uint64_t)layout << 61);
}

__device__ __forceinline__ void mma_commit(unsigned mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          mbar)
      : "memory");
}

// 32 lanes x 32 consecutive FP32 columns from TMEM into v[0..31].
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int e = 0; e < 32; ++e) v[e] = __uint_as_float(r[e]);
}

// TMA tile copies (5-D tensor maps) and their completion mechanisms.
__device__ __forceinline__ void tma_load5(unsigned dst, const CUtensorMap *m, int c0, int c1,
                                          int c2, int c3, int c4, unsigned mbar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
      "{%2, %3, %4, %5, %6}], [%7];\n" ::"r"(dst),
      "l"(m), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void tma_load4(unsigned dst, const CUtensorMap *m, int c0, int c1,
                                          int c2, int c3, unsigned mbar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
      "{%2, %3, %4, %5}], [%6];\n" ::"r"(dst),
      "l"(m), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void tma_store5(const CUtensorMap *m, unsigned src, int c0, int c1,
                                           int c2, int c3, int c4) {
  asm volatile(
      "cp.async.bulk.tensor.5d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5, %6}], "
      "[%1];\n" ::"l"(m),
      "r"(src), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
      : "memory");
}
__device__ __forceinline__ void tma_store3(const CUtensorMap *m, unsigned src, int c0, int c1,
                                           int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];\n" ::"l"(m),
      "r"(src), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}
__device__ __forceinline__ void expect_tx(unsigned mbar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read0() {
  asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}
// All but the most recent bulk group have read their shared memory.
__device__ __forceinline__ void bulk_wait_read1() {
  asm volatile("cp.async.bulk.wait_group.read 1;\n" ::: "memory");
}
// Barrier of the epilogue warps that also ORs a flag over them: the abort
// decision stays uniform, so no epilogue thread is left at a barrier.
// (Named barrier 1 + g belongs to epilogue group g of NT threads.)
template <int NT>
__device__ __forceinline__ bool epi_any(bool v, int g) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((unsigned)v), "r"(1 + g), "n"(NT)
      : "memory");
  return r != 0;
}
template <int NT>
__device__ __forceinline__ void epi_sync(int g) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(1 + g), "n"(NT) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
}

// Walk over chunks t0, t0 + step, ...: t = c cpr + w (right-hand side c,
// chunk w of it), advanced by an addition and at most one carry per step.
struct ChunkWalk {
  int64_t t, c, w, dc, dw, cpr;
  __device__ ChunkWalk(int64_t t0, int64_t step, int64_t cpr_)
      : t(t0), c(t0 / cpr_), w(t0 % cpr_), dc(step / cpr_), dw(step % cpr_), cpr(cpr_) {}
  __device__ void next() {
    t += dc * cpr + dw;
    c += dc;
    w += dw;
    if (w >= cpr) {
      w -= cpr;
      ++c;
    }
  }
};

__device__ __forceinline__ void mbar_arrive(unsigned a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(a) : "memory");
}
// Bounded wait that also gives up once another role raised the abort flag.
__device__ __forceinline__ bool wait_bar(unsigned a, unsigned parity, volatile int *abort,
                                         long long budget = kWaitBudget) {
  const long long t0 = clock64();
  for (;;) {
    if (mbar_try(a, parity)) return true;
    if (*abort) return false;
    if (clock64() - t0 > budget) {
      *abort = 1;
      return false;
    }
  }
}

// Shared-memory plan (byte offsets from a 1024-aligned base).
// Core matrix M (Mp x Kp) as the K-major operand, 128-byte swizzle: K in
// atoms of 64 (Mp rows of 128 bytes each), row r of atom ka at
// ka Mp 128 + r 128, its 16-byte chunk c at (c ^ r % 8).
__host__ __device__ inline unsigned a_bytes(int Mp, int Kp) {
  return (unsigned)((Kp + 63) / 64) * (unsigned)Mp * 128u;
}
__device__ __forceinline__ unsigned a_offset(int Mp, int r, int kc) {
  return (unsigned)(kc >> 3) * (unsigned)Mp * 128u + (unsigned)r * 128u +
         ((unsigned)((kc & 7) ^ (r & 7)) << 4);
}

// 1024-byte alignment of a shared-memory offset (the 128-byte swizzle repeats
// every 8 rows of 128 bytes).
__host__ __device__ inline unsigned up1k(unsigned v) { return (v + 1023u) & ~1023u; }

// The driver's tensor-map encoder, looked up through the runtime (the library
// does not link libcuda, so it loads on machines without a driver).
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  return encode;
}

}  // namespace tcx
}  // namespace qtt
