// BF16 core step on the tensor cores (mma.sync m16n8k16, FP32 accumulate).
//
// One step of Algorithm 2 is the product phi_k = M_k b_k of the
// (2 r_{k+1}) x (2 r_k) core matrix with the (2 r_k) x (N/2 x nrhs) matrix of
// position pairs; with BF16 operands this is a real dense contraction, so it
// runs on the tensor cores:
//   A = M_k, rows (b, i) -> 2b + i, columns (a, j) -> 2a + j, padded to
//       multiples of 16 with zeros, resident in shared memory for the whole
//       (persistent) CTA;
//   B = the input chunk of 128 position pairs, K-major in shared memory
//       ([2a + j][pair]), copied with 16-byte cp.async (8 consecutive pairs
//       of one (a, j) are 8 consecutive positions once k >= 3), three chunks
//       in flight so the next ones stream in while this one multiplies;
//   fragments by ldmatrix (B transposed), mma.sync accumulates in FP32, the
//       epilogue rounds to BF16 and writes rows (b, i) to positions p0 | i 2^k.
// The numerics equal the CUDA-core BF16 step up to FP32 summation order.
// The step moves (r_k + r_{k+1}) x 2 bytes per position for 4 r_k r_{k+1}
// flops, so it is HBM-bound for r <~ 200; the persistent grid keeps the
// copies of the next chunk in flight behind the current chunk's MMAs.
#include <cuda_bf16.h>

#include "qtt_internal.h"
#include "step_mma.h"

namespace qtt {
namespace {

constexpr int kThreads = 256;  // 8 warps
constexpr int kPadB = 8;       // bf16 padding per smem row (16 B)
constexpr int kStages = 3;     // chunks in flight per CTA

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(unsigned dst, const void *src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src),
               "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ void ldsm_x4(unsigned addr, unsigned &r0, unsigned &r1, unsigned &r2,
                                        unsigned &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned addr, unsigned &r0, unsigned &r1, unsigned &r2,
                                          unsigned &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2_t(unsigned addr, unsigned &r0, unsigned &r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r0), "=r"(r1)
               : "r"(addr));
}
__device__ __forceinline__ void mma_bf16(float (&c)[4], unsigned a0, unsigned a1, unsigned a2,
                                         unsigned a3, unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Issue the cp.async copies of chunk (c, q0) into B buffer `sb`.  Thread t
// copies piece ch = t % 16 (8 consecutive pairs = 16 bytes) of rows
// t / 16, t / 16 + 16, ...; the position of its piece is computed once.
template <int kBN>
__device__ __forceinline__ void load_chunk(const StepMMA &s, __nv_bfloat16 *sb, int64_t c,
                                           int64_t q0) {
  const int rows = 2 * s.rin;  // valid K rows; padding rows stay zero
  constexpr int PIECES = kBN / 8;
  const int ch = threadIdx.x % PIECES, r0 = threadIdx.x / PIECES;
  const int64_t bit = (int64_t)1 << s.k, low = bit - 1;
  const int64_t q = q0 + 8 * ch;
  const bool ok = q < (s.N >> 1);
  const __nv_bfloat16 *base = s.in + c * s.in_rhs_stride + (((q & ~low) << 1) | (q & low));
  const unsigned dst0 = smem_u32(sb + 8 * ch);
  for (int kk = r0; kk < rows; kk += kThreads / PIECES) {
    const __nv_bfloat16 *src = base + (int64_t)(kk >> 1) * s.N + ((kk & 1) ? bit : 0);
    cp_async16(dst0 + (unsigned)(kk * (kBN + kPadB) * 2), ok ? src : s.in, ok ? 16 : 0);
  }
}

template <int MT, int NT>
__global__ void __launch_bounds__(kThreads) step_mma_bf16_kernel(StepMMA s) {
  constexpr int kBN = 64 * NT;  // pairs per chunk (8 NT per warp)
  extern __shared__ __align__(16) unsigned char smraw[];
  const int Kp = s.Kp, Mp = MT * 16;
  const int lda = Kp + kPadB;
  const size_t bstage = (size_t)Kp * (kBN + kPadB);
  __nv_bfloat16 *sA = reinterpret_cast<__nv_bfloat16 *>(smraw);
  __nv_bfloat16 *sB = sA + (size_t)Mp * lda;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // zero the K-padding rows of every B stage once; load A (already padded)
  for (int e = tid; e < (Kp - 2 * s.rin) * (kBN + kPadB); e += kThreads) {
    const int r = 2 * s.rin + e / (kBN + kPadB), cidx = e % (kBN + kPadB);
#pragma unroll
    for (int st = 0; st < kStages; ++st)
      sB[st * bstage + (size_t)r * (kBN + kPadB) + cidx] = __float2bfloat16(0.0f);
  }
  for (int e = tid; e < Mp * (Kp / 8); e += kThreads) {
    const int r = e / (Kp / 8), ch = e % (Kp / 8);
    cp_async16(smem_u32(sA + (size_t)r * lda + 8 * ch), s.A + (size_t)r * Kp + 8 * ch, 16);
  }
  const int64_t npairs = s.N >> 1;
  const int64_t chunks_per_rhs = (npairs + kBN - 1) / kBN;
  const int64_t nchunks = chunks_per_rhs * s.nrhs;
  const int64_t G = gridDim.x;
  // prologue: chunks 0 .. kStages-2 of this CTA
#pragma unroll
  for (int st = 0; st < kStages - 1; ++st) {
    const int64_t t = blockIdx.x + st * G;
    if (t < nchunks)
      load_chunk<kBN>(s, sB + st * bstage, t / chunks_per_rhs, (t % chunks_per_rhs) * kBN);
    cp_async_commit();
  }

  const int64_t bit = (int64_t)1 << s.k, low = bit - 1;
  const int n0 = warp * 8 * NT;
  const int g = lane >> 2, tq = lane & 3;
  const int mi = lane >> 3, rr = lane & 7;
  // ldmatrix row offsets (elements) of this lane
  const int b_off = (rr + ((mi & 1) ? 8 : 0)) * (kBN + kPadB) + n0 + ((mi & 2) && NT == 2 ? 8 : 0);
  const int a_off = (rr + ((mi & 1) ? 8 : 0)) * lda + ((mi & 2) ? 8 : 0);
  int stage = 0;
  for (int64_t t = blockIdx.x; t < nchunks; t += G) {
    {
      const int64_t tn = t + (kStages - 1) * G;
      const int ns = (stage + kStages - 1) % kStages;
      if (tn < nchunks)
        load_chunk<kBN>(s, sB + ns * bstage, tn / chunks_per_rhs, (tn % chunks_per_rhs) * kBN);
      cp_async_commit();
    }
    cp_async_wait<kStages - 1>();
    __syncthreads();
    const __nv_bfloat16 *cur = sB + stage * bstage;

    float acc[MT][NT][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.0f;
    const unsigned bbase = smem_u32(cur + b_off);
    const unsigned abase = smem_u32(sA + a_off);
    for (int k0 = 0; k0 < Kp; k0 += 16) {
      unsigned b0, b1, b2 = 0, b3 = 0;
      if constexpr (NT == 2)
        ldsm_x4_t(bbase + (unsigned)(k0 * (kBN + kPadB) * 2), b0, b1, b2, b3);
      else
        ldsm_x2_t(bbase + (unsigned)(k0 * (kBN + kPadB) * 2), b0, b1);
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
        unsigned a0, a1, a2, a3;
        ldsm_x4(abase + (unsigned)((mt * 16 * lda + k0) * 2), a0, a1, a2, a3);
        mma_bf16(acc[mt][0], a0, a1, a2, a3, b0, b1);
        if constexpr (NT == 2) mma_bf16(acc[mt][1], a0, a1, a2, a3, b2, b3);
      }
    }
    // epilogue: rows (b, i), columns = pairs; positions computed once
    const int64_t c = t / chunks_per_rhs;
    const int64_t q0 = (t % chunks_per_rhs) * kBN;
    __nv_bfloat16 *out = s.out + c * s.out_rhs_stride;
    int64_t pos[NT];
    bool okq[NT];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      const int64_t q = q0 + n0 + nt * 8 + 2 * tq;
      okq[nt] = q < npairs;
      pos[nt] = ((q & ~low) << 1) | (q & low);
    }
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = mt * 16 + g + 8 * h;
        const int b = row >> 1;
        if (b >= s.rout) continue;
        __nv_bfloat16 *ob = out + (int64_t)b * s.N + ((row & 1) ? bit : 0);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          if (!okq[nt]) continue;
          *reinterpret_cast<__nv_bfloat162 *>(ob + pos[nt]) =
              __floats2bfloat162_rn(acc[mt][nt][2 * h], acc[mt][nt][2 * h + 1]);
        }
      }
    __syncthreads();  // everyone done with this stage before it is refilled
    stage = (stage + 1) % kStages;
  }
  cp_async_wait<0>();
}

template <int MT, int NT>
size_t smem_bytes(int Kp) {
  return sizeof(__nv_bfloat16) *
         ((size_t)MT * 16 * (Kp + kPadB) + (size_t)kStages * Kp * (64 * NT + kPadB));
}

template <int MT, int NT>
cudaError_t launch_mt(const StepMMA &s, cudaStream_t st) {
  // The dynamic shared-memory limit is a property of the kernel shared by all
  // host threads: raise it once to the largest this instantiation can use
  // (Kp = 2 x 64), never per call, so concurrent launches cannot lower it
  // under each other.
  static cudaError_t attr = cudaFuncSetAttribute(
      step_mma_bf16_kernel<MT, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)smem_bytes<MT, NT>(2 * kMmaMaxRank));
  if (attr != cudaSuccess) return attr;
  const size_t smem = smem_bytes<MT, NT>(s.Kp);
  int per_sm = 1, dev = 0, sms = 148;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_mma_bf16_kernel<MT, NT>, kThreads,
                                                smem);
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t npairs = s.N >> 1;
  const int64_t nchunks = (npairs + 64 * NT - 1) / (64 * NT) * s.nrhs;
  int64_t grid = (int64_t)(per_sm < 1 ? 1 : per_sm) * sms;
  if (grid > nchunks) grid = nchunks;
  step_mma_bf16_kernel<MT, NT><<<(unsigned)grid, kThreads, smem, st>>>(s);
  count_launches(1);
  return cudaGetLastError();
}

// 128-pair chunks (two n8 tiles per warp); one n8 tile per warp (64-pair
// chunks, more CTAs per SM) measured 22 % slower on GB300.
template <int MT>
cudaError_t launch_nt(const StepMMA &s, cudaStream_t st) {
  return launch_mt<MT, 2>(s, st);
}

}  // namespace

bool mma_step_eligible(int k, int rin, int rout, int64_t N) {
  return k >= 3 && rin >= 4 && rout >= 4 && rin <= kMmaMaxRank && rout <= kMmaMaxRank &&
         (N >> 1) % 8 == 0;
}

cudaError_t launch_step_mma_bf16(const StepMMA &s, cudaStream_t st) {
  switch ((s.Mp + 15) / 16) {
    case 1: return launch_nt<1>(s, st);
    case 2: return launch_nt<2>(s, st);
    case 3: return launch_nt<3>(s, st);
    case 4: return launch_nt<4>(s, st);
    case 5: return launch_nt<5>(s, st);
    case 6: return launch_nt<6>(s, st);
    case 7: return launch_nt<7>(s, st);
    case 8: return launch_nt<8>(s, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace qtt
