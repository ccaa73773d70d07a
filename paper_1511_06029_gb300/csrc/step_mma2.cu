// Two consecutive BF16 core steps fused on the tensor cores (mma.sync).  The
// apply uses it for pairs the tcgen05 pair kernel (step_tc2.cu) does not
// take: k = 3, or ranks with r_k % 8 != 0, in [16, 48].
//
// Steps k and k+1 of Algorithm 2 only mix position bits k and k+1, so the
// four positions of a "quad" (bits k, k+1 free, the others fixed) are closed
// under both steps.  A chunk of 64 quads is read once, both contractions run
// on chip, and only the result of step k+1 goes back to HBM: the r_{k+1}
// planes in between never leave the SM, which halves the bytes of a pair of
// middle steps.
//
//   stage (B of step k):   rows (a, j_k) -> 2a + j_k,
//                          columns (j_{k+1}, quad) -> 64 j_{k+1} + quad
//   C1 = M_k x stage:      rows (b, i_k), columns (j_{k+1}, quad)
//   T  (B of step k+1):    rows (b, j_{k+1}) -> 2b + j_{k+1},
//                          columns (i_k, quad) -> 72 i_k + quad (8 pad so the
//                          two halves fall on different banks)
//   C2 = M_{k+1} x T:      rows (c, i_{k+1}), columns (i_k, quad)
//                          -> position base(quad) | i_k 2^k | i_{k+1} 2^(k+1)
// C1 is rounded to BF16 when it is written to T (the same rounding the
// unfused path applies when it stores the intermediate), so the result equals
// the unfused BF16 sweep up to FP32 summation order.  Both core matrices stay
// in shared memory for the persistent CTA; input chunks stream through a
// three-deep cp.async ring (8 consecutive quads are 8 consecutive positions
// once k >= 3).
#include <cuda_bf16.h>

#include "qtt_internal.h"
#include "step_mma.h"

namespace qtt {
namespace {

constexpr int kThreads = 256;
constexpr int kQ = 64;          // quads per chunk
constexpr int kCols = 2 * kQ;   // columns of both B operands
constexpr int kLdS = kCols + 8; // stage row stride (bf16)
constexpr int kHalfT = kQ + 8;  // T: one i_k half plus padding
constexpr int kLdT = 2 * kHalfT + 8;
constexpr int kStages = 3;

__device__ __forceinline__ unsigned su32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cpa16(unsigned dst, const void *src, int n) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(n));
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cpa_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}
__device__ __forceinline__ void ldsm4(unsigned a, unsigned &r0, unsigned &r1, unsigned &r2,
                                      unsigned &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(a));
}
__device__ __forceinline__ void ldsm4t(unsigned a, unsigned &r0, unsigned &r1, unsigned &r2,
                                       unsigned &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(a));
}
__device__ __forceinline__ void mma16816(float (&c)[4], unsigned a0, unsigned a1, unsigned a2,
                                         unsigned a3, unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Quad q -> position with bits k and k+1 cleared.
__device__ __forceinline__ int64_t quad_base(int64_t q, int k) {
  const int64_t low = ((int64_t)1 << k) - 1;
  return ((q & ~low) << 2) | (q & low);
}

__device__ __forceinline__ void load_chunk2(const StepMMA2 &s, __nv_bfloat16 *sb, int64_t c,
                                            int64_t q0) {
  const int rows = 2 * s.r0;
  const int64_t bit = (int64_t)1 << s.k, nq = s.N >> 2;
  const __nv_bfloat16 *in = s.in + c * s.in_rhs_stride;
  // thread -> 16-byte piece (8 quads) `pc` of column half `jh`, rows r0, r0+16, ...
  const int piece = threadIdx.x & 15, jh = piece >> 3, pc = piece & 7;
  const int64_t q = q0 + 8 * pc;
  const bool ok = q < nq;
  const __nv_bfloat16 *base = in + quad_base(q, s.k) + (jh ? 2 * bit : 0);
  const unsigned dst0 = su32(sb + jh * kQ + 8 * pc);
  for (int kk = threadIdx.x >> 4; kk < rows; kk += kThreads / 16) {
    const __nv_bfloat16 *src = base + (int64_t)(kk >> 1) * s.N + ((kk & 1) ? bit : 0);
    cpa16(dst0 + (unsigned)(kk * kLdS * 2), ok ? src : s.in, ok ? 16 : 0);
  }
}

template <int MT1, int MT2>
__global__ void __launch_bounds__(kThreads, 1) step_mma2_kernel(StepMMA2 s) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int Kp1 = s.Kp1, Kp2 = MT1 * 16;  // step k+1 contracts over the rows of C1
  const int lda1 = Kp1 + 8, lda2 = Kp2 + 8;
  __nv_bfloat16 *sA1 = reinterpret_cast<__nv_bfloat16 *>(smraw);
  __nv_bfloat16 *sA2 = sA1 + (size_t)MT1 * 16 * lda1;
  __nv_bfloat16 *sT = sA2 + (size_t)MT2 * 16 * lda2;
  __nv_bfloat16 *sS = sT + (size_t)Kp2 * kLdT;
  const size_t sstage = (size_t)Kp1 * kLdS;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // zero: K-padding rows of every stage, all of T (its padding rows stay 0)
  for (int e = tid; e < (Kp1 - 2 * s.r0) * kLdS; e += kThreads) {
    const int r = 2 * s.r0 + e / kLdS, cc = e % kLdS;
#pragma unroll
    for (int st = 0; st < kStages; ++st) sS[st * sstage + (size_t)r * kLdS + cc] = __float2bfloat16(0.f);
  }
  for (int e = tid; e < Kp2 * kLdT; e += kThreads) sT[e] = __float2bfloat16(0.f);
  for (int e = tid; e < MT1 * 16 * (Kp1 / 8); e += kThreads) {
    const int r = e / (Kp1 / 8), ch = e % (Kp1 / 8);
    cpa16(su32(sA1 + (size_t)r * lda1 + 8 * ch), s.A1 + (size_t)r * Kp1 + 8 * ch, 16);
  }
  for (int e = tid; e < MT2 * 16 * (Kp2 / 8); e += kThreads) {
    const int r = e / (Kp2 / 8), ch = e % (Kp2 / 8);
    cpa16(su32(sA2 + (size_t)r * lda2 + 8 * ch), s.A2 + (size_t)r * Kp2 + 8 * ch, 16);
  }
  const int64_t nq = s.N >> 2;
  const int64_t cpr = (nq + kQ - 1) / kQ;
  const int64_t nchunks = cpr * s.nrhs;
  const int64_t G = gridDim.x;
#pragma unroll
  for (int st = 0; st < kStages - 1; ++st) {
    const int64_t t = blockIdx.x + st * G;
    if (t < nchunks) load_chunk2(s, sS + st * sstage, t / cpr, (t % cpr) * kQ);
    cpa_commit();
  }
  const int64_t bit = (int64_t)1 << s.k;
  const int g = lane >> 2, tq = lane & 3, mi = lane >> 3, rr = lane & 7;
  const int n0 = warp * 16;                      // this warp's 16 columns
  const int half = n0 / kQ, qn0 = n0 % kQ;       // j_{k+1} (step 1) or i_k (step 2)
  // ldmatrix lane offsets (elements)
  const int bS = (rr + ((mi & 1) ? 8 : 0)) * kLdS + n0 + ((mi & 2) ? 8 : 0);
  const int bT = (rr + ((mi & 1) ? 8 : 0)) * kLdT + half * kHalfT + qn0 + ((mi & 2) ? 8 : 0);
  const int a1o = (rr + ((mi & 1) ? 8 : 0)) * lda1 + ((mi & 2) ? 8 : 0);
  const int a2o = (rr + ((mi & 1) ? 8 : 0)) * lda2 + ((mi & 2) ? 8 : 0);
  int cur = 0;
  for (int64_t t = blockIdx.x; t < nchunks; t += G) {
    {
      const int64_t tn = t + (kStages - 1) * G;
      if (tn < nchunks)
        load_chunk2(s, sS + ((cur + kStages - 1) % kStages) * sstage, tn / cpr, (tn % cpr) * kQ);
      cpa_commit();
    }
    cpa_wait<kStages - 1>();
    __syncthreads();
    // ---- step k: C1 = M_k x stage, rounded into T
    {
      float acc[MT1][2][4];
#pragma unroll
      for (int m = 0; m < MT1; ++m)
#pragma unroll
        for (int n = 0; n < 2; ++n)
#pragma unroll
          for (int e = 0; e < 4; ++e) acc[m][n][e] = 0.f;
      const unsigned bb = su32(sS + cur * sstage + bS), ab = su32(sA1 + a1o);
      for (int k0 = 0; k0 < Kp1; k0 += 16) {
        unsigned b0, b1, b2, b3;
        ldsm4t(bb + (unsigned)(k0 * kLdS * 2), b0, b1, b2, b3);
#pragma unroll
        for (int m = 0; m < MT1; ++m) {
          unsigned a0, a1, a2, a3;
          ldsm4(ab + (unsigned)((m * 16 * lda1 + k0) * 2), a0, a1, a2, a3);
          mma16816(acc[m][0], a0, a1, a2, a3, b0, b1);
          mma16816(acc[m][1], a0, a1, a2, a3, b2, b3);
        }
      }
      // C1[(b, i)][(j', qq)] -> T[(b, j')][(i, qq)]
#pragma unroll
      for (int m = 0; m < MT1; ++m)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int row = m * 16 + g + 8 * h;
          const int b = row >> 1, i = row & 1;
          if (b >= s.r1) continue;
#pragma unroll
          for (int n = 0; n < 2; ++n) {
            const int qq = qn0 + 8 * n + 2 * tq;
            *reinterpret_cast<__nv_bfloat162 *>(sT + (2 * b + half) * kLdT + i * kHalfT + qq) =
                __floats2bfloat162_rn(acc[m][n][2 * h], acc[m][n][2 * h + 1]);
          }
        }
    }
    __syncthreads();
    // ---- step k+1: C2 = M_{k+1} x T, written to HBM
    {
      float acc[MT2][2][4];
#pragma unroll
      for (int m = 0; m < MT2; ++m)
#pragma unroll
        for (int n = 0; n < 2; ++n)
#pragma unroll
          for (int e = 0; e < 4; ++e) acc[m][n][e] = 0.f;
      const unsigned bb = su32(sT + bT), ab = su32(sA2 + a2o);
      for (int k0 = 0; k0 < Kp2; k0 += 16) {
        unsigned b0, b1, b2, b3;
        ldsm4t(bb + (unsigned)(k0 * kLdT * 2), b0, b1, b2, b3);
#pragma unroll
        for (int m = 0; m < MT2; ++m) {
          unsigned a0, a1, a2, a3;
          ldsm4(ab + (unsigned)((m * 16 * lda2 + k0) * 2), a0, a1, a2, a3);
          mma16816(acc[m][0], a0, a1, a2, a3, b0, b1);
          mma16816(acc[m][1], a0, a1, a2, a3, b2, b3);
        }
      }
      const int64_t c = t / cpr, q0 = (t % cpr) * kQ;
      __nv_bfloat16 *out = s.out + c * s.out_rhs_stride;
      int64_t pos[2];
      bool okq[2];
#pragma unroll
      for (int n = 0; n < 2; ++n) {
        const int64_t q = q0 + qn0 + 8 * n + 2 * tq;
        okq[n] = q < nq;
        pos[n] = quad_base(q, s.k) + (half ? bit : 0);  // + i_k 2^k
      }
#pragma unroll
      for (int m = 0; m < MT2; ++m)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int row = m * 16 + g + 8 * h;
          const int cc = row >> 1, i2 = row & 1;
          if (cc >= s.r2) continue;
          __nv_bfloat16 *oc = out + (int64_t)cc * s.N + (i2 ? 2 * bit : 0);
#pragma unroll
          for (int n = 0; n < 2; ++n) {
            if (!okq[n]) continue;
            *reinterpret_cast<__nv_bfloat162 *>(oc + pos[n]) =
                __floats2bfloat162_rn(acc[m][n][2 * h], acc[m][n][2 * h + 1]);
          }
        }
    }
    __syncthreads();  // T and this stage are rewritten next iteration
    cur = (cur + 1) % kStages;
  }
  cpa_wait<0>();
}

template <int MT1, int MT2>
size_t smem2(int Kp1) {
  const int Kp2 = MT1 * 16;
  return sizeof(__nv_bfloat16) *
         ((size_t)MT1 * 16 * (Kp1 + 8) + (size_t)MT2 * 16 * (Kp2 + 8) + (size_t)Kp2 * kLdT +
          (size_t)kStages * Kp1 * kLdS);
}

template <int MT1, int MT2>
cudaError_t launch2(const StepMMA2 &s, cudaStream_t st) {
  // raised once to the largest footprint of this instantiation (Kp1 = 96)
  static cudaError_t attr = cudaFuncSetAttribute(
      step_mma2_kernel<MT1, MT2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)smem2<MT1, MT2>(2 * kMma2MaxRank));
  if (attr != cudaSuccess) return attr;
  const size_t smem = smem2<MT1, MT2>(s.Kp1);
  int per_sm = 1, dev = 0, sms = 148;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_mma2_kernel<MT1, MT2>, kThreads,
                                                smem);
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t nchunks = ((s.N >> 2) + kQ - 1) / kQ * s.nrhs;
  int64_t grid = (int64_t)(per_sm < 1 ? 1 : per_sm) * sms;
  if (grid > nchunks) grid = nchunks;
  step_mma2_kernel<MT1, MT2><<<(unsigned)grid, kThreads, smem, st>>>(s);
  count_launches(1);
  return cudaGetLastError();
}

template <int MT1>
cudaError_t launch2_mt2(const StepMMA2 &s, cudaStream_t st) {
  switch (s.Mp2 / 16) {
    case 2: return launch2<MT1, 2>(s, st);
    case 3: return launch2<MT1, 3>(s, st);
    case 4: return launch2<MT1, 4>(s, st);
    case 5: return launch2<MT1, 5>(s, st);
    case 6: return launch2<MT1, 6>(s, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

bool mma2_steps_eligible(int k, int r0, int r1, int r2, int64_t N) {
  // both steps on the tensor cores, every rank in [16, 48], 8 consecutive
  // quads contiguous (k >= 3), whole 8-quad pieces
  return k >= 3 && r0 >= 16 && r1 >= 16 && r2 >= 16 && r0 <= kMma2MaxRank &&
         r1 <= kMma2MaxRank && r2 <= kMma2MaxRank && (N >> 2) % 8 == 0;
}

cudaError_t launch_step_mma2_bf16(const StepMMA2 &s, cudaStream_t st) {
  switch (s.Mp1 / 16) {
    case 2: return launch2_mt2<2>(s, st);
    case 3: return launch2_mt2<3>(s, st);
    case 4: return launch2_mt2<4>(s, st);
    case 5: return launch2_mt2<5>(s, st);
    case 6: return launch2_mt2<6>(s, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace qtt
