// FP32 / TF32 core step on the FP32 pipe with staged inputs (intermediate to
// intermediate steps with k >= 2).
//
// Same contraction as step_lp.cu, reorganised so that memory latency is
// hidden: a persistent CTA keeps the packed core M_k in shared memory and
// streams chunks of 128 position pairs through a three-deep cp.async ring
// ([2a + j][pair] rows of 16-byte pieces; 4 consecutive pairs are 4
// consecutive positions once k >= 2), while its eight warps multiply the
// current chunk: warp w owns output ranks w*TB .. w*TB+TB-1 (TB = 2 ceil(r_out
// / 16)) for all 128 pairs (4 consecutive per lane), so each (a, j) costs one
// 16-byte shared load of the input, TB/2 16-byte broadcast loads of the core
// and 8 TB FMAs.
// TF32 mode: the cores are packed TF32-rounded and the intermediates were
// stored TF32-rounded by the previous step (rounding at the store instead of
// at every use gives the same products), so no rounding happens here except
// on the stored result.
#include "checked.cuh"
#include "qtt_internal.h"
#include "step_lp.h"

namespace qtt {
namespace {

constexpr int kThreads = 256;
constexpr int kPC = 128;      // pairs per chunk
constexpr int kStages = 3;
constexpr int kMaxRankF32s = 48;

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

__device__ __forceinline__ float tf32_round(float x) {
  unsigned u = __float_as_uint(x);
  if ((u & 0x7f800000u) != 0x7f800000u) {
    u += 0x0fffu + ((u >> 13) & 1u);
    u &= 0xffffe000u;
  }
  return __uint_as_float(u);
}

__device__ __forceinline__ void load_chunk(const StepLP &s, float *sb, int64_t c, int64_t q0) {
  const int rows = 2 * s.rin;
  const int64_t bit = (int64_t)1 << s.k, low = bit - 1, npairs = s.N >> 1;
  const float *in = static_cast<const float *>(s.in) + c * s.in_rhs_stride;
  const int pc = threadIdx.x & 31;  // piece: pairs 4 pc .. 4 pc + 3
  const int64_t q = q0 + 4 * pc;
  const bool ok = q < npairs;
  const float *base = in + (((q & ~low) << 1) | (q & low));
  for (int kk = threadIdx.x >> 5; kk < rows; kk += kThreads / 32) {
    const float *src = base + (int64_t)(kk >> 1) * s.N + ((kk & 1) ? bit : 0);
    cpa16(su32(sb + kk * kPC + 4 * pc), ok ? src : s.in, ok ? 16 : 0);
  }
}

// Lane `lane` owns the 4 consecutive pairs 4 lane .. 4 lane + 3 of the chunk
// (one 16-byte shared load per (a, j)); the warp owns output ranks b0 ..
// b0 + TB - 1 (TB even), read two at a time as one 16-byte broadcast load
// ((b, i=0), (b, i=1), (b+1, i=0), (b+1, i=1)).  Per (a, j): 1 + TB/2 loads
// for 8 TB FMAs.  Results leave as 16-byte stores (4 consecutive positions).
template <int TB>
__device__ __forceinline__ void chunk_block(const float *sb, const float *sG, const StepLP &s,
                                            int b0, int lane, float *out, int64_t q0,
                                            bool tf32) {
  // acc[t][m] = (output i = 0, output i = 1) of rank b0 + t at the lane's
  // pair m: the coefficients (b, 0), (b, 1) sit side by side in the core
  // row, so each multiply-add is one two-lane FP32 FMA (each lane rounded
  // as fmaf) with the input value in both lanes
  float2 acc[TB][4];
#pragma unroll
  for (int t = 0; t < TB; ++t)
#pragma unroll
    for (int m = 0; m < 4; ++m) acc[t][m] = make_float2(0.0f, 0.0f);
  const int rpad = s.rout_pad;
#pragma unroll 4
  for (int kk = 0; kk < 2 * s.rin; ++kk) {
    const float4 v = *reinterpret_cast<const float4 *>(sb + kk * kPC + 4 * lane);
    const float2 vv[4] = {make_float2(v.x, v.x), make_float2(v.y, v.y), make_float2(v.z, v.z),
                          make_float2(v.w, v.w)};
    const float4 *g4 = reinterpret_cast<const float4 *>(sG + (kk * rpad + b0) * 2);
#pragma unroll
    for (int t2 = 0; t2 < TB / 2; ++t2) {
      // ranks past the padded row contribute nothing (rpad is a multiple of 4)
      const float4 g = b0 + 2 * t2 < rpad ? g4[t2] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float2 gp[2] = {make_float2(g.x, g.y), make_float2(g.z, g.w)};
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int m = 0; m < 4; ++m) acc[2 * t2 + h][m] = __ffma2_rn(gp[h], vv[m], acc[2 * t2 + h][m]);
    }
  }
  const int64_t bit = (int64_t)1 << s.k, low = bit - 1, npairs = s.N >> 1;
  const int64_t q = q0 + 4 * lane;
  if (q >= npairs) return;
  const int64_t p0 = QTT_CK(((q & ~low) << 1) | (q & low), s.N - bit, 203);
#pragma unroll
  for (int t = 0; t < TB; ++t) {
    const int b = b0 + t;
    if (b >= s.rout) break;
    float *ob = out + (int64_t)b * s.N + p0;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      float4 o = i ? make_float4(acc[t][0].y, acc[t][1].y, acc[t][2].y, acc[t][3].y)
                   : make_float4(acc[t][0].x, acc[t][1].x, acc[t][2].x, acc[t][3].x);
      if (tf32) {
        o.x = tf32_round(o.x);
        o.y = tf32_round(o.y);
        o.z = tf32_round(o.z);
        o.w = tf32_round(o.w);
      }
      *reinterpret_cast<float4 *>(ob + (i ? bit : 0)) = o;
    }
  }
}

__global__ void __launch_bounds__(kThreads) step_f32s_kernel(StepLP s) {
  extern __shared__ __align__(16) float smf[];
  const int rows = 2 * s.rin, rpad = s.rout_pad;
  const int gfl = (rows * 2 * rpad + 3) / 4 * 4;  // core floats, 16-byte aligned end
  float *sG = smf;
  float *sB = smf + gfl;
  const size_t stage = (size_t)rows * kPC;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool tf32 = s.mode == LP_TF32;
  const float *G = static_cast<const float *>(s.M);
  for (int e = tid; e < rows * 2 * rpad; e += kThreads) sG[e] = __ldg(G + e);

  const int64_t npairs = s.N >> 1;
  const int64_t cpr = (npairs + kPC - 1) / kPC;
  const int64_t nchunks = cpr * s.nrhs;
  const int64_t Gs = gridDim.x;
#pragma unroll
  for (int st = 0; st < kStages - 1; ++st) {
    const int64_t t = blockIdx.x + st * Gs;
    if (t < nchunks) load_chunk(s, sB + st * stage, t / cpr, (t % cpr) * kPC);
    cpa_commit();
  }
  const int TB = 2 * ((s.rout + 15) / 16);  // even; 8 warps x TB >= r_out
  const int b0 = warp * TB;
  int cur = 0;
  for (int64_t t = blockIdx.x; t < nchunks; t += Gs) {
    {
      const int64_t tn = t + (kStages - 1) * Gs;
      if (tn < nchunks)
        load_chunk(s, sB + ((cur + kStages - 1) % kStages) * stage, tn / cpr, (tn % cpr) * kPC);
      cpa_commit();
    }
    cpa_wait<kStages - 1>();
    __syncthreads();
    const float *sb = sB + cur * stage;
    const int64_t c = QTT_CK(t / cpr, s.nrhs, 204), q0 = (t % cpr) * kPC;
    float *out = static_cast<float *>(s.out) + c * s.out_rhs_stride;
    if (b0 < s.rout) {
      switch (TB) {
        case 2: chunk_block<2>(sb, sG, s, b0, lane, out, q0, tf32); break;
        case 4: chunk_block<4>(sb, sG, s, b0, lane, out, q0, tf32); break;
        default: chunk_block<6>(sb, sG, s, b0, lane, out, q0, tf32); break;
      }
    }
    __syncthreads();  // the stage is refilled next iteration
    cur = (cur + 1) % kStages;
  }
  cpa_wait<0>();
}

size_t f32s_smem(int rin, int rpad) {
  const int rows = 2 * rin;
  const size_t gfl = (size_t)(rows * 2 * rpad + 3) / 4 * 4;
  return sizeof(float) * (gfl + (size_t)kStages * rows * kPC);
}

}  // namespace

bool f32s_step_eligible(const StepLP &s) {
  // ranks <= 48 keep the core plus three stages within one CTA's shared memory
  return (s.mode == LP_F32 || s.mode == LP_TF32) && s.k >= 2 && s.in_type == QTT_F32 &&
         s.out_type == QTT_F32 && !s.epi && s.rin <= kMaxRankF32s &&
         s.rout <= kMaxRankF32s && s.rout >= 2 && (s.N >> 1) % 4 == 0;
}

cudaError_t launch_step_f32s(const StepLP &s, cudaStream_t st) {
  // the kernel's shared-memory limit is raised once to the largest footprint
  static cudaError_t attr = cudaFuncSetAttribute(
      step_f32s_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)f32s_smem(kMaxRankF32s, (kMaxRankF32s + 3) / 4 * 4));
  if (attr != cudaSuccess) return attr;
  const size_t smem = f32s_smem(s.rin, s.rout_pad);
  int per_sm = 1, dev = 0, sms = 148;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_f32s_kernel, kThreads, smem);
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t nchunks = ((s.N >> 1) + kPC - 1) / kPC * s.nrhs;
  int64_t grid = (int64_t)(per_sm < 1 ? 1 : per_sm) * sms;
  if (grid > nchunks) grid = nchunks;
  step_f32s_kernel<<<(unsigned)grid, kThreads, smem, st>>>(s);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace qtt
