// Reduced-precision core step of the QTT apply (Algorithm 2, one k) on the
// FP32 pipe: FP32 multiply-adds with operands in FP32, TF32 or BF16.
//
//   out[b][p_i] = sum_{a, j} G_k(a, i, j, b) in[a][p_j]   (p_j = p0 | j 2^k)
//
// Numerics per mode (round to nearest even on every conversion):
//   F32  : FP32 cores, FP32 intermediates, FP32 accumulation.
//   TF32 : cores and each input rounded to TF32 (10-bit mantissa) before the
//          multiply, so every product is exact in FP32; FP32 accumulation and
//          FP32 intermediates (the tensor-core TF32 contract).
//   BF16 : BF16 cores, inputs rounded to BF16 when read, intermediates stored
//          in BF16; products exact in FP32, FP32 accumulation (the tensor-core
//          BF16 contract).
// The first step may read FP64/FP32/BF16 vectors and the last step may write
// FP64/FP32/BF16 with an epilogue out = s_acc acc + s_u u (u of the output
// type; u = out gives the in-place update x += P r of refinement, in FP64).
//
// Register tiling: a thread owns TB output ranks x 2 row bits x TN position
// pairs (2 TB TN FP32 accumulators); the 32 lanes of a warp share the rank
// block (broadcast core loads, 2 x 16-byte loads per (a, j)) and read 32
// consecutive pairs (coalesced).  Cores are packed [a][j][b padded to TB][i]
// so the TB x 2 values of one (a, j) are contiguous.
#include "checked.cuh"
#include "qtt_internal.h"
#include "step_lp.h"

namespace qtt {
namespace {

constexpr int kTB = 4;       // output ranks per thread
constexpr int kTN = 4;       // position pairs per thread
constexpr int kWarpsY = 8;   // rank blocks per CTA

__device__ __forceinline__ float tf32_rne(float x) {
  // Round to nearest even at 13 dropped mantissa bits (finite values).
  unsigned u = __float_as_uint(x);
  if ((u & 0x7f800000u) != 0x7f800000u) {
    u += 0x0fffu + ((u >> 13) & 1u);
    u &= 0xffffe000u;
  }
  return __uint_as_float(u);
}

__device__ __forceinline__ float bf16_rne(float x) {
  return __bfloat162float(__float2bfloat16_rn(x));
}

template <int MODE>
__device__ __forceinline__ float round_in(float v) {
  if (MODE == LP_TF32) return tf32_rne(v);
  if (MODE == LP_BF16) return bf16_rne(v);
  return v;
}

__device__ __forceinline__ float ld_as_float(const double *p) { return (float)__ldg(p); }
__device__ __forceinline__ float ld_as_float(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ld_as_float(const __nv_bfloat16 *p) {
  return __bfloat162float(__ldg(p));
}

__device__ __forceinline__ void st_from_float(double *p, float v) { *p = (double)v; }
__device__ __forceinline__ void st_from_float(float *p, float v) { *p = v; }
__device__ __forceinline__ void st_from_float(__nv_bfloat16 *p, float v) {
  *p = __float2bfloat16_rn(v);
}

// Epilogue value s_v v + s_u u + s_acc acc in the output type's precision
// (FP64 for FP64 outputs, FP32 otherwise).
__device__ __forceinline__ double epi_val(const double *u, const double *v, int64_t p,
                                          const StepLP &s, float acc) {
  double t = v ? s.s_v * v[p] : 0.0;
  if (u) t += s.s_u * u[p];
  return t + s.s_acc * (double)acc;
}
__device__ __forceinline__ float epi_val(const float *u, const float *v, int64_t p,
                                         const StepLP &s, float acc) {
  float t = v ? (float)s.s_v * v[p] : 0.0f;
  if (u) t += (float)s.s_u * u[p];
  return t + (float)s.s_acc * acc;
}
__device__ __forceinline__ float epi_val(const __nv_bfloat16 *u, const __nv_bfloat16 *v,
                                         int64_t p, const StepLP &s, float acc) {
  float t = v ? (float)s.s_v * __bfloat162float(v[p]) : 0.0f;
  if (u) t += (float)s.s_u * __bfloat162float(u[p]);
  return t + (float)s.s_acc * acc;
}
__device__ __forceinline__ void st_val(double *p, double v) { *p = v; }
__device__ __forceinline__ void st_val(float *p, float v) { *p = v; }
__device__ __forceinline__ void st_val(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }

// 8 consecutive core values (TB = 4 ranks x 2 row bits) as floats.
__device__ __forceinline__ void ld_core8(const float *g, float (&o)[8]) {
  const float4 a = __ldg(reinterpret_cast<const float4 *>(g));
  const float4 b = __ldg(reinterpret_cast<const float4 *>(g) + 1);
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
  o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
}
__device__ __forceinline__ void ld_core8(const __nv_bfloat16 *g, float (&o)[8]) {
  const uint4 raw = __ldg(reinterpret_cast<const uint4 *>(g));
  const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&raw);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float2 f = __bfloat1622float2(h[q]);
    o[2 * q] = f.x;
    o[2 * q + 1] = f.y;
  }
}

template <int MODE, typename TIN, typename TOUT, typename TCORE>
__global__ void __launch_bounds__(32 * kWarpsY)
step_lp_kernel(StepLP s) {
  // blockIdx.x = pair tile * rank-block groups + group (adjacent CTAs share
  // the input tile through L2)
  const int ngrp = ((s.rout + kTB - 1) / kTB + blockDim.y - 1) / blockDim.y;
  const int bb = (int)(blockIdx.x % ngrp) * blockDim.y + threadIdx.y;  // rank block
  const int b0 = bb * kTB;
  if (b0 >= s.rout) return;
  const int64_t c = QTT_CK(blockIdx.z, s.nrhs, 201);
  const int64_t npairs = s.N >> 1;
  const int64_t bit = (int64_t)1 << s.k;
  const int64_t low = bit - 1;
  const int64_t q0 = (int64_t)(blockIdx.x / ngrp) * (32 * kTN) + threadIdx.x;
  int64_t p0[kTN];
  bool ok[kTN];
#pragma unroll
  for (int m = 0; m < kTN; ++m) {
    const int64_t q = q0 + 32 * m;
    ok[m] = q < npairs;
    p0[m] = ((q & ~low) << 1) | (q & low);
    if (ok[m]) p0[m] = QTT_CK(p0[m], s.N - bit, 202);  // p0 and p0 + 2^k in range
  }
  const TIN *in = static_cast<const TIN *>(s.in) + c * s.in_rhs_stride;
  const TCORE *G = static_cast<const TCORE *>(s.M);
  const int rpad = s.rout_pad;

  float acc[kTB][2][kTN];
#pragma unroll
  for (int t = 0; t < kTB; ++t)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int m = 0; m < kTN; ++m) acc[t][i][m] = 0.0f;

  for (int a = 0; a < s.rin; ++a) {
    const TIN *ina = in + (int64_t)a * s.N;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      float g[8];
      ld_core8(G + ((int64_t)(2 * a + j) * rpad + b0) * 2, g);
      const int64_t sh = j ? bit : 0;
      float v[kTN];
#pragma unroll
      for (int m = 0; m < kTN; ++m)
        v[m] = ok[m] ? round_in<MODE>(ld_as_float(ina + p0[m] + sh)) : 0.0f;
#pragma unroll
      for (int t = 0; t < kTB; ++t)
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int m = 0; m < kTN; ++m) acc[t][i][m] = fmaf(g[2 * t + i], v[m], acc[t][i][m]);
    }
  }

  TOUT *out = static_cast<TOUT *>(s.out) + c * s.out_rhs_stride;
  const TOUT *u = s.epi && s.u ? static_cast<const TOUT *>(s.u) + c * s.u_rhs_stride : nullptr;
  const TOUT *vv = s.epi && s.v ? static_cast<const TOUT *>(s.v) + c * s.u_rhs_stride : nullptr;
#pragma unroll
  for (int t = 0; t < kTB; ++t) {
    const int b = b0 + t;
    if (b >= s.rout) break;
    TOUT *ob = out + (int64_t)b * s.N;
#pragma unroll
    for (int m = 0; m < kTN; ++m) {
      if (!ok[m]) continue;
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int64_t p = p0[m] + (i ? bit : 0);
        if (s.epi)
          st_val(ob + p, epi_val(u, vv, p, s, acc[t][i][m]));
        else if (MODE == LP_TF32 && s.round_tf32_out)
          st_from_float(ob + p, tf32_rne(acc[t][i][m]));
        else
          st_from_float(ob + p, acc[t][i][m]);
      }
    }
  }
}

template <int MODE, typename TIN, typename TOUT, typename TCORE>
cudaError_t launch_t(const StepLP &s, cudaStream_t st) {
  const int64_t npairs = s.N >> 1;
  const int nbb = (s.rout + kTB - 1) / kTB;
  const int by = nbb < kWarpsY ? nbb : kWarpsY;
  const int64_t gx = (npairs + 32 * kTN - 1) / (32 * kTN);
  const int64_t gy = (nbb + by - 1) / by;
  for (int64_t c0 = 0; c0 < s.nrhs; c0 += 65535) {
    StepLP t = s;
    const int64_t nc = (s.nrhs - c0) < 65535 ? (s.nrhs - c0) : 65535;
    t.in = static_cast<const TIN *>(s.in) + c0 * s.in_rhs_stride;
    t.out = static_cast<TOUT *>(s.out) + c0 * s.out_rhs_stride;
    if (t.u) t.u = static_cast<const TOUT *>(s.u) + c0 * s.u_rhs_stride;
    if (t.v) t.v = static_cast<const TOUT *>(s.v) + c0 * s.u_rhs_stride;
    step_lp_kernel<MODE, TIN, TOUT, TCORE>
        <<<dim3((unsigned)(gx * gy), 1, (unsigned)nc), dim3(32, by), 0, st>>>(t);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int MODE, typename TCORE, typename TMID>
cudaError_t dispatch_io(const StepLP &s, cudaStream_t st) {
  // in: x type on the first step, TMID afterwards; out: TMID except the last.
  auto by_out = [&](auto in_tag) -> cudaError_t {
    using TI = decltype(in_tag);
    switch (s.out_type) {
      case QTT_F64: return launch_t<MODE, TI, double, TCORE>(s, st);
      case QTT_BF16: return launch_t<MODE, TI, __nv_bfloat16, TCORE>(s, st);
      default: return launch_t<MODE, TI, float, TCORE>(s, st);
    }
  };
  switch (s.in_type) {
    case QTT_F64: return by_out(double());
    case QTT_BF16: return by_out(__nv_bfloat16());
    default: return by_out(float());
  }
}

}  // namespace

int lp_rank_pad(int r) { return (r + kTB - 1) / kTB * kTB; }

cudaError_t launch_step_lp(const StepLP &s, cudaStream_t st) {
  switch (s.mode) {
    case LP_F32: return dispatch_io<LP_F32, float, float>(s, st);
    case LP_TF32: return dispatch_io<LP_TF32, float, float>(s, st);
    case LP_BF16: return dispatch_io<LP_BF16, __nv_bfloat16, __nv_bfloat16>(s, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace qtt
