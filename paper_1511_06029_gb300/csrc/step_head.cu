// The first m core steps (m = 2 or 3, every rank r_1 .. r_m <= 8) of a
// reduced-precision apply in one launch.
//
// Steps 0 .. m-1 of Algorithm 2 mix only position bits 0 .. m-1, so the 2^m
// consecutive positions 2^m g .. 2^m g + 2^m - 1 are closed under them.  Two
// lanes share a group (2^(m-1) positions each): steps 0 .. m-2 run in each
// lane's registers, step m-1 (bit m-1 = the lane parity) exchanges the
// partner's half with one shuffle per value.  Each lane writes r_m planes of
// 2^(m-1) values (one vector store each).  The apply reads x once and writes
// y_m once instead of moving y_1 .. y_{m-1} through HBM, and a warp's
// accesses are contiguous.
//
// The cores travel by value in the launch parameters, so every multiply
// takes its core value as a constant-bank operand (no load instruction).
//
// Numerics are those of the one-step kernel (step_lp.cu) step by step: the
// input rounded to the mode's precision when read, each intermediate rounded
// to it (BF16 or TF32) as the one-step kernel stores it, FP32 sums over
// (a, j) in the same order -- so the result is bitwise that of m separate
// launches.
#include <cuda_bf16.h>

#include <atomic>

#include "checked.cuh"
#include "qtt_internal.h"
#include "step_lp.h"
#include "tc_common.cuh"
#include "tf32.cuh"

namespace qtt {
namespace {

constexpr int kR = kHeadMaxRank;  // register tile bound on every rank
constexpr int kThreads = 256;

template <int MODE>
__device__ __forceinline__ float round_mode(float v) {
  if (MODE == LP_TF32) return tf32_rn(v);
  if (MODE == LP_BF16) return __bfloat162float(__float2bfloat16_rn(v));
  return v;
}
// Two multiply-adds as one two-lane FP32 FMA, each lane rounded as fmaf:
// (z0, z1) += (g.x, g.y) v, and (z0, z1) += g (v0, v1).
__device__ __forceinline__ void fma_pair(float2 g, float v, float &z0, float &z1) {
  const float2 r = __ffma2_rn(g, make_float2(v, v), make_float2(z0, z1));
  z0 = r.x;
  z1 = r.y;
}
__device__ __forceinline__ void fma_both(float g, float v0, float v1, float &z0, float &z1) {
  const float2 r = __ffma2_rn(make_float2(g, g), make_float2(v0, v1), make_float2(z0, z1));
  z0 = r.x;
  z1 = r.y;
}
__device__ __forceinline__ float to_f(double v) { return (float)v; }
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
// T consecutive input values: one vector load when the address allows it
// (the caller's x may have any leading dimension), else scalar loads.
template <int T, typename TIN>
__device__ __forceinline__ void load_vec(const TIN *p, TIN (&v)[T]) {
  constexpr int bytes = T * (int)sizeof(TIN);
  if (bytes >= 4 && (reinterpret_cast<uintptr_t>(p) & (bytes > 16 ? 15 : bytes - 1)) == 0) {
    if (bytes <= 16) {
      if (bytes == 16) {
        const uint4 w = __ldg(reinterpret_cast<const uint4 *>(p));
        memcpy(v, &w, 16);
      } else if (bytes == 8) {
        const uint2 w = __ldg(reinterpret_cast<const uint2 *>(p));
        memcpy(v, &w, 8);
      } else {
        const unsigned w = __ldg(reinterpret_cast<const unsigned *>(p));
        memcpy(v, &w, 4);
      }
    } else {
#pragma unroll
      for (int q = 0; q < bytes / 16; ++q) {
        const uint4 w = __ldg(reinterpret_cast<const uint4 *>(p) + q);
        memcpy(reinterpret_cast<char *>(v) + 16 * q, &w, 16);
      }
    }
    return;
  }
#pragma unroll
  for (int q = 0; q < T; ++q) v[q] = p[q];
}

// T consecutive values as one vector store (T = 2 or 4; the scratch planes
// are 16-byte aligned and T divides every plane offset used).
template <int T>
__device__ __forceinline__ void store_vec(float *o, const float *v) {
  if (T == 4)
    *reinterpret_cast<float4 *>(o) = make_float4(v[0], v[1], v[2], v[3]);
  else
    *reinterpret_cast<float2 *>(o) = make_float2(v[0], v[1]);
}
template <int T>
__device__ __forceinline__ void store_vec(__nv_bfloat16 *o, const float *v) {
  __nv_bfloat162 h0 = __floats2bfloat162_rn(v[0], v[1]);
  if (T == 4) {
    __nv_bfloat162 h1 = __floats2bfloat162_rn(v[2], v[3]);
    *reinterpret_cast<uint2 *>(o) =
        make_uint2(*reinterpret_cast<unsigned *>(&h0), *reinterpret_cast<unsigned *>(&h1));
  } else {
    *reinterpret_cast<__nv_bfloat162 *>(o) = h0;
  }
}

// HALF: the ranks are 1, 2, 4, 8 (M = 3), known at compile time, so the
// loops over ranks unroll without bounds tests and no dead plane is zeroed
// or rounded; otherwise they come from s.r (every rank <= 8).
template <int MODE, typename TIN, typename TMID, int M, bool HALF>
__global__ void __launch_bounds__(kThreads, 2) step_head_kernel(const __grid_constant__ StepHead s) {
  static_assert(!HALF || M == 3, "the halving profile has three steps");
  constexpr int P = 1 << M;   // positions of a group
  constexpr int T = P / 2;    // positions per thread: two lanes share a group
  // lane pair (2 g, 2 g + 1) holds group g: the lane with h = 1 the positions
  // with bit M-1 set.  Inactive lanes (past the end) still take part in the
  // shuffles of the last step.
  const int64_t groups = s.N >> M;
  const int64_t tidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = tidx < 2 * groups;
  const int h = (int)(tidx & 1);
  const int64_t c = QTT_CK(blockIdx.y, s.nrhs, 205);
  int64_t pbase = (tidx >> 1) * P + h * T;  // first position of this thread
  if (active) pbase = QTT_CK(pbase, s.N - T + 1, 206);  // pbase .. pbase + T - 1
  float y[kR][T], z[kR][T];
  {
    const TIN *in = static_cast<const TIN *>(s.in) + c * s.in_rhs_stride + pbase;
    TIN xv[T];
    if (active) load_vec<T>(in, xv);
#pragma unroll
    for (int q = 0; q < T; ++q) y[0][q] = active ? round_mode<MODE>(to_f(xv[q])) : 0.0f;
  }
  int rin = 1;
#pragma unroll
  for (int k = 0; k < M; ++k) {
    const int rout = HALF ? 2 << k : s.r[k + 1];
#pragma unroll
    for (int b = 0; b < kR; ++b)
#pragma unroll
      for (int q = 0; q < T; ++q) z[b][q] = 0.0f;
    if (k < M - 1) {
      // bit k lies inside the thread's T positions
#pragma unroll
      for (int a = 0; a < kR; ++a) {
        if (a >= rin) break;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
#pragma unroll
          for (int b = 0; b < kR; ++b) {
            if (b >= rout) break;
            const float2 g = make_float2(s.G[k][2 * a + j][b][0], s.G[k][2 * a + j][b][1]);
#pragma unroll
            for (int q = 0; q < T; ++q) {
              if (((q >> k) & 1) != 0) continue;  // q = pair base (bit k clear)
              const float v = y[a][q | (j << k)];
              fma_pair(g, v, z[b][q], z[b][q | (1 << k)]);
            }
          }
        }
      }
    } else {
      // bit M-1 is the lane parity: the partner lane holds the other half;
      // every output of this lane has i = h
#pragma unroll
      for (int a = 0; a < kR; ++a) {
        if (a >= rin) break;  // uniform over the warp: rin is the same everywhere
        float other[T];
#pragma unroll
        for (int q = 0; q < T; ++q) other[q] = __shfl_xor_sync(0xffffffffu, y[a][q], 1);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
#pragma unroll
          for (int b = 0; b < kR; ++b) {
            if (b >= rout) break;
            const float g = h ? s.G[k][2 * a + j][b][1] : s.G[k][2 * a + j][b][0];
#pragma unroll
            for (int q = 0; q < T; q += 2)
              fma_both(g, j == h ? y[a][q] : other[q], j == h ? y[a][q + 1] : other[q + 1],
                       z[b][q], z[b][q + 1]);
          }
        }
      }
    }
#pragma unroll
    for (int b = 0; b < kR; ++b)
#pragma unroll
      for (int q = 0; q < T; ++q) y[b][q] = round_mode<MODE>(z[b][q]);
    rin = rout;
  }
  if (!active) return;
  TMID *out = static_cast<TMID *>(s.out) + c * s.out_rhs_stride + pbase;
#pragma unroll
  for (int b = 0; b < kR; ++b) {
    if (b >= rin) break;
    store_vec<T>(out + (int64_t)b * s.N, y[b]);
  }
}

template <int MODE, typename TIN, typename TMID>
cudaError_t launch_m(const StepHead &s, cudaStream_t st) {
  const int64_t groups = s.N >> s.m;
  const unsigned gx = (unsigned)((2 * groups + kThreads - 1) / kThreads);
  for (int64_t c0 = 0; c0 < s.nrhs; c0 += 65535) {
    StepHead t = s;
    const int64_t nc = (s.nrhs - c0) < 65535 ? (s.nrhs - c0) : 65535;
    t.in = static_cast<const TIN *>(s.in) + c0 * s.in_rhs_stride;
    t.out = static_cast<TMID *>(s.out) + c0 * s.out_rhs_stride;
    if (s.m == 2)
      step_head_kernel<MODE, TIN, TMID, 2, false><<<dim3(gx, (unsigned)nc), kThreads, 0, st>>>(t);
    else if (s.r[1] == 2 && s.r[2] == 4 && s.r[3] == 8)
      step_head_kernel<MODE, TIN, TMID, 3, true><<<dim3(gx, (unsigned)nc), kThreads, 0, st>>>(t);
    else
      step_head_kernel<MODE, TIN, TMID, 3, false><<<dim3(gx, (unsigned)nc), kThreads, 0, st>>>(t);
    count_launches(1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int MODE, typename TMID>
cudaError_t by_input(const StepHead &s, cudaStream_t st) {
  switch (s.in_type) {
    case QTT_F64: return launch_m<MODE, double, TMID>(s, st);
    case QTT_BF16: return launch_m<MODE, __nv_bfloat16, TMID>(s, st);
    default: return launch_m<MODE, float, TMID>(s, st);
  }
}

// ------------------------------------------------------------------ tail
// Steps d-m .. d-1 mix only position bits d-m .. d-1 (the top bits), so the
// 2^m positions p + t 2^(d-m) (t < 2^m) are closed under them.  As in the
// head, a lane pair holds one such group (the lane parity is the top bit),
// steps d-m .. d-2 run in registers and step d-1 exchanges halves by
// shuffles; the last step's FP32 result goes to y through the one-step
// kernel's output conversion and epilogue, so the result is bitwise that of
// m separate launches.

// s_v v + s_u u + s_acc acc in the output type's precision (FP64 for FP64
// outputs, FP32 otherwise), as the one-step kernel's last step computes it.
__device__ __forceinline__ double tail_epi(const double *u, const double *v, int64_t p,
                                           const StepTail &s, float acc) {
  double t = v ? s.s_v * v[p] : 0.0;
  if (u) t += s.s_u * u[p];
  return t + s.s_acc * (double)acc;
}
__device__ __forceinline__ float tail_epi(const float *u, const float *v, int64_t p,
                                          const StepTail &s, float acc) {
  float t = v ? (float)s.s_v * v[p] : 0.0f;
  if (u) t += (float)s.s_u * u[p];
  return t + (float)s.s_acc * acc;
}
__device__ __forceinline__ float tail_epi(const __nv_bfloat16 *u, const __nv_bfloat16 *v,
                                          int64_t p, const StepTail &s, float acc) {
  float t = v ? (float)s.s_v * __bfloat162float(v[p]) : 0.0f;
  if (u) t += (float)s.s_u * __bfloat162float(u[p]);
  return t + (float)s.s_acc * acc;
}
__device__ __forceinline__ void st_out(double *p, double v) { *p = v; }
__device__ __forceinline__ void st_out(float *p, float v) { *p = v; }
__device__ __forceinline__ void st_out(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void st_acc(double *p, float v) { *p = (double)v; }
__device__ __forceinline__ void st_acc(float *p, float v) { *p = v; }
__device__ __forceinline__ void st_acc(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }

// Steps d-m .. d-1 on one lane's half of a group: y[a][q] holds plane a of
// y_{d-m} (rounded to the mode's precision) at the lane's positions
// p + (q + h T) 2^(d-m); on return z[0][q] is the FP32 sum of the last step
// (r_d = 1) at those positions.  Steps d-m .. d-2 run in registers, step d-1
// (the top bit, = h) exchanges halves with the partner lane by shuffles, so
// all 32 lanes of the warp call it together.  Every output is summed over
// (a, j) in ascending order, intermediates rounded as the one-step kernel
// stores them.
// HALF: the ranks are 8, 4, 2, 1 (M = 3), known at compile time (as in the
// head kernel); otherwise they come from s.r (every rank <= 8).
template <int MODE, int M, bool HALF>
__device__ __forceinline__ void tail_math(const StepTail &s, int h, float (&y)[kR][1 << (M - 1)],
                                          float (&z)[kR][1 << (M - 1)]) {
  constexpr int T = 1 << (M - 1);
  int rin = HALF ? 8 : s.r[0];
#pragma unroll
  for (int k = 0; k < M; ++k) {
    const int rout = HALF ? 4 >> k : s.r[k + 1];
#pragma unroll
    for (int b = 0; b < kR; ++b)
#pragma unroll
      for (int q = 0; q < T; ++q) z[b][q] = 0.0f;
    if (k < M - 1) {
#pragma unroll
      for (int a = 0; a < kR; ++a) {
        if (a >= rin) break;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
#pragma unroll
          for (int b = 0; b < kR; ++b) {
            if (b >= rout) break;
            const float2 g = make_float2(s.G[k][2 * a + j][b][0], s.G[k][2 * a + j][b][1]);
#pragma unroll
            for (int q = 0; q < T; ++q) {
              if (((q >> k) & 1) != 0) continue;  // q = pair base (bit k clear)
              const float v = y[a][q | (j << k)];
              fma_pair(g, v, z[b][q], z[b][q | (1 << k)]);
            }
          }
        }
      }
#pragma unroll
      for (int b = 0; b < kR; ++b)
#pragma unroll
        for (int q = 0; q < T; ++q) y[b][q] = round_mode<MODE>(z[b][q]);
    } else {
#pragma unroll
      for (int a = 0; a < kR; ++a) {
        if (a >= rin) break;
        float other[T];
#pragma unroll
        for (int q = 0; q < T; ++q) other[q] = __shfl_xor_sync(0xffffffffu, y[a][q], 1);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
#pragma unroll
          for (int b = 0; b < kR; ++b) {
            if (b >= rout) break;
            const float g = h ? s.G[k][2 * a + j][b][1] : s.G[k][2 * a + j][b][0];
#pragma unroll
            for (int q = 0; q < T; q += 2)
              fma_both(g, j == h ? y[a][q] : other[q], j == h ? y[a][q + 1] : other[q + 1],
                       z[b][q], z[b][q + 1]);
          }
        }
      }
    }
    rin = rout;
  }
}

// The last step's accumulator z at position p of right-hand side c, through
// the one-step kernel's output conversion and epilogue.
template <typename TOUT>
__device__ __forceinline__ void tail_store(const StepTail &s, int64_t c, int64_t p, float z) {
  TOUT *out = static_cast<TOUT *>(s.out) + c * s.out_rhs_stride;
  if (s.epi) {
    const TOUT *u = s.u ? static_cast<const TOUT *>(s.u) + c * s.u_rhs_stride : nullptr;
    const TOUT *v = s.v ? static_cast<const TOUT *>(s.v) + c * s.u_rhs_stride : nullptr;
    st_out(out + p, tail_epi(u, v, p, s, z));
  } else {
    st_acc(out + p, z);
  }
}

// One thread per (low position, half), plain loads: the form for small
// problems and unaligned intermediates.  The intermediate arrives in the
// mode's precision (every kernel that writes one rounds it), so it is read
// as it is.
template <int MODE, typename TMID, typename TOUT, int M, bool HALF>
__global__ void __launch_bounds__(kThreads, 2) step_tail_kernel(const __grid_constant__ StepTail s) {
  static_assert(!HALF || M == 3, "the halving profile has three steps");
  constexpr int P = 1 << M;
  constexpr int T = P / 2;
  const int64_t lowN = (int64_t)1 << s.k0;      // positions below the tail's bits
  const int64_t tidx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = tidx < 2 * lowN;
  const int h = (int)(tidx & 1);
  const int64_t plow = active ? QTT_CK(tidx >> 1, lowN, 208) : tidx >> 1;
  const int64_t c = QTT_CK(blockIdx.y, s.nrhs, 207);
  auto pos = [&](int q) { return plow + ((int64_t)(q + h * T) << s.k0); };
  float y[kR][T], z[kR][T];
  {
    const TMID *in = static_cast<const TMID *>(s.in) + c * s.in_rhs_stride;
#pragma unroll
    for (int a = 0; a < kR; ++a)
#pragma unroll
      for (int q = 0; q < T; ++q)
        y[a][q] = active && a < (HALF ? 8 : s.r[0]) ? to_f(in[(int64_t)a * s.N + pos(q)]) : 0.0f;
  }
  tail_math<MODE, M, HALF>(s, h, y, z);
  if (!active) return;
  // r_d = 1: the last step's accumulators z[0][q] are y at pos(q)
#pragma unroll
  for (int q = 0; q < T; ++q) tail_store<TOUT>(s, c, pos(q), z[0][q]);
}

// ------------------------------------------------------- staged tail
// The plain tail kernel reads, per warp, 2^m r_{d-m} runs of 64 bytes that
// lie 2^(d-m) positions apart; with every SM doing the same, the DRAM serves
// short runs from many rows at once.  The staged form is persistent: a tile
// is kTailPos consecutive low positions of one right-hand side, and one
// producer thread per CTA brings all of its r_{d-m} 2^m runs into shared
// memory with one TMA load of a 4-D box (positions, top bits, planes, one
// right-hand side), `stages` tiles ahead.  The box is a few positions wider
// than the tile (the next tile's first values, or zeros past the end) so
// that its rows land 64/T bytes further apart than kTailPos elements.  Two or three CTAs share an SM (as registers
// allow), so their compute warps, which all wake on the same barrier within
// a CTA, do not all wait at once.  The compute warps take lane pairs as the
// plain kernel does, read their values from shared memory and run the same
// arithmetic (tail_math), so the two forms agree bitwise.
//
// The intermediate arrives in the mode's precision (every kernel that
// writes one rounds it: BF16 storage, TF32-rounded FP32), so it is not
// rounded again when read.
//
// Every wait is bounded; a compute warp decides uniformly (all lanes) to
// stop, and the producer, once stopped, waits (bounded) for its copies in
// flight before the CTA leaves.  A timeout is recorded in g_tail_status.
constexpr int kTailPos = 128;                    // low positions per tile
constexpr int kTailCompute = 2 * kTailPos;       // two lanes per position
constexpr int kTailThreads = kTailCompute + 32;  // + the producer warp
constexpr int kTailMaxStages = 8;
constexpr unsigned kTailSmemPerSM = 210 * 1024;  // shared by the CTAs of an SM

__device__ int g_tail_status = 0;

// Row pitch of a staged run: kTailPos elements plus 64/T bytes, so that the
// two lanes of a pair (rows T apart) read banks 16 words apart.
template <typename TMID, int T>
__host__ __device__ constexpr unsigned tail_row_bytes() {
  return kTailPos * (unsigned)sizeof(TMID) + 64u / T;
}

// Box width in elements (kTailPos plus the row pad).
template <typename TMID, int T>
__host__ __device__ constexpr unsigned tail_box_x() {
  return tail_row_bytes<TMID, T>() / (unsigned)sizeof(TMID);
}

template <int MODE, typename TMID, typename TOUT, int M, bool HALF>
__global__ void __launch_bounds__(kTailThreads, 2)
    step_tail_staged_kernel(const __grid_constant__ CUtensorMap tin,
                            const __grid_constant__ StepTail s, int stages, int64_t tiles) {
  using namespace tcx;
  static_assert(!HALF || M == 3, "the halving profile has three steps");
  constexpr int P = 1 << M;
  constexpr int T = P / 2;
  constexpr unsigned row = tail_row_bytes<TMID, T>();
  extern __shared__ __align__(128) unsigned char tile_smem[];
  __shared__ __align__(8) uint64_t full[kTailMaxStages], empty[kTailMaxStages];
  __shared__ int abort_flag;
  const int r0 = HALF ? 8 : s.r[0];
  const unsigned stage_bytes = (unsigned)(r0 * P) * row;
  const int64_t tpr = ((int64_t)1 << s.k0) / kTailPos;  // tiles per right-hand side
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int i = 0; i < stages; ++i) {
      mbar_init(su32(&full[i]), 1);
      mbar_init(su32(&empty[i]), kTailCompute / 32);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  volatile int *abort = &abort_flag;
  const unsigned sbase = (su32(tile_smem) + 127u) & ~127u;  // TMA destinations: 128-byte aligned
  const unsigned char *tiles_base = tile_smem + (sbase - su32(tile_smem));

  if (tid >= kTailCompute) {
    if (tid != kTailCompute) return;
    // producer: tile t = (c, w), runs (a, q) at a N + q 2^k0 + w kTailPos
    int64_t n = 0;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x, ++n) {
      const int st = (int)(n % stages);
      if (n >= stages && !wait_bar(su32(&empty[st]), (unsigned)(n / stages - 1) & 1u, abort)) break;
      const int64_t c = QTT_CK(t / tpr, s.nrhs, 209);
      const int64_t w = t % tpr;
      const unsigned fb = su32(&full[st]);
      expect_tx(fb, stage_bytes);  // the whole box, zeros past the end included
      tma_load4(sbase + (unsigned)st * stage_bytes, &tin, (int)(w * kTailPos), 0, 0, (int)c, fb);
    }
    if (*abort) {
      volatile int never = 0;
      for (int64_t m = n - stages < 0 ? 0 : n - stages; m < n; ++m)
        wait_bar(su32(&full[m % stages]), (unsigned)(m / stages) & 1u, &never);
      atomicCAS(&g_tail_status, 0, (int)QTT_ERR_TIMEOUT);
    }
    return;
  }
  // compute lanes: pair (2 l, 2 l + 1) holds low position l of the tile
  const int h = tid & 1;
  const int pl = tid >> 1;
  int64_t n = 0;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x, ++n) {
    const int st = (int)(n % stages);
    const bool ok = wait_bar(su32(&full[st]), (unsigned)(n / stages) & 1u, abort);
    if (!__all_sync(0xffffffffu, ok)) {
      *abort = 1;
      break;
    }
    const unsigned char *stg = tiles_base + (size_t)st * stage_bytes + (size_t)pl * sizeof(TMID);
    float y[kR][T], z[kR][T];
#pragma unroll
    for (int a = 0; a < kR; ++a)
#pragma unroll
      for (int q = 0; q < T; ++q)
        y[a][q] = a < r0 ? to_f(*reinterpret_cast<const TMID *>(
                               stg + (size_t)(a * P + q + h * T) * row))
                         : 0.0f;
    __syncwarp();
    if ((tid & 31) == 0) mbar_arrive(su32(&empty[st]));
    tail_math<MODE, M, HALF>(s, h, y, z);
    const int64_t c = t / tpr;
    const int64_t plow = (t % tpr) * kTailPos + pl;
#pragma unroll
    for (int q = 0; q < T; ++q)
      tail_store<TOUT>(s, c, plow + ((int64_t)(q + h * T) << s.k0), z[0][q]);
  }
  if (*abort && tid == 0) atomicCAS(&g_tail_status, 0, (int)QTT_ERR_TIMEOUT);
}

template <int MODE, typename TMID, typename TOUT, int M, bool HALF>
cudaError_t launch_tail_staged(const StepTail &s, cudaStream_t st) {
  constexpr int T = 1 << (M - 1);
  auto kern = step_tail_staged_kernel<MODE, TMID, TOUT, M, HALF>;
  const int r0 = HALF ? 8 : s.r[0];
  const unsigned stage_bytes = (unsigned)(r0 * 2 * T) * tail_row_bytes<TMID, T>();
  static cudaError_t attr = cudaFuncSetAttribute(
      kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemPerSM / 2 + 128);
  if (attr != cudaSuccess) return attr;
  // 4-D view of the intermediate: positions below bit k0, the m top bits,
  // the r_{d-m} planes, the right-hand sides
  CUtensorMap tin;
  {
    const cuuint64_t es = sizeof(TMID);
    const cuuint64_t dims[4] = {(cuuint64_t)1 << s.k0, (cuuint64_t)(2 * T), (cuuint64_t)r0,
                                (cuuint64_t)s.nrhs};
    const cuuint64_t strides[3] = {((cuuint64_t)1 << s.k0) * es, (cuuint64_t)s.N * es,
                                   (cuuint64_t)s.in_rhs_stride * es};
    const cuuint32_t box[4] = {tail_box_x<TMID, T>(), (cuuint32_t)(2 * T), (cuuint32_t)r0, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const PFN_cuTensorMapEncodeTiled_v12000 encode = tcx::tensor_map_encoder();
    if (!encode ||
        encode(&tin,
               sizeof(TMID) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
               4, const_cast<void *>(s.in), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorNotSupported;
  }
  // CTAs per SM as registers allow (at most 3), then the stages that fit
  // their share of shared memory; worked out once per rank r_{d-m} (the
  // occupancy query costs more host time than a small tail's kernel)
  static std::atomic<int> plan_for_r0[kR + 1];
  int per_sm = 0, stages = 0;
  const int cached = plan_for_r0[r0].load(std::memory_order_relaxed);
  if (cached) {
    per_sm = cached >> 8;
    stages = cached & 255;
  } else {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, kern, kTailThreads, 2 * (size_t)stage_bytes + 128);
    if (e != cudaSuccess) return e;
    if (per_sm > 3) per_sm = 3;
    for (; per_sm >= 1; --per_sm) {
      stages = (int)(kTailSmemPerSM / (unsigned)per_sm / stage_bytes);
      if (stages > kTailMaxStages) stages = kTailMaxStages;
      if ((size_t)stages * stage_bytes > kTailSmemPerSM / 2)
        stages = (int)(kTailSmemPerSM / 2 / stage_bytes);
      if (stages >= 2) break;
    }
    if (per_sm < 1 || stages < 2) return cudaErrorNotSupported;
    plan_for_r0[r0].store(per_sm << 8 | stages, std::memory_order_relaxed);
  }
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles = (((int64_t)1 << s.k0) / kTailPos) * s.nrhs;
  const int64_t cap = (int64_t)sms * per_sm;
  const unsigned grid = (unsigned)(tiles < cap ? tiles : cap);
  kern<<<grid, kTailThreads, (size_t)stages * stage_bytes + 128, st>>>(tin, s, stages, tiles);
  count_launches(1);
  return cudaGetLastError();
}

// The staged form needs whole tiles (2^k0 a multiple of kTailPos) and every
// run 16-byte aligned: the intermediate's base, plane and right-hand-side
// strides in bytes multiples of 16.
template <typename TMID>
bool tail_staged_eligible(const StepTail &s) {
  const int64_t e = (int64_t)sizeof(TMID);
  return s.k0 >= 7 && (reinterpret_cast<uintptr_t>(s.in) & 15) == 0 && (s.N * e) % 16 == 0 &&
         (s.in_rhs_stride * e) % 16 == 0 && s.nrhs >= 1;
}

template <int MODE, typename TMID, typename TOUT>
cudaError_t launch_tail_t(const StepTail &s, cudaStream_t st) {
  if (tail_staged_eligible<TMID>(s)) {
    if (s.m == 2) return launch_tail_staged<MODE, TMID, TOUT, 2, false>(s, st);
    if (s.r[0] == 8 && s.r[1] == 4 && s.r[2] == 2)
      return launch_tail_staged<MODE, TMID, TOUT, 3, true>(s, st);
    return launch_tail_staged<MODE, TMID, TOUT, 3, false>(s, st);
  }
  const int64_t lanes = (int64_t)2 << s.k0;
  const unsigned gx = (unsigned)((lanes + kThreads - 1) / kThreads);
  for (int64_t c0 = 0; c0 < s.nrhs; c0 += 65535) {
    StepTail t = s;
    const int64_t nc = (s.nrhs - c0) < 65535 ? (s.nrhs - c0) : 65535;
    t.in = static_cast<const TMID *>(s.in) + c0 * s.in_rhs_stride;
    t.out = static_cast<TOUT *>(s.out) + c0 * s.out_rhs_stride;
    if (t.u) t.u = static_cast<const TOUT *>(s.u) + c0 * s.u_rhs_stride;
    if (t.v) t.v = static_cast<const TOUT *>(s.v) + c0 * s.u_rhs_stride;
    if (s.m == 2)
      step_tail_kernel<MODE, TMID, TOUT, 2, false><<<dim3(gx, (unsigned)nc), kThreads, 0, st>>>(t);
    else if (s.r[0] == 8 && s.r[1] == 4 && s.r[2] == 2)
      step_tail_kernel<MODE, TMID, TOUT, 3, true><<<dim3(gx, (unsigned)nc), kThreads, 0, st>>>(t);
    else
      step_tail_kernel<MODE, TMID, TOUT, 3, false><<<dim3(gx, (unsigned)nc), kThreads, 0, st>>>(t);
    count_launches(1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int MODE, typename TMID>
cudaError_t tail_by_output(const StepTail &s, cudaStream_t st) {
  switch (s.out_type) {
    case QTT_F64: return launch_tail_t<MODE, TMID, double>(s, st);
    case QTT_BF16: return launch_tail_t<MODE, TMID, __nv_bfloat16>(s, st);
    default: return launch_tail_t<MODE, TMID, float>(s, st);
  }
}

}  // namespace

int tail_steps(const int *ranks, int d, int head) {
  int m = 0;
  while (m < 3 && d - (m + 1) >= 1 && d - (m + 1) >= head && ranks[d - m - 1] <= kHeadMaxRank)
    ++m;
  return m >= 2 ? m : 0;
}

cudaError_t launch_step_tail(const StepTail &s, cudaStream_t st) {
  if (s.m < 2 || s.m > 3) return cudaErrorInvalidValue;
  switch (s.mode) {
    case LP_F32: return tail_by_output<LP_F32, float>(s, st);
    case LP_TF32: return tail_by_output<LP_TF32, float>(s, st);
    case LP_BF16: return tail_by_output<LP_BF16, __nv_bfloat16>(s, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t tail_status_take(int *status) {
  int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(status, g_tail_status, sizeof(int));
  if (e == cudaSuccess && *status != 0) e = cudaMemcpyToSymbol(g_tail_status, &zero, sizeof(int));
  return e;
}

int head_steps(const int *ranks, int d) {
  int m = 0;
  while (m < 3 && m + 1 < d && ranks[m + 1] <= kHeadMaxRank) ++m;
  return m >= 2 ? m : 0;
}

cudaError_t launch_step_head(const StepHead &s, cudaStream_t st) {
  if (s.m < 2 || s.m > 3) return cudaErrorInvalidValue;
  switch (s.mode) {
    case LP_F32: return by_input<LP_F32, float>(s, st);
    case LP_TF32: return by_input<LP_TF32, float>(s, st);
    case LP_BF16: return by_input<LP_BF16, __nv_bfloat16>(s, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace qtt
