// FP64 core step of the QTT apply (Algorithm 2, one iteration of the sweep).
//
// Step k maps the intermediate y_k (r_k planes of N positions) to y_{k+1}
// (r_{k+1} planes).  Position p keeps its bits; bit k holds the column bit
// j_k on input and the row bit i_k on output, so the column merge and row
// split of Algorithm 2 are pure addressing.  For every pair of positions
// (p0, p1 = p0 | 2^k) and every output rank b:
//   out[b][p_i] = sum_{a, j} G_k(a, i, j, b) in[a][p_j]      (i, j in {0,1})
// which is phi_k = M_k b_k for the column of that pair.  The flop count is
// 4 r_k r_{k+1} N (Sec. 4.2).
//
// On GB300 the FP64 pipe is the limit by a wide margin (the step moves
// (r_k + r_{k+1}) x 8 bytes per position against 4 r_k r_{k+1} flops), so
// the kernel is shaped for DFMA issue, not bandwidth: each thread owns one
// output rank b (both row bits) and TN position pairs, giving 2 TN
// independent FMA chains; the warp shares b, so each core element is a
// broadcast load, and the 32 lanes read 32 consecutive pairs (coalesced).
#include "checked.cuh"
#include "qtt_internal.h"

namespace qtt {
namespace {

constexpr int kTN = 4;       // position pairs per thread
constexpr int kWarpsY = 8;   // output ranks per CTA (one per warp)

// The body of one CTA of the step: `cta` = pair tile * rank blocks + rank
// block, `by` ranks per block, thread (ty, tx) = (rank in the block, lane),
// right-hand side c.  Shared by the single-operator kernel and the grouped
// kernel of the serving loop, so a step's arithmetic is the same in both.
template <int TN>
__device__ __forceinline__ void step_f64_tn_body(const StepF64 &s, int64_t cta, int by,
                                                 int64_t c, int ty, int tx) {
  // CTAs that share a pair tile (and so its input) run back to back and
  // meet it in L2
  const int nrb = (s.rout + by - 1) / by;
  const int b = (int)(cta % nrb) * by + ty;
  if (b >= s.rout) return;
  c = QTT_CK(c, s.nrhs, 101);
  const int64_t npairs = s.N >> 1;
  const int64_t bit = (int64_t)1 << s.k;
  const int64_t low = bit - 1;
  const int64_t q0 = (cta / nrb) * (32 * TN) + tx;

  int64_t p0[TN];
  bool ok[TN];
#pragma unroll
  for (int m = 0; m < TN; ++m) {
    const int64_t q = q0 + 32 * m;
    ok[m] = q < npairs;
    p0[m] = ((q & ~low) << 1) | (q & low);
    if (ok[m]) p0[m] = QTT_CK(p0[m], s.N - bit, 102);  // p0 and p0 + 2^k in range
  }
  const double *in = s.in + c * s.in_rhs_stride;
  const double2 *Mb = reinterpret_cast<const double2 *>(s.M) + (int64_t)b * 2 * s.rin;

  double acc0[TN], acc1[TN];
#pragma unroll
  for (int m = 0; m < TN; ++m) acc0[m] = acc1[m] = 0.0;

  for (int a = 0; a < s.rin; ++a) {
    const double *ina = in + (int64_t)a * s.N;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const double2 g = __ldg(Mb + 2 * a + j);  // (i = 0, i = 1)
      const int64_t sh = j ? bit : 0;
#pragma unroll
      for (int m = 0; m < TN; ++m) {
        const double v = ok[m] ? __ldg(ina + p0[m] + sh) : 0.0;
        acc0[m] = fma(g.x, v, acc0[m]);
        acc1[m] = fma(g.y, v, acc1[m]);
      }
    }
  }

  double *out = s.out + c * s.out_rhs_stride + (int64_t)b * s.N;
  if (s.epi) {
    const double *u = s.u ? s.u + c * s.uv_rhs_stride : nullptr;
    const double *v = s.v ? s.v + c * s.uv_rhs_stride : nullptr;
#pragma unroll
    for (int m = 0; m < TN; ++m) {
      if (!ok[m]) continue;
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int64_t p = p0[m] + (i ? bit : 0);
        double t = v ? s.s_v * v[p] : 0.0;
        if (u) t += s.s_u * u[p];
        out[p] = t + s.s_acc * (i ? acc1[m] : acc0[m]);
      }
    }
  } else {
#pragma unroll
    for (int m = 0; m < TN; ++m) {
      if (!ok[m]) continue;
      out[p0[m]] = acc0[m];
      out[p0[m] + bit] = acc1[m];
    }
  }
}

template <int TN>
__global__ void __launch_bounds__(32 * kWarpsY)
step_f64_kernel(StepF64 s) {
  step_f64_tn_body<TN>(s, blockIdx.x, blockDim.y, blockIdx.z, threadIdx.y, threadIdx.x);
}

// Small steps (few pair tiles, e.g. the 8^3 volume operator with N = 512):
// the same contraction with the sum over (a, j) split among KS warps, so a
// CTA of 8 warps covers 8 / KS output ranks of 32 pairs and the grid has
// KS times more CTAs with KS times shorter FMA chains.  The KS partial sums
// meet in shared memory and are added in a fixed order (deterministic).
// One CTA of the split-sum form (every thread of the CTA calls it: it holds
// a CTA-wide barrier); part is the CTA's shared scratch.
template <int KS>
__device__ __forceinline__ void step_f64_small_body(const StepF64 &s, int64_t cta, int64_t c,
                                                    int warp, int lane,
                                                    double (*part)[2][32]) {
  constexpr int RPC = kWarpsY / KS;  // output ranks per CTA
  const int nrg = (s.rout + RPC - 1) / RPC;
  const int b = (int)(cta % nrg) * RPC + warp / KS;
  const int split = warp % KS;
  const int64_t npairs = s.N >> 1;
  const int64_t bit = (int64_t)1 << s.k;
  const int64_t low = bit - 1;
  const int64_t q = (cta / nrg) * 32 + lane;
  const bool ok = q < npairs && b < s.rout;
  c = QTT_CK(c, s.nrhs, 103);
  int64_t p0 = ((q & ~low) << 1) | (q & low);
  if (ok) p0 = QTT_CK(p0, s.N - bit, 104);
  double acc0 = 0.0, acc1 = 0.0;
  if (ok) {
    const double *in = s.in + c * s.in_rhs_stride;
    const double2 *Mb = reinterpret_cast<const double2 *>(s.M) + (int64_t)b * 2 * s.rin;
    const int per = (s.rin + KS - 1) / KS;
    const int a0 = split * per, a1 = min(s.rin, a0 + per);
    for (int a = a0; a < a1; ++a) {
      const double *ina = in + (int64_t)a * s.N + p0;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const double2 g = __ldg(Mb + 2 * a + j);
        const double v = __ldg(ina + (j ? bit : 0));
        acc0 = fma(g.x, v, acc0);
        acc1 = fma(g.y, v, acc1);
      }
    }
  }
  part[warp][0][lane] = acc0;
  part[warp][1][lane] = acc1;
  __syncthreads();
  if (split != 0 || !ok) return;
  acc0 = acc1 = 0.0;
#pragma unroll
  for (int t = 0; t < KS; ++t) {
    acc0 += part[warp + t][0][lane];
    acc1 += part[warp + t][1][lane];
  }
  double *out = s.out + c * s.out_rhs_stride + (int64_t)b * s.N;
  if (s.epi) {
    const double *u = s.u ? s.u + c * s.uv_rhs_stride : nullptr;
    const double *v = s.v ? s.v + c * s.uv_rhs_stride : nullptr;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int64_t p = p0 + (i ? bit : 0);
      double t = v ? s.s_v * v[p] : 0.0;
      if (u) t += s.s_u * u[p];
      out[p] = t + s.s_acc * (i ? acc1 : acc0);
    }
  } else {
    out[p0] = acc0;
    out[p0 + bit] = acc1;
  }
}

template <int KS>
__global__ void __launch_bounds__(32 * kWarpsY)
step_f64_small_kernel(StepF64 s) {
  __shared__ double part[kWarpsY][2][32];
  step_f64_small_body<KS>(s, blockIdx.x, blockIdx.z, threadIdx.x >> 5, threadIdx.x & 31, part);
}

// Grouped steps: one launch runs, for each descriptor, one step of one
// operator (its own sizes, buffers and epilogue).  CTA blockIdx.x belongs to
// the descriptor whose range [cta0, cta0 + ctas) holds it; inside that range
// it is CTA (cta, c) of the single-operator launch, with the same body and
// the same form (split-sum or pairs-per-lane) that launch would take.
__global__ void __launch_bounds__(32 * kWarpsY)
step_f64_grouped_kernel(const GroupedStepF64 *g, int n) {
  __shared__ double part[kWarpsY][2][32];
  int lo = 0, hi = n - 1;
  const int64_t bx = blockIdx.x;
  while (lo < hi) {  // last descriptor with cta0 <= bx
    const int mid = (lo + hi + 1) >> 1;
    if (g[mid].cta0 <= bx) lo = mid;
    else hi = mid - 1;
  }
  const GroupedStepF64 &d = g[lo];
  const int64_t local = bx - d.cta0;
  const int64_t c = local / d.ctas_per_rhs, cta = local - c * d.ctas_per_rhs;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (d.small)
    step_f64_small_body<4>(d.s, cta, c, warp, lane, part);
  else
    step_f64_tn_body<kTN>(d.s, cta, kWarpsY, c, warp, lane);
}

}  // namespace

namespace {

cudaError_t launch_small(const StepF64 &s, cudaStream_t stream) {
  constexpr int KS = 4, RPC = kWarpsY / KS;
  const int64_t gx = ((s.N >> 1) + 31) / 32 * ((s.rout + RPC - 1) / RPC);
  for (int64_t c0 = 0; c0 < s.nrhs; c0 += 65535) {
    StepF64 t = s;
    const int64_t nc = (s.nrhs - c0) < 65535 ? (s.nrhs - c0) : 65535;
    t.in += c0 * s.in_rhs_stride;
    t.out += c0 * s.out_rhs_stride;
    if (t.u) t.u += c0 * s.uv_rhs_stride;
    if (t.v) t.v += c0 * s.uv_rhs_stride;
    if (gx > 0x7fffffffLL) return cudaErrorInvalidValue;
    step_f64_small_kernel<KS><<<dim3((unsigned)gx, 1, (unsigned)nc), 32 * kWarpsY, 0, stream>>>(t);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int TN>
cudaError_t launch_tn(const StepF64 &s, cudaStream_t stream) {
  const int64_t npairs = s.N >> 1;
  const int by = s.rout < kWarpsY ? s.rout : kWarpsY;
  const int64_t gx = (npairs + 32 * TN - 1) / (32 * TN);
  const int64_t gy = (s.rout + by - 1) / by;
  dim3 block(32, by, 1);
  for (int64_t c0 = 0; c0 < s.nrhs; c0 += 65535) {
    StepF64 t = s;
    const int64_t nc = (s.nrhs - c0) < 65535 ? (s.nrhs - c0) : 65535;
    t.in += c0 * s.in_rhs_stride;
    t.out += c0 * s.out_rhs_stride;
    if (t.u) t.u += c0 * s.uv_rhs_stride;
    if (t.v) t.v += c0 * s.uv_rhs_stride;
    if (gx * gy > 0x7fffffffLL) return cudaErrorInvalidValue;
    dim3 grid((unsigned)(gx * gy), 1, (unsigned)nc);
    step_f64_kernel<TN><<<grid, block, 0, stream>>>(t);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

// Small steps (the 8^3 volume operator has N = 512) would give a few CTAs
// with 4 pairs per lane and leave most SMs idle: the split-sum kernel then
// gives 16x the CTAs (one pair per lane, the (a, j) sum over 4 warps).  The
// choice depends on one right-hand side's work only (not on nrhs): the two
// forms sum in different orders, and a right-hand side must get the same
// bits whatever else shares its launch (chunked applies, batched solves, the
// server's grouped steps).
bool f64_step_small(int64_t N, int rout) {
  static const int sms = [] {
    int dev = 0, n = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
  }();
  const int64_t ctas_per_rhs = ((N >> 1) + 127) / 128 * ((rout + kWarpsY - 1) / kWarpsY);
  return ctas_per_rhs < 2 * sms;
}

cudaError_t launch_step_f64(const StepF64 &s, cudaStream_t stream) {
  if (f64_step_small(s.N, s.rout)) return launch_small(s, stream);
  return launch_tn<kTN>(s, stream);
}

int64_t f64_step_ctas_per_rhs(const StepF64 &s, bool small) {
  const int64_t npairs = s.N >> 1;
  if (small) return (npairs + 31) / 32 * ((s.rout + 1) / 2);
  return (npairs + 32 * kTN - 1) / (32 * kTN) * ((s.rout + kWarpsY - 1) / kWarpsY);
}

cudaError_t launch_step_f64_grouped(const GroupedStepF64 *dev_table, int n, int64_t total_ctas,
                                    cudaStream_t stream) {
  if (n <= 0 || total_ctas <= 0) return cudaSuccess;
  if (total_ctas > 0x7fffffffLL) return cudaErrorInvalidValue;
  step_f64_grouped_kernel<<<(unsigned)total_ctas, 32 * kWarpsY, 0, stream>>>(dev_table, n);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace qtt
