// FP64 dense building blocks (see dense.h).  On GB300 the FP64 pipe issues
// about two fused multiply-adds per clock per SM, so these kernels are
// bound by DFMA issue as soon as their operands sit in shared memory or L2;
// they are written for that: register tiles for the GEMM, one pass over
// the trailing matrix per Householder step, and every reduction in a fixed
// order (results do not depend on the launch shape).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "dense.h"

namespace qtt {
namespace dense {
namespace {

constexpr int kThreads = 256;

// ------------------------------------------------------------------- GEMM
// 64 x 64 tile of C per CTA, K in slices of 16 through shared memory; thread
// (ty, tx) of 16 x 16 owns rows ty + 16 s and columns tx + 16 t (s, t < 4),
// so shared-memory reads are conflict-free and C stores coalesced.
constexpr int BM = 64, BN = 64, BK = 16;

struct GemmArgs {
  const double *A, *B;
  double *C;
  int64_t m, n, k, lda, ldb, ldc, sa, sb, sc;
  double alpha, beta;
  int ta, tb;
  // split-K: blockIdx.z = batch * splits + split; split s sums k in
  // [s kchunk, (s + 1) kchunk) into part[(s batch + b) m n] (alpha applied)
  int splits;
  int64_t kchunk, batch;
  double *part;
};

__global__ void __launch_bounds__(kThreads) gemm_kernel(GemmArgs g) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t z = blockIdx.z;
  const int64_t bz = z / g.splits, sp = z - bz * g.splits;
  const double *A = g.A + bz * g.sa;
  const double *B = g.B + bz * g.sb;
  double *C = g.C + bz * g.sc;
  const int64_t i0 = (int64_t)blockIdx.y * BM, j0 = (int64_t)blockIdx.x * BN;
  const int64_t klo = sp * g.kchunk, khi = min(g.k, klo + g.kchunk);
  double acc[4][4];
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int t = 0; t < 4; ++t) acc[s][t] = 0.0;
  for (int64_t k0 = klo; k0 < khi; k0 += BK) {
    for (int e = tid; e < BM * BK; e += kThreads) {
      // consecutive threads read consecutive addresses of A
      const int ii = g.ta ? e % BM : e / BK, kk = g.ta ? e / BM : e % BK;
      const int64_t gi = i0 + ii, gk = k0 + kk;
      double v = 0.0;
      if (gi < g.m && gk < khi) v = g.ta ? A[gk * g.lda + gi] : A[gi * g.lda + gk];
      As[kk][ii] = v;
    }
    for (int e = tid; e < BN * BK; e += kThreads) {
      const int jj = g.tb ? e / BK : e % BN, kk = g.tb ? e % BK : e / BN;
      const int64_t gj = j0 + jj, gk = k0 + kk;
      double v = 0.0;
      if (gj < g.n && gk < khi) v = g.tb ? B[gj * g.ldb + gk] : B[gk * g.ldb + gj];
      Bs[kk][jj] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int s = 0; s < 4; ++s) a[s] = As[kk][ty + 16 * s];
#pragma unroll
      for (int t = 0; t < 4; ++t) b[t] = Bs[kk][tx + 16 * t];
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int t = 0; t < 4; ++t) acc[s][t] = fma(a[s], b[t], acc[s][t]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int64_t i = i0 + ty + 16 * s;
    if (i >= g.m) continue;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int64_t j = j0 + tx + 16 * t;
      if (j >= g.n) continue;
      if (g.splits > 1) {
        g.part[(sp * g.batch + bz) * g.m * g.n + i * g.n + j] = g.alpha * acc[s][t];
        continue;
      }
      double *c = C + i * g.ldc + j;
      *c = g.beta == 0.0 ? g.alpha * acc[s][t] : fma(g.alpha, acc[s][t], g.beta * *c);
    }
  }
}

// C = sum over the splits, in split order, of the partial products (+ beta C).
__global__ void __launch_bounds__(kThreads) gemm_reduce_kernel(GemmArgs g) {
  const int64_t mn = g.m * g.n, total = mn * g.batch;
  for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * kThreads) {
    const int64_t bz = e / mn, r = e - bz * mn, i = r / g.n, j = r - i * g.n;
    double s = 0.0;
    for (int sp = 0; sp < g.splits; ++sp) s += g.part[((int64_t)sp * g.batch + bz) * mn + r];
    double *c = g.C + bz * g.sc + i * g.ldc + j;
    *c = g.beta == 0.0 ? s : fma(g.beta, *c, s);
  }
}

// ---------------------------------------------------------------- permute
struct PermArgs {
  const double *in;
  double *out;
  int64_t dims[8], stride[8];
  int64_t total;
  int nd;
  double scale;
};

__global__ void __launch_bounds__(kThreads) permute_kernel(PermArgs a) {
  for (int64_t o = (int64_t)blockIdx.x * kThreads + threadIdx.x; o < a.total;
       o += (int64_t)gridDim.x * kThreads) {
    int64_t rem = o, src = 0;
    for (int t = a.nd - 1; t >= 0; --t) {
      const int64_t q = rem / a.dims[t];
      src += (rem - q * a.dims[t]) * a.stride[t];
      rem = q;
    }
    a.out[o] = a.scale == 1.0 ? a.in[src] : a.scale * a.in[src];
  }
}

// ------------------------------------------------------------------ sumsq
constexpr int kSumBlocks = 256;

__global__ void __launch_bounds__(kThreads) sumsq_part_kernel(const double *x, int64_t n,
                                                              double *part) {
  __shared__ double red[kThreads];
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * per, hi = min(n, lo + per);
  double s = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += kThreads) s = fma(x[i], x[i], s);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void sumsq_final_kernel(const double *part, int nb, double *out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[b];
    *out = s;
  }
}

// ------------------------------------------------------------ gather_rows
__global__ void __launch_bounds__(kThreads) gather_rows_kernel(const double *in, int64_t ldi,
                                                               const int *idx, const double *scale,
                                                               int64_t nr, int64_t nc, double *out,
                                                               int64_t ldo, int divide) {
  const int64_t total = nr * nc;
  for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * kThreads) {
    const int64_t r = e / nc, c = e - r * nc;
    const int src = idx[r];
    double v = in[(int64_t)src * ldi + c];
    // a zero singular value (an all-zero unfolding) gives a zero row, not NaN
    if (scale) v = divide ? (scale[src] != 0.0 ? v / scale[src] : 0.0) : v * scale[src];
    out[r * ldo + c] = v;
  }
}

unsigned grid_for(int64_t work) {
  const int64_t g = (work + kThreads - 1) / kThreads;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 32));
}

}  // namespace

cudaError_t gemm(bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha,
                 const double *A, int64_t lda, int64_t sa, const double *B, int64_t ldb,
                 int64_t sb, double beta, double *C, int64_t ldc, int64_t sc, int64_t batch,
                 cudaStream_t st) {
  if (m <= 0 || n <= 0 || batch <= 0) return cudaSuccess;
  GemmArgs g{A, B, C, m, n, k, lda, ldb, ldc, sa, sb, sc, alpha, beta, ta ? 1 : 0, tb ? 1 : 0,
             1, std::max<int64_t>(k, 1), 1, nullptr};
  const int64_t gx = (n + BN - 1) / BN, gy = (m + BM - 1) / BM;
  if (gy > 65535 || gx > 0x7fffffffLL) return cudaErrorInvalidValue;
  // Split-K when the output tiles leave most SMs idle and K is long: S
  // splits (a function of the shape only, so results are reproducible) sum
  // into partial products that a second launch adds in split order.
  const int64_t tiles = gx * gy * batch;
  int S = 1;
  if (batch <= 65535 && tiles < 2 * 152 && k >= 8 * BK) {
    S = (int)std::min<int64_t>({(2 * 152 + tiles - 1) / tiles, k / (4 * BK), 64});
    if (tiles * S > 65535 * gx * gy) S = 1;
  }
  if (S > 1) {
    void *part = nullptr;
    if (scratch_alloc(&part, (size_t)S * batch * m * n * sizeof(double), st) != QTT_OK) {
      S = 1;  // no room: the single pass below
    } else {
      g.splits = S;
      g.kchunk = ((k + S - 1) / S + BK - 1) / BK * BK;
      g.batch = batch;
      g.part = static_cast<double *>(part);
      gemm_kernel<<<dim3((unsigned)gx, (unsigned)gy, (unsigned)(batch * S)), kThreads, 0, st>>>(g);
      gemm_reduce_kernel<<<grid_for(m * n * batch), kThreads, 0, st>>>(g);
      count_launches(2);
      const cudaError_t e = cudaGetLastError();
      scratch_free(part, st);
      return e;
    }
  }
  for (int64_t b0 = 0; b0 < batch; b0 += 65535) {
    GemmArgs h = g;
    h.A += b0 * sa;
    h.B += b0 * sb;
    h.C += b0 * sc;
    const int64_t nb = std::min<int64_t>(65535, batch - b0);
    gemm_kernel<<<dim3((unsigned)gx, (unsigned)gy, (unsigned)nb), kThreads, 0, st>>>(h);
    count_launches(1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t permute(const double *in, double *out, int nd, const int64_t *dims,
                    const int64_t *stride, double scale, cudaStream_t st) {
  if (nd < 1 || nd > 8) return cudaErrorInvalidValue;
  PermArgs a;
  std::memset(&a, 0, sizeof(a));
  a.in = in;
  a.out = out;
  a.nd = nd;
  a.scale = scale;
  a.total = 1;
  for (int t = 0; t < nd; ++t) {
    a.dims[t] = dims[t];
    a.stride[t] = stride[t];
    a.total *= dims[t];
  }
  if (a.total == 0) return cudaSuccess;
  permute_kernel<<<grid_for(a.total), kThreads, 0, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

size_t sumsq_work_doubles(int64_t) { return kSumBlocks; }

cudaError_t sumsq(const double *x, int64_t n, double *out, double *work, cudaStream_t st) {
  sumsq_part_kernel<<<kSumBlocks, kThreads, 0, st>>>(x, n, work);
  sumsq_final_kernel<<<1, 32, 0, st>>>(work, kSumBlocks, out);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t gather_rows(const double *in, int64_t ldi, const int *idx, const double *scale,
                        int64_t nr, int64_t ncols, double *out, int64_t ldo, bool divide,
                        cudaStream_t st) {
  if (nr <= 0 || ncols <= 0) return cudaSuccess;
  gather_rows_kernel<<<grid_for(nr * ncols), kThreads, 0, st>>>(in, ldi, idx, scale, nr, ncols,
                                                                out, ldo, divide ? 1 : 0);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace dense
}  // namespace qtt
