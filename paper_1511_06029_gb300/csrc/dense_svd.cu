// One-sided Jacobi SVD on the device (dense.h), the truncation step of TT
// rounding and of TT-SVD (Algorithm 1).
//
// Hestenes' method: the columns of B (here the rows of Bt, so that each is
// contiguous) are made mutually orthogonal by plane rotations; for a pair
// (u, v) with a = |u|^2, b = |v|^2, c = u.v, the rotation with
// zeta = (b - a) / (2 c), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
// cs = 1 / sqrt(1 + t^2), sn = cs t  makes  cs u - sn v  and  sn u + cs v
// orthogonal, and the same rotation applied to the rows of Vt accumulates V.
// The pairs of one round are disjoint (the round-robin ordering of Brent and
// Luk), so a round is one launch with one warp per pair; sweeps repeat until
// no pair needed a rotation.  The result has high relative accuracy in the
// small singular values, which the truncation thresholds of TT rounding
// (down to eps ~ 1e-8 of the norm) depend on.  Every sum is a fixed
// butterfly over the warp, so the factorisation is the same run to run.
#include <algorithm>
#include <cmath>
#include <vector>

#include "dense.h"

namespace qtt {
namespace dense {
namespace {

constexpr int kT = 256;
constexpr int kWarps = kT / 32;
constexpr int kMaxSweeps = 60;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kT) jacobi_round_kernel(double *Bt, int64_t ldb, int64_t len,
                                                          double *Vt, int64_t ldv, int64_t p,
                                                          const int2 *pairs, int npairs,
                                                          double tol, int *rotations) {
  const int w = blockIdx.x * kWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (w >= npairs) return;
  const int2 pr = pairs[w];
  if (pr.x >= p || pr.y >= p) return;  // the padding index of an odd p
  double *u = Bt + (int64_t)pr.x * ldb, *v = Bt + (int64_t)pr.y * ldb;
  double a = 0.0, b = 0.0, c = 0.0;
  for (int64_t r = lane; r < len; r += 32) {
    const double x = u[r], y = v[r];
    a = fma(x, x, a);
    b = fma(y, y, b);
    c = fma(x, y, c);
  }
  a = warp_sum(a);
  b = warp_sum(b);
  c = warp_sum(c);
  if (a == 0.0 || b == 0.0 || !(fabs(c) > tol * sqrt(a) * sqrt(b))) return;
  const double zeta = (b - a) / (2.0 * c);
  const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + hypot(1.0, zeta));
  const double cs = 1.0 / sqrt(fma(t, t, 1.0)), sn = cs * t;
  for (int64_t r = lane; r < len; r += 32) {
    const double x = u[r], y = v[r];
    u[r] = fma(cs, x, -sn * y);
    v[r] = fma(sn, x, cs * y);
  }
  double *vu = Vt + (int64_t)pr.x * ldv, *vv = Vt + (int64_t)pr.y * ldv;
  for (int64_t r = lane; r < p; r += 32) {
    const double x = vu[r], y = vv[r];
    vu[r] = fma(cs, x, -sn * y);
    vv[r] = fma(sn, x, cs * y);
  }
  if (lane == 0) atomicAdd(rotations, 1);
}

__global__ void __launch_bounds__(kT) row_norms_kernel(const double *Bt, int64_t ldb, int64_t len,
                                                       int64_t p, double *sigma) {
  const int64_t i = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= p) return;
  double s = 0.0;
  for (int64_t r = lane; r < len; r += 32) s = fma(Bt[i * ldb + r], Bt[i * ldb + r], s);
  s = warp_sum(s);
  if (lane == 0) sigma[i] = sqrt(s);
}

__global__ void __launch_bounds__(kT) eye_sq_kernel(double *V, int64_t ldv, int64_t p) {
  const int64_t total = p * p;
  for (int64_t e = (int64_t)blockIdx.x * kT + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * kT) {
    const int64_t i = e / p, c = e - i * p;
    V[i * ldv + c] = i == c ? 1.0 : 0.0;
  }
}

}  // namespace

size_t jacobi_work_ints(int64_t p) {
  const int64_t q = p + (p & 1);
  return (size_t)std::max<int64_t>(1, (q - 1) * (q / 2)) * 2 + 2;
}

qtt_status jacobi_svd(int64_t p, int64_t len, double *Bt, int64_t ldb, double *Vt, int64_t ldv,
                      double *sigma, int *work, cudaStream_t st, int *sweeps) {
  if (sweeps) *sweeps = 0;
  if (p <= 0) return QTT_OK;
  int *counter = work;
  int2 *pairs = reinterpret_cast<int2 *>(work + 2);
  const int64_t q = p + (p & 1);
  const int npairs = (int)(q / 2);
  const int rounds = (int)std::max<int64_t>(1, q - 1);
  // round-robin schedule: index q-1 stays, the others rotate by one per round
  std::vector<int> tab((size_t)rounds * npairs * 2);
  for (int r = 0; r < rounds; ++r) {
    if (q == 1) break;
    for (int k = 0; k < npairs; ++k) {
      int i, j;
      if (k == 0) {
        i = (int)(q - 1);
        j = r;
      } else {
        i = (int)((r + k) % (q - 1));
        j = (int)((r - k + (q - 1)) % (q - 1));
      }
      if (i > j) std::swap(i, j);
      tab[((size_t)r * npairs + k) * 2] = i;
      tab[((size_t)r * npairs + k) * 2 + 1] = j;
    }
  }
  QTT_CUDA_TRY(cudaMemcpyAsync(pairs, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice,
                               st));
  eye_sq_kernel<<<(unsigned)std::min<int64_t>((p * p + kT - 1) / kT, 4096), kT, 0, st>>>(Vt, ldv, p);
  count_launches(1);
  const double tol = std::max(1e-15, std::sqrt((double)std::max<int64_t>(len, 1)) * 1.2e-16);
  const unsigned grid = (unsigned)((npairs + kWarps - 1) / kWarps);
  int done_sweeps = 0;
  if (p > 1) {
    for (int sw = 0; sw < kMaxSweeps; ++sw) {
      QTT_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int), st));
      for (int r = 0; r < rounds; ++r)
        jacobi_round_kernel<<<grid, kT, 0, st>>>(Bt, ldb, len, Vt, ldv, p,
                                                 pairs + (size_t)r * npairs, npairs, tol, counter);
      count_launches((uint64_t)rounds);
      QTT_CUDA_TRY(cudaGetLastError());
      int h = 0;
      QTT_CUDA_TRY(cudaMemcpyAsync(&h, counter, sizeof(int), cudaMemcpyDeviceToHost, st));
      QTT_CUDA_TRY(cudaStreamSynchronize(st));
      ++done_sweeps;
      if (h == 0) break;
    }
  }
  row_norms_kernel<<<(unsigned)((p + kWarps - 1) / kWarps), kT, 0, st>>>(Bt, ldb, len, p, sigma);
  count_launches(1);
  QTT_CUDA_TRY(cudaGetLastError());
  if (sweeps) *sweeps = done_sweeps;
  return QTT_OK;
}

}  // namespace dense
}  // namespace qtt
