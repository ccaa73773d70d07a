// Householder QR on the device (dense.h): the orthogonalisation step of TT
// rounding and of the SVDs of tall unfoldings.
//
// Column j of an m x n row-major matrix is reduced by H_j = I - tau v v^T,
// v = (1, x_1 / (alpha - beta), ...), beta = -sign(alpha) ||x||, tau =
// (beta - alpha) / beta (Householder's reflector in LAPACK's normalisation),
// in three launches over the trailing matrix:
//   dots    each thread one column c >= j, each CTA a block of rows i > j:
//           partial sums of x_i A(i, c)                (c = j gives ||x_1..||^2)
//   reduce  per column, the partial sums in row-block order -> w_c =
//           tau (A(j, c) + s_c / (alpha - beta)); other CTAs scale x into v
//   update  A(i, c) -= v_i w_c for i >= j, c > j; beta goes on the diagonal
// Threads own columns and walk rows, so every access of a row-major matrix
// is coalesced across a warp; each row block's partial sums are added in one
// fixed order, so the result does not depend on the grid.  The thin Q is
// accumulated backwards from [I; 0] with the same three launches.
#include <algorithm>
#include <cmath>

#include "dense.h"

namespace qtt {
namespace dense {
namespace {

constexpr int kT = 256;
constexpr int kMaxRowBlocks = 512;

struct Blocks {
  int64_t r0, nrows, rows_per;
  int R;           // row blocks
  int64_t c0, nc;  // columns c0 .. c0 + nc - 1
  int cb;          // column blocks of kT columns
};

Blocks blocks_for(int64_t r0, int64_t m, int64_t c0, int64_t n) {
  Blocks b;
  b.r0 = r0;
  b.nrows = std::max<int64_t>(0, m - r0);
  b.c0 = c0;
  b.nc = std::max<int64_t>(0, n - c0);
  b.cb = (int)std::max<int64_t>(1, (b.nc + kT - 1) / kT);
  // about four CTAs per SM in all, at least 32 rows per block
  int64_t R = std::max<int64_t>(1, (608 + b.cb - 1) / b.cb);
  R = std::min<int64_t>(R, std::max<int64_t>(1, (b.nrows + 31) / 32));
  R = std::min<int64_t>(R, kMaxRowBlocks);
  b.rows_per = std::max<int64_t>(1, (b.nrows + R - 1) / R);
  b.R = (int)std::max<int64_t>(1, (b.nrows + b.rows_per - 1) / b.rows_per);
  return b;
}

// part[rb * nc + (c - c0)] = sum over the block's rows i of v_i M(i, c), with
// v_i = V(i, vcol) and, when unit_row >= 0, v = 1 at row unit_row.
__global__ void __launch_bounds__(kT) dots_kernel(const double *V, int64_t ldv, int64_t vcol,
                                                  const double *M, int64_t ldm, Blocks b,
                                                  int64_t unit_row, double *part) {
  const int64_t c = b.c0 + (int64_t)blockIdx.x * kT + threadIdx.x;
  if (c >= b.c0 + b.nc) return;
  const int64_t lo = b.r0 + (int64_t)blockIdx.y * b.rows_per;
  const int64_t hi = min(b.r0 + b.nrows, lo + b.rows_per);
  double s = 0.0;
  for (int64_t i = lo; i < hi; ++i) {
    const double v = i == unit_row ? 1.0 : V[i * ldv + vcol];
    s = fma(v, M[i * ldm + c], s);
  }
  part[(int64_t)blockIdx.y * b.nc + (c - b.c0)] = s;
}

// The reflector of column j from the partial sums of ||x_{j+1..}||^2.
struct Refl {
  double tau, scale, beta;
};
__device__ __forceinline__ Refl reflector(const double *part, int R, int64_t nc, double alpha) {
  double x2 = 0.0;
  for (int r = 0; r < R; ++r) x2 += part[(int64_t)r * nc];  // column j is index 0
  Refl f;
  if (x2 == 0.0) {
    f.tau = 0.0;
    f.scale = 0.0;
    f.beta = alpha;
  } else {
    const double nrm = sqrt(fma(alpha, alpha, x2));
    f.beta = alpha >= 0.0 ? -nrm : nrm;
    f.tau = (f.beta - alpha) / f.beta;
    f.scale = 1.0 / (alpha - f.beta);
  }
  return f;
}

// geqrf reduce step: blocks [0, cb) compute w_c for c > j; blocks [cb, ..)
// scale x_{j+1..} into v (column j) and store tau_j and beta (beta goes on
// the diagonal in the update launch: every block here reads alpha there).
__global__ void __launch_bounds__(kT) qr_reduce_kernel(double *A, int64_t lda, int64_t m,
                                                       int64_t j, Blocks b, const double *part,
                                                       double *w, double *tau, double *beta) {
  const Refl f = reflector(part, b.R, b.nc, A[j * lda + j]);
  if ((int)blockIdx.x < b.cb) {
    const int64_t c = b.c0 + (int64_t)blockIdx.x * kT + threadIdx.x;
    if (c <= j || c >= b.c0 + b.nc) return;
    double s = 0.0;
    for (int r = 0; r < b.R; ++r) s += part[(int64_t)r * b.nc + (c - b.c0)];
    w[c] = f.tau * fma(f.scale, s, A[j * lda + c]);
  } else {
    const int64_t i = j + 1 + (int64_t)(blockIdx.x - b.cb) * kT + threadIdx.x;
    if (i < m) A[i * lda + j] *= f.scale;
    if (blockIdx.x == (unsigned)b.cb && threadIdx.x == 0) {
      *beta = f.beta;
      tau[j] = f.tau;
    }
  }
}

// M(i, c) -= v_i w_c for the block's rows i and columns c in (cmin, c0 + nc);
// v = 1 at unit_row, V(i, vcol) elsewhere.  When diag is given, the first
// thread also stores *diag at M(unit_row, vcol) (geqrf's beta).
__global__ void __launch_bounds__(kT) update_kernel(const double *V, int64_t ldv, int64_t vcol,
                                                    double *M, int64_t ldm, Blocks b,
                                                    int64_t unit_row, int64_t cmin,
                                                    const double *w, const double *diag) {
  if (diag && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
    M[unit_row * ldm + vcol] = *diag;
  const int64_t c = b.c0 + (int64_t)blockIdx.x * kT + threadIdx.x;
  if (c <= cmin || c >= b.c0 + b.nc) return;
  const double wc = w[c];
  if (wc == 0.0) return;
  const int64_t lo = b.r0 + (int64_t)blockIdx.y * b.rows_per;
  const int64_t hi = min(b.r0 + b.nrows, lo + b.rows_per);
  for (int64_t i = lo; i < hi; ++i) {
    const double v = i == unit_row ? 1.0 : V[i * ldv + vcol];
    M[i * ldm + c] = fma(-v, wc, M[i * ldm + c]);
  }
}

// orgqr reduce step: w_c = tau_j sum of the partial sums, for c >= j.
__global__ void __launch_bounds__(kT) q_reduce_kernel(Blocks b, const double *part,
                                                      const double *tau, int64_t j, double *w) {
  const int64_t c = b.c0 + (int64_t)blockIdx.x * kT + threadIdx.x;
  if (c >= b.c0 + b.nc) return;
  double s = 0.0;
  for (int r = 0; r < b.R; ++r) s += part[(int64_t)r * b.nc + (c - b.c0)];
  w[c] = tau[j] * s;
}

__global__ void __launch_bounds__(kT) eye_kernel(double *Q, int64_t ldq, int64_t m, int64_t p) {
  const int64_t total = m * p;
  for (int64_t e = (int64_t)blockIdx.x * kT + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * kT) {
    const int64_t i = e / p, c = e - i * p;
    Q[i * ldq + c] = i == c ? 1.0 : 0.0;
  }
}

__global__ void __launch_bounds__(kT) copy_r_kernel(const double *A, int64_t lda, int64_t p,
                                                    int64_t n, double *R, int64_t ldr) {
  const int64_t total = p * n;
  for (int64_t e = (int64_t)blockIdx.x * kT + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * kT) {
    const int64_t i = e / n, c = e - i * n;
    R[i * ldr + c] = c >= i ? A[i * lda + c] : 0.0;
  }
}

unsigned grid1(int64_t work) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + kT - 1) / kT, 152 * 32));
}

}  // namespace

size_t qr_work_doubles(int64_t m, int64_t n) {
  (void)m;
  return (size_t)kMaxRowBlocks * (size_t)std::max<int64_t>(n, 1) + (size_t)std::max<int64_t>(n, 1) +
         2;
}

cudaError_t geqrf(int64_t m, int64_t n, double *A, int64_t lda, double *tau, double *work,
                  cudaStream_t st) {
  const int64_t p = std::min(m, n);
  double *w = work;                                   // n
  double *beta = work + std::max<int64_t>(n, 1);      // 1
  double *part = beta + 2;                            // kMaxRowBlocks x n
  for (int64_t j = 0; j < p; ++j) {
    const Blocks b = blocks_for(j + 1, m, j, n);  // rows below the diagonal, columns >= j
    dots_kernel<<<dim3(b.cb, b.R), kT, 0, st>>>(A, lda, j, A, lda, b, -1, part);
    const int64_t scale_blocks = std::max<int64_t>(1, (m - j - 1 + kT - 1) / kT);
    qr_reduce_kernel<<<(unsigned)(b.cb + scale_blocks), kT, 0, st>>>(A, lda, m, j, b, part, w,
                                                                     tau, beta);
    // rows >= j, columns > j (none for the last column: the launch then only
    // stores beta)
    const Blocks u = blocks_for(j, m, j + 1, n);
    update_kernel<<<dim3(u.cb, u.R), kT, 0, st>>>(A, lda, j, A, lda, u, j, j, w, beta);
    count_launches(3);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t orgqr(int64_t m, int64_t n, const double *A, int64_t lda, const double *tau,
                  double *Q, int64_t ldq, double *work, cudaStream_t st) {
  const int64_t p = std::min(m, n);
  if (p <= 0) return cudaSuccess;
  double *w = work;
  double *part = work + std::max<int64_t>(n, 1) + 2;
  eye_kernel<<<grid1(m * p), kT, 0, st>>>(Q, ldq, m, p);
  count_launches(1);
  for (int64_t j = p - 1; j >= 0; --j) {
    const Blocks b = blocks_for(j, m, j, p);  // rows >= j, columns j .. p-1
    dots_kernel<<<dim3(b.cb, b.R), kT, 0, st>>>(A, lda, j, Q, ldq, b, j, part);
    q_reduce_kernel<<<b.cb, kT, 0, st>>>(b, part, tau, j, w);
    update_kernel<<<dim3(b.cb, b.R), kT, 0, st>>>(A, lda, j, Q, ldq, b, j, j - 1, w, nullptr);
    count_launches(3);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t copy_r(int64_t m, int64_t n, const double *A, int64_t lda, double *R, int64_t ldr,
                   cudaStream_t st) {
  const int64_t p = std::min(m, n);
  if (p <= 0 || n <= 0) return cudaSuccess;
  copy_r_kernel<<<grid1(p * n), kT, 0, st>>>(A, lda, p, n, R, ldr);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace dense
}  // namespace qtt
