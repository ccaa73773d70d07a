// Whole-core QTT operations on the device, built on the FP64 dense layer
// (dense.h):
//   qtt_tt_round     TT rounding (orthogonalisation, then truncated SVDs with
//                    the threshold of Algorithm 1), e.g. of the compressed
//                    product c = A b of Sec. 4.2, whose ranks multiply
//   qtt_tt_svd       Algorithm 1: the QTT decomposition of a dense matrix
//   qtt_local_apply  the three-core product of the inversion's local systems
//                    (appendix on local linear systems)
// Only the truncation decision runs on the host: it reads the singular
// values of one unfolding (a few hundred numbers), sorts them and picks the
// rank; every product, factorisation and reordering is a kernel.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "dense.h"

namespace qtt {
namespace {

// Stream-ordered scratch that is returned on every exit.
struct Pool {
  cudaStream_t st;
  std::vector<void *> held;
  explicit Pool(cudaStream_t s) : st(s) {}
  ~Pool() {
    for (void *p : held) scratch_free(p, st);
  }
  template <class T>
  qtt_status get(T **out, size_t n) {
    void *p = nullptr;
    const qtt_status s = scratch_alloc(&p, std::max<size_t>(n, 1) * sizeof(T), st);
    if (s != QTT_OK) return s;
    held.push_back(p);
    *out = static_cast<T *>(p);
    return QTT_OK;
  }
  void put(void *p) {
    auto it = std::find(held.begin(), held.end(), p);
    if (it != held.end()) {
      scratch_free(p, st);
      held.erase(it);
    }
  }
};

#define TT_TRY(x)                               \
  do {                                          \
    const qtt_status s_ = (x);                  \
    if (s_ != QTT_OK) return s_;                \
  } while (0)
#define TT_CUDA(x, what)                        \
  do {                                          \
    const cudaError_t e_ = (x);                 \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

// 2-D transpose: out (cols x rows) = in (rows x cols)^T, times scale.
cudaError_t transpose(const double *in, int64_t rows, int64_t cols, double *out, cudaStream_t st,
                      double scale = 1.0) {
  const int64_t dims[2] = {cols, rows}, stride[2] = {1, cols};
  return dense::permute(in, out, 2, dims, stride, scale, st);
}

// Singular values read back, sorted in decreasing order (ties by index) and
// cut by the rule of Algorithm 1: the smallest rank whose discarded values
// have 2-norm <= delta, at least 1.  Returns the kept indices, uploaded.
qtt_status truncate(Pool &P, const double *sigma_dev, int64_t p, double delta, int **idx_dev,
                    std::vector<double> *kept_sigma) {
  std::vector<double> s((size_t)p);
  TT_CUDA(cudaMemcpyAsync(s.data(), sigma_dev, (size_t)p * sizeof(double), cudaMemcpyDeviceToHost,
                          P.st),
          "truncate: read singular values");
  TT_CUDA(cudaStreamSynchronize(P.st), "truncate: sync");
  std::vector<int> order((size_t)p);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return s[a] > s[b]; });
  int64_t keep = p;
  // tail[t] = sum of the squares of the sorted values t .. p-1
  std::vector<double> tail((size_t)p + 1, 0.0);
  for (int64_t t = p - 1; t >= 0; --t) tail[t] = tail[t + 1] + s[order[t]] * s[order[t]];
  while (keep > 1 && std::sqrt(tail[keep - 1]) <= delta) --keep;
  order.resize((size_t)keep);
  if (kept_sigma) {
    kept_sigma->clear();
    for (int i : order) kept_sigma->push_back(s[i]);
  }
  TT_TRY(P.get(idx_dev, (size_t)keep));
  TT_CUDA(cudaMemcpyAsync(*idx_dev, order.data(), (size_t)keep * sizeof(int),
                          cudaMemcpyHostToDevice, P.st),
          "truncate: upload indices");
  TT_CUDA(cudaStreamSynchronize(P.st), "truncate: sync");
  return QTT_OK;
}

// QR of the m x n matrix M (overwritten): Q (m x p) and R (p x n), p =
// min(m, n), both newly taken from the pool.
qtt_status qr(Pool &P, double *M, int64_t m, int64_t n, double **Q, double **R) {
  const int64_t p = std::min(m, n);
  double *tau, *work;
  TT_TRY(P.get(&tau, (size_t)p));
  TT_TRY(P.get(&work, dense::qr_work_doubles(m, n)));
  TT_TRY(P.get(Q, (size_t)(m * p)));
  TT_TRY(P.get(R, (size_t)(p * n)));
  TT_CUDA(dense::geqrf(m, n, M, n, tau, work, P.st), "qr: geqrf");
  TT_CUDA(dense::copy_r(m, n, M, n, *R, n, P.st), "qr: copy R");
  TT_CUDA(dense::orgqr(m, n, M, n, tau, *Q, p, work, P.st), "qr: orgqr");
  P.put(tau);
  P.put(work);
  return QTT_OK;
}

// Jacobi SVD of B given as Bt (p x len, rows = columns of B): Vt (p x p)
// and sigma (p) newly taken from the pool; Bt is overwritten by Sigma U^T.
qtt_status svd(Pool &P, double *Bt, int64_t p, int64_t len, double **Vt, double **sigma) {
  int *iw;
  TT_TRY(P.get(Vt, (size_t)(p * p)));
  TT_TRY(P.get(sigma, (size_t)p));
  TT_TRY(P.get(&iw, dense::jacobi_work_ints(p)));
  TT_TRY(dense::jacobi_svd(p, len, Bt, len, *Vt, p, *sigma, iw, P.st, nullptr));
  P.put(iw);
  return QTT_OK;
}

bool round_args_ok(int d, const int *ranks, int n) {
  if (d < 1 || d > 64 || !ranks || n < 1 || n > 256) return false;
  if (ranks[0] != 1 || ranks[d] != 1) return false;
  for (int k = 0; k <= d; ++k)
    if (ranks[k] < 1 || ranks[k] > 32768) return false;
  for (int k = 0; k < d; ++k)
    if ((double)ranks[k] * n * ranks[k + 1] > 4.0e9) return false;
  return true;
}

}  // namespace
}  // namespace qtt

using namespace qtt;

extern "C" qtt_status qtt_tt_round(int d, const int *ranks, int n, const double *cores_in,
                                   double eps, int *ranks_out, double *cores_out, void *stream) {
  if (!round_args_ok(d, ranks, n))
    return fail(QTT_ERR_INVALID_ARG,
                "qtt_tt_round: need 1 <= d <= 64, ranks[0] = ranks[d] = 1, ranks in [1, 32768], "
                "1 <= n <= 256 and cores of at most 4e9 entries");
  if (!cores_in || !cores_out || !ranks_out)
    return fail(QTT_ERR_INVALID_ARG, "qtt_tt_round: NULL pointer");
  if (!(eps >= 0.0)) return fail(QTT_ERR_INVALID_ARG, "qtt_tt_round: eps must be >= 0");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Pool P(st);
  std::vector<int64_t> r(ranks, ranks + d + 1);
  std::vector<double *> core((size_t)d, nullptr);
  {
    int64_t off = 0;
    for (int k = 0; k < d; ++k) {
      const int64_t sz = r[k] * n * r[k + 1];
      TT_TRY(P.get(&core[k], (size_t)sz));
      TT_CUDA(cudaMemcpyAsync(core[k], cores_in + off, (size_t)sz * sizeof(double),
                              cudaMemcpyDeviceToDevice, st),
              "qtt_tt_round: copy in");
      off += sz;
    }
  }
  // left to right: core k = Q (left-orthonormal), core k+1 = R core k+1
  for (int k = 0; k + 1 < d; ++k) {
    const int64_t m = r[k] * n, nb = r[k + 1], p = std::min(m, nb);
    double *Q, *R;
    TT_TRY(qr(P, core[k], m, nb, &Q, &R));
    double *next;
    const int64_t ncols = n * r[k + 2];
    TT_TRY(P.get(&next, (size_t)(p * ncols)));
    TT_CUDA(dense::gemm(false, false, p, ncols, nb, 1.0, R, nb, 0, core[k + 1], ncols, 0, 0.0, next,
                        ncols, 0, 1, st),
            "qtt_tt_round: R x next core");
    P.put(core[k]);
    P.put(core[k + 1]);
    P.put(R);
    core[k] = Q;
    core[k + 1] = next;
    r[k + 1] = p;
  }
  // ||t||_F is the norm of the last core now; the threshold of Algorithm 1
  double delta = 0.0;
  {
    double *work, *acc;
    TT_TRY(P.get(&work, dense::sumsq_work_doubles(0)));
    TT_TRY(P.get(&acc, 1));
    TT_CUDA(dense::sumsq(core[d - 1], r[d - 1] * n, acc, work, st), "qtt_tt_round: norm");
    double h = 0.0;
    TT_CUDA(cudaMemcpyAsync(&h, acc, sizeof(double), cudaMemcpyDeviceToHost, st), "norm read");
    TT_CUDA(cudaStreamSynchronize(st), "norm sync");
    delta = eps * std::sqrt(h) / std::sqrt((double)std::max(d - 1, 1));
    P.put(work);
    P.put(acc);
  }
  // right to left: truncated SVD of the unfolding ra x (n rb) of core k
  for (int k = d - 1; k >= 1; --k) {
    const int64_t ra = r[k], q = n * r[k + 1];
    double *X = nullptr;        // ra x keep, multiplies core k-1 from the right
    bool x_transposed = false;  // X given as its transpose (keep x ra)
    double *newk = nullptr;
    int64_t keep = 0;
    if (ra >= q) {
      double *Q1, *R;
      TT_TRY(qr(P, core[k], ra, q, &Q1, &R));  // Q1 ra x q, R q x q
      double *Bt;
      TT_TRY(P.get(&Bt, (size_t)(q * q)));
      TT_CUDA(transpose(R, q, q, Bt, st), "transpose R");  // B = R
      P.put(R);
      double *Vt, *sig;
      TT_TRY(svd(P, Bt, q, q, &Vt, &sig));  // R = U_R S V^T, Bt = S U_R^T
      int *idx;
      std::vector<double> ks;
      TT_TRY(truncate(P, sig, q, delta, &idx, &ks));
      keep = (int64_t)ks.size();
      TT_TRY(P.get(&newk, (size_t)(keep * q)));
      TT_CUDA(dense::gather_rows(Vt, q, idx, nullptr, keep, q, newk, q, false, st), "V^T rows");
      double *Bk;
      TT_TRY(P.get(&Bk, (size_t)(keep * q)));
      TT_CUDA(dense::gather_rows(Bt, q, idx, nullptr, keep, q, Bk, q, false, st), "S U^T rows");
      TT_TRY(P.get(&X, (size_t)(ra * keep)));
      TT_CUDA(dense::gemm(false, true, ra, keep, q, 1.0, Q1, q, 0, Bk, q, 0, 0.0, X, keep, 0, 1, st),
              "Q1 U S");
      P.put(Q1);
      P.put(Bt);
      P.put(Vt);
      P.put(sig);
      P.put(Bk);
    } else {
      double *Mt;
      TT_TRY(P.get(&Mt, (size_t)(q * ra)));
      TT_CUDA(transpose(core[k], ra, q, Mt, st), "transpose unfolding");
      double *Q2, *R2;
      TT_TRY(qr(P, Mt, q, ra, &Q2, &R2));  // Q2 q x ra, R2 ra x ra
      P.put(Mt);
      double *Vt, *sig;
      TT_TRY(svd(P, R2, ra, ra, &Vt, &sig));  // B = R2^T = U S W^T; R2 becomes S U^T
      int *idx;
      std::vector<double> ks;
      TT_TRY(truncate(P, sig, ra, delta, &idx, &ks));
      keep = (int64_t)ks.size();
      double *Wk;
      TT_TRY(P.get(&Wk, (size_t)(keep * ra)));
      TT_CUDA(dense::gather_rows(Vt, ra, idx, nullptr, keep, ra, Wk, ra, false, st), "W^T rows");
      TT_TRY(P.get(&newk, (size_t)(keep * q)));
      TT_CUDA(dense::gemm(false, true, keep, q, ra, 1.0, Wk, ra, 0, Q2, ra, 0, 0.0, newk, q, 0, 1,
                          st),
              "W^T Q2^T");
      TT_TRY(P.get(&X, (size_t)(keep * ra)));
      TT_CUDA(dense::gather_rows(R2, ra, idx, nullptr, keep, ra, X, ra, false, st), "S U^T rows");
      x_transposed = true;
      P.put(Q2);
      P.put(R2);
      P.put(Vt);
      P.put(sig);
      P.put(Wk);
    }
    // core k-1 (r_{k-1} n x ra) times X (ra x keep)
    const int64_t mrows = r[k - 1] * n;
    double *prev;
    TT_TRY(P.get(&prev, (size_t)(mrows * keep)));
    TT_CUDA(dense::gemm(false, x_transposed, mrows, keep, ra, 1.0, core[k - 1], ra, 0, X,
                        x_transposed ? ra : keep, 0, 0.0, prev, keep, 0, 1, st),
            "core k-1 x U S");
    P.put(X);
    P.put(core[k - 1]);
    P.put(core[k]);
    core[k - 1] = prev;
    core[k] = newk;
    r[k] = keep;
  }
  int64_t off = 0;
  for (int k = 0; k < d; ++k) {
    const int64_t sz = r[k] * n * r[k + 1];
    TT_CUDA(cudaMemcpyAsync(cores_out + off, core[k], (size_t)sz * sizeof(double),
                            cudaMemcpyDeviceToDevice, st),
            "qtt_tt_round: copy out");
    off += sz;
  }
  TT_CUDA(cudaStreamSynchronize(st), "qtt_tt_round: sync");
  for (int k = 0; k <= d; ++k) ranks_out[k] = (int)r[k];
  return QTT_OK;
}

namespace qtt {
namespace {

// T[(i_0 j_0), (i_1 j_1), ..., (i_{d-1} j_{d-1})] (C order, mode 0 slowest,
// mode value 2 i_k + j_k) = A(i, j) with i = sum_k i_k 2^k, j likewise: the
// tensor whose first unfolding Algorithm 1 splits.
__global__ void __launch_bounds__(256) modes_kernel(const double *A, int d, double *T) {
  const int64_t N = (int64_t)1 << d, total = N * N;
  for (int64_t t = (int64_t)blockIdx.x * 256 + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * 256) {
    int64_t i = 0, j = 0, rem = t;
    for (int k = d - 1; k >= 0; --k) {
      const int mk = (int)(rem & 3);
      rem >>= 2;
      i |= (int64_t)(mk >> 1) << k;
      j |= (int64_t)(mk & 1) << k;
    }
    T[t] = A[i * N + j];
  }
}

}  // namespace
}  // namespace qtt

extern "C" qtt_status qtt_tt_svd(int d, const double *A, double eps, int *ranks_out,
                                 double *cores_out, int64_t capacity, int64_t *n_out,
                                 void *stream) {
  if (d < 1 || d > 13) return fail(QTT_ERR_INVALID_ARG, "qtt_tt_svd: d must be in [1, 13]");
  if (!A || !ranks_out || !n_out) return fail(QTT_ERR_INVALID_ARG, "qtt_tt_svd: NULL pointer");
  if (!(eps >= 0.0)) return fail(QTT_ERR_INVALID_ARG, "qtt_tt_svd: eps must be >= 0");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Pool P(st);
  const int64_t N = (int64_t)1 << d, total = N * N;
  double *M;
  TT_TRY(P.get(&M, (size_t)total));
  {
    const unsigned g = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32);
    modes_kernel<<<g, 256, 0, st>>>(A, d, M);
    count_launches(1);
    TT_CUDA(cudaGetLastError(), "qtt_tt_svd: mode order");
  }
  double delta = 0.0;
  {
    double *work, *acc;
    TT_TRY(P.get(&work, dense::sumsq_work_doubles(total)));
    TT_TRY(P.get(&acc, 1));
    TT_CUDA(dense::sumsq(M, total, acc, work, st), "qtt_tt_svd: norm");
    double h = 0.0;
    TT_CUDA(cudaMemcpyAsync(&h, acc, sizeof(double), cudaMemcpyDeviceToHost, st), "norm read");
    TT_CUDA(cudaStreamSynchronize(st), "norm sync");
    delta = eps * std::sqrt(h) / std::sqrt((double)std::max(d - 1, 1));
    P.put(work);
    P.put(acc);
  }
  std::vector<int64_t> r{1};
  std::vector<double *> core;
  int64_t cols = total / 4;
  for (int k = 0; k + 1 < d; ++k) {
    const int64_t rows = 4 * r.back();  // M is rows x cols
    double *U = nullptr, *next = nullptr;
    int64_t keep = 0;
    if (rows <= cols) {
      // wide: QR of M^T; M = R2^T Q2^T, R2^T = U S W^T, M = U S (Q2 W)^T
      double *Mt;
      TT_TRY(P.get(&Mt, (size_t)(rows * cols)));
      TT_CUDA(transpose(M, rows, cols, Mt, st), "transpose unfolding");
      P.put(M);
      double *Q2, *R2;
      TT_TRY(qr(P, Mt, cols, rows, &Q2, &R2));  // Q2 cols x rows, R2 rows x rows
      P.put(Mt);
      double *Vt, *sig;
      TT_TRY(svd(P, R2, rows, rows, &Vt, &sig));
      int *idx;
      std::vector<double> ks;
      TT_TRY(truncate(P, sig, rows, delta, &idx, &ks));
      keep = (int64_t)ks.size();
      // core k = U[:, kept]: rows of R2 (S U^T) divided by sigma, transposed
      double *Ut;
      TT_TRY(P.get(&Ut, (size_t)(keep * rows)));
      TT_CUDA(dense::gather_rows(R2, rows, idx, sig, keep, rows, Ut, rows, true, st), "U^T rows");
      TT_TRY(P.get(&U, (size_t)(rows * keep)));
      TT_CUDA(transpose(Ut, keep, rows, U, st), "U");
      // next = S W^T Q2^T (keep x cols)
      double *SW;
      TT_TRY(P.get(&SW, (size_t)(keep * rows)));
      TT_CUDA(dense::gather_rows(Vt, rows, idx, sig, keep, rows, SW, rows, false, st), "S W^T");
      TT_TRY(P.get(&next, (size_t)(keep * cols)));
      TT_CUDA(dense::gemm(false, true, keep, cols, rows, 1.0, SW, rows, 0, Q2, rows, 0, 0.0, next,
                          cols, 0, 1, st),
              "S W^T Q2^T");
      for (void *p : {(void *)Q2, (void *)R2, (void *)Vt, (void *)sig, (void *)Ut, (void *)SW})
        P.put(p);
    } else {
      // tall: M = Q1 R, R = U_R S V^T, M = (Q1 U_R) S V^T
      double *Q1, *R;
      TT_TRY(qr(P, M, rows, cols, &Q1, &R));  // Q1 rows x cols, R cols x cols
      P.put(M);
      double *Bt;
      TT_TRY(P.get(&Bt, (size_t)(cols * cols)));
      TT_CUDA(transpose(R, cols, cols, Bt, st), "transpose R");
      P.put(R);
      double *Vt, *sig;
      TT_TRY(svd(P, Bt, cols, cols, &Vt, &sig));
      int *idx;
      std::vector<double> ks;
      TT_TRY(truncate(P, sig, cols, delta, &idx, &ks));
      keep = (int64_t)ks.size();
      double *Ut;
      TT_TRY(P.get(&Ut, (size_t)(keep * cols)));
      TT_CUDA(dense::gather_rows(Bt, cols, idx, sig, keep, cols, Ut, cols, true, st), "U_R^T rows");
      TT_TRY(P.get(&U, (size_t)(rows * keep)));
      TT_CUDA(dense::gemm(false, true, rows, keep, cols, 1.0, Q1, cols, 0, Ut, cols, 0, 0.0, U, keep,
                          0, 1, st),
              "Q1 U_R");
      TT_TRY(P.get(&next, (size_t)(keep * cols)));
      TT_CUDA(dense::gather_rows(Vt, cols, idx, sig, keep, cols, next, cols, false, st), "S V^T");
      for (void *p : {(void *)Q1, (void *)Bt, (void *)Vt, (void *)sig, (void *)Ut}) P.put(p);
    }
    core.push_back(U);  // rows (alpha_k, i_k, j_k) x keep: [alpha][i][j][alpha']
    r.push_back(keep);
    M = next;           // keep x cols = (4 keep) x (cols / 4), the next unfolding
    cols /= 4;
  }
  core.push_back(M);  // (4 r_{d-1}) x 1
  r.push_back(1);
  int64_t need = 0;
  for (int k = 0; k < d; ++k) need += 4 * r[k] * r[k + 1];
  *n_out = need;
  for (int k = 0; k <= d; ++k) ranks_out[k] = (int)r[k];
  if (!cores_out || capacity < need) {
    TT_CUDA(cudaStreamSynchronize(st), "qtt_tt_svd: sync");
    return fail(QTT_ERR_INVALID_ARG, "qtt_tt_svd: cores_out holds " + std::to_string(capacity) +
                                         " doubles, the decomposition needs " +
                                         std::to_string(need) + " (see *n_out)");
  }
  int64_t off = 0;
  for (int k = 0; k < d; ++k) {
    const int64_t sz = 4 * r[k] * r[k + 1];
    TT_CUDA(cudaMemcpyAsync(cores_out + off, core[k], (size_t)sz * sizeof(double),
                            cudaMemcpyDeviceToDevice, st),
            "qtt_tt_svd: copy out");
    off += sz;
  }
  TT_CUDA(cudaStreamSynchronize(st), "qtt_tt_svd: sync");
  return QTT_OK;
}

// y[beta][i][p][B] = sum Psi[a][beta][g] G[a][i][j][A] Phi[A][B][C] W[g][j][p][C]
// as three GEMMs:
//   T1[a beta][j p C]  = Psi[(a beta)][g] W[g][(j p C)]
//   T1' = T1 reordered [beta][p][C][a][j];  G' = G reordered [a][j][i][A]
//   T2[(beta p C)][(i A)] = T1'[(beta p C)][(a j)] G'[(a j)][(i A)]
//   T2' = T2 reordered [beta][i][p][A][C];  Phi' = Phi reordered [A][C][B]
//   y[(beta i p)][B] = T2'[(beta i p)][(A C)] Phi'[(A C)][B]
extern "C" qtt_status qtt_local_apply(int ra, int ra2, int rx, int rx2, const double *psi,
                                      const double *G, const double *phi, const double *W,
                                      double *y, int64_t nvec, void *stream) {
  if (ra < 1 || ra2 < 1 || rx < 1 || rx2 < 1 || ra > 4096 || ra2 > 4096 || rx > 4096 ||
      rx2 > 4096)
    return fail(QTT_ERR_INVALID_ARG, "qtt_local_apply: ranks must be in [1, 4096]");
  if (nvec < 0) return fail(QTT_ERR_INVALID_ARG, "qtt_local_apply: nvec < 0");
  if (nvec == 0) return QTT_OK;
  if (!psi || !G || !phi || !W || !y) return fail(QTT_ERR_INVALID_ARG, "qtt_local_apply: NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Pool P(st);
  const int64_t a = ra, A2 = ra2, b = rx, B2 = rx2;
  const int64_t wsz = b * 4 * B2;  // one W and one y
  double *Gp, *Phip, *T1, *T1p, *T2, *T2p;
  TT_TRY(P.get(&Gp, (size_t)(a * 4 * A2)));
  TT_TRY(P.get(&Phip, (size_t)(A2 * B2 * B2)));
  TT_TRY(P.get(&T1, (size_t)(a * b * 4 * B2)));
  TT_TRY(P.get(&T1p, (size_t)(a * b * 4 * B2)));
  TT_TRY(P.get(&T2, (size_t)(b * 4 * B2 * A2)));
  TT_TRY(P.get(&T2p, (size_t)(b * 4 * B2 * A2)));
  {
    // G'[a][j][i][A] = G[a][i][j][A]
    const int64_t dims[4] = {a, 2, 2, A2}, str[4] = {4 * A2, A2, 2 * A2, 1};
    TT_CUDA(dense::permute(G, Gp, 4, dims, str, 1.0, st), "reorder G");
    // Phi'[A][C][B] = Phi[A][B][C]
    const int64_t d2[3] = {A2, B2, B2}, s2[3] = {B2 * B2, 1, B2};
    TT_CUDA(dense::permute(phi, Phip, 3, d2, s2, 1.0, st), "reorder Phi");
  }
  for (int64_t v = 0; v < nvec; ++v) {
    const double *Wv = W + v * wsz;
    double *yv = y + v * wsz;
    TT_CUDA(dense::gemm(false, false, a * b, 4 * B2, b, 1.0, psi, b, 0, Wv, 4 * B2, 0, 0.0, T1,
                        4 * B2, 0, 1, st),
            "Psi W");
    {
      // T1'[beta][p][C][a][j] = T1[a][beta][j][p][C]
      const int64_t dims[5] = {b, 2, B2, a, 2};
      const int64_t str[5] = {4 * B2, B2, 1, b * 4 * B2, 2 * B2};
      TT_CUDA(dense::permute(T1, T1p, 5, dims, str, 1.0, st), "reorder T1");
    }
    TT_CUDA(dense::gemm(false, false, b * 2 * B2, 2 * A2, 2 * a, 1.0, T1p, 2 * a, 0, Gp, 2 * A2, 0,
                        0.0, T2, 2 * A2, 0, 1, st),
            "T1 G");
    {
      // T2'[beta][i][p][A][C] = T2[beta][p][C][i][A]
      const int64_t dims[5] = {b, 2, 2, A2, B2};
      const int64_t str[5] = {2 * B2 * 2 * A2, A2, B2 * 2 * A2, 1, 2 * A2};
      TT_CUDA(dense::permute(T2, T2p, 5, dims, str, 1.0, st), "reorder T2");
    }
    TT_CUDA(dense::gemm(false, false, b * 4, B2, A2 * B2, 1.0, T2p, A2 * B2, 0, Phip, B2, 0, 0.0, yv,
                        B2, 0, 1, st),
            "T2 Phi");
  }
  return QTT_OK;
}
