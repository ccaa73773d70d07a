// FP64 dense linear algebra on the device, for the parts of the QTT method
// that work on whole cores: TT rounding (orthogonalisation by QR, truncation
// by SVD), TT-SVD (Algorithm 1), and the local systems of the inversion
// sweeps.  Every matrix is row-major: element (i, j) of a matrix with
// leading dimension ld is p[i * ld + j].
#pragma once

#include <cstdint>
#include <vector>

#include "qtt_internal.h"

namespace qtt {
namespace dense {

// C = alpha op(A) op(B) + beta C for `batch` independent problems (element
// strides sa, sb, sc between them).  op(A) is m x k (A itself k x m when ta),
// op(B) is k x n (B itself n x k when tb).  beta = 0 never reads C.
cudaError_t gemm(bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha,
                 const double *A, int64_t lda, int64_t sa, const double *B, int64_t ldb,
                 int64_t sb, double beta, double *C, int64_t ldc, int64_t sc, int64_t batch,
                 cudaStream_t st);

// out (contiguous, C order over dims[0..nd-1], nd <= 8) gathers
// out[i_0, ..., i_{nd-1}] = scale * in[sum_t i_t stride[t]]: transposes,
// axis permutations and reshapes of a tensor in one pass.
cudaError_t permute(const double *in, double *out, int nd, const int64_t *dims,
                    const int64_t *stride, double scale, cudaStream_t st);

// Householder QR of the m x n matrix A (any shape), p = min(m, n) reflectors
// H_j = I - tau_j v_j v_j^T with v_j(j) = 1: on return the upper triangle of
// A holds R and the entries below the diagonal the v_j (LAPACK's layout).
// tau: device, p entries.  work: device, qr_work_doubles(m, n) doubles.
size_t qr_work_doubles(int64_t m, int64_t n);
cudaError_t geqrf(int64_t m, int64_t n, double *A, int64_t lda, double *tau, double *work,
                  cudaStream_t st);
// The thin factor Q = H_0 ... H_{p-1} [I_p; 0] (m x p) from geqrf's output.
cudaError_t orgqr(int64_t m, int64_t n, const double *A, int64_t lda, const double *tau,
                  double *Q, int64_t ldq, double *work, cudaStream_t st);
// R (p x n, upper trapezoidal) copied out of geqrf's output, zeros below.
cudaError_t copy_r(int64_t m, int64_t n, const double *A, int64_t lda, double *R, int64_t ldr,
                   cudaStream_t st);

// One-sided Jacobi SVD (Hestenes' method, with the round-robin ordering of
// Brent and Luk) of the matrix B whose p COLUMNS are the p rows of Bt (each
// of length len): plane rotations of row pairs of Bt, accumulated in Vt
// (p x p, initialised to I here), until every pair is orthogonal to
// relative tolerance.  On return row i of Bt is sigma_i u_i^T and row i of
// Vt is v_i^T, so B = U diag(sigma) V^T; sigma (device, p) holds the row
// norms, unsorted.  work: device, jacobi_work_ints(p) ints.  Synchronises
// `st` once per sweep (the convergence test).  Returns the sweeps run in
// *sweeps (at most 60).
size_t jacobi_work_ints(int64_t p);
qtt_status jacobi_svd(int64_t p, int64_t len, double *Bt, int64_t ldb, double *Vt, int64_t ldv,
                      double *sigma, int *work, cudaStream_t st, int *sweeps);

// Sum of squares of n doubles (deterministic order), into *out (device).
cudaError_t sumsq(const double *x, int64_t n, double *out, double *work, cudaStream_t st);
size_t sumsq_work_doubles(int64_t n);

// out rows r = 0..nr-1 take in row idx[r] (device idx), times scale[idx[r]]
// when scale is given (the selection and ordering of singular triplets).
cudaError_t gather_rows(const double *in, int64_t ldi, const int *idx, const double *scale,
                        int64_t nr, int64_t ncols, double *out, int64_t ldo, bool divide,
                        cudaStream_t st);

}  // namespace dense
}  // namespace qtt
