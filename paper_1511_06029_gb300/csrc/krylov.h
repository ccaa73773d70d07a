// Batched FP64 vector kernels used by the solves.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace qtt {

// A set of vectors: vector i of right-hand side c starts at
// ptr + i * vec_stride + c * ld.
struct VecSet {
  double *ptr;
  int64_t ld;
  int64_t vec_stride;
};

inline VecSet vecs(const double *p, int64_t ld, int64_t vec_stride = 0) {
  return VecSet{const_cast<double *>(p), ld, vec_stride};
}

// Number of partial sums per right-hand side (fixed by N alone).
int blocks_for(int64_t N);

// out[i * nrhs + c] = <V_i[c], W[c]> for i < nv (written if out != NULL;
// added into accumulate_into if that is not NULL).  `partial` must hold
// nv * min(nrhs, 65535) * blocks_for(N) doubles.
cudaError_t vec_dots(VecSet V, int nv, VecSet W, int64_t N, int64_t nrhs, double *partial,
                     double *out, double *accumulate_into, cudaStream_t st);
// W[c] -= sum_{i < nv} h[i * nrhs + c] V_i[c]
cudaError_t vec_gs_update(VecSet W, VecSet V, int nv, const double *h, int64_t N, int64_t nrhs,
                          cudaStream_t st);
// U[c] = sum_{i < nv} y[i * nrhs + c] V_i[c]
cudaError_t vec_combine(VecSet U, VecSet V, int nv, const double *y, int64_t N, int64_t nrhs,
                        cudaStream_t st);
// D[c] = S[c] / sqrt(sumsq[c]) (0 where sumsq[c] == 0)
cudaError_t vec_normalize(VecSet D, VecSet S, const double *sumsq, int64_t N, int64_t nrhs,
                          cudaStream_t st);
// D[c] = S[c] * scale[c]
cudaError_t vec_scale(VecSet D, VecSet S, const double *scale, int64_t N, int64_t nrhs,
                      cudaStream_t st);
// D[c] += alpha S[c]
cudaError_t vec_axpy(VecSet D, VecSet S, double alpha, int64_t N, int64_t nrhs,
                     cudaStream_t st);
cudaError_t vec_copy(VecSet D, VecSet S, int64_t N, int64_t nrhs, cudaStream_t st);

}  // namespace qtt
