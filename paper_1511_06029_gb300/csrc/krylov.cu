// Vector kernels of the solves (FP64): Gram-Schmidt dots and updates, norms,
// basis combinations and axpys, batched over right-hand sides.
//
// Every reduction has a fixed order that depends only on N: right-hand side
// c is cut into B = blocks_for(N) equal chunks, each chunk summed by one
// 256-thread block in a fixed strided order and a fixed shared-memory tree,
// and the B partials summed sequentially.  A right-hand side therefore gets
// bitwise the same dots whatever else is in the batch.
#include "qtt_internal.h"
#include "krylov.h"

namespace qtt {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double block_sum(double v, double *sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  return sh[0];
}

// partial[(i * nrhs + c) * B + blk] = sum over chunk blk of V_i[c] . W[c]
__global__ void __launch_bounds__(kThreads)
dots_partial_kernel(VecSet V, int nv, VecSet W, int64_t N, int B, double *partial) {
  __shared__ double sh[kThreads];
  const int blk = blockIdx.x;
  const int64_t c = blockIdx.y;
  const int i = blockIdx.z;
  const int64_t nrhs = gridDim.y;
  const int64_t chunk = N / B;
  const double *v = V.ptr + (int64_t)i * V.vec_stride + c * V.ld;
  const double *w = W.ptr + c * W.ld;
  double s = 0.0;
  for (int64_t t = (int64_t)blk * chunk + threadIdx.x; t < (int64_t)(blk + 1) * chunk; t += kThreads)
    s = fma(v[t], w[t], s);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partial[((int64_t)i * nrhs + c) * B + blk] = s;
  (void)nv;
}

// partial[(i * nc + c) * B + b] -> out[i * nrhs + c0 + c] (sum over b in order)
__global__ void reduce_partials_kernel(const double *partial, int B, int64_t nc, int nv,
                                       int64_t nrhs, int64_t c0, double *out, double *out2) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nc * nv) return;
  double s = 0.0;
  for (int b = 0; b < B; ++b) s += partial[idx * B + b];
  const int64_t i = idx / nc, c = idx % nc;
  const int64_t o = i * nrhs + c0 + c;
  if (out2) out2[o] += s;  // accumulate (second Gram-Schmidt pass)
  if (out) out[o] = s;
}

// W[c] -= sum_i h[i * nrhs + c] V_i[c]
__global__ void gs_update_kernel(VecSet W, VecSet V, int nv, const double *h, int64_t N) {
  const int64_t c = blockIdx.y;
  const int64_t nrhs = gridDim.y;
  double *w = W.ptr + c * W.ld;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    double acc = w[t];
    for (int i = 0; i < nv; ++i)
      acc -= h[(int64_t)i * nrhs + c] * V.ptr[(int64_t)i * V.vec_stride + c * V.ld + t];
    w[t] = acc;
  }
}

// U[c] = sum_i y[i * nrhs + c] V_i[c]
__global__ void combine_kernel(VecSet U, VecSet V, int nv, const double *y, int64_t N) {
  const int64_t c = blockIdx.y;
  const int64_t nrhs = gridDim.y;
  double *u = U.ptr + c * U.ld;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < nv; ++i)
      acc += y[(int64_t)i * nrhs + c] * V.ptr[(int64_t)i * V.vec_stride + c * V.ld + t];
    u[t] = acc;
  }
}

// D[c] = S[c] / sqrt(sumsq[c])   (0 if sumsq[c] == 0)
__global__ void normalize_kernel(VecSet D, VecSet S, const double *sumsq, int64_t N) {
  const int64_t c = blockIdx.y;
  const double q = sumsq[c];
  const double inv = q > 0.0 ? 1.0 / sqrt(q) : 0.0;
  const double *s = S.ptr + c * S.ld;
  double *dd = D.ptr + c * D.ld;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x)
    dd[t] = s[t] * inv;
}

// D[c] = S[c] * scale[c]
__global__ void scale_kernel(VecSet D, VecSet S, const double *scale, int64_t N) {
  const int64_t c = blockIdx.y;
  const double a = scale[c];
  const double *s = S.ptr + c * S.ld;
  double *dd = D.ptr + c * D.ld;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x)
    dd[t] = s[t] * a;
}

__global__ void copy_kernel(VecSet D, VecSet S, int64_t N) {
  const int64_t c = blockIdx.y;
  const double *s = S.ptr + c * S.ld;
  double *dd = D.ptr + c * D.ld;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x)
    dd[t] = s[t];
}

// D[c] += alpha S[c]
__global__ void axpy_kernel(VecSet D, VecSet S, double alpha, int64_t N) {
  const int64_t c = blockIdx.y;
  const double *s = S.ptr + c * S.ld;
  double *dd = D.ptr + c * D.ld;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x)
    dd[t] += alpha * s[t];
}

unsigned grid_x(int64_t N) {
  int64_t g = (N + kThreads - 1) / kThreads;
  if (g > 4096) g = 4096;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

int blocks_for(int64_t N) {
  int64_t B = N / 4096;
  if (B < 1) B = 1;
  if (B > 256) B = 256;
  return (int)B;  // N and B are powers of two, so B divides N
}

cudaError_t vec_dots(VecSet V, int nv, VecSet W, int64_t N, int64_t nrhs, double *partial,
                     double *out, double *accumulate_into, cudaStream_t st) {
  if (nv <= 0 || nrhs <= 0) return cudaSuccess;
  const int B = blocks_for(N);
  for (int64_t c0 = 0; c0 < nrhs; c0 += 65535) {
    const int64_t nc = nrhs - c0 < 65535 ? nrhs - c0 : 65535;
    VecSet Vc = V, Wc = W;
    Vc.ptr += c0 * V.ld;
    Wc.ptr += c0 * W.ld;
    // partial layout uses the chunk's own nrhs; reduce it into out[i*nrhs+c]
    dots_partial_kernel<<<dim3(B, (unsigned)nc, nv), kThreads, 0, st>>>(Vc, nv, Wc, N, B, partial);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t count = nc * nv;
    reduce_partials_kernel<<<(unsigned)((count + 127) / 128), 128, 0, st>>>(
        partial, B, nc, nv, nrhs, c0, out, accumulate_into);
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t vec_gs_update(VecSet W, VecSet V, int nv, const double *h, int64_t N, int64_t nrhs,
                          cudaStream_t st) {
  if (nv <= 0 || nrhs <= 0) return cudaSuccess;
  if (nrhs > 65535) return cudaErrorInvalidValue;
  gs_update_kernel<<<dim3(grid_x(N), (unsigned)nrhs), kThreads, 0, st>>>(W, V, nv, h, N);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t vec_combine(VecSet U, VecSet V, int nv, const double *y, int64_t N, int64_t nrhs,
                        cudaStream_t st) {
  if (nrhs <= 0) return cudaSuccess;
  if (nrhs > 65535) return cudaErrorInvalidValue;
  combine_kernel<<<dim3(grid_x(N), (unsigned)nrhs), kThreads, 0, st>>>(U, V, nv, y, N);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t vec_normalize(VecSet D, VecSet S, const double *sumsq, int64_t N, int64_t nrhs,
                          cudaStream_t st) {
  if (nrhs <= 0) return cudaSuccess;
  if (nrhs > 65535) return cudaErrorInvalidValue;
  normalize_kernel<<<dim3(grid_x(N), (unsigned)nrhs), kThreads, 0, st>>>(D, S, sumsq, N);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t vec_scale(VecSet D, VecSet S, const double *scale, int64_t N, int64_t nrhs,
                      cudaStream_t st) {
  if (nrhs <= 0) return cudaSuccess;
  if (nrhs > 65535) return cudaErrorInvalidValue;
  scale_kernel<<<dim3(grid_x(N), (unsigned)nrhs), kThreads, 0, st>>>(D, S, scale, N);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t vec_axpy(VecSet D, VecSet S, double alpha, int64_t N, int64_t nrhs,
                     cudaStream_t st) {
  if (nrhs <= 0) return cudaSuccess;
  if (nrhs > 65535) return cudaErrorInvalidValue;
  axpy_kernel<<<dim3(grid_x(N), (unsigned)nrhs), kThreads, 0, st>>>(D, S, alpha, N);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t vec_copy(VecSet D, VecSet S, int64_t N, int64_t nrhs, cudaStream_t st) {
  if (nrhs <= 0) return cudaSuccess;
  if (nrhs > 65535) return cudaErrorInvalidValue;
  copy_kernel<<<dim3(grid_x(N), (unsigned)nrhs), kThreads, 0, st>>>(D, S, N);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace qtt
