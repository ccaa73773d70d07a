// BF16 tensor-core core step -- see step_mma.cu.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace qtt {

constexpr int kMmaMaxRank = 64;

struct StepMMA {
  const __nv_bfloat16 *in;   // y_k, planar [rhs][a][position], BF16
  int64_t in_rhs_stride;
  __nv_bfloat16 *out;        // y_{k+1}
  int64_t out_rhs_stride;
  const __nv_bfloat16 *A;    // M_k as [Mp][Kp], row 2b+i, column 2a+j, zero padded
  int k, rin, rout, Mp, Kp;
  int64_t N, nrhs;
};

// Steps the tensor-core kernel takes (others use the CUDA-core step).
bool mma_step_eligible(int k, int rin, int rout, int64_t N);
cudaError_t launch_step_mma_bf16(const StepMMA &s, cudaStream_t st);

}  // namespace qtt
