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

// Two consecutive steps k, k+1 in one launch (step_mma2.cu): the r_{k+1}
// planes between them stay in shared memory.
constexpr int kMma2MaxRank = 48;

struct StepMMA2 {
  const __nv_bfloat16 *in;   // y_k, planar [rhs][a][position], BF16
  int64_t in_rhs_stride;
  __nv_bfloat16 *out;        // y_{k+2}
  int64_t out_rhs_stride;
  const __nv_bfloat16 *A1;   // M_k as [Mp1][Kp1]
  const __nv_bfloat16 *A2;   // M_{k+1} as [Mp2][Mp1] (its K padding equals M_k's row padding)
  int k, r0, r1, r2, Mp1, Kp1, Mp2;
  int64_t N, nrhs;
  int groups_cap = 0;        // tcgen05 pairs: 0 = as many epilogue groups as fit, 2 = two
};

bool mma2_steps_eligible(int k, int r0, int r1, int r2, int64_t N);
cudaError_t launch_step_mma2_bf16(const StepMMA2 &s, cudaStream_t st);

// The same fused pair on the tcgen05 tensor cores (step_tc2.cu): TMA tile
// loads and stores, MMAs from shared-memory descriptors into TMEM.  Returns
// cudaErrorNotSupported (nothing launched) when the shapes do not fit its
// tile views; the caller then runs the two steps another way.
constexpr int kTc2MaxRank = 56;
bool tc2_steps_eligible(int k, int r0, int r1, int r2, int64_t N);
cudaError_t launch_step_tc2_bf16(const StepMMA2 &s, cudaStream_t st);
// Two consecutive TF32 steps on the tcgen05 tensor cores (step_tc2f.cu,
// kind::tf32): FP32 planar buffers holding TF32-rounded values.  Cores as
// TF32 matrices: A1 = M_k as [128][K1] (K1 = 2 r_k rounded up to 8; rows
// 2b + i, columns 2a + j; rows past 2 r_{k+1} zero), A2 = M_{k+1} as
// [80][2 r'] (r' = r_{k+1} rounded up to 4; rows 2c + i, columns j r' + b;
// rows past 2 r_{k+2} zero).  cudaErrorNotSupported (nothing launched) when
// the shapes do not fit.
struct StepTF2 {
  const float *in;           // y_k, planar [rhs][a][position]
  int64_t in_rhs_stride;
  float *out;                // y_{k+2}
  int64_t out_rhs_stride;
  const float *A1;           // M_k as [128][K1], columns 2a + j
  const float *A2;           // M_{k+1} as [80][2 r'], columns j r' + b
  int k, r0, r1, r2;
  int64_t N, nrhs;
};
bool tc2f_steps_eligible(int k, int r0, int r1, int r2, int64_t N);
cudaError_t launch_step_tc2_tf32(const StepTF2 &s, cudaStream_t st);
cudaError_t tcf_status_take(int *status);

// Device status word of the tcgen05 kernels (QTT_ERR_TIMEOUT after a bounded
// wait gave up); returns it and clears it.
cudaError_t tc_status_take(int *status);
// Launch a kernel whose bounded wait runs out after about `seconds` (the
// failure path of the tcgen05 kernels, exercised without a GPU fault).
cudaError_t wait_selftest(double seconds, cudaStream_t st);

}  // namespace qtt
