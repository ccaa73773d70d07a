// Reduced-precision core step (FP32 pipe) -- see step_lp.cu.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/qtt.h"

namespace qtt {

enum LpMode { LP_F32 = 0, LP_TF32 = 1, LP_BF16 = 2 };

struct StepLP {
  const void *in;          // element type in_type
  int64_t in_rhs_stride;
  void *out;               // element type out_type
  int64_t out_rhs_stride;
  const void *M;           // packed core k: [a][j][rout_pad][i], float or bf16
  int k, rin, rout, rout_pad;
  int64_t N, nrhs;
  int mode;                // LpMode
  qtt_dtype in_type, out_type;
  // Epilogue (last step): out = s_v v + s_u u + s_acc acc; u, v of out_type
  // (either may be NULL; u may be out itself).
  int epi;
  const void *u;
  const void *v;
  int64_t u_rhs_stride;  // also the stride of v
  double s_acc, s_u, s_v;
  // TF32 mode: round the stored intermediate to TF32 (set for k < d-1), so
  // that later steps may use it without rounding again.
  int round_tf32_out;
};

// Rank padding of the packed reduced-precision cores (multiple of the
// per-thread rank tile).
int lp_rank_pad(int r);
cudaError_t launch_step_lp(const StepLP &s, cudaStream_t st);

// The first m = 2 or 3 steps in one launch (step_head.cu), when r_1 .. r_m
// are all <= kHeadMaxRank: reads x once, writes y_m.
constexpr int kHeadMaxRank = 8;
struct StepHead {
  const void *in;          // x, element type in_type, rhs stride in elements
  int64_t in_rhs_stride;
  void *out;               // y_m (intermediate type of the mode), planar
  int64_t out_rhs_stride;
  int r[4];                // ranks r_0 .. r_m
  int64_t N, nrhs;
  int m, mode;
  qtt_dtype in_type;
  // cores 0 .. m-1 by value (the kernel reads them as constant-bank operands):
  // G[k][2a + j][b][i], zero beyond the ranks, values of the mode's packed copy
  float G[3][2 * kHeadMaxRank][kHeadMaxRank][2];
};
// Steps the head kernel takes for this rank profile (0: none).
int head_steps(const int *ranks, int d);
cudaError_t launch_step_head(const StepHead &s, cudaStream_t st);

// The last m = 2 or 3 steps in one launch (step_head.cu), when r_{d-m} ..
// r_d are all <= kHeadMaxRank: reads y_{d-m} once and writes y (any output
// type, with the last step's epilogue).
struct StepTail {
  const void *in;          // y_{d-m}, the mode's intermediate type, planar
  int64_t in_rhs_stride;
  void *out;               // y, element type out_type, rhs stride (ld)
  int64_t out_rhs_stride;
  int r[4];                // ranks r_{d-m} .. r_d
  int64_t N, nrhs;
  int k0, m, mode;
  qtt_dtype out_type;
  // out = s_v v + s_u u + s_acc acc when epi (u, v of out_type, may be NULL)
  int epi;
  const void *u;
  const void *v;
  int64_t u_rhs_stride;
  double s_acc, s_u, s_v;
  float G[3][2 * kHeadMaxRank][kHeadMaxRank][2];  // cores d-m .. d-1, as for StepHead
};
// Steps the tail kernel takes (0: none), given the head's steps.
int tail_steps(const int *ranks, int d, int head);
cudaError_t launch_step_tail(const StepTail &s, cudaStream_t st);
// Reads and clears the staged tail kernel's timeout word (0: none).
cudaError_t tail_status_take(int *status);

// Staged (cp.async, persistent) FP32/TF32 step for intermediate-to-
// intermediate steps with k >= 2 -- see step_f32s.cu.
bool f32s_step_eligible(const StepLP &s);
cudaError_t launch_step_f32s(const StepLP &s, cudaStream_t st);

}  // namespace qtt
