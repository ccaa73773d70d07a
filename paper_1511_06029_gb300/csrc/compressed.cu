// qtt_apply_tt: the compressed matrix-vector product c = A b of Sec. 4.2,
// for a right-hand side b that is itself a QTT vector.
//
// Core k of c merges the rank pairs (alpha, beta) of A and b into one index
// alpha s_k + beta and sums over the column bit:
//   C_k[alpha s + beta][i][alpha' s' + beta'] =
//       sum_j A_k[alpha][i][j][alpha'] b_k[beta][j][beta'],
// so c's ranks are the products r_k s_k (no rounding here).  Every output
// entry is two products and one addition, written once (sum_k 2 r_k s_k
// r_{k+1} s_{k+1} doubles); the small cores of A and b are read once per row
// into shared memory.  Each entry is fma(a_1, b_1, fl(a_0 b_0)): within
// u (|a_0 b_0| + |a_0 b_0 + a_1 b_1|) of the exact sum.
#include <vector>

#include "qtt_internal.h"

namespace qtt {
namespace {

constexpr int kThreads = 256;

// One core of c, one output row per CTA.  M: A's FP64 core as packed at
// qtt_create, [a'][a][j][i]; B: b's core [beta][j][beta']; C: c's core
// [a s + beta][i][a' s' + beta'].  Row blockIdx.x = (a s + beta) 2 + i fixes
// A's slice (a, i) and b's slice beta: the CTA stages A(a, i, j, a') for both
// j and b(beta, j, beta') for both j in shared memory, then its threads walk
// the row's r' s' columns -- column = a' s' + beta', the pair (a', beta')
// advanced by counters, no division per entry -- and each writes
// fma(A_1, b_1, fl(A_0 b_0)).  On GB300 the FP64 pipe issues two
// instructions per clock per SM, so an entry's two FP64 instructions (a
// multiply and a fused multiply-add) for its 8 stored bytes -- not the
// store itself -- set the limit: 152 x 2 x 2.07e9 / 2 = 3.1e11 entries/s,
// 2.5 TB/s of output.
__global__ void __launch_bounds__(kThreads) compressed_core_kernel(
    const double *__restrict__ M, const double *__restrict__ B, double *__restrict__ C, int ra,
    int rb, int s, int s2) {
  extern __shared__ double sm[];
  double *sa = sm;            // [a'][j]: 2 rb
  double *sb = sm + 2 * rb;   // [j][beta']: 2 s2
  const unsigned row2 = blockIdx.x;  // (a s + beta) 2 + i
  const int i = (int)(row2 & 1u);
  const unsigned row = row2 >> 1;
  const int a = (int)(row / (unsigned)s), beta = (int)(row % (unsigned)s);
  for (int t = threadIdx.x; t < rb; t += kThreads) {
    const double *m = M + ((int64_t)t * ra + a) * 4 + i;  // (a' = t, a, j = 0, i)
    sa[2 * t] = __ldg(m);
    sa[2 * t + 1] = __ldg(m + 2);
  }
  for (int t = threadIdx.x; t < 2 * s2; t += kThreads) sb[t] = __ldg(B + (int64_t)beta * 2 * s2 + t);
  __syncthreads();
  const unsigned cols = (unsigned)rb * (unsigned)s2;
  double *crow = C + (int64_t)row2 * cols;
  unsigned a2 = threadIdx.x / (unsigned)s2, b2 = threadIdx.x % (unsigned)s2;
  const unsigned da = kThreads / (unsigned)s2, db = kThreads % (unsigned)s2;
  for (unsigned col = threadIdx.x; col < cols; col += kThreads) {
    crow[col] = fma(sa[2 * a2 + 1], sb[s2 + b2], __dmul_rn(sa[2 * a2], sb[b2]));
    a2 += da;
    b2 += db;
    if (b2 >= (unsigned)s2) {
      b2 -= (unsigned)s2;
      ++a2;
    }
  }
}

bool sizes(const qtt_op *A, const int *b_ranks, std::vector<int64_t> *boff,
           std::vector<int64_t> *coff) {
  const int d = A->d;
  if (b_ranks[0] != 1 || b_ranks[d] != 1) return false;
  boff->assign(d + 1, 0);
  coff->assign(d + 1, 0);
  for (int k = 0; k < d; ++k) {
    const int64_t s = b_ranks[k], s2 = b_ranks[k + 1];
    if (s < 1 || s2 < 1 || s > 4096 || s2 > 4096) return false;
    const int64_t rows = (int64_t)A->ranks[k] * s, cols = (int64_t)A->ranks[k + 1] * s2;
    // rows: 2 r_k s_k blocks of the grid's y dimension (<= 65535); cols: one
    // 32-bit column index
    if (rows > 32767 || cols > (1 << 20)) return false;
    (*boff)[k + 1] = (*boff)[k] + 2 * s * s2;
    (*coff)[k + 1] = (*coff)[k] + 2 * rows * cols;
    if ((*coff)[k + 1] > ((int64_t)1 << 40)) return false;
  }
  return true;
}

}  // namespace
}  // namespace qtt

using namespace qtt;

extern "C" qtt_status qtt_apply_tt_size(const qtt_op *A, const int *b_ranks, int64_t *n_elems) {
  if (!A || !b_ranks || !n_elems) return fail(QTT_ERR_INVALID_ARG, "qtt_apply_tt_size: NULL argument");
  std::vector<int64_t> boff, coff;
  if (!sizes(A, b_ranks, &boff, &coff))
    return fail(QTT_ERR_INVALID_ARG,
                "qtt_apply_tt_size: vector ranks must start and end with 1, lie in [1, 4096], "
                "and keep every product rank r_k s_k <= 32767");
  *n_elems = coff[A->d];
  return QTT_OK;
}

extern "C" qtt_status qtt_apply_tt(const qtt_op *A, const int *b_ranks, const double *b_cores,
                                   double *c_cores, void *stream) {
  if (!A || !b_ranks || !b_cores || !c_cores)
    return fail(QTT_ERR_INVALID_ARG, "qtt_apply_tt: NULL argument");
  if (qtt_status ds = check_device(A, "qtt_apply_tt")) return ds;
  std::vector<int64_t> boff, coff;
  if (!sizes(A, b_ranks, &boff, &coff))
    return fail(QTT_ERR_INVALID_ARG,
                "qtt_apply_tt: vector ranks must start and end with 1, lie in [1, 4096], "
                "and keep every product rank r_k s_k <= 32767");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // shared memory of the largest core: 2 (r' + s') doubles (<= 128 KB)
  static const cudaError_t attr = cudaFuncSetAttribute(
      compressed_core_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * (4096 + 4096) * 8);
  if (attr != cudaSuccess) return cuda_fail(attr, "qtt_apply_tt: shared memory attribute");
  for (int k = 0; k < A->d; ++k) {
    const int64_t rows2 = (int64_t)A->ranks[k] * b_ranks[k] * 2;  // <= 65534
    const size_t smem = (size_t)2 * (A->ranks[k + 1] + b_ranks[k + 1]) * sizeof(double);
    compressed_core_kernel<<<(unsigned)rows2, kThreads, smem, st>>>(
        A->m64 + A->off[k], b_cores + boff[k], c_cores + coff[k], A->ranks[k], A->ranks[k + 1],
        b_ranks[k], b_ranks[k + 1]);
    count_launches(1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      note_use(A, st);
      return cuda_fail(e, "qtt_apply_tt: launch");
    }
  }
  note_use(A, st);
  return QTT_OK;
}
