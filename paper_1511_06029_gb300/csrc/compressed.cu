// qtt_apply_tt: the compressed matrix-vector product c = A b of Sec. 4.2,
// for a right-hand side b that is itself a QTT vector.
//
// Core k of c merges the rank pairs (alpha, beta) of A and b into one index
// alpha s_k + beta and sums over the column bit:
//   C_k[alpha s + beta][i][alpha' s' + beta'] =
//       sum_j A_k[alpha][i][j][alpha'] b_k[beta][j][beta'],
// so c's ranks are the products r_k s_k (no rounding here).  Every output
// entry is two products and one addition, written once: the kernel streams
// the output (sum_k 2 r_k s_k r_{k+1} s_{k+1} doubles) and reads the small
// cores of A and b through L1/L2.  Each entry is the separately rounded
// fl(fl(a_0 b_0) + fl(a_1 b_1)) (no fused multiply-add), the evaluation of
// the definition written out.
#include <vector>

#include "qtt_internal.h"

namespace qtt {
namespace {

constexpr int kThreads = 256;

// One core of c.  M: A's FP64 core as packed at qtt_create, [a'][a][j][i];
// B: b's core [beta][j][beta']; C: c's core [a s + beta][i][a' s' + beta'].
// Block row blockIdx.y = (a s + beta) 2 + i (one output row, its A and b
// slices fixed); threads stride over the row's rb s' columns, so each entry
// costs one 32-bit division (col -> a', beta') and one coalesced store.
__global__ void __launch_bounds__(kThreads) compressed_core_kernel(
    const double *__restrict__ M, const double *__restrict__ B, double *__restrict__ C, int ra,
    int rb, int s, int s2) {
  const unsigned row2 = blockIdx.y;  // (a s + beta) 2 + i
  const int i = (int)(row2 & 1u);
  const unsigned row = row2 >> 1;
  const int a = (int)(row / (unsigned)s), beta = (int)(row % (unsigned)s);
  const unsigned cols = (unsigned)rb * (unsigned)s2;
  const double *mrow = M + (int64_t)a * 4 + i;                  // + a' ra 4; j at +2
  const double *brow = B + (int64_t)beta * 2 * s2;              // + beta'; j at +s2
  double *crow = C + (int64_t)row2 * cols;
  const int64_t mstride = (int64_t)ra * 4;
  for (unsigned col = blockIdx.x * kThreads + threadIdx.x; col < cols;
       col += gridDim.x * kThreads) {
    const unsigned a2 = col / (unsigned)s2, beta2 = col - a2 * (unsigned)s2;
    const double *m = mrow + a2 * mstride;
    const double *bb = brow + beta2;
    crow[col] = __dadd_rn(__dmul_rn(__ldg(m), __ldg(bb)), __dmul_rn(__ldg(m + 2), __ldg(bb + s2)));
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
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (int k = 0; k < A->d; ++k) {
    const int64_t rows2 = (int64_t)A->ranks[k] * b_ranks[k] * 2;       // <= 65534
    const int64_t cols = (int64_t)A->ranks[k + 1] * b_ranks[k + 1];     // <= 2^20
    // enough blocks per row that the grid covers every SM several times
    int64_t bx = (cols + kThreads - 1) / kThreads;
    const int64_t want = ((int64_t)sms * 8 + rows2 - 1) / rows2;
    if (bx > want) bx = want < 1 ? 1 : want;
    const dim3 grid((unsigned)bx, (unsigned)rows2);
    compressed_core_kernel<<<grid, kThreads, 0, st>>>(A->m64 + A->off[k], b_cores + boff[k],
                                                      c_cores + coff[k], A->ranks[k],
                                                      A->ranks[k + 1], b_ranks[k],
                                                      b_ranks[k + 1]);
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
