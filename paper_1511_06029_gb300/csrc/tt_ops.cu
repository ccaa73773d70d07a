// Exact QTT arithmetic on the device: the product of two QTT matrices and
// the weighted sum of QTT tensors, the building blocks of preconditioners
// such as round(I - K + K^2) and of the product preconditioners of Sec. 4.2.
//   qtt_op_product  C = A B core by core (Sec. 4.2's compressed product with
//                   a matrix on the right): rank pairs (a, b) merge into
//                   a s + b and the inner mode is summed,
//                     C_k[a s + b][i][p][a' s' + b'] =
//                         sum_j A_k[a][i][j][a'] B_k[b][j][p][b'],
//                   each entry evaluated as fl(fl(A_0 B_0) + fl(A_1 B_1));
//   qtt_tt_sum      sum_t c_t T_t by concatenating the ranks (Sec. 3.3): the
//                   first cores side by side, the middle ones block-diagonal,
//                   the last ones stacked and scaled by c_t.
// Both write every output entry once (memory-bound, no rounding beyond the
// stated products and sums), with the sizes checked before any launch.
#include <algorithm>
#include <vector>

#include "qtt_internal.h"

namespace qtt {
namespace {

constexpr int kT = 256;

unsigned grid_for(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + kT - 1) / kT, 152 * 32));
}

// One core of C = A B.  mA, mB: the operators' FP64 cores as packed by
// qtt_create, [a'][a][j][i] (element G(a, i, j, a')).
__global__ void __launch_bounds__(kT) product_core_kernel(const double *__restrict__ mA,
                                                          const double *__restrict__ mB, int ra,
                                                          int ra2, int rb, int rb2,
                                                          double *__restrict__ C) {
  const int64_t R2 = (int64_t)ra2 * rb2;
  const int64_t total = (int64_t)ra * rb * 4 * R2;
  for (int64_t e = (int64_t)blockIdx.x * kT + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * kT) {
    const int64_t col = e % R2;
    const int64_t rest = e / R2;  // ((a rb + b) 2 + i) 2 + p
    const int p = (int)(rest & 1), i = (int)((rest >> 1) & 1);
    const int64_t row = rest >> 2;
    const int a = (int)(row / rb), b = (int)(row % rb);
    const int a2 = (int)(col / rb2), b2 = (int)(col % rb2);
    const double *ga = mA + (((int64_t)a2 * ra + a) * 2) * 2 + i;  // + 2 j
    const double *gb = mB + (((int64_t)b2 * rb + b) * 2 + p) * 2;  // + j
    C[e] = __dadd_rn(__dmul_rn(__ldg(ga), __ldg(gb)), __dmul_rn(__ldg(ga + 2), __ldg(gb + 1)));
  }
}

// out[(r0 + a)][m][(c0 + b)] += s in[a][m][b] for one block of a sum's core.
__global__ void __launch_bounds__(kT) place_kernel(const double *__restrict__ in, int ra, int n,
                                                   int rb, double s, double *__restrict__ out,
                                                   int64_t r0, int64_t c0, int64_t RB) {
  const int64_t total = (int64_t)ra * n * rb;
  for (int64_t e = (int64_t)blockIdx.x * kT + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * kT) {
    const int64_t b = e % rb, am = e / rb;
    const int64_t m = am % n, a = am / n;
    double *o = out + ((r0 + a) * n + m) * RB + (c0 + b);
    *o = *o + (s == 1.0 ? in[e] : s * in[e]);
  }
}

}  // namespace
}  // namespace qtt

using namespace qtt;

extern "C" qtt_status qtt_op_product(const qtt_op *A, const qtt_op *B, double *c_cores,
                                     int64_t capacity, int *c_ranks, void *stream) {
  if (!A || !B || !c_cores || !c_ranks)
    return fail(QTT_ERR_INVALID_ARG, "qtt_op_product: NULL argument");
  if (A->d != B->d) return fail(QTT_ERR_INVALID_ARG, "qtt_op_product: operators differ in d");
  if (qtt_status ds = check_device(A, "qtt_op_product")) return ds;
  if (qtt_status ds = check_device(B, "qtt_op_product")) return ds;
  const int d = A->d;
  std::vector<int64_t> off(d + 1, 0);
  for (int k = 0; k <= d; ++k) {
    const int64_t r = (int64_t)A->ranks[k] * B->ranks[k];
    if (r > 32768)
      return fail(QTT_ERR_INVALID_ARG, "qtt_op_product: a product rank exceeds 32768");
    c_ranks[k] = (int)r;
  }
  for (int k = 0; k < d; ++k) off[k + 1] = off[k] + 4 * (int64_t)c_ranks[k] * c_ranks[k + 1];
  if (capacity < off[d])
    return fail(QTT_ERR_INVALID_ARG, "qtt_op_product: c_cores holds " + std::to_string(capacity) +
                                         " doubles, the product needs " + std::to_string(off[d]));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int k = 0; k < d; ++k) {
    const int64_t total = off[k + 1] - off[k];
    product_core_kernel<<<grid_for(total), kT, 0, st>>>(A->m64 + A->off[k], B->m64 + B->off[k],
                                                        A->ranks[k], A->ranks[k + 1], B->ranks[k],
                                                        B->ranks[k + 1], c_cores + off[k]);
    count_launches(1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      note_use(A, st);
      note_use(B, st);
      return cuda_fail(e, "qtt_op_product: launch");
    }
  }
  note_use(A, st);
  note_use(B, st);
  return QTT_OK;
}

extern "C" qtt_status qtt_tt_sum(int d, int n, int nterms, const int *const *ranks,
                                 const double *const *cores, const double *coefs,
                                 int *ranks_out, double *cores_out, int64_t capacity,
                                 void *stream) {
  if (d < 1 || d > 64 || n < 1 || n > 256 || nterms < 1 || !ranks || !cores || !coefs ||
      !ranks_out || !cores_out)
    return fail(QTT_ERR_INVALID_ARG, "qtt_tt_sum: bad sizes or NULL argument");
  std::vector<int64_t> R(d + 1, 0);
  R[0] = R[d] = 1;
  for (int t = 0; t < nterms; ++t) {
    if (!ranks[t] || !cores[t]) return fail(QTT_ERR_INVALID_ARG, "qtt_tt_sum: NULL term");
    if (ranks[t][0] != 1 || ranks[t][d] != 1)
      return fail(QTT_ERR_INVALID_ARG, "qtt_tt_sum: every term needs ranks[0] = ranks[d] = 1");
    for (int k = 1; k < d; ++k) {
      if (ranks[t][k] < 1) return fail(QTT_ERR_INVALID_ARG, "qtt_tt_sum: ranks must be >= 1");
      R[k] += ranks[t][k];
    }
  }
  for (int k = 0; k <= d; ++k)
    if (R[k] > 32768) return fail(QTT_ERR_INVALID_ARG, "qtt_tt_sum: a summed rank exceeds 32768");
  std::vector<int64_t> off(d + 1, 0);
  for (int k = 0; k < d; ++k) off[k + 1] = off[k] + R[k] * n * R[k + 1];
  if (capacity < off[d])
    return fail(QTT_ERR_INVALID_ARG, "qtt_tt_sum: cores_out holds " + std::to_string(capacity) +
                                         " doubles, the sum needs " + std::to_string(off[d]));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(cores_out, 0, (size_t)off[d] * sizeof(double), st);
  if (e != cudaSuccess) return cuda_fail(e, "qtt_tt_sum: clear");
  std::vector<int64_t> toff(nterms, 0);  // element offset of core k in term t
  std::vector<int64_t> r0(nterms, 0), c0(nterms, 0);
  for (int k = 0; k < d; ++k) {
    int64_t rowpos = 0, colpos = 0;
    for (int t = 0; t < nterms; ++t) {
      const int ra = ranks[t][k], rb = ranks[t][k + 1];
      const int64_t rs = k > 0 ? rowpos : 0, cs = k < d - 1 ? colpos : 0;
      const double s = k == d - 1 ? coefs[t] : 1.0;
      place_kernel<<<grid_for((int64_t)ra * n * rb), kT, 0, st>>>(
          cores[t] + toff[t], ra, n, rb, s, cores_out + off[k], rs, cs, R[k + 1]);
      count_launches(1);
      e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(e, "qtt_tt_sum: launch");
      toff[t] += (int64_t)ra * n * rb;
      rowpos += ra;
      colpos += rb;
    }
  }
  for (int k = 0; k <= d; ++k) ranks_out[k] = (int)R[k];
  return QTT_OK;
}
