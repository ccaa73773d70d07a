// QTT matrices with general mode sizes: core k is G_k(alpha_k, i_k, j_k,
// alpha_{k+1}) with a row mode i_k < m_k and a column mode j_k < n_k (the
// tensorisation of Sec. 3.1 with m_k x n_k modes), so the matrix is
// (prod m_k) x (prod n_k) -- rectangular when the products differ -- and
// y = A x (or y = A^T x) is the sweep of Algorithm 2 with mixed-radix
// positions.
//
// Index convention (first mode fastest, as for the binary operators): the
// column index is j = sum_k j_k prod_{l<k} n_l and the row index i = sum_k
// i_k prod_{l<k} m_l.  Before step k the intermediate holds, per right-hand
// side and per rank alpha_k, the positions t = low + L (j_k + n_k high) with
// low < L = prod_{l<k} m_l (row modes already produced) and high < H =
// prod_{l>k} n_l (column modes still to contract); step k replaces the
// column mode j_k by the row mode i_k:
//   out[b][low + L (i + m_k high)] = sum_{a, j} G_k(a, i, j, b) in[a][low + L (j + n_k high)].
// A transposed apply runs the same sweep with the roles of i and j (and of
// m and n) exchanged, from a second packed copy of the cores.
//
// The step is FP64-pipe-bound for the ranks of interest (r_in n FMAs per
// output against one load), so it is shaped like the binary FP64 step: each
// warp owns one output rank b (the core values are warp-wide broadcast
// loads), each lane owns TN columns (low, high) and keeps m accumulators per
// column, 32 lanes take 32 consecutive columns (consecutive positions once
// L >= 32).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "qtt_internal.h"

// A general-mode QTT matrix resident on the device.
struct qtt_gop {
  int d = 0;
  int device = 0;
  std::vector<int> ranks, m, n;
  std::vector<int64_t> off;  // element offset of core k in the packed copies
  int64_t rows = 1, cols = 1;
  double flops_per_rhs = 0.0;
  // packed [b][a][j][i] (forward: input mode j, output mode i) and
  // [b][a][i][j] (transposed)
  double *fwd = nullptr, *tr = nullptr;
  std::mutex use_mu;
  std::vector<std::pair<cudaStream_t, cudaEvent_t>> uses;
};

namespace qtt {
namespace {

constexpr int kWarps = 8;     // output ranks per CTA (one per warp)
constexpr int kMaxMode = 16;  // largest m_k, n_k

struct GStep {
  const double *in;
  double *out;
  const double *M;  // packed core: [b][a][jin][iout]
  int64_t in_rhs_stride, out_rhs_stride;
  int64_t L, H;     // produced-mode and pending-mode extents
  int rin, rout, nin, mout;
};

// MOUT = compile-time bound on the output mode size (accumulators per
// column); TN columns per lane.
template <int MOUT, int TN>
__global__ void __launch_bounds__(32 * kWarps) gstep_kernel(GStep s) {
  const int nrb = (s.rout + kWarps - 1) / kWarps;
  const int b = (int)(blockIdx.x % nrb) * kWarps + threadIdx.y;
  if (b >= s.rout) return;
  const int64_t ncol = s.L * s.H;
  const int64_t c0 = (int64_t)(blockIdx.x / nrb) * (32 * TN) + threadIdx.x;
  const double *in = s.in + (int64_t)blockIdx.z * s.in_rhs_stride;
  double *out = s.out + (int64_t)blockIdx.z * s.out_rhs_stride;
  int64_t pin[TN], pout[TN];
  bool ok[TN];
#pragma unroll
  for (int t = 0; t < TN; ++t) {
    const int64_t c = c0 + 32 * t;
    ok[t] = c < ncol;
    const int64_t high = ok[t] ? c / s.L : 0, low = ok[t] ? c - high * s.L : 0;
    pin[t] = low + s.L * s.nin * high;
    pout[t] = low + s.L * s.mout * high;
  }
  double acc[TN][MOUT];
#pragma unroll
  for (int t = 0; t < TN; ++t)
#pragma unroll
    for (int i = 0; i < MOUT; ++i) acc[t][i] = 0.0;
  const int64_t plane = s.L * s.nin * s.H;  // input positions per rank
  const double *Mb = s.M + (int64_t)b * s.rin * s.nin * s.mout;
  for (int a = 0; a < s.rin; ++a) {
    const double *ina = in + (int64_t)a * plane;
    for (int j = 0; j < s.nin; ++j) {
      double v[TN];
#pragma unroll
      for (int t = 0; t < TN; ++t) v[t] = ok[t] ? __ldg(ina + pin[t] + s.L * j) : 0.0;
      const double *g = Mb + ((int64_t)a * s.nin + j) * s.mout;
#pragma unroll
      for (int i = 0; i < MOUT; ++i) {
        if (i < s.mout) {
          const double gi = __ldg(g + i);
#pragma unroll
          for (int t = 0; t < TN; ++t) acc[t][i] = fma(gi, v[t], acc[t][i]);
        }
      }
    }
  }
  const int64_t oplane = s.L * s.mout * s.H;
  double *ob = out + (int64_t)b * oplane;
#pragma unroll
  for (int t = 0; t < TN; ++t) {
    if (!ok[t]) continue;
#pragma unroll
    for (int i = 0; i < MOUT; ++i)
      if (i < s.mout) ob[pout[t] + s.L * i] = acc[t][i];
  }
}

template <int MOUT, int TN>
cudaError_t launch_g(const GStep &s, int64_t nrhs, cudaStream_t st) {
  const int64_t ncol = s.L * s.H;
  const int64_t gx = (ncol + 32 * TN - 1) / (32 * TN) * ((s.rout + kWarps - 1) / kWarps);
  if (gx > 0x7fffffffLL) return cudaErrorInvalidValue;
  for (int64_t r0 = 0; r0 < nrhs; r0 += 65535) {
    GStep t = s;
    t.in += r0 * s.in_rhs_stride;
    t.out += r0 * s.out_rhs_stride;
    const int64_t nr = std::min<int64_t>(65535, nrhs - r0);
    gstep_kernel<MOUT, TN><<<dim3((unsigned)gx, 1, (unsigned)nr), dim3(32, kWarps), 0, st>>>(t);
    count_launches(1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_gstep(const GStep &s, int64_t nrhs, cudaStream_t st) {
  // 8 accumulators per lane: TN columns x MOUT output modes
  if (s.mout <= 2) return launch_g<2, 4>(s, nrhs, st);
  if (s.mout <= 4) return launch_g<4, 2>(s, nrhs, st);
  if (s.mout <= 8) return launch_g<8, 1>(s, nrhs, st);
  return launch_g<16, 1>(s, nrhs, st);
}

void gnote_use(const qtt_gop *A, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return;
  }
  qtt_gop *G = const_cast<qtt_gop *>(A);
  std::lock_guard<std::mutex> lk(G->use_mu);
  cudaEvent_t ev = nullptr;
  for (auto &u : G->uses)
    if (u.first == st) ev = u.second;
  if (!ev) {
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    G->uses.emplace_back(st, ev);
  }
  cudaEventRecord(ev, st);
}

}  // namespace
}  // namespace qtt

using namespace qtt;

extern "C" {

qtt_status qtt_gcreate(qtt_gop **out, int d, const int *ranks, const int *m, const int *n,
                       const double *cores, void *stream) {
  if (!out) return fail(QTT_ERR_INVALID_ARG, "qtt_gcreate: out is NULL");
  *out = nullptr;
  if (d < 1 || d > 60) return fail(QTT_ERR_INVALID_ARG, "qtt_gcreate: d must be in [1, 60]");
  if (!ranks || !m || !n || !cores)
    return fail(QTT_ERR_INVALID_ARG, "qtt_gcreate: NULL ranks, modes or cores");
  if (ranks[0] != 1 || ranks[d] != 1)
    return fail(QTT_ERR_INVALID_ARG, "qtt_gcreate: ranks[0] and ranks[d] must be 1");
  double rows = 1.0, cols = 1.0;
  for (int k = 0; k <= d; ++k)
    if (ranks[k] < 1 || ranks[k] > 4096)
      return fail(QTT_ERR_INVALID_ARG, "qtt_gcreate: ranks must be in [1, 4096]");
  for (int k = 0; k < d; ++k) {
    if (m[k] < 1 || m[k] > kMaxMode || n[k] < 1 || n[k] > kMaxMode)
      return fail(QTT_ERR_INVALID_ARG, "qtt_gcreate: mode sizes must be in [1, 16]");
    rows *= m[k];
    cols *= n[k];
  }
  if (rows > 4.0e12 || cols > 4.0e12)
    return fail(QTT_ERR_INVALID_ARG, "qtt_gcreate: matrix dimensions above 4e12");
  qtt_gop *A = new (std::nothrow) qtt_gop();
  if (!A) return fail(QTT_ERR_OOM, "qtt_gcreate: host allocation failed");
  A->d = d;
  cudaGetDevice(&A->device);
  A->ranks.assign(ranks, ranks + d + 1);
  A->m.assign(m, m + d);
  A->n.assign(n, n + d);
  A->rows = (int64_t)rows;
  A->cols = (int64_t)cols;
  A->off.assign(d + 1, 0);
  for (int k = 0; k < d; ++k)
    A->off[k + 1] = A->off[k] + (int64_t)ranks[k] * m[k] * n[k] * ranks[k + 1];
  // flops of y = A x per right-hand side: step k has L H columns, each
  // 2 r_k m_k n_k r_{k+1} flops (Sec. 4.2's 2 m_k n_k r_k r_{k+1} per column)
  {
    double f = 0.0;
    for (int k = 0; k < d; ++k) {
      double L = 1.0, H = 1.0;
      for (int l = 0; l < k; ++l) L *= m[l];
      for (int l = k + 1; l < d; ++l) H *= n[l];
      f += 2.0 * ranks[k] * (double)m[k] * n[k] * ranks[k + 1] * L * H;
    }
    A->flops_per_rhs = f;
  }
  const int64_t total = A->off[d];
  std::vector<double> pf((size_t)total), pt((size_t)total);
  for (int k = 0; k < d; ++k) {
    const int ra = ranks[k], rb = ranks[k + 1], mk = m[k], nk = n[k];
    const double *G = cores + A->off[k];
    double *F = pf.data() + A->off[k], *T = pt.data() + A->off[k];
    for (int a = 0; a < ra; ++a)
      for (int i = 0; i < mk; ++i)
        for (int j = 0; j < nk; ++j)
          for (int b = 0; b < rb; ++b) {
            const double g = G[(((size_t)a * mk + i) * nk + j) * rb + b];
            F[(((size_t)b * ra + a) * nk + j) * mk + i] = g;
            T[(((size_t)b * ra + a) * mk + i) * nk + j] = g;
          }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)total * sizeof(double);
  qtt_status s = persistent_alloc(reinterpret_cast<void **>(&A->fwd), bytes, st);
  if (s == QTT_OK) s = persistent_alloc(reinterpret_cast<void **>(&A->tr), bytes, st);
  if (s == QTT_OK) {
    cudaError_t e = cudaMemcpyAsync(A->fwd, pf.data(), bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(A->tr, pt.data(), bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_fail(e, "qtt_gcreate: upload");
  }
  if (s != QTT_OK) {
    release_after({A->fwd, A->tr}, {});
    delete A;
    return s;
  }
  *out = A;
  return QTT_OK;
}

qtt_status qtt_gdestroy(qtt_gop *A) {
  if (!A) return QTT_OK;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != A->device) cudaSetDevice(A->device);
  std::vector<cudaEvent_t> evs;
  {
    std::lock_guard<std::mutex> lk(A->use_mu);
    for (auto &u : A->uses) evs.push_back(u.second);
    A->uses.clear();
  }
  release_after({A->fwd, A->tr}, evs);
  for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
  if (cur >= 0 && cur != A->device) cudaSetDevice(cur);
  delete A;
  return QTT_OK;
}

int64_t qtt_gop_rows(const qtt_gop *A) { return A ? A->rows : -1; }
int64_t qtt_gop_cols(const qtt_gop *A) { return A ? A->cols : -1; }
double qtt_gop_flops(const qtt_gop *A, int transpose) {
  if (!A) return 0.0;
  if (!transpose) return A->flops_per_rhs;
  double f = 0.0;
  for (int k = 0; k < A->d; ++k) {
    double L = 1.0, H = 1.0;
    for (int l = 0; l < k; ++l) L *= A->n[l];
    for (int l = k + 1; l < A->d; ++l) H *= A->m[l];
    f += 2.0 * A->ranks[k] * (double)A->m[k] * A->n[k] * A->ranks[k + 1] * L * H;
  }
  return f;
}

qtt_status qtt_gapply(const qtt_gop *A, const double *x, double *y, int64_t nrhs, int64_t ldx,
                      int64_t ldy, int transpose, void *stream) {
  if (!A) return fail(QTT_ERR_INVALID_ARG, "qtt_gapply: NULL operator");
  {
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != A->device)
      return fail(QTT_ERR_INVALID_ARG, "qtt_gapply: the operator lives on another device");
  }
  if (transpose != 0 && transpose != 1)
    return fail(QTT_ERR_INVALID_ARG, "qtt_gapply: transpose must be 0 or 1");
  const int d = A->d;
  const std::vector<int> &mo = transpose ? A->n : A->m;  // output modes
  const std::vector<int> &mi = transpose ? A->m : A->n;  // input modes
  const int64_t nin = transpose ? A->rows : A->cols, nout = transpose ? A->cols : A->rows;
  if (nrhs < 0) return fail(QTT_ERR_INVALID_ARG, "qtt_gapply: nrhs < 0");
  if (nrhs == 0) return QTT_OK;
  if (ldx < nin || ldy < nout)
    return fail(QTT_ERR_INVALID_ARG, "qtt_gapply: ldx < input length or ldy < output length");
  if (!x || !y) return fail(QTT_ERR_INVALID_ARG, "qtt_gapply: NULL vector");
  {
    const char *xb = reinterpret_cast<const char *>(x), *yb = reinterpret_cast<const char *>(y);
    const size_t sx = ((size_t)(nrhs - 1) * (size_t)ldx + (size_t)nin) * sizeof(double);
    const size_t sy = ((size_t)(nrhs - 1) * (size_t)ldy + (size_t)nout) * sizeof(double);
    if (xb < yb + sy && yb < xb + sx)
      return fail(QTT_ERR_INVALID_ARG, "qtt_gapply: x and y overlap");
  }
  // intermediate after step k (k < d-1): r_{k+1} prod_{l<=k} mo_l prod_{l>k} mi_l
  int64_t per_rhs_half = 0;
  {
    double L = 1.0;
    for (int k = 0; k + 1 < d; ++k) {
      L *= mo[k];
      double H = 1.0;
      for (int l = k + 1; l < d; ++l) H *= mi[l];
      per_rhs_half = std::max<int64_t>(per_rhs_half, (int64_t)(A->ranks[k + 1] * L * H));
    }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t per_rhs = (size_t)2 * (size_t)per_rhs_half * sizeof(double);
  int64_t chunk = nrhs;
  if (per_rhs) {
    const int64_t fit = (int64_t)(scratch_available_at_least(per_rhs * (size_t)nrhs) / per_rhs);
    if (fit < 1)
      return fail(QTT_ERR_OOM, "qtt_gapply: scratch for one right-hand side does not fit");
    chunk = std::min<int64_t>(nrhs, fit);
  }
  void *scratch = nullptr;
  qtt_status s = scratch_alloc(&scratch, per_rhs * (size_t)chunk, st);
  if (s != QTT_OK) return s;
  double *buf[2] = {static_cast<double *>(scratch),
                    scratch ? static_cast<double *>(scratch) + (size_t)per_rhs_half * chunk
                            : nullptr};
  const double *cores = transpose ? A->tr : A->fwd;
  for (int64_t c0 = 0; c0 < nrhs && s == QTT_OK; c0 += chunk) {
    const int64_t nc = std::min<int64_t>(chunk, nrhs - c0);
    int64_t L = 1;
    for (int k = 0; k < d; ++k) {
      int64_t H = 1;
      for (int l = k + 1; l < d; ++l) H *= mi[l];
      GStep g;
      g.rin = A->ranks[k];
      g.rout = A->ranks[k + 1];
      g.nin = mi[k];
      g.mout = mo[k];
      g.L = L;
      g.H = H;
      g.M = cores + A->off[k];
      if (k == 0) {
        g.in = x + c0 * ldx;
        g.in_rhs_stride = ldx;
      } else {
        g.in = buf[(k - 1) & 1];
        g.in_rhs_stride = (int64_t)g.rin * L * g.nin * H;
      }
      if (k == d - 1) {
        g.out = y + c0 * ldy;
        g.out_rhs_stride = ldy;
      } else {
        g.out = buf[k & 1];
        g.out_rhs_stride = (int64_t)g.rout * L * g.mout * H;
      }
      const cudaError_t e = launch_gstep(g, nc, st);
      if (e != cudaSuccess) {
        s = cuda_fail(e, "qtt_gapply: step launch");
        break;
      }
      L *= mo[k];
    }
  }
  scratch_free(scratch, st);
  gnote_use(A, st);
  return s;
}

}  // extern "C"
