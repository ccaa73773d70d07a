// qtt_solve: direct solve by a QTT inverse, right-preconditioned GMRES(m) and
// mixed-precision iterative refinement for (a I + K) x = f, batched over
// right-hand sides.  Host control loop; every vector operation is a kernel.
//
//   DIRECT : x = P f                     (Tables 1-2, "Solve" column)
//   GMRES  : A P u = f, x = P u, x0 = 0  (Sec. 5.3: a QTT approximate inverse
//            as preconditioner inside GMRES; right preconditioning so the
//            true FP64 residual decides convergence), in the flexible form:
//            Z_j = P v_j is kept and x += Z y, which stays consistent when
//            P is applied in reduced precision (not exactly linear)
//   REFINE : x0 = P f; x <- x + P (f - A x)
// The residual f - A x is always the FP64 apply of K with the subtraction
// fused into its last step; P may be applied in FP64, FP32, TF32 or BF16.
//
// GMRES orthogonalises by classical Gram-Schmidt applied twice (CGS2): two
// rounds of (dots against the basis, one update) per Arnoldi step, with the
// deterministic reductions of krylov.cu; Givens rotations and the small
// triangular solve run on the host.  Right-hand sides advance in lockstep;
// each keeps its own Hessenberg matrix, rotations and residual estimate.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "krylov.h"
#include "qtt_internal.h"
#include "solve_internal.h"

namespace qtt {
namespace {

struct Scratch {
  cudaStream_t st;
  std::vector<void *> blocks;
  qtt_status get(double **p, size_t n) {
    void *q = nullptr;
    qtt_status s = scratch_alloc(&q, n * sizeof(double), st);
    if (s != QTT_OK) return s;
    blocks.push_back(q);
    *p = static_cast<double *>(q);
    return QTT_OK;
  }
  ~Scratch() {
    for (void *q : blocks) scratch_free(q, st);
  }
};

#define QTT_TRY(expr)                 \
  do {                                \
    qtt_status s_ = (expr);           \
    if (s_ != QTT_OK) return s_;      \
  } while (0)

#define QTT_CUDA_OK(expr, where)                     \
  do {                                               \
    cudaError_t e_ = (expr);                         \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

struct Ctx {
  const qtt_op *K, *P;
  double a;
  qtt_dtype pc;
  int64_t N, nrhs;
  cudaStream_t st;
};

// out = P in (FP64 in/out, arithmetic pc); accumulate: out += P in.
qtt_status apply_P(const Ctx &c, const double *in, int64_t ld_in, double *out, int64_t ld_out,
                   bool accumulate) {
  if (!c.P) {
    if (accumulate)
      QTT_CUDA_OK(vec_axpy(vecs(out, ld_out), vecs(in, ld_in), 1.0, c.N, c.nrhs, c.st), "axpy");
    else
      QTT_CUDA_OK(vec_copy(vecs(out, ld_out), vecs(in, ld_in), c.N, c.nrhs, c.st), "copy");
    return QTT_OK;
  }
  if (ld_in != ld_out) {
    // the apply takes one leading dimension: stage through a contiguous copy
    return fail(QTT_ERR_INVALID_ARG, "apply_P: leading dimensions differ");
  }
  if (c.pc == QTT_F64) {
    Epilogue e;
    if (accumulate) {
      e.on = true;
      e.u = out;
      e.s_u = 1.0;
      e.s_acc = 1.0;
    }
    return apply_f64(c.P, in, out, c.nrhs, ld_in, c.st, e);
  }
  LpEpilogue e;
  if (accumulate) {
    e.on = true;
    e.u = out;
    e.s_u = 1.0;
    e.s_acc = 1.0;
  }
  return apply_lp(c.P, c.pc, in, QTT_F64, out, QTT_F64, c.nrhs, ld_in, c.st, e);
}

// out = a z + K z (FP64)
qtt_status apply_A(const Ctx &c, const double *z, double *out, int64_t ld) {
  Epilogue e;
  e.on = true;
  e.u = z;
  e.s_u = c.a;
  e.s_acc = 1.0;
  return apply_f64(c.K, z, out, c.nrhs, ld, c.st, e);
}

// out = rhs + s_z z - K z with K in the low precision c.pc (FP64 vectors;
// FP64 K when c.pc is FP64).
qtt_status apply_K_lowp(const Ctx &c, const double *z, double *out, const double *rhs,
                        double s_z) {
  if (c.pc == QTT_F64) {
    Epilogue e;
    e.on = true;
    e.v = rhs;
    e.s_v = 1.0;
    e.u = z;
    e.s_u = s_z;
    e.s_acc = -1.0;
    return apply_f64(c.K, z, out, c.nrhs, c.N, c.st, e);
  }
  LpEpilogue e;
  e.on = true;
  e.v = rhs;
  e.s_v = 1.0;
  e.u = z;
  e.s_u = s_z;
  e.s_acc = -1.0;
  return apply_lp(c.K, c.pc, z, QTT_F64, out, QTT_F64, c.nrhs, c.N, c.st, e);
}

// z = M rhs, the correction operator: z0 = P rhs (P = I if absent), then
// `inner` Richardson steps z <- z + P (rhs - (a z + K z)) with K and P in the
// low precision c.pc and all vectors and updates in FP64.  tmp (and tmp2 when
// there is no P) are N x nrhs work buffers; every buffer has leading dim N.
qtt_status apply_M(const Ctx &c, int inner, const double *rhs, double *z, double *tmp,
                   double *tmp2) {
  QTT_TRY(apply_P(c, rhs, c.N, z, c.N, false));
  for (int s = 0; s < inner; ++s) {
    if (c.P) {
      QTT_TRY(apply_K_lowp(c, z, tmp, rhs, -c.a));  // tmp = rhs - a z - K z
      QTT_TRY(apply_P(c, tmp, c.N, z, c.N, true));  // z += P tmp
    } else {
      QTT_TRY(apply_K_lowp(c, z, tmp2, rhs, 1.0 - c.a));  // rhs + (1 - a) z - K z
      QTT_CUDA_OK(vec_copy(vecs(z, c.N), vecs(tmp2, c.N), c.N, c.nrhs, c.st), "copy");
    }
  }
  return QTT_OK;
}

// r = f - (a x + K x) (FP64, fused)
qtt_status residual(const Ctx &c, const double *f, const double *x, int64_t ld, double *r) {
  Epilogue e;
  e.on = true;
  e.v = f;
  e.s_v = 1.0;
  e.u = x;
  e.s_u = -c.a;
  e.s_acc = -1.0;
  return apply_f64(c.K, x, r, c.nrhs, ld, c.st, e);
}

// host copy of per-RHS sums of squares
qtt_status sumsq(const Ctx &c, const double *v, int64_t ld, double *partial, double *dev_out,
                 std::vector<double> &host) {
  QTT_CUDA_OK(vec_dots(vecs(v, ld), 1, vecs(v, ld), c.N, c.nrhs, partial, dev_out, nullptr, c.st),
              "dots");
  host.resize(c.nrhs);
  QTT_CUDA_OK(cudaMemcpyAsync(host.data(), dev_out, sizeof(double) * c.nrhs,
                              cudaMemcpyDeviceToHost, c.st), "memcpy");
  QTT_CUDA_OK(cudaStreamSynchronize(c.st), "sync");
  return QTT_OK;
}

qtt_status copy_strided(const Ctx &c, double *dst, int64_t ldd, const double *src, int64_t lds) {
  QTT_CUDA_OK(vec_copy(vecs(dst, ldd), vecs(src, lds), c.N, c.nrhs, c.st), "copy");
  return QTT_OK;
}

// ------------------------------------------------------------------ GMRES
qtt_status gmres(const Ctx &c, const double *f, double *x, int64_t ld, const qtt_solve_params &prm,
                 const std::vector<double> &fn, qtt_solve_info *info) {
  const int64_t N = c.N, nr = c.nrhs;
  const int m = prm.restart;
  Scratch S{c.st, {}};
  double *V, *Z = nullptr, *w, *z, *partial, *h1, *h2, *ss, *ydev;
  const int64_t nrc = std::min<int64_t>(nr, 65535);
  QTT_TRY(S.get(&V, (size_t)(m + 1) * N * nr));
  // Flexible GMRES: keep Z_j = P v_j, so that A Z = V H holds exactly for
  // the preconditioner as applied (a reduced-precision P is not exactly
  // linear), and update x with Z y.
  const int inner = prm.inner_iters;
  const bool flex = c.P || inner > 0;  // z_j = M v_j differs from v_j
  if (flex) QTT_TRY(S.get(&Z, (size_t)m * N * nr));
  double *t1 = nullptr, *t2 = nullptr;
  if (inner > 0) {
    QTT_TRY(S.get(&t1, (size_t)N * nr));
    QTT_TRY(S.get(&t2, (size_t)N * nr));
  }
  QTT_TRY(S.get(&w, (size_t)N * nr));
  QTT_TRY(S.get(&z, (size_t)N * nr));
  QTT_TRY(S.get(&partial, (size_t)(m + 1) * nrc * blocks_for(N)));
  QTT_TRY(S.get(&h1, (size_t)(m + 1) * nr));
  QTT_TRY(S.get(&h2, (size_t)(m + 1) * nr));
  QTT_TRY(S.get(&ss, (size_t)nr));
  QTT_TRY(S.get(&ydev, (size_t)m * nr));
  const int64_t vstride = N * nr;  // basis vector i of RHS c: V + i*vstride + c*N

  QTT_CUDA_OK(cudaMemset2DAsync(x, ld * sizeof(double), 0, N * sizeof(double), nr, c.st),
              "memset x");
  std::vector<double> H((size_t)nr * (m + 1) * m), cs((size_t)nr * m), sn((size_t)nr * m),
      g((size_t)nr * (m + 1)), hv1, hv2, hs, beta, y((size_t)m * nr);
  std::vector<double> rel(nr, 0.0);
  int iters = 0;
  bool first = true;
  for (;;) {
    // true residual r = f - A x into w (x = 0 on the first cycle: r = f)
    if (first)
      QTT_TRY(copy_strided(c, w, N, f, ld));
    else {
      // residual needs f, x with the same ld; r goes to w (ld = N) via z
      if (ld == N) {
        QTT_TRY(residual(c, f, x, ld, w));
      } else {
        QTT_TRY(copy_strided(c, z, N, x, ld));
        QTT_TRY(copy_strided(c, V, N, f, ld));  // V_0 is free at this point
        QTT_TRY(residual(c, V, z, N, w));
      }
    }
    first = false;
    QTT_TRY(sumsq(c, w, N, partial, ss, beta));
    bool all = true;
    for (int64_t r = 0; r < nr; ++r) {
      const double b = std::sqrt(beta[r]);
      rel[r] = fn[r] > 0.0 ? b / fn[r] : 0.0;
      if (fn[r] > 0.0 && rel[r] > prm.tol) all = false;
    }
    if (all || iters >= prm.max_iter) break;
    QTT_CUDA_OK(vec_normalize(vecs(V, N), vecs(w, N), ss, N, nr, c.st), "normalize");
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    for (int64_t r = 0; r < nr; ++r) g[(size_t)r * (m + 1)] = std::sqrt(beta[r]);
    int jl = 0;
    for (int j = 0; j < m && iters < prm.max_iter; ++j) {
      double *Vj = V + (int64_t)j * vstride;
      double *Zj = flex ? Z + (int64_t)j * vstride : Vj;
      if (flex) QTT_TRY(apply_M(c, inner, Vj, Zj, t1, t2));
      QTT_TRY(apply_A(c, Zj, w, N));
      const int nv = j + 1;
      QTT_CUDA_OK(vec_dots(vecs(V, N, vstride), nv, vecs(w, N), N, nr, partial, h1, nullptr, c.st),
                  "dots");
      QTT_CUDA_OK(vec_gs_update(vecs(w, N), vecs(V, N, vstride), nv, h1, N, nr, c.st), "gs");
      QTT_CUDA_OK(vec_dots(vecs(V, N, vstride), nv, vecs(w, N), N, nr, partial, h2, nullptr, c.st),
                  "dots");
      QTT_CUDA_OK(vec_gs_update(vecs(w, N), vecs(V, N, vstride), nv, h2, N, nr, c.st), "gs");
      QTT_CUDA_OK(vec_dots(vecs(w, N), 1, vecs(w, N), N, nr, partial, ss, nullptr, c.st), "dots");
      QTT_CUDA_OK(vec_normalize(vecs(V + (int64_t)(j + 1) * vstride, N), vecs(w, N), ss, N, nr,
                                c.st), "normalize");
      hv1.resize((size_t)nv * nr);
      hv2.resize((size_t)nv * nr);
      hs.resize(nr);
      QTT_CUDA_OK(cudaMemcpyAsync(hv1.data(), h1, sizeof(double) * nv * nr,
                                  cudaMemcpyDeviceToHost, c.st), "memcpy");
      QTT_CUDA_OK(cudaMemcpyAsync(hv2.data(), h2, sizeof(double) * nv * nr,
                                  cudaMemcpyDeviceToHost, c.st), "memcpy");
      QTT_CUDA_OK(cudaMemcpyAsync(hs.data(), ss, sizeof(double) * nr, cudaMemcpyDeviceToHost,
                                  c.st), "memcpy");
      QTT_CUDA_OK(cudaStreamSynchronize(c.st), "sync");
      ++iters;
      jl = j + 1;
      const bool done = gmres_host_step(nr, m, j, hv1.data(), hv2.data(), hs.data(), fn, prm.tol,
                                        H, cs, sn, g);
      if (done) break;
    }
    // y = H^{-1} g per RHS, x += P (V y)
    gmres_back_solve(nr, m, jl, H, g, y.data());
    QTT_CUDA_OK(cudaMemcpyAsync(ydev, y.data(), sizeof(double) * jl * nr, cudaMemcpyHostToDevice,
                                c.st), "memcpy");
    // x += Z y (Z = V without a preconditioner)
    QTT_CUDA_OK(vec_combine(vecs(z, N), vecs(flex ? Z : V, N, vstride), jl, ydev, N, nr, c.st),
                "combine");
    QTT_CUDA_OK(vec_axpy(vecs(x, ld), vecs(z, N), 1.0, N, nr, c.st), "axpy");
  }
  for (int64_t r = 0; r < nr; ++r) {
    info[r].iters = iters;
    info[r].rel_residual = rel[r];
    info[r].status = rel[r] <= prm.tol ? QTT_OK : QTT_ERR_NOT_CONVERGED;
  }
  return QTT_OK;
}

// -------------------------------------------------------------- refinement
qtt_status refine(const Ctx &c, const double *f, double *x, int64_t ld,
                  const qtt_solve_params &prm, const std::vector<double> &fn,
                  qtt_solve_info *info) {
  const int64_t N = c.N, nr = c.nrhs;
  Scratch S{c.st, {}};
  double *r, *partial, *ss, *fc = nullptr, *xc = nullptr;
  QTT_TRY(S.get(&r, (size_t)N * nr));
  QTT_TRY(S.get(&partial, (size_t)std::min<int64_t>(nr, 65535) * blocks_for(N)));
  QTT_TRY(S.get(&ss, (size_t)nr));
  // Work on contiguous copies when ld != N (the fused kernels take one ld).
  const double *F = f;
  double *X = x;
  if (ld != N) {
    QTT_TRY(S.get(&fc, (size_t)N * nr));
    QTT_TRY(S.get(&xc, (size_t)N * nr));
    QTT_TRY(copy_strided(c, fc, N, f, ld));
    F = fc;
    X = xc;
  }
  const int64_t L = ld != N ? N : ld;
  const int inner = prm.inner_iters;
  double *zA = nullptr, *zB = nullptr, *w = nullptr;
  if (inner > 0) {
    QTT_TRY(S.get(&zA, (size_t)N * nr));
    QTT_TRY(S.get(&zB, (size_t)N * nr));
    QTT_TRY(S.get(&w, (size_t)N * nr));
  }
  auto correction = [&](const double *rhs) -> qtt_status {
    return apply_M(c, inner, rhs, zA, w, zB);
  };
  if (inner > 0) {
    QTT_TRY(correction(F));
    QTT_TRY(copy_strided(c, X, L, zA, N));  // x0 = M f
  } else {
    QTT_TRY(apply_P(c, F, L, X, L, false));  // x0 = P f
  }
  int iters = 1;
  std::vector<double> q, rel(nr, 0.0);
  for (;;) {
    QTT_TRY(residual(c, F, X, L, r));
    QTT_TRY(sumsq(c, r, N, partial, ss, q));
    bool all = true;
    for (int64_t k = 0; k < nr; ++k) {
      rel[k] = fn[k] > 0.0 ? std::sqrt(q[k]) / fn[k] : 0.0;
      if (rel[k] > prm.tol) all = false;
    }
    if (all || iters >= prm.max_iter) break;
    if (inner > 0) {
      QTT_TRY(correction(r));
      QTT_CUDA_OK(vec_axpy(vecs(X, L), vecs(zA, N), 1.0, N, nr, c.st), "axpy");  // FP64 update
    } else {
      QTT_TRY(apply_P(c, r, N, X, L, true));  // x += P r (FP64 update)
    }
    ++iters;
  }
  if (ld != N) QTT_TRY(copy_strided(c, x, ld, X, N));
  QTT_CUDA_OK(cudaStreamSynchronize(c.st), "sync");
  for (int64_t k = 0; k < nr; ++k) {
    info[k].iters = iters;
    info[k].rel_residual = rel[k];
    info[k].status = rel[k] <= prm.tol ? QTT_OK : QTT_ERR_NOT_CONVERGED;
  }
  return QTT_OK;
}

qtt_status direct(const Ctx &c, const double *f, double *x, int64_t ld,
                  const std::vector<double> &fn, qtt_solve_info *info) {
  const int64_t N = c.N, nr = c.nrhs;
  QTT_TRY(apply_P(c, f, ld, x, ld, false));
  std::vector<double> rel(nr, -1.0);
  if (c.K) {
    Scratch S{c.st, {}};
    double *r, *partial, *ss;
    QTT_TRY(S.get(&r, (size_t)N * nr));
    QTT_TRY(S.get(&partial, (size_t)std::min<int64_t>(nr, 65535) * blocks_for(N)));
    QTT_TRY(S.get(&ss, (size_t)nr));
    if (ld == N) {
      QTT_TRY(residual(c, f, x, ld, r));
      std::vector<double> q;
      QTT_TRY(sumsq(c, r, N, partial, ss, q));
      for (int64_t k = 0; k < nr; ++k) rel[k] = fn[k] > 0.0 ? std::sqrt(q[k]) / fn[k] : 0.0;
    }
  }
  QTT_CUDA_OK(cudaStreamSynchronize(c.st), "sync");
  for (int64_t k = 0; k < nr; ++k) {
    info[k].iters = 1;
    info[k].rel_residual = rel[k];
    info[k].status = QTT_OK;
  }
  return QTT_OK;
}

}  // namespace
}  // namespace qtt

using namespace qtt;

extern "C" qtt_status qtt_solve(const qtt_op *K, const qtt_op *P, const double *f, double *x,
                                int64_t nrhs, int64_t ld, const qtt_solve_params *prm,
                                qtt_solve_info *info, void *stream) {
  if (!prm) return fail(QTT_ERR_INVALID_ARG, "qtt_solve: NULL params");
  if (prm->kind != QTT_SOLVE_DIRECT && prm->kind != QTT_SOLVE_GMRES &&
      prm->kind != QTT_SOLVE_REFINE)
    return fail(QTT_ERR_INVALID_ARG, "qtt_solve: unknown kind");
  if (prm->kind == QTT_SOLVE_DIRECT && !P)
    return fail(QTT_ERR_INVALID_ARG, "qtt_solve: DIRECT needs P");
  if (prm->kind != QTT_SOLVE_DIRECT && !K)
    return fail(QTT_ERR_INVALID_ARG, "qtt_solve: GMRES and REFINE need K");
  if (K && P && K->d != P->d) return fail(QTT_ERR_INVALID_ARG, "qtt_solve: K and P differ in d");
  for (const qtt_op *A : {K, P})
    if (A)
      if (qtt_status ds = check_device(A, "qtt_solve")) return ds;
  const qtt_op *any = K ? K : P;
  const int64_t N = (int64_t)1 << any->d;
  if (nrhs < 0) return fail(QTT_ERR_INVALID_ARG, "qtt_solve: nrhs < 0");
  if (nrhs == 0) return QTT_OK;
  if (nrhs > 65535) return fail(QTT_ERR_INVALID_ARG, "qtt_solve: nrhs > 65535");
  if (ld < N) return fail(QTT_ERR_INVALID_ARG, "qtt_solve: ld < N");
  if (!f || !x || !info) return fail(QTT_ERR_INVALID_ARG, "qtt_solve: NULL f, x or info");
  if (!(prm->tol >= 0.0)) return fail(QTT_ERR_INVALID_ARG, "qtt_solve: tol must be >= 0");
  if (prm->max_iter < 1) return fail(QTT_ERR_INVALID_ARG, "qtt_solve: max_iter < 1");
  if (prm->kind == QTT_SOLVE_GMRES && (prm->restart < 1 || prm->restart > 1000))
    return fail(QTT_ERR_INVALID_ARG, "qtt_solve: restart must be in [1, 1000]");
  const qtt_dtype pc = prm->precond_compute;
  if (pc != QTT_F64 && pc != QTT_F32 && pc != QTT_TF32 && pc != QTT_BF16)
    return fail(QTT_ERR_INVALID_ARG, "qtt_solve: unknown precond_compute");
  auto packed = [&](const qtt_op *A) -> bool {
    return pc == QTT_F32 ? A->m32 != nullptr
           : pc == QTT_TF32 ? A->mtf32 != nullptr : A->mbf16 != nullptr;
  };
  if (P && pc != QTT_F64 && !packed(P))
    return fail(QTT_ERR_INVALID_ARG, "qtt_solve: P lacks the packed copy for precond_compute");
  if (prm->inner_iters < 0 || prm->inner_iters > 1000)
    return fail(QTT_ERR_INVALID_ARG, "qtt_solve: inner_iters must be in [0, 1000]");
  if (prm->kind != QTT_SOLVE_DIRECT && prm->inner_iters > 0 && pc != QTT_F64 && !packed(K))
    return fail(QTT_ERR_INVALID_ARG,
                "qtt_solve: inner iterations need K packed for precond_compute");
  {
    const size_t span = ((size_t)(nrhs - 1) * (size_t)ld + (size_t)N) * sizeof(double);
    const char *fb = reinterpret_cast<const char *>(f), *xb = reinterpret_cast<const char *>(x);
    if (fb < xb + span && xb < fb + span)
      return fail(QTT_ERR_INVALID_ARG, "qtt_solve: f and x overlap");
  }
  Ctx c{K, P, prm->a, pc, N, nrhs, static_cast<cudaStream_t>(stream)};
  // ||f|| per right-hand side
  std::vector<double> fn(nrhs);
  {
    Scratch S{c.st, {}};
    double *partial, *ss;
    QTT_TRY(S.get(&partial, (size_t)nrhs * blocks_for(N)));
    QTT_TRY(S.get(&ss, (size_t)nrhs));
    std::vector<double> q;
    QTT_TRY(sumsq(c, f, ld, partial, ss, q));
    for (int64_t k = 0; k < nrhs; ++k) fn[k] = std::sqrt(q[k]);
  }
  qtt_status s;
  switch (prm->kind) {
    case QTT_SOLVE_DIRECT: s = direct(c, f, x, ld, fn, info); break;
    case QTT_SOLVE_GMRES: s = gmres(c, f, x, ld, *prm, fn, info); break;
    default: s = refine(c, f, x, ld, *prm, fn, info); break;
  }
  if (s != QTT_OK) return s;
  if (prm->kind != QTT_SOLVE_DIRECT)
    for (int64_t k = 0; k < nrhs; ++k)
      if (info[k].status != QTT_OK)
        return fail(QTT_ERR_NOT_CONVERGED,
                    "qtt_solve: right-hand side " + std::to_string(k) + " ended at relative residual " +
                        std::to_string(info[k].rel_residual) + " after " +
                        std::to_string(info[k].iters) + " iterations");
  return QTT_OK;
}

namespace qtt {

qtt_status solve_apply_M(const SolveCtx &c, int inner, const double *rhs, double *z, double *tmp,
                         double *tmp2) {
  return apply_M(Ctx{c.K, c.P, c.a, c.pc, c.N, c.nrhs, c.st}, inner, rhs, z, tmp, tmp2);
}

qtt_status solve_apply_P(const SolveCtx &c, const double *in, double *out, bool accumulate) {
  return apply_P(Ctx{c.K, c.P, c.a, c.pc, c.N, c.nrhs, c.st}, in, c.N, out, c.N, accumulate);
}

bool gmres_host_step(int64_t nr, int m, int j, const double *hv1, const double *hv2,
                     const double *hs, const std::vector<double> &fn, double tol,
                     std::vector<double> &H, std::vector<double> &cs, std::vector<double> &sn,
                     std::vector<double> &g) {
  bool done = true;
  for (int64_t r = 0; r < nr; ++r) {
    double *Hr = H.data() + (size_t)r * (m + 1) * m;
    double *csr = cs.data() + (size_t)r * m, *snr = sn.data() + (size_t)r * m;
    double *gr = g.data() + (size_t)r * (m + 1);
    for (int i = 0; i <= j; ++i) Hr[i * m + j] = hv1[(size_t)i * nr + r] + hv2[(size_t)i * nr + r];
    Hr[(j + 1) * m + j] = std::sqrt(hs[r]);
    for (int i = 0; i < j; ++i) {
      const double a0 = Hr[i * m + j], a1 = Hr[(i + 1) * m + j];
      Hr[i * m + j] = csr[i] * a0 + snr[i] * a1;
      Hr[(i + 1) * m + j] = -snr[i] * a0 + csr[i] * a1;
    }
    const double a0 = Hr[j * m + j], a1 = Hr[(j + 1) * m + j];
    const double den = std::sqrt(a0 * a0 + a1 * a1);
    csr[j] = den == 0.0 ? 1.0 : a0 / den;
    snr[j] = den == 0.0 ? 0.0 : a1 / den;
    Hr[j * m + j] = den;
    Hr[(j + 1) * m + j] = 0.0;
    gr[j + 1] = -snr[j] * gr[j];
    gr[j] = csr[j] * gr[j];
    if (fn[r] > 0.0 && std::fabs(gr[j + 1]) / fn[r] > tol && hs[r] > 0.0) done = false;
  }
  return done;
}

void gmres_back_solve(int64_t nr, int m, int jl, const std::vector<double> &H,
                      const std::vector<double> &g, double *y) {
  for (int64_t r = 0; r < nr; ++r) {
    const double *Hr = H.data() + (size_t)r * (m + 1) * m;
    const double *gr = g.data() + (size_t)r * (m + 1);
    double yy[1024];
    for (int i = jl - 1; i >= 0; --i) {
      double s = gr[i];
      for (int l = i + 1; l < jl; ++l) s -= Hr[i * m + l] * yy[l];
      yy[i] = Hr[i * m + i] != 0.0 ? s / Hr[i * m + i] : 0.0;
    }
    for (int i = 0; i < jl; ++i) y[(size_t)i * nr + r] = yy[i];
  }
}

}  // namespace qtt
