/*
 * QTT oracle: plain, slow, obviously correct FP64 reference for the QTT
 * matrix x dense-vector product and the solves built on it.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or helper
 * with the CUDA path.
 *
 * Conventions (Corona, Rahimian, Zorin, "A Tensor-Train accelerated solver
 * for integral equations in complex geometries"):
 *   - A matrix in QTT format has d cores; core k (0-based here, k = 0..d-1)
 *     is G_k(alpha_k, i_k, j_k, alpha_{k+1}) with ranks r[k], r[k+1],
 *     r[0] = r[d] = 1 (Sec. 2.2, eq. (TTdeccores) and the dummy-rank remark;
 *     matrix tensorisation on the product tree, Sec. 3.1).
 *   - Storage: all cores concatenated in one array; core k is C-order
 *     [r[k]][2 (row bit i)][2 (column bit j)][r[k+1]].
 *   - Linear index, least-significant bit first: i = sum_k i_k 2^k, core 0
 *     acting on the finest level of the tree (Sec. 2.4 numbers the finest
 *     level first; Matlab reshape order, Sec. 2.1).
 *   - Entry: A(i, j) = G_0[i_0, j_0] G_1[i_1, j_1] ... G_{d-1}[i_{d-1}, j_{d-1}]
 *     where G_k[i_k, j_k] is the r[k] x r[k+1] slice.
 *
 * The apply here contracts cores from the LAST to the FIRST (the reverse of
 * the paper's Algorithm 2); summation over the rank indices is associative,
 * so it reaches the same product up to rounding.  Every output is a plain
 * sequential sum; OpenMP only distributes independent outputs over threads.
 *
 * Parity of each function is pinned by tests that do not reuse its code:
 * dense brute force, the identity, Kronecker products, integer-exact cases,
 * algebraic invariants (sum, product, transpose) and the TT-SVD error bound.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define QO_OK 0
#define QO_EINVAL 1
#define QO_ENOMEM 2
#define QO_ENOTCONV 4

static int64_t core_offset(const int *r, int k) {
  int64_t off = 0;
  for (int l = 0; l < k; ++l) off += (int64_t)4 * r[l] * r[l + 1];
  return off;
}

static int check_tt(int d, const int *r) {
  if (d < 1 || d > 30) return QO_EINVAL;
  if (r[0] != 1 || r[d] != 1) return QO_EINVAL;
  for (int k = 0; k <= d; ++k)
    if (r[k] < 1) return QO_EINVAL;
  return QO_OK;
}

int qo_num_params(int d, const int *r) { return (int)core_offset(r, d); }

static void set_threads(int threads) {
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#else
  (void)threads;
#endif
}

/* ------------------------------------------------------------------------ */
/* y = A x, contracting cores d-1 down to 0 (see header).                    */
/*                                                                            */
/* State after cores k..d-1: Z_k(alpha_k, t), t in [0, N); bits 0..k-1 of t  */
/* are still column bits j, bits k..d-1 are already row bits i.               */
/*   Z_d(0, t) = x(t)                                                          */
/*   Z_k(a, t) = sum_{b, j} G_k(a, bit_k(t), j, b) Z_{k+1}(b, t with bit k = j) */
/*   y(t) = Z_0(0, t)                                                         */
/* ------------------------------------------------------------------------ */
#define DEFINE_APPLY(NAME, REAL)                                               \
  int NAME(int d, const int *r, const double *G, int64_t nrhs,               \
           const double *x, int64_t ldx, double *y, int64_t ldy,             \
           int threads) {                                                    \
    int st = check_tt(d, r);                                                 \
    if (st) return st;                                                       \
    const int64_t N = (int64_t)1 << d;                                       \
    if (nrhs < 0 || ldx < N || ldy < N) return QO_EINVAL;                    \
    int rmax = 1;                                                            \
    for (int k = 0; k <= d; ++k)                                             \
      if (r[k] > rmax) rmax = r[k];                                          \
    REAL *Zin = (REAL *)malloc(sizeof(REAL) * (size_t)rmax * (size_t)N);     \
    REAL *Zout = (REAL *)malloc(sizeof(REAL) * (size_t)rmax * (size_t)N);    \
    if (!Zin || !Zout) {                                                     \
      free(Zin);                                                             \
      free(Zout);                                                            \
      return QO_ENOMEM;                                                      \
    }                                                                        \
    set_threads(threads);                                                    \
    for (int64_t c = 0; c < nrhs; ++c) {                                     \
      for (int64_t t = 0; t < N; ++t) Zin[t] = (REAL)x[c * ldx + t];         \
      for (int k = d - 1; k >= 0; --k) {                                     \
        const double *Gk = G + core_offset(r, k);                            \
        const int ra = r[k], rb = r[k + 1];                                  \
        const int64_t bit = (int64_t)1 << k;                                 \
        _Pragma("omp parallel for schedule(static)")                         \
        for (int64_t at = 0; at < (int64_t)ra * N; ++at) {                   \
          const int a = (int)(at / N);                                       \
          const int64_t t = at % N;                                          \
          const int i = (int)((t >> k) & 1);                                 \
          REAL s = 0;                                                        \
          for (int b = 0; b < rb; ++b)                                       \
            for (int j = 0; j < 2; ++j) {                                    \
              const int64_t src = (t & ~bit) | ((int64_t)j << k);            \
              const REAL g = (REAL)Gk[((a * 2 + i) * 2 + j) * rb + b];       \
              s += g * Zin[(int64_t)b * N + src];                            \
            }                                                                \
          Zout[at] = s;                                                      \
        }                                                                    \
        REAL *tmp = Zin;                                                     \
        Zin = Zout;                                                          \
        Zout = tmp;                                                          \
      }                                                                      \
      for (int64_t t = 0; t < N; ++t) y[c * ldy + t] = (double)Zin[t];       \
    }                                                                        \
    free(Zin);                                                               \
    free(Zout);                                                              \
    return QO_OK;                                                            \
  }

DEFINE_APPLY(qo_apply, double)
/* Check mode: the same sweep carried in long double (80-bit on x86, 128-bit
 * on aarch64) to bound the FP64 oracle's own rounding error. */
DEFINE_APPLY(qo_apply_ld, long double)

/* ------------------------------------------------------------------------ */
/* Dense reconstruction A(i, j) (row-major, N x N) straight from the entry    */
/* formula: A(i, j) = G_0[i_0,j_0] G_1[i_1,j_1] ... (Sec. 2.2 eq.             */
/* (TTdeccores) with the product-tree indices of Sec. 3.1).  The chain of     */
/* slice products is evaluated left to right; pairs of (i, j) that share the  */
/* low bits share the prefix product (depth-first over the levels).           */
/* ------------------------------------------------------------------------ */
static void dense_rec(int d, const int *r, const double *G, int k,
                      int64_t i, int64_t j, const double *v, double *work,
                      double *A, int64_t N) {
  if (k == d) {
    A[i * N + j] = v[0];
    return;
  }
  const double *Gk = G + core_offset(r, k);
  const int ra = r[k], rb = r[k + 1];
  double *w = work; /* r[k+1] doubles for this level */
  for (int ik = 0; ik < 2; ++ik)
    for (int jk = 0; jk < 2; ++jk) {
      for (int b = 0; b < rb; ++b) {
        double s = 0.0;
        for (int a = 0; a < ra; ++a) s += v[a] * Gk[((a * 2 + ik) * 2 + jk) * rb + b];
        w[b] = s;
      }
      dense_rec(d, r, G, k + 1, i | ((int64_t)ik << k), j | ((int64_t)jk << k),
                w, work + rb, A, N);
    }
}

int qo_dense(int d, const int *r, const double *G, double *A) {
  int st = check_tt(d, r);
  if (st) return st;
  if (d > 13) return QO_EINVAL;
  const int64_t N = (int64_t)1 << d;
  int64_t need = 1;
  for (int k = 0; k <= d; ++k) need += r[k];
  double *work = (double *)malloc(sizeof(double) * (size_t)need);
  if (!work) return QO_ENOMEM;
  double one = 1.0;
  dense_rec(d, r, G, 0, 0, 0, &one, work, A, N);
  free(work);
  return QO_OK;
}

/* Brute-force dense product y = A x, A row-major N x N. */
int qo_dense_matvec(int64_t N, const double *A, int64_t nrhs, const double *x,
                    int64_t ldx, double *y, int64_t ldy) {
  for (int64_t c = 0; c < nrhs; ++c)
    for (int64_t i = 0; i < N; ++i) {
      double s = 0.0;
      for (int64_t j = 0; j < N; ++j) s += A[i * N + j] * x[c * ldx + j];
      y[c * ldy + i] = s;
    }
  return QO_OK;
}

/* ------------------------------------------------------------------------ */
/* Structural operations on QTT matrices (used to build test operators and   */
/* the invariants).                                                          */
/* ------------------------------------------------------------------------ */

/* Transpose: A^T(i, j) = A(j, i), i.e. swap the row and column bit in every
 * core. */
int qo_transpose(int d, const int *r, const double *G, double *GT) {
  int st = check_tt(d, r);
  if (st) return st;
  for (int k = 0; k < d; ++k) {
    const double *Gk = G + core_offset(r, k);
    double *Tk = GT + core_offset(r, k);
    const int ra = r[k], rb = r[k + 1];
    for (int a = 0; a < ra; ++a)
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
          for (int b = 0; b < rb; ++b)
            Tk[((a * 2 + i) * 2 + j) * rb + b] = Gk[((a * 2 + j) * 2 + i) * rb + b];
  }
  return QO_OK;
}

/* Sum C = A + B: ranks add; the first core is the row block [A_0 B_0], the
 * last the column block [A_{d-1}; B_{d-1}], the others block diagonal (the
 * rank-addition argument behind Corollary 1, Sec. 3.3).  rc must hold
 * rA[k] + rB[k] for 0 < k < d and 1 at both ends. */
int qo_sum(int d, const int *rA, const double *GA, const int *rB,
           const double *GB, int *rc, double *GC) {
  int st = check_tt(d, rA);
  if (st) return st;
  st = check_tt(d, rB);
  if (st) return st;
  rc[0] = 1;
  rc[d] = 1;
  for (int k = 1; k < d; ++k) rc[k] = rA[k] + rB[k];
  if (d == 1) {
    for (int e = 0; e < 4; ++e) GC[e] = GA[e] + GB[e];
    return QO_OK;
  }
  for (int k = 0; k < d; ++k) {
    const double *Ak = GA + core_offset(rA, k);
    const double *Bk = GB + core_offset(rB, k);
    double *Ck = GC + core_offset(rc, k);
    const int ca = rc[k], cb = rc[k + 1];
    memset(Ck, 0, sizeof(double) * (size_t)4 * ca * cb);
    /* A block at (0, 0); B block at row offset (k>0 ? rA[k] : 0) and column
     * offset (k<d-1 ? rA[k+1] : 0). */
    const int boff_a = (k > 0) ? rA[k] : 0;
    const int boff_b = (k < d - 1) ? rA[k + 1] : 0;
    for (int a = 0; a < rA[k]; ++a)
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
          for (int b = 0; b < rA[k + 1]; ++b)
            Ck[((a * 2 + i) * 2 + j) * cb + b] = Ak[((a * 2 + i) * 2 + j) * rA[k + 1] + b];
    for (int a = 0; a < rB[k]; ++a)
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
          for (int b = 0; b < rB[k + 1]; ++b)
            Ck[(((a + boff_a) * 2 + i) * 2 + j) * cb + (b + boff_b)] =
                Bk[((a * 2 + i) * 2 + j) * rB[k + 1] + b];
  }
  return QO_OK;
}

/* Product C = A B, core by core: C_k[(a,a'),(i),(j),(b,b')] =
 * sum_l A_k[a][i][l][b] B_k[a'][l][j][b'] -- the core-wise contraction over
 * the inner mode index with merged rank pairs (Sec. 4.2, compressed product;
 * ranks multiply, Corollary 1).  Merged rank index (a, a') -> a * rB + a'. */
int qo_product(int d, const int *rA, const double *GA, const int *rB,
               const double *GB, int *rc, double *GC) {
  int st = check_tt(d, rA);
  if (st) return st;
  st = check_tt(d, rB);
  if (st) return st;
  for (int k = 0; k <= d; ++k) rc[k] = rA[k] * rB[k];
  for (int k = 0; k < d; ++k) {
    const double *Ak = GA + core_offset(rA, k);
    const double *Bk = GB + core_offset(rB, k);
    double *Ck = GC + core_offset(rc, k);
    const int pa = rA[k], pb = rB[k], qa = rA[k + 1], qb = rB[k + 1];
    const int cb = rc[k + 1];
    for (int a = 0; a < pa; ++a)
      for (int a2 = 0; a2 < pb; ++a2)
        for (int i = 0; i < 2; ++i)
          for (int j = 0; j < 2; ++j)
            for (int b = 0; b < qa; ++b)
              for (int b2 = 0; b2 < qb; ++b2) {
                double s = 0.0;
                for (int l = 0; l < 2; ++l)
                  s += Ak[((a * 2 + i) * 2 + l) * qa + b] * Bk[((a2 * 2 + l) * 2 + j) * qb + b2];
                Ck[(((a * pb + a2) * 2 + i) * 2 + j) * cb + (b * qb + b2)] = s;
              }
  }
  return QO_OK;
}

/* ------------------------------------------------------------------------ */
/* Solves for (a I + K) x = f with an optional QTT preconditioner P.          */
/* ------------------------------------------------------------------------ */
typedef struct {
  int d;
  const int *r;
  const double *G;
} qo_tt;

static double dot(int64_t n, const double *u, const double *v) {
  double s = 0.0;
  for (int64_t t = 0; t < n; ++t) s += u[t] * v[t];
  return s;
}

/* out = (a I + K) v ; K may be absent (d == 0 marker) */
static int apply_A(const qo_tt *K, double a, const double *v, double *out,
                   int64_t N, int threads) {
  if (K->G) {
    int st = qo_apply(K->d, K->r, K->G, 1, v, N, out, N, threads);
    if (st) return st;
  } else {
    for (int64_t t = 0; t < N; ++t) out[t] = 0.0;
  }
  for (int64_t t = 0; t < N; ++t) out[t] += a * v[t];
  return QO_OK;
}

static int apply_P(const qo_tt *P, const double *v, double *out, int64_t N,
                   int threads) {
  if (P->G) return qo_apply(P->d, P->r, P->G, 1, v, N, out, N, threads);
  memcpy(out, v, sizeof(double) * (size_t)N);
  return QO_OK;
}

/* Direct solve: x = P f (the "Solve" column of Tables 1 and 2: the QTT
 * inverse applied to a dense right-hand side). */
int qo_solve_direct(int d, const int *rP, const double *GP, int64_t nrhs,
                    const double *f, double *x, int threads) {
  const int64_t N = (int64_t)1 << d;
  return qo_apply(d, rP, GP, nrhs, f, N, x, N, threads);
}

/* Iterative refinement: x_0 = P f, then x <- x + P (f - A x) until
 * ||f - A x|| <= tol ||f||.  iters[c] counts applications of P. */
int qo_solve_refine(int d, double a, const int *rK, const double *GK,
                    const int *rP, const double *GP, int64_t nrhs,
                    const double *f, double *x, double tol, int max_iter,
                    int *iters, double *relres, int threads) {
  const int64_t N = (int64_t)1 << d;
  qo_tt K = {d, rK, GK}, P = {d, rP, GP};
  double *res = (double *)malloc(sizeof(double) * (size_t)N);
  double *z = (double *)malloc(sizeof(double) * (size_t)N);
  if (!res || !z) {
    free(res);
    free(z);
    return QO_ENOMEM;
  }
  int status = QO_OK;
  for (int64_t c = 0; c < nrhs; ++c) {
    const double *fc = f + c * N;
    double *xc = x + c * N;
    const double fn = sqrt(dot(N, fc, fc));
    if (fn == 0.0) {
      memset(xc, 0, sizeof(double) * (size_t)N);
      iters[c] = 0;
      relres[c] = 0.0;
      continue;
    }
    int it = 0, st;
    st = apply_P(&P, fc, xc, N, threads);
    if (st) { status = st; break; }
    ++it;
    double rr = 0.0;
    for (;;) {
      st = apply_A(&K, a, xc, res, N, threads);
      if (st) { status = st; break; }
      for (int64_t t = 0; t < N; ++t) res[t] = fc[t] - res[t];
      rr = sqrt(dot(N, res, res)) / fn;
      if (rr <= tol || it >= max_iter) break;
      st = apply_P(&P, res, z, N, threads);
      if (st) { status = st; break; }
      for (int64_t t = 0; t < N; ++t) xc[t] += z[t];
      ++it;
    }
    if (status) break;
    iters[c] = it;
    relres[c] = rr;
    if (rr > tol) status = QO_ENOTCONV;
  }
  free(res);
  free(z);
  return status;
}

/* Right-preconditioned restarted GMRES(m): A P u = f, x = P u, x_0 = 0.
 * Arnoldi by modified Gram-Schmidt, least squares by Givens rotations.  The
 * true residual ||f - A x|| is recomputed at every restart and decides
 * convergence; within a cycle the Givens residual estimate ends the cycle
 * early.  iters[c] counts Arnoldi steps (one A and one P apply each). */
int qo_solve_gmres(int d, double a, const int *rK, const double *GK,
                   const int *rP, const double *GP, int64_t nrhs,
                   const double *f, double *x, double tol, int m,
                   int max_iter, int *iters, double *relres, int threads) {
  const int64_t N = (int64_t)1 << d;
  if (m < 1) return QO_EINVAL;
  qo_tt K = {d, rK, GK}, P = {d, rP, GP};
  double *V = (double *)malloc(sizeof(double) * (size_t)(m + 1) * (size_t)N);
  double *w = (double *)malloc(sizeof(double) * (size_t)N);
  double *z = (double *)malloc(sizeof(double) * (size_t)N);
  double *H = (double *)calloc((size_t)(m + 1) * m, sizeof(double));
  double *cs = (double *)malloc(sizeof(double) * m);
  double *sn = (double *)malloc(sizeof(double) * m);
  double *g = (double *)malloc(sizeof(double) * (m + 1));
  double *yv = (double *)malloc(sizeof(double) * m);
  if (!V || !w || !z || !H || !cs || !sn || !g || !yv) {
    free(V); free(w); free(z); free(H); free(cs); free(sn); free(g); free(yv);
    return QO_ENOMEM;
  }
  int status = QO_OK;
  for (int64_t c = 0; c < nrhs && !status; ++c) {
    const double *fc = f + c * N;
    double *xc = x + c * N;
    memset(xc, 0, sizeof(double) * (size_t)N);
    const double fn = sqrt(dot(N, fc, fc));
    iters[c] = 0;
    relres[c] = 0.0;
    if (fn == 0.0) continue;
    int it = 0;
    double rr = 1.0;
    for (;;) {
      /* true residual */
      int st = apply_A(&K, a, xc, w, N, threads);
      if (st) { status = st; break; }
      for (int64_t t = 0; t < N; ++t) w[t] = fc[t] - w[t];
      const double beta = sqrt(dot(N, w, w));
      rr = beta / fn;
      if (rr <= tol || it >= max_iter) break;
      for (int64_t t = 0; t < N; ++t) V[t] = w[t] / beta;
      memset(H, 0, sizeof(double) * (size_t)(m + 1) * m);
      for (int i = 0; i <= m; ++i) g[i] = 0.0;
      g[0] = beta;
      int jl = 0; /* number of Arnoldi columns completed in this cycle */
      for (int j = 0; j < m && it < max_iter; ++j) {
        double *vj = V + (int64_t)j * N;
        st = apply_P(&P, vj, z, N, threads);
        if (st) break;
        st = apply_A(&K, a, z, w, N, threads);
        if (st) break;
        for (int i = 0; i <= j; ++i) {
          double *vi = V + (int64_t)i * N;
          const double h = dot(N, w, vi);
          H[i * m + j] = h;
          for (int64_t t = 0; t < N; ++t) w[t] -= h * vi[t];
        }
        const double hn = sqrt(dot(N, w, w));
        H[(j + 1) * m + j] = hn;
        if (hn > 0.0) {
          double *vn = V + (int64_t)(j + 1) * N;
          for (int64_t t = 0; t < N; ++t) vn[t] = w[t] / hn;
        }
        for (int i = 0; i < j; ++i) { /* previous rotations */
          const double h0 = H[i * m + j], h1 = H[(i + 1) * m + j];
          H[i * m + j] = cs[i] * h0 + sn[i] * h1;
          H[(i + 1) * m + j] = -sn[i] * h0 + cs[i] * h1;
        }
        const double h0 = H[j * m + j], h1 = H[(j + 1) * m + j];
        const double den = sqrt(h0 * h0 + h1 * h1);
        cs[j] = (den == 0.0) ? 1.0 : h0 / den;
        sn[j] = (den == 0.0) ? 0.0 : h1 / den;
        H[j * m + j] = den;
        H[(j + 1) * m + j] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        ++it;
        jl = j + 1;
        if (fabs(g[j + 1]) / fn <= tol || hn == 0.0) break;
      }
      if (st) { status = st; break; }
      /* back substitution H(0:jl,0:jl) y = g(0:jl) */
      for (int i = jl - 1; i >= 0; --i) {
        double s = g[i];
        for (int l = i + 1; l < jl; ++l) s -= H[i * m + l] * yv[l];
        yv[i] = (H[i * m + i] != 0.0) ? s / H[i * m + i] : 0.0;
      }
      /* x += P (V y) */
      memset(w, 0, sizeof(double) * (size_t)N);
      for (int i = 0; i < jl; ++i) {
        const double *vi = V + (int64_t)i * N;
        for (int64_t t = 0; t < N; ++t) w[t] += yv[i] * vi[t];
      }
      st = apply_P(&P, w, z, N, threads);
      if (st) { status = st; break; }
      for (int64_t t = 0; t < N; ++t) xc[t] += z[t];
    }
    iters[c] = it;
    relres[c] = rr;
    if (!status && rr > tol) status = QO_ENOTCONV;
  }
  free(V); free(w); free(z); free(H); free(cs); free(sn); free(g); free(yv);
  return status;
}

/* Spectral norm estimate ||K||_2 by power iteration on K^T K, started from
 * the caller's vector v0 (length N).  Stops after max_iter iterations or when
 * the estimate changes by less than rtol (relative).  Returns the estimate in
 * *sigma and the iteration count in *iters. */
int qo_power_norm(int d, const int *r, const double *G, const double *v0,
                  int max_iter, double rtol, double *sigma, int *iters,
                  int threads) {
  int st = check_tt(d, r);
  if (st) return st;
  const int64_t N = (int64_t)1 << d;
  const int64_t np = core_offset(r, d);
  double *GT = (double *)malloc(sizeof(double) * (size_t)np);
  double *v = (double *)malloc(sizeof(double) * (size_t)N);
  double *u = (double *)malloc(sizeof(double) * (size_t)N);
  double *w = (double *)malloc(sizeof(double) * (size_t)N);
  if (!GT || !v || !u || !w) {
    free(GT); free(v); free(u); free(w);
    return QO_ENOMEM;
  }
  qo_transpose(d, r, G, GT);
  double nv = sqrt(dot(N, v0, v0));
  for (int64_t t = 0; t < N; ++t) v[t] = v0[t] / nv;
  double lam = 0.0;
  int it = 0;
  for (it = 0; it < max_iter; ++it) {
    st = qo_apply(d, r, G, 1, v, N, u, N, threads);
    if (st) break;
    st = qo_apply(d, r, GT, 1, u, N, w, N, threads);
    if (st) break;
    const double nw = sqrt(dot(N, w, w)); /* ||K^T K v|| with ||v|| = 1 */
    const double prev = lam;
    lam = nw;
    for (int64_t t = 0; t < N; ++t) v[t] = w[t] / nw;
    if (it > 0 && fabs(lam - prev) <= rtol * lam) {
      ++it;
      break;
    }
  }
  *sigma = sqrt(lam);
  *iters = it;
  free(GT); free(v); free(u); free(w);
  return st;
}

/* Single entries A(I[n], J[n]) by the entry formula: the chain of slice
 * products G_0[i_0, j_0] ... G_{d-1}[i_{d-1}, j_{d-1}] (Sec. 2.2), evaluated
 * left to right; O(d r^2) per entry, so entries of a full-size operator can
 * be checked one by one. */
int qo_entries(int d, const int *r, const double *G, int64_t n,
               const int64_t *I, const int64_t *J, double *out) {
  int st = check_tt(d, r);
  if (st) return st;
  int rmax = 1;
  for (int k = 0; k <= d; ++k)
    if (r[k] > rmax) rmax = r[k];
  double *v = (double *)malloc(sizeof(double) * rmax);
  double *w = (double *)malloc(sizeof(double) * rmax);
  if (!v || !w) {
    free(v);
    free(w);
    return QO_ENOMEM;
  }
  for (int64_t e = 0; e < n; ++e) {
    v[0] = 1.0;
    for (int k = 0; k < d; ++k) {
      const double *Gk = G + core_offset(r, k);
      const int ra = r[k], rb = r[k + 1];
      const int i = (int)((I[e] >> k) & 1), j = (int)((J[e] >> k) & 1);
      for (int b = 0; b < rb; ++b) {
        double s = 0.0;
        for (int a = 0; a < ra; ++a) s += v[a] * Gk[((a * 2 + i) * 2 + j) * rb + b];
        w[b] = s;
      }
      for (int b = 0; b < rb; ++b) v[b] = w[b];
    }
    out[e] = v[0];
  }
  free(v);
  free(w);
  return QO_OK;
}
