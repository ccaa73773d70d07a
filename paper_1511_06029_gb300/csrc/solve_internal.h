// Pieces of the solves shared by qtt_solve and the serving loop, so that a
// request served in the loop runs exactly the arithmetic of qtt_solve.
#pragma once

#include <vector>

#include "qtt_internal.h"

namespace qtt {

struct SolveCtx {
  const qtt_op *K, *P;
  double a;
  qtt_dtype pc;
  int64_t N, nrhs;
  cudaStream_t st;
};

// z = M rhs: P rhs (P = identity when absent), then `inner` Richardson
// steps z <- z + P (rhs - (a z + K z)) with K and P in the low precision;
// vectors FP64 with leading dimension N; tmp, tmp2 work buffers.
qtt_status solve_apply_M(const SolveCtx &c, int inner, const double *rhs, double *z, double *tmp,
                         double *tmp2);
// out = P in, or out += P in (accumulate), leading dimension N.
qtt_status solve_apply_P(const SolveCtx &c, const double *in, double *out, bool accumulate);

// Host part of Arnoldi step j of GMRES(m) for nr right-hand sides: column j
// of each Hessenberg matrix from the CGS2 coefficients hv1 + hv2 and the new
// norm sqrt(hs), the previous Givens rotations applied, a new rotation
// computed, and the residual estimate g updated.  Returns true when every
// right-hand side has met tol (or lost its Krylov space).
bool gmres_host_step(int64_t nr, int m, int j, const double *hv1, const double *hv2,
                     const double *hs, const std::vector<double> &fn, double tol,
                     std::vector<double> &H, std::vector<double> &cs, std::vector<double> &sn,
                     std::vector<double> &g);
// y = H^{-1} g for the first jl Arnoldi steps of each right-hand side,
// stored y[i * nr + r].
void gmres_back_solve(int64_t nr, int m, int jl, const std::vector<double> &H,
                      const std::vector<double> &g, double *y);

}  // namespace qtt
