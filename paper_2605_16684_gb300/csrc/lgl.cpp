// lgl.cpp -- Legendre-Gauss-Lobatto nodes, weights and differentiation matrix
// for the device tables (Section 3: tensor-product LGL collocation).
//
// Interior nodes are the roots of P_N'; P_N' and P_N'' come from the
// derivative recurrences P'_{k+1} = P'_{k-1} + (2k+1) P_k and
// P''_{k+1} = P''_{k-1} + (2k+1) P'_k, refined by Newton's method in long
// double.  Weights are 2 / (N (N+1) P_N(x)^2).  D uses barycentric weights
// lambda_j = 1 / prod_{k != j} (x_j - x_k): D_ij = (lambda_j / lambda_i) / (x_i - x_j),
// D_ii = -sum_{j != i} D_ij.  Dt = 2D - W^-1 B has zero diagonal by construction.
#include <cmath>
#include <cstring>

#include "esdg_internal.cuh"

namespace {

void legendre_all(int N, long double x, long double* P, long double* dP, long double* d2P) {
  long double p[ESDG_MAXNQ + 1], dp[ESDG_MAXNQ + 1], d2p[ESDG_MAXNQ + 1];
  p[0] = 1.0L;
  dp[0] = 0.0L;
  d2p[0] = 0.0L;
  p[1] = x;
  dp[1] = 1.0L;
  d2p[1] = 0.0L;
  for (int k = 1; k < N; k++) {
    p[k + 1] = ((2 * k + 1) * x * p[k] - k * p[k - 1]) / (k + 1);
    dp[k + 1] = dp[k - 1] + (2 * k + 1) * p[k];
    d2p[k + 1] = d2p[k - 1] + (2 * k + 1) * dp[k];
  }
  *P = p[N];
  *dP = dp[N];
  *d2P = d2p[N];
}

}  // namespace

int esdg_lgl_build(int N, EsdgLGL* out) {
  if (N < 1 || N + 1 > ESDG_MAXNQ) return -1;
  std::memset(out, 0, sizeof(*out));
  const int Nq = N + 1;
  long double x[ESDG_MAXNQ];
  const long double pi = 3.141592653589793238462643383279502884L;
  x[0] = -1.0L;
  x[N] = 1.0L;
  for (int k = 1; k < N; k++) {
    // start from the Chebyshev-Gauss-Lobatto point and polish with Newton
    long double t = -std::cos(pi * (long double)k / (long double)N);
    for (int it = 0; it < 100; it++) {
      long double P, dP, d2P;
      legendre_all(N, t, &P, &dP, &d2P);
      const long double step = dP / d2P;
      t -= step;
      if (std::fabs((double)step) < 1e-20) break;
    }
    x[k] = t;
  }
  long double lam[ESDG_MAXNQ];
  for (int j = 0; j < Nq; j++) {
    long double prod = 1.0L;
    for (int k = 0; k < Nq; k++)
      if (k != j) prod *= (x[j] - x[k]);
    lam[j] = 1.0L / prod;
  }
  out->N = N;
  for (int i = 0; i < Nq; i++) {
    long double P, dP, d2P;
    legendre_all(N, x[i], &P, &dP, &d2P);
    out->xi[i] = (double)x[i];
    out->xi_lo[i] = (double)(x[i] - (long double)out->xi[i]);
    out->w[i] = (double)(2.0L / ((long double)N * (N + 1) * P * P));
    long double diag = 0.0L;
    for (int j = 0; j < Nq; j++) {
      if (j == i) continue;
      const long double dij = (lam[j] / lam[i]) / (x[i] - x[j]);
      out->D[i][j] = (double)dij;
      out->D_lo[i][j] = (double)(dij - (long double)out->D[i][j]);
      out->Dt[i][j] = (double)(2.0L * dij);
      diag -= dij;
    }
    out->D[i][i] = (double)diag;
    out->D_lo[i][i] = (double)(diag - (long double)out->D[i][i]);
    out->Dt[i][i] = 0.0;
  }
  return 0;
}
