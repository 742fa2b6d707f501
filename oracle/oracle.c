/*
 * CPU FP64 oracle kernels (plain C, OpenMP).
 *
 * TEST INFRASTRUCTURE ONLY.  This file belongs to the oracle: only tests/,
 * __graft_entry__.smoke() and bench.py's cpu_baseline / reference leg may
 * load the library built from it.  It shares no code with the CUDA path.
 *
 * 1. oracle_jacobi_eig: eigen-decomposition of a dense symmetric matrix by the
 *    cyclic Jacobi method with the symmetric 2x2 Schur rotation of Golub & Van
 *    Loan (Matrix Computations, 4th ed., Sec. 8.5: Alg. 8.5.1 "symSchur2" and
 *    Alg. 8.5.3 "cyclic Jacobi").  The n(n-1)/2 rotations of a sweep are
 *    visited in the round-robin ("tournament") order of Brent & Luk (1985),
 *    which groups them into n-1 rounds of disjoint (p,q) pairs; the rotations
 *    of one round commute, so a round is applied as one orthogonal similarity
 *    and the pairs run in parallel.  The eigen-decomposition X = Q diag(l) Q^T
 *    is what the PSD projection of the paper is defined through (Sec. 1,
 *    Higham's closed form, and the spectral operator F(X) = Q diag(f(l)) Q^T).
 *
 * 2. oracle_efloat_scan: the discretised error of Sec. 3.2 (Eq. "e_float"):
 *    the maximum, over every float32 value x in [-1, 1], of an error of the
 *    composite polynomial g = f_T o ... o f_1 evaluated in FP64.  Both the
 *    ReLU error |x(1+g(x))/2 - max(x,0)| and the doubled form |x g(x) - |x||
 *    are returned (see the Python wrapper for why both).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* One cyclic-Jacobi eigen-decomposition.
 *   n      order
 *   A      n*n row-major symmetric matrix, overwritten (ends near-diagonal)
 *   w      out: n eigenvalues (unsorted; the Python side sorts)
 *   V      out: n*n row-major, column k is the eigenvector of w[k]
 *   max_sweeps, tol: stop when off(A) <= tol * ||A||_F or after max_sweeps.
 * Returns the number of sweeps used (> max_sweeps means no convergence).
 */
int oracle_jacobi_eig(int n, double *A, double *w, double *V, int max_sweeps,
                      double tol) {
  if (n <= 0) return 0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[(size_t)i * n + j] = (i == j) ? 1.0 : 0.0;
  if (n == 1) {
    w[0] = A[0];
    return 0;
  }
  /* Round-robin tournament on m players (m even); player n is a bye when n
   * is odd.  Player 0 stays fixed, the others rotate one place per round. */
  const int m = (n % 2 == 0) ? n : n + 1;
  const int half = m / 2;
  int *players = (int *)malloc(sizeof(int) * m);
  int *P = (int *)malloc(sizeof(int) * half);
  int *Qi = (int *)malloc(sizeof(int) * half);
  double *C = (double *)malloc(sizeof(double) * half);
  double *S = (double *)malloc(sizeof(double) * half);
  for (int i = 0; i < m; ++i) players[i] = i;

  double frob2 = 0.0;
  for (size_t k = 0; k < (size_t)n * n; ++k) frob2 += A[k] * A[k];
  const double frob = sqrt(frob2);

  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    double off2 = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        if (i != j) off2 += A[(size_t)i * n + j] * A[(size_t)i * n + j];
    if (sqrt(off2) <= tol * frob) break;

    for (int round = 0; round < m - 1; ++round) {
      /* pairs of this round */
      for (int k = 0; k < half; ++k) {
        int p = players[k], q = players[m - 1 - k];
        if (p > q) { int t = p; p = q; q = t; }
        P[k] = p;
        Qi[k] = q;
      }
      /* rotation parameters from the current 2x2 blocks (disjoint pairs, so
       * no block is touched by another pair's rotation in this round) */
      for (int k = 0; k < half; ++k) {
        int p = P[k], q = Qi[k];
        C[k] = 1.0;
        S[k] = 0.0;
        if (q >= n) continue; /* bye */
        double apq = A[(size_t)p * n + q];
        if (apq == 0.0) continue;
        double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
        /* symSchur2: tau = (a_qq - a_pp) / (2 a_pq), t = sign(tau)/(|tau| + sqrt(1+tau^2)) */
        double tau = (aqq - app) / (2.0 * apq);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t);
        C[k] = c;
        S[k] = t * c;
      }
      /* A <- J^T A : rows p, q of every pair */
#pragma omp parallel for schedule(static)
      for (int k = 0; k < half; ++k) {
        int p = P[k], q = Qi[k];
        if (q >= n || S[k] == 0.0) continue;
        double c = C[k], s = S[k];
        double *rp = A + (size_t)p * n, *rq = A + (size_t)q * n;
        for (int j = 0; j < n; ++j) {
          double x = rp[j], y = rq[j];
          rp[j] = c * x - s * y;
          rq[j] = s * x + c * y;
        }
      }
      /* A <- A J and V <- V J : columns p, q, row by row */
#pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i) {
        double *ra = A + (size_t)i * n, *rv = V + (size_t)i * n;
        for (int k = 0; k < half; ++k) {
          int p = P[k], q = Qi[k];
          if (q >= n || S[k] == 0.0) continue;
          double c = C[k], s = S[k];
          double x = ra[p], y = ra[q];
          ra[p] = c * x - s * y;
          ra[q] = s * x + c * y;
          x = rv[p];
          y = rv[q];
          rv[p] = c * x - s * y;
          rv[q] = s * x + c * y;
        }
      }
      /* the rotation zeroes a_pq in exact arithmetic */
      for (int k = 0; k < half; ++k) {
        int p = P[k], q = Qi[k];
        if (q >= n || S[k] == 0.0) continue;
        A[(size_t)p * n + q] = 0.0;
        A[(size_t)q * n + p] = 0.0;
      }
      /* rotate players 1..m-1 by one place */
      int last = players[m - 1];
      for (int i = m - 1; i > 1; --i) players[i] = players[i - 1];
      players[1] = last;
    }
  }
  for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
  free(players);
  free(P);
  free(Qi);
  free(C);
  free(S);
  return sweep;
}

/* Composite g(x) = s_T^-1 f_T( ... s_1^-1 f_1(x)) with f_t(x) = a x + b x^3 + c x^5. */
static double composite(double x, int T, const double *coef, const double *inv_s) {
  for (int t = 0; t < T; ++t) {
    double a = coef[3 * t], b = coef[3 * t + 1], c = coef[3 * t + 2];
    double x2 = x * x;
    x = x * (a + x2 * (b + x2 * c));
    x *= inv_s[t];
  }
  return x;
}

/* Maximum errors over every float32 value in [0, 1] (the errors are even
 * functions of x because g is odd, so this covers [-1, 1]).
 *   out[0] = max |x (1 + g(x)) / 2 - max(x, 0)|   (ReLU error)
 *   out[1] = max |x g(x) - |x||                    (doubled form)
 *   out[2] = the float32 x at which out[0] is attained
 *   out[3] = number of float32 values visited in [0, 1]
 */
void oracle_efloat_scan(int T, const double *coef, const double *inv_s, double *out) {
  const uint32_t last = 0x3F800000u; /* bits of 1.0f */
  double best = 0.0, best2 = 0.0, bestx = 0.0;
#pragma omp parallel
  {
    double lb = 0.0, lb2 = 0.0, lx = 0.0;
#pragma omp for schedule(static)
    for (int64_t b = 0; b <= (int64_t)last; ++b) {
      uint32_t bits = (uint32_t)b;
      float xf;
      memcpy(&xf, &bits, sizeof(float));
      double x = (double)xf;
      double g = composite(x, T, coef, inv_s);
      double e = fabs(0.5 * x * (1.0 + g) - x);
      double e2 = fabs(x * g - x);
      if (e > lb) { lb = e; lx = x; }
      if (e2 > lb2) lb2 = e2;
    }
#pragma omp critical
    {
      if (lb > best || (lb == best && lx < bestx)) { best = lb; bestx = lx; }
      if (lb2 > best2) best2 = lb2;
    }
  }
  out[0] = best;
  out[1] = best2;
  out[2] = bestx;
  out[3] = (double)last + 1.0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
