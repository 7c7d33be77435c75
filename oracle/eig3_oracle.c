/*
 * eig3_oracle.c -- plain, slow, scalar FP64 oracle for the closed-form 3x3
 * eigenvalue method of Habera & Zilian, "Numerically stable evaluation of
 * closed-form expressions for eigenvalues of 3x3 matrices" (arXiv 2511.00292).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA library is checked against.  It shares no code, header, constant or
 * helper with the CUDA path, and the product path never loads it.  Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark use it.
 *
 * Rules followed here:
 *   - every operation is one IEEE-754 binary64 operation, compiled with
 *     -ffp-contract=off (no FMA contraction), evaluated in the order the
 *     paper writes it (left to right for sums and products);
 *   - divisions by the integers 3, 6 and 27 are real divisions;
 *   - no blocking, fusion, common-subexpression rewriting or reordering.
 *
 * Matrices are 9 doubles, row-major, A[3*i+j] = A_ij with 0-based indices as
 * in the paper (Section "Invariant I1").  Symmetric 6-entry inputs are in the
 * order (A00, A11, A22, A12, A02, A01) and are expanded to 9 entries first.
 *
 * Readings of the paper that this file takes (each also listed in the design
 * notes):
 *   R1  Algorithm 5, r10: the second term is +M02*M21*d2.  As printed
 *       (-M02*M21*d2) the 14-term sum is not the discriminant 4J2^3-27J3^2;
 *       with the sign flipped it is an exact polynomial identity.
 *   R2  Algorithm 6: phi = arctan(t) with t = sqrt(27 Delta)/(27 J3) is read
 *       as phi = atan2(sqrt(27 Delta), 27 J3), in [0, pi].  A one-argument
 *       arctan returns phi - pi whenever J3 < 0, which breaks the ordering
 *       lambda_1 <= lambda_2 <= lambda_3 the paper states in the introduction.
 *   R3  Negative computed J2 or Delta (possible for nonsymmetric input) are
 *       clamped to zero before the square roots; the paper is silent.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <pthread.h>

#define A00 A[0]
#define A01 A[1]
#define A02 A[2]
#define A10 A[3]
#define A11 A[4]
#define A12 A[5]
#define A20 A[6]
#define A21 A[7]
#define A22 A[8]

/* ---------------------------------------------------------------------- */
/* Layout helper                                                           */
/* ---------------------------------------------------------------------- */

/* Expand the symmetric order (A00, A11, A22, A12, A02, A01) to row-major 9. */
void eig3o_sym6_to_general9(const double *s, double *A) {
  A[0] = s[0]; A[1] = s[5]; A[2] = s[4];
  A[3] = s[5]; A[4] = s[1]; A[5] = s[3];
  A[6] = s[4]; A[7] = s[3]; A[8] = s[2];
}

/* ---------------------------------------------------------------------- */
/* Algorithm 1: I1 = A00 + A11 + A22 (Section "Invariant I1").             */
/* ---------------------------------------------------------------------- */
double eig3o_I1(const double *A) { return (A00 + A11) + A22; }

/* ---------------------------------------------------------------------- */
/* Algorithm 2: stable J2 (Section "Invariant J2").                        */
/*   d0 = A00-A11, d1 = A00-A22, d2 = A11-A22                              */
/*   offdiag = A01 A10 + A02 A20 + A12 A21                                 */
/*   diag    = (d0^2 + d1^2 + d2^2) / 6                                    */
/*   J2      = diag + offdiag                                              */
/* ---------------------------------------------------------------------- */
double eig3o_J2(const double *A) {
  double d0 = A00 - A11;
  double d1 = A00 - A22;
  double d2 = A11 - A22;
  double offdiag = (A01 * A10 + A02 * A20) + A12 * A21;
  double diag = ((d0 * d0 + d1 * d1) + d2 * d2) / 6.0;
  return diag + offdiag;
}

/* ---------------------------------------------------------------------- */
/* Algorithm 4: stable J3 (Section "Invariant J3").                        */
/*   t1 = d1 + d2, t2 = d0 - d2, t3 = -d0 - d1                             */
/*   offdiag = A01 A12 A20 + A02 A10 A21                                   */
/*   mixed   = (A01 A10 t1 + A02 A20 t2 + A12 A21 t3) / 3                  */
/*   diag    = t1 t2 t3 / 27                                               */
/*   J3      = offdiag + mixed - diag                                      */
/* ---------------------------------------------------------------------- */
double eig3o_J3(const double *A) {
  double d0 = A00 - A11;
  double d1 = A00 - A22;
  double d2 = A11 - A22;
  double t1 = d1 + d2;
  double t2 = d0 - d2;
  double t3 = -d0 - d1;
  double offdiag = A01 * A12 * A20 + A02 * A10 * A21;
  double mixed = ((A01 * A10 * t1 + A02 * A20 * t2) + A12 * A21 * t3) / 3.0;
  double diag = t1 * t2 * t3 / 27.0;
  return (offdiag + mixed) - diag;
}

/* ---------------------------------------------------------------------- */
/* Algorithm 5: discriminant as the 14-term sum of products                */
/* (Section "Discriminant Delta", Eq. sum-of-products).  M is A or A^T,    */
/* addressed through the element accessor so that dx(A^T) uses            */
/* M_ij = A_ji with the same diagonal differences.  Reading R1 applies to  */
/* r10.                                                                    */
/* ---------------------------------------------------------------------- */
static void dx(const double *A, int transpose, double d0, double d1, double d2,
               double *r) {
#define M(i, j) (transpose ? A[3 * (j) + (i)] : A[3 * (i) + (j)])
  double M01 = M(0, 1), M02 = M(0, 2), M10 = M(1, 0);
  double M12 = M(1, 2), M20 = M(2, 0), M21 = M(2, 1);
#undef M
  r[0] = M01 * M12 * M20 - M02 * M10 * M21;
  r[1] = (-M01 * M02 * d2 + M01 * M01 * M12) - M02 * M02 * M21;
  r[2] = (M01 * M21 * d1 - M01 * M01 * M20) + M02 * M21 * M21;
  r[3] = (M02 * M12 * d0 + M01 * M12 * M12) - M02 * M02 * M10;
  r[4] = (M01 * M12 * d1 - M01 * M02 * M10) + M02 * M12 * M21;
  r[5] = (M02 * M21 * d0 - M01 * M02 * M20) + M01 * M12 * M21;
  r[6] = (-M02 * M10 * d2 + M01 * M10 * M12) - M02 * M12 * M20;
  r[7] = ((M12 * d0 * d1 - M02 * M10 * d1) + M01 * M10 * M12) - M12 * M12 * M21;
  r[8] = ((M12 * d0 * d1 - M02 * M10 * d0) + M02 * M12 * M20) - M12 * M12 * M21;
  r[9] = ((M01 * d1 * d2 + M02 * M21 * d2) + M01 * M02 * M20) - M01 * M01 * M10;
  r[10] = ((M01 * d1 * d2 + M02 * M21 * d1) + M01 * M12 * M21) - M01 * M01 * M10;
  r[11] = ((-M02 * d0 * d2 + M01 * M12 * d0) + M02 * M12 * M21) - M02 * M02 * M20;
  r[12] = ((M02 * d0 * d2 + M01 * M12 * d2) - M01 * M02 * M10) + M02 * M02 * M20;
  r[13] = ((d0 * d1 * d2 - M01 * M10 * d0) + M02 * M20 * d1) - M12 * M21 * d2;
}

static const double W14[14] = {9, 6, 6, 6, 8, 8, 8, 2, 2, 2, 2, 2, 2, 1};

double eig3o_Delta(const double *A) {
  double d0 = A00 - A11;
  double d1 = A00 - A22;
  double d2 = A11 - A22;
  double u[14], v[14];
  dx(A, 0, d0, d1, d2, u);
  dx(A, 1, d0, d1, d2, v);
  double s = 0.0;
  for (int i = 0; i < 14; ++i) s = s + W14[i] * u[i] * v[i];
  return s;
}

/* All four invariants, out = (I1, J2, J3, Delta). */
void eig3o_invariants(const double *A, double *out) {
  out[0] = eig3o_I1(A);
  out[1] = eig3o_J2(A);
  out[2] = eig3o_J3(A);
  out[3] = eig3o_Delta(A);
}

/* ---------------------------------------------------------------------- */
/* Algorithm 6: eigenvalues from (I1, J2, J3, Delta) (Section              */
/* "Eigenvalues", with the trigonometric formula of the introduction):     */
/*   phi      = atan2(sqrt(27 Delta), 27 J3)            (reading R2)       */
/*   lambda_k = (I1 + 2 sqrt(3 J2) cos((phi + 2 pi k)/3)) / 3, k = 1,2,3   */
/* J2 and Delta are clamped at zero first (reading R3).  The result is     */
/* ascending: lambda_1 <= lambda_2 <= lambda_3.                            */
/* ---------------------------------------------------------------------- */
static const double TWO_PI = 6.283185307179586476925286766559;

void eig3o_eigvals_from_invariants(const double *inv, double *lam) {
  double I1 = inv[0], J2 = inv[1], J3 = inv[2], D = inv[3];
  if (J2 < 0.0) J2 = 0.0;
  if (D < 0.0) D = 0.0;
  double phi = atan2(sqrt(27.0 * D), 27.0 * J3);
  double rad = 2.0 * sqrt(3.0 * J2);
  for (int k = 1; k <= 3; ++k)
    lam[k - 1] = (I1 + rad * cos((phi + TWO_PI * k) / 3.0)) / 3.0;
}

void eig3o_eigvals(const double *A, double *lam) {
  double inv[4];
  eig3o_invariants(A, inv);
  eig3o_eigvals_from_invariants(inv, lam);
}

/* ---------------------------------------------------------------------- */
/* Naive variants, used only by tests that reproduce the paper's           */
/* comparison: Algorithm 3 (naive J2, monomial sum), the naive J3 monomial */
/* sum, and Delta = 4 J2^3 - 27 J3^2 from them (Sections J2, J3, Delta).   */
/* ---------------------------------------------------------------------- */
double eig3o_J2_naive(const double *A) {
  return (A00 * A00 - A00 * A11 - A00 * A22 + 3.0 * A01 * A10 + 3.0 * A02 * A20 +
          A11 * A11 - A11 * A22 + 3.0 * A12 * A21 + A22 * A22) / 3.0;
}

double eig3o_J3_naive(const double *A) {
  double s = 2.0 * A00 * A00 * A00 - 3.0 * A00 * A00 * A11 - 3.0 * A00 * A00 * A22 +
             9.0 * A00 * A01 * A10 + 9.0 * A00 * A02 * A20 - 3.0 * A00 * A11 * A11 +
             12.0 * A00 * A11 * A22 - 18.0 * A00 * A12 * A21 - 3.0 * A00 * A22 * A22 +
             9.0 * A01 * A10 * A11 - 18.0 * A01 * A10 * A22 + 27.0 * A01 * A12 * A20 +
             27.0 * A02 * A10 * A21 - 18.0 * A02 * A11 * A20 + 9.0 * A02 * A20 * A22 +
             2.0 * A11 * A11 * A11 - 3.0 * A11 * A11 * A22 + 9.0 * A11 * A12 * A21 -
             3.0 * A11 * A22 * A22 + 9.0 * A12 * A21 * A22 + 2.0 * A22 * A22 * A22;
  return s / 27.0;
}

void eig3o_invariants_naive(const double *A, double *out) {
  out[0] = eig3o_I1(A);
  out[1] = eig3o_J2_naive(A);
  out[2] = eig3o_J3_naive(A);
  out[3] = 4.0 * out[1] * out[1] * out[1] - 27.0 * out[2] * out[2];
}

/* ---------------------------------------------------------------------- */
/* comparison: the "naive tensor" invariants of Sections J2, J3 and Delta:  */
/*   S = A - (tr(A)/3) I,  J2 = tr(S S)/2,  J3 = det S,                     */
/*   Delta = 4 J2^3 - 27 J3^2.                                              */
/* tr(S S) = sum_i (S S)_ii with (S S)_ii = sum_k S_ik S_ki (a matrix       */
/* product and its trace); det S by cofactor expansion along the first     */
/* row (the paper takes numpy's LU-based determinant here).                */
/* ---------------------------------------------------------------------- */
void eig3o_invariants_naive_tensor(const double *A, double *out) {
  double tr = (A00 + A11) + A22;
  double m = tr / 3.0;
  double S[9];
  for (int j = 0; j < 9; ++j) S[j] = A[j];
  S[0] = S[0] - m;
  S[4] = S[4] - m;
  S[8] = S[8] - m;
  double t = 0.0;
  for (int i = 0; i < 3; ++i) {
    double sii = (S[3 * i + 0] * S[0 * 3 + i] + S[3 * i + 1] * S[1 * 3 + i]) + S[3 * i + 2] * S[2 * 3 + i];
    t = (i == 0) ? sii : t + sii;
  }
  double J2 = 0.5 * t;
  double J3 = S[0] * (S[4] * S[8] - S[5] * S[7]) - S[1] * (S[3] * S[8] - S[5] * S[6]) +
              S[2] * (S[3] * S[7] - S[4] * S[6]);
  out[0] = tr;
  out[1] = J2;
  out[2] = J3;
  out[3] = 4.0 * J2 * J2 * J2 - 27.0 * J3 * J3;
}

/* ---------------------------------------------------------------------- */
/* Eigenvalue gradient, plain definition (Section 1: E_k^T = d lambda_k/dA).*/
/* For a simple eigenvalue lambda with right eigenvector r ((A-lambda I)r=0)*/
/* and left eigenvector l (l^T (A-lambda I) = 0),                          */
/*   d lambda / dA_ij = l_i r_j / (l^T r).                                 */
/* r is the largest cross product of two rows of A - lambda I; l the       */
/* largest cross product of two columns.  This is deliberately not the     */
/* invariant chain rule that the CUDA adjoint uses.                        */
/* ---------------------------------------------------------------------- */
static void cross3(const double *a, const double *b, double *c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

static double norm2_3(const double *a) { return a[0] * a[0] + a[1] * a[1] + a[2] * a[2]; }

/* Null vector of the 3x3 matrix M (row-major) from its rows, or of M^T. */
static void null_vector(const double *M, int use_columns, double *out) {
  double v[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) v[i][j] = use_columns ? M[3 * j + i] : M[3 * i + j];
  double c[3][3];
  cross3(v[0], v[1], c[0]);
  cross3(v[0], v[2], c[1]);
  cross3(v[1], v[2], c[2]);
  int best = 0;
  double bn = norm2_3(c[0]);
  for (int i = 1; i < 3; ++i) {
    double n = norm2_3(c[i]);
    if (n > bn) { bn = n; best = i; }
  }
  for (int j = 0; j < 3; ++j) out[j] = c[best][j];
}

/* d lambda_k / dA for k = 0,1,2 (ascending lambda), 27 doubles: G[k*9 + 3i + j]. */
void eig3o_eigval_jacobians(const double *A, double *G) {
  double lam[3];
  eig3o_eigvals(A, lam);
  for (int k = 0; k < 3; ++k) {
    double M[9];
    for (int i = 0; i < 9; ++i) M[i] = A[i];
    M[0] = M[0] - lam[k];
    M[4] = M[4] - lam[k];
    M[8] = M[8] - lam[k];
    double r[3], l[3];
    null_vector(M, 0, r);
    null_vector(M, 1, l);
    double lr = l[0] * r[0] + l[1] * r[1] + l[2] * r[2];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) G[9 * k + 3 * i + j] = l[i] * r[j] / lr;
  }
}

/* Gradient of L = sum_k gbar_k lambda_k with respect to the 9 entries. */
void eig3o_eigvals_grad(const double *A, const double *gbar, double *gA) {
  double G[27];
  eig3o_eigval_jacobians(A, G);
  for (int i = 0; i < 9; ++i)
    gA[i] = gbar[0] * G[i] + gbar[1] * G[9 + i] + gbar[2] * G[18 + i];
}

/* ---------------------------------------------------------------------- */
/* First-order stability bounds with C = 1, Frobenius norm, unit roundoff  */
/* u (the lines drawn in the paper's error figures):                       */
/*   I1:     ||A|| u                                    (Section I1)       */
/*   J2:     ||dev A||^2 u                              (Theorem, J2)      */
/*   J3:     ||dev cof dev A|| ||dev A|| u              (Lemma, J3)        */
/*   Delta:  ||dev(12 J2^2 A^T - 54 J3 cof dev A)|| ||dev A|| u            */
/*   lambda: kappa ||A|| u                              (Bauer-Fike lemma) */
/* out = (b_I1, b_J2, b_J3, b_Delta, b_lambda).                            */
/* ---------------------------------------------------------------------- */
static double frob(const double *M) {
  double s = 0.0;
  for (int i = 0; i < 9; ++i) s = s + M[i] * M[i];
  return sqrt(s);
}

static void dev9(const double *M, double *S) {
  double tr3 = ((M[0] + M[4]) + M[8]) / 3.0;
  for (int i = 0; i < 9; ++i) S[i] = M[i];
  S[0] = S[0] - tr3;
  S[4] = S[4] - tr3;
  S[8] = S[8] - tr3;
}

static void cof9(const double *S, double *C) {
  C[0] = S[4] * S[8] - S[5] * S[7];
  C[1] = S[5] * S[6] - S[3] * S[8];
  C[2] = S[3] * S[7] - S[4] * S[6];
  C[3] = S[2] * S[7] - S[1] * S[8];
  C[4] = S[0] * S[8] - S[2] * S[6];
  C[5] = S[1] * S[6] - S[0] * S[7];
  C[6] = S[1] * S[5] - S[2] * S[4];
  C[7] = S[2] * S[3] - S[0] * S[5];
  C[8] = S[0] * S[4] - S[1] * S[3];
}

void eig3o_bounds(const double *A, double kappa, double u, double *out) {
  double S[9], C[9], dC[9], T[9], dT[9];
  dev9(A, S);
  cof9(S, C);
  dev9(C, dC);
  double nA = frob(A), nS = frob(S);
  double J2 = eig3o_J2(A), J3 = eig3o_J3(A);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      T[3 * i + j] = 12.0 * J2 * J2 * A[3 * j + i] - 54.0 * J3 * C[3 * i + j];
  dev9(T, dT);
  out[0] = nA * u;
  out[1] = nS * nS * u;
  out[2] = frob(dC) * nS * u;
  out[3] = frob(dT) * nS * u;
  out[4] = kappa * nA * u;
}

/* ---------------------------------------------------------------------- */
/* Mohr-Coulomb yield function (Section "Application"):                    */
/*   f = (1/S_yc) ((m+1)/2) max_{i<j} (|s_i - s_j| + K (s_i + s_j)) - 1,    */
/*   K = (m-1)/(m+1), s_k the principal stresses (the eigenvalues).         */
/* The gradient is d f/d s_k of the maximising pair chained with           */
/* d lambda_k / dA (eigenvector form).  out_grad may be NULL.              */
/* ---------------------------------------------------------------------- */
double eig3o_mohr_coulomb(const double *A, double s_yc, double m, double *out_grad) {
  double s[3];
  eig3o_eigvals(A, s);
  double K = (m - 1.0) / (m + 1.0);
  double best = -INFINITY;
  int bi = 0, bj = 1;
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j) {
      double v = fabs(s[i] - s[j]) + K * (s[i] + s[j]);
      if (v > best) { best = v; bi = i; bj = j; }
    }
  double c = (m + 1.0) / 2.0 / s_yc;
  if (out_grad) {
    double g[3] = {0.0, 0.0, 0.0};
    double sg = (s[bi] - s[bj] >= 0.0) ? 1.0 : -1.0;   /* d|s_i - s_j| */
    g[bi] = c * (sg + K);
    g[bj] = c * (-sg + K);
    eig3o_eigvals_grad(A, g, out_grad);
  }
  return c * best - 1.0;
}

/* ---------------------------------------------------------------------- */
/* Batched entry points (layout 0 = 9 entries, 1 = symmetric 6 entries).   */
/* ---------------------------------------------------------------------- */
static void load(const double *X, int64_t i, int layout, double *A) {
  if (layout == 0) {
    for (int j = 0; j < 9; ++j) A[j] = X[9 * i + j];
  } else {
    eig3o_sym6_to_general9(X + 6 * i, A);
  }
}

void eig3o_invariants_batch(const double *X, int64_t n, int layout, double *out) {
  double A[9];
  for (int64_t i = 0; i < n; ++i) {
    load(X, i, layout, A);
    eig3o_invariants(A, out + 4 * i);
  }
}

void eig3o_invariants_naive_batch(const double *X, int64_t n, int layout, double *out) {
  double A[9];
  for (int64_t i = 0; i < n; ++i) {
    load(X, i, layout, A);
    eig3o_invariants_naive(A, out + 4 * i);
  }
}

void eig3o_invariants_naive_tensor_batch(const double *X, int64_t n, int layout, double *out) {
  double A[9];
  for (int64_t i = 0; i < n; ++i) {
    load(X, i, layout, A);
    eig3o_invariants_naive_tensor(A, out + 4 * i);
  }
}

void eig3o_eigvals_naive_tensor_batch(const double *X, int64_t n, int layout, double *lam) {
  double A[9], inv[4];
  for (int64_t i = 0; i < n; ++i) {
    load(X, i, layout, A);
    eig3o_invariants_naive_tensor(A, inv);
    eig3o_eigvals_from_invariants(inv, lam + 3 * i);
  }
}

void eig3o_eigvals_batch(const double *X, int64_t n, int layout, double *lam) {
  double A[9];
  for (int64_t i = 0; i < n; ++i) {
    load(X, i, layout, A);
    eig3o_eigvals(A, lam + 3 * i);
  }
}

void eig3o_eigvals_naive_batch(const double *X, int64_t n, int layout, double *lam) {
  double A[9], inv[4];
  for (int64_t i = 0; i < n; ++i) {
    load(X, i, layout, A);
    eig3o_invariants_naive(A, inv);
    eig3o_eigvals_from_invariants(inv, lam + 3 * i);
  }
}

/* Gradient with respect to the stored entries: 9 per matrix for layout 0;
 * for the symmetric layout the stored off-diagonal entry stands for both
 * A_ij and A_ji, so its gradient is G_ij + G_ji. */
void eig3o_eigvals_grad_batch(const double *X, const double *gbar, int64_t n, int layout,
                              double *gX) {
  double A[9], G[9];
  for (int64_t i = 0; i < n; ++i) {
    load(X, i, layout, A);
    eig3o_eigvals_grad(A, gbar + 3 * i, G);
    if (layout == 0) {
      for (int j = 0; j < 9; ++j) gX[9 * i + j] = G[j];
    } else {
      double *g = gX + 6 * i;
      g[0] = G[0];
      g[1] = G[4];
      g[2] = G[8];
      g[3] = G[5] + G[7];
      g[4] = G[2] + G[6];
      g[5] = G[1] + G[3];
    }
  }
}

/* d lambda_k / dA for every matrix: 27 doubles per matrix, k-major, row-major
 * 3x3 blocks (with respect to the 9 entries of the expanded matrix). */
void eig3o_eigval_jacobians_batch(const double *X, int64_t n, int layout, double *out) {
  double A[9];
  for (int64_t i = 0; i < n; ++i) {
    load(X, i, layout, A);
    eig3o_eigval_jacobians(A, out + 27 * i);
  }
}

/* Mohr-Coulomb value per matrix, and its gradient with respect to the stored
 * entries (layout as eig3o_eigvals_grad_batch) when gX is not NULL. */
void eig3o_mohr_coulomb_batch(const double *X, int64_t n, int layout, double s_yc, double m,
                              double *f, double *gX) {
  double A[9], G[9];
  for (int64_t i = 0; i < n; ++i) {
    load(X, i, layout, A);
    f[i] = eig3o_mohr_coulomb(A, s_yc, m, gX ? G : 0);
    if (!gX) continue;
    if (layout == 0) {
      for (int j = 0; j < 9; ++j) gX[9 * i + j] = G[j];
    } else {
      double *g = gX + 6 * i;
      g[0] = G[0];
      g[1] = G[4];
      g[2] = G[8];
      g[3] = G[5] + G[7];
      g[4] = G[2] + G[6];
      g[5] = G[1] + G[3];
    }
  }
}

void eig3o_bounds_batch(const double *X, const double *kappa, int64_t n, int layout, double u,
                        double *out) {
  double A[9];
  for (int64_t i = 0; i < n; ++i) {
    load(X, i, layout, A);
    eig3o_bounds(A, kappa ? kappa[i] : 1.0, u, out + 5 * i);
  }
}

/* Threaded forward, for timing the oracle on the host cores: contiguous
 * chunks, one POSIX thread each.  Returns the number of threads used. */
typedef struct {
  const double *X;
  int64_t lo, hi;
  int layout;
  double *lam;
} eig3o_job;

static void *eig3o_worker(void *p) {
  eig3o_job *j = (eig3o_job *)p;
  double A[9];
  for (int64_t i = j->lo; i < j->hi; ++i) {
    load(j->X, i, j->layout, A);
    eig3o_eigvals(A, j->lam + 3 * i);
  }
  return 0;
}

int eig3o_eigvals_batch_mt(const double *X, int64_t n, int layout, double *lam, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 1024) nthreads = 1024;
  pthread_t tid[1024];
  eig3o_job jobs[1024];
  int started = 0;
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].X = X;
    jobs[t].lo = n * t / nthreads;
    jobs[t].hi = n * (t + 1) / nthreads;
    jobs[t].layout = layout;
    jobs[t].lam = lam;
    if (pthread_create(&tid[t], 0, eig3o_worker, &jobs[t]) == 0) {
      ++started;
    } else {
      eig3o_worker(&jobs[t]);
      tid[t] = 0;
    }
  }
  for (int t = 0; t < nthreads; ++t)
    if (tid[t]) pthread_join(tid[t], 0);
  return started > 0 ? started : 1;
}
