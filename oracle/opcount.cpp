// opcount.cpp -- the oracle's own source (eig3_oracle.c), compiled with its
// binary64 scalar replaced by a type that counts every operation it performs.
//
// TEST INFRASTRUCTURE ONLY (part of the oracle package; nothing of the CUDA
// path).  The counts are the arithmetic of the paper's algorithms as the oracle
// writes them (Algorithms 1, 2, 4, 5 and 6, one rounded operation each, no
// sharing of products): the method's literal operation count, against which
// the kernels' own counts (shared products, fused multiply-adds) are compared.
//
// The value of every operation is the binary64 result the oracle computes, so
// a counted run also returns the oracle's results.  Counted separately:
// additions and subtractions, multiplications, divisions, negations, square
// roots, two-argument arctangents, cosines, comparisons, absolute values.
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

#include <cmath>

namespace {

struct Counts {
  long long add, mul, div, neg, sqrt_, atan2_, cos_, cmp, abs_;
};
thread_local Counts g_counts;

// A binary64 value whose operations are counted.  No conversion back to
// double, so every use of the oracle's arithmetic goes through these operators.
struct Real {
  double v;
  Real() : v(0.0) {}
  Real(double x) : v(x) {}  // NOLINT: literals and array initialisers convert implicitly
};

Real operator+(Real a, Real b) { ++g_counts.add; return Real(a.v + b.v); }
Real operator-(Real a, Real b) { ++g_counts.add; return Real(a.v - b.v); }
Real operator*(Real a, Real b) { ++g_counts.mul; return Real(a.v * b.v); }
Real operator/(Real a, Real b) { ++g_counts.div; return Real(a.v / b.v); }
Real operator-(Real a) { ++g_counts.neg; return Real(-a.v); }
bool operator<(Real a, Real b) { ++g_counts.cmp; return a.v < b.v; }
bool operator>(Real a, Real b) { ++g_counts.cmp; return a.v > b.v; }
bool operator<=(Real a, Real b) { ++g_counts.cmp; return a.v <= b.v; }
bool operator>=(Real a, Real b) { ++g_counts.cmp; return a.v >= b.v; }
bool operator==(Real a, Real b) { ++g_counts.cmp; return a.v == b.v; }
bool operator!=(Real a, Real b) { ++g_counts.cmp; return a.v != b.v; }
Real sqrt(Real a) { ++g_counts.sqrt_; return Real(std::sqrt(a.v)); }
Real atan2(Real y, Real x) { ++g_counts.atan2_; return Real(std::atan2(y.v, x.v)); }
Real cos(Real a) { ++g_counts.cos_; return Real(std::cos(a.v)); }
Real fabs(Real a) { ++g_counts.abs_; return Real(std::fabs(a.v)); }

}  // namespace

// The oracle, unchanged, with its scalar type counted.
#define double Real
#include "eig3_oracle.c"
#undef double

namespace {

void reset() { g_counts = Counts{0, 0, 0, 0, 0, 0, 0, 0, 0}; }

void store(long long *out) {
  const Counts &c = g_counts;
  const long long v[9] = {c.add, c.mul, c.div, c.neg, c.sqrt_, c.atan2_, c.cos_, c.cmp, c.abs_};
  for (int i = 0; i < 9; ++i) out[i] = v[i];
}

void load9(const double *a, Real *A) {
  for (int i = 0; i < 9; ++i) A[i] = Real(a[i]);
}

}  // namespace

extern "C" {

// Counts of one oracle function on the general 9-entry matrix a (row-major):
//   which 0 eigvals, 1 invariants, 2 I1, 3 J2, 4 J3, 5 Delta,
//         6 eigvals_from_invariants (a[0..3] = I1, J2, J3, Delta).
// counts[0..8] = additions (and subtractions), multiplications, divisions,
// negations, square roots, atan2, cos, comparisons, absolute values;
// result[0..3] receives the function's binary64 results (as many as it has).
// Returns 0, or -1 for an unknown `which`.
int eig3o_opcount(int which, const double *a, long long *counts, double *result) {
  Real A[9], out[4];
  load9(a, A);
  reset();
  int nres = 0;
  switch (which) {
    case 0: eig3o_eigvals(A, out); nres = 3; break;
    case 1: eig3o_invariants(A, out); nres = 4; break;
    case 2: out[0] = eig3o_I1(A); nres = 1; break;
    case 3: out[0] = eig3o_J2(A); nres = 1; break;
    case 4: out[0] = eig3o_J3(A); nres = 1; break;
    case 5: out[0] = eig3o_Delta(A); nres = 1; break;
    case 6: eig3o_eigvals_from_invariants(A, out); nres = 3; break;
    default: return -1;
  }
  store(counts);
  for (int i = 0; i < nres; ++i) result[i] = out[i].v;
  return 0;
}

}  // extern "C"
