// eig3_variants.cu -- the invariant evaluations the paper compares the method
// against (Sections J2, J3, Delta and Eigenvalues), in binary64 on the GPU, so
// that their stability can be measured at the scale of the real batches:
//
//   naive         Algorithm 3 (J2 as a monomial sum) and the naive J3
//                 monomial sum, Delta = 4 J2^3 - 27 J3^2;
//   naive tensor  S = A - (tr A / 3) I, J2 = tr(S S)/2, J3 = det S (first-row
//                 cofactor expansion), Delta = 4 J2^3 - 27 J3^2;
//   present       Algorithms 1, 2, 4, 5 (the library's own invariants).
//
// Each is followed by Algorithm 6 (the library's trigonometric step).  The
// comparison variants are evaluated exactly as printed: every monomial left
// to right (coefficient first), the sums left to right, with explicitly
// rounded multiplies and adds (no contraction into FMAs), so they round like
// any other left-to-right binary64 evaluation of the printed formulas.  This
// path is for measurement and comparison, not for use.
#include <cstdint>

#include "eig3_f64.cuh"
#include "eig3_internal.h"
#include "eig3_tile.cuh"

namespace eig3 {
namespace {

__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }

// One monomial c x y (z), multiplied left to right, coefficient first.  A
// subtracted monomial is added with a negative coefficient: negation is exact,
// so s + (-c x y) rounds exactly as s - (c x y).
__device__ __forceinline__ double mono(double c, double x, double y) { return mul(mul(c, x), y); }
__device__ __forceinline__ double mono(double c, double x, double y, double z) {
  return mul(mul(mul(c, x), y), z);
}

__device__ __forceinline__ double discriminant_naive(double J2, double J3) {
  return sub(mul(mul(mul(4.0, J2), J2), J2), mul(mul(27.0, J3), J3));
}

__device__ __forceinline__ Inv invariants_naive(const double (&A)[9]) {
  const double A00 = A[0], A01 = A[1], A02 = A[2], A10 = A[3], A11 = A[4], A12 = A[5],
               A20 = A[6], A21 = A[7], A22 = A[8];
  Inv v;
  v.e = 0;
  v.I1 = add(add(A00, A11), A22);
  // Algorithm 3: 3 J2 as a monomial sum
  double s = mono(1.0, A00, A00);
  s = add(s, mono(-1.0, A00, A11));
  s = add(s, mono(-1.0, A00, A22));
  s = add(s, mono(3.0, A01, A10));
  s = add(s, mono(3.0, A02, A20));
  s = add(s, mono(1.0, A11, A11));
  s = add(s, mono(-1.0, A11, A22));
  s = add(s, mono(3.0, A12, A21));
  s = add(s, mono(1.0, A22, A22));
  v.J2 = __ddiv_rn(s, 3.0);
  // the naive J3: 27 J3 as a monomial sum
  double q = mono(2.0, A00, A00, A00);
  q = add(q, mono(-3.0, A00, A00, A11));
  q = add(q, mono(-3.0, A00, A00, A22));
  q = add(q, mono(9.0, A00, A01, A10));
  q = add(q, mono(9.0, A00, A02, A20));
  q = add(q, mono(-3.0, A00, A11, A11));
  q = add(q, mono(12.0, A00, A11, A22));
  q = add(q, mono(-18.0, A00, A12, A21));
  q = add(q, mono(-3.0, A00, A22, A22));
  q = add(q, mono(9.0, A01, A10, A11));
  q = add(q, mono(-18.0, A01, A10, A22));
  q = add(q, mono(27.0, A01, A12, A20));
  q = add(q, mono(27.0, A02, A10, A21));
  q = add(q, mono(-18.0, A02, A11, A20));
  q = add(q, mono(9.0, A02, A20, A22));
  q = add(q, mono(2.0, A11, A11, A11));
  q = add(q, mono(-3.0, A11, A11, A22));
  q = add(q, mono(9.0, A11, A12, A21));
  q = add(q, mono(-3.0, A11, A22, A22));
  q = add(q, mono(9.0, A12, A21, A22));
  q = add(q, mono(2.0, A22, A22, A22));
  v.J3 = __ddiv_rn(q, 27.0);
  v.D = discriminant_naive(v.J2, v.J3);
  return v;
}

__device__ __forceinline__ Inv invariants_naive_tensor(const double (&A)[9]) {
  Inv v;
  v.e = 0;
  const double tr = add(add(A[0], A[4]), A[8]);
  const double m = __ddiv_rn(tr, 3.0);
  double S[9];
#pragma unroll
  for (int j = 0; j < 9; ++j) S[j] = A[j];
  S[0] = sub(S[0], m);
  S[4] = sub(S[4], m);
  S[8] = sub(S[8], m);
  // tr(S S) = sum_i sum_k S_ik S_ki, inner sums first
  double t = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double sii =
        add(add(mul(S[3 * i], S[i]), mul(S[3 * i + 1], S[3 + i])), mul(S[3 * i + 2], S[6 + i]));
    t = (i == 0) ? sii : add(t, sii);
  }
  v.I1 = tr;
  v.J2 = mul(0.5, t);
  v.J3 = add(sub(mul(S[0], sub(mul(S[4], S[8]), mul(S[5], S[7]))),
                 mul(S[1], sub(mul(S[3], S[8]), mul(S[5], S[6])))),
             mul(S[2], sub(mul(S[3], S[7]), mul(S[4], S[6]))));
  v.D = discriminant_naive(v.J2, v.J3);
  return v;
}

template <int N>
__device__ __forceinline__ void to_general(const double (&a)[N], double (&A)[9]) {
  if constexpr (N == 9) {
#pragma unroll
    for (int j = 0; j < 9; ++j) A[j] = a[j];
  } else {  // (A00, A11, A22, A12, A02, A01)
    A[0] = a[0];
    A[1] = a[5];
    A[2] = a[4];
    A[3] = a[5];
    A[4] = a[1];
    A[5] = a[3];
    A[6] = a[4];
    A[7] = a[3];
    A[8] = a[2];
  }
}

template <int LAYOUT, typename T, int VARIANT>
__global__ void __launch_bounds__(kThreads)
    k_variant(const T *__restrict__ A, int64_t n, double *__restrict__ inv, T *__restrict__ lam) {
  constexpr int N = (LAYOUT == EIG3_GENERAL9) ? 9 : 6;
  __shared__ __align__(16) T sA[2][kTile * N];
  for_each_row<N, T>(A, n, sA, [&](int64_t i, const T *row) {
    double a[N];
#pragma unroll
    for (int j = 0; j < N; ++j) a[j] = (double)row[j];
    Inv v;
    if constexpr (VARIANT == EIG3_VARIANT_PRESENT) {
      if constexpr (LAYOUT == EIG3_GENERAL9) {
        v = invariants_general(a);
      } else {
        v = invariants_sym(a);
      }
    } else {
      double G[9];
      to_general<N>(a, G);
      v = (VARIANT == EIG3_VARIANT_NAIVE) ? invariants_naive(G) : invariants_naive_tensor(G);
    }
    if (inv) {
      double *o = inv + 4 * i;
      o[0] = v.I1;
      o[1] = v.e == 0 ? v.J2 : ldexp(v.J2, 2 * v.e);  // back from 2^-e A
      o[2] = v.e == 0 ? v.J3 : ldexp(v.J3, 3 * v.e);
      o[3] = v.e == 0 ? v.D : ldexp(v.D, 6 * v.e);
    }
    if (lam) {
      const Eig e = eigvals_from_inv(v);
      lam[3 * i + 0] = (T)e.l1;
      lam[3 * i + 1] = (T)e.l2;
      lam[3 * i + 2] = (T)e.l3;
    }
  });
}

template <int LAYOUT, typename T, int VARIANT>
cudaError_t launch3(const void *A, int64_t n, double *inv, void *lam, cudaStream_t s) {
  auto k = k_variant<LAYOUT, T, VARIANT>;
  k<<<grid_for((const void *)k, kThreads, 0, n), kThreads, 0, s>>>((const T *)A, n, inv, (T *)lam);
  return cudaGetLastError();
}

template <int LAYOUT, typename T>
cudaError_t launch2(const void *A, int variant, int64_t n, double *inv, void *lam,
                    cudaStream_t s) {
  switch (variant) {
    case EIG3_VARIANT_NAIVE: return launch3<LAYOUT, T, EIG3_VARIANT_NAIVE>(A, n, inv, lam, s);
    case EIG3_VARIANT_NAIVE_TENSOR:
      return launch3<LAYOUT, T, EIG3_VARIANT_NAIVE_TENSOR>(A, n, inv, lam, s);
    default: return launch3<LAYOUT, T, EIG3_VARIANT_PRESENT>(A, n, inv, lam, s);
  }
}

}  // namespace

cudaError_t launch_variant_f64(const void *A, int layout, int dtype, int variant, int64_t n,
                               double *inv, void *lam, cudaStream_t s) {
  if (layout == EIG3_GENERAL9)
    return dtype == EIG3_F64 ? launch2<EIG3_GENERAL9, double>(A, variant, n, inv, lam, s)
                             : launch2<EIG3_GENERAL9, float>(A, variant, n, inv, lam, s);
  return dtype == EIG3_F64 ? launch2<EIG3_SYM6, double>(A, variant, n, inv, lam, s)
                           : launch2<EIG3_SYM6, float>(A, variant, n, inv, lam, s);
}

}  // namespace eig3
