// eig3_guard.cu -- the guarded binary64 path (EIG3_PREC_F64_GUARDED) for
// general matrices whose eigenbasis may be ill-conditioned.
//
// Sections J3, Delta and Eigenvalues find that Algorithms 4 and 5 (and so the
// eigenvalues) meet their first-order bounds for well-conditioned or
// orthogonal eigenbases but not for nearly singular ones, where an iterative
// method (LAPACK DGEEV) does.  The error comes from cancellation in the sums
// of products that form J3 and Delta: for an eigenbasis of condition kappa
// the terms exceed Delta by up to about kappa^6 times the eigenvalue scale,
// beyond what even doubled working precision resolves near a repeated
// eigenvalue.  The guard therefore switches method instead of precision:
//
//   1. evaluate the invariants as the binary64 path does;
//   2. measure the departure from normality of S = dev(A),
//        rho = ||S||_F^2 / tr(S^2) = ||S||_F^2 / (2 J2)  >= 1,
//      equal to 1 exactly for normal S (Schur), growing like kappa(V)^2 for
//      an ill-conditioned eigenbasis V (measured: rho <= 0.46 kappa^2);
//   3. when rho > 32 (or J2 <= 0 while S != 0), compute the eigenvalues by
//      the shifted QR algorithm on the 3x3 matrix in this thread: one plane
//      rotation to Hessenberg form, QR steps with the Wilkinson shift (the
//      eigenvalue of the trailing 2x2 block nearer its last diagonal entry)
//      until a subdiagonal entry is negligible, and the remaining 2x2 block
//      in closed form.  Orthogonal similarity transformations make this
//      backward stable, so its error follows the first-order bound
//      kappa ||A|| u, as the paper reports for DGEEV.
//
// Matrices with rho <= 32 get exactly the binary64 path's results: up to
// there that path stays within its bound (measured maximum 1.7 bounds for
// rho <= 64, against the tolerance of 8).  Symmetric matrices have rho = 1
// and are never switched; their launches use the binary64 kernels directly.
// The adjoint inputs (r, sigma1, sigma2) of a switched matrix follow from its
// eigenvalue gaps g12 = lambda2 - lambda1, g23 = lambda3 - lambda2:
//   r^2 = g12^2 + g12 g23 + g23^2, sigma1 = (sqrt3/2) g12 / r,
//   sigma2 = (sqrt3/2) g23 / r
// (the gaps of the trigonometric formula are (2r/sqrt3) sigma1 and
// (2r/sqrt3) sigma2).
#include <cstdint>

#include "eig3_f64.cuh"
#include "eig3_internal.h"
#include "eig3_stats.cuh"
#include "eig3_tile.cuh"

namespace eig3 {
namespace {

constexpr double kGuardRho = 32.0;
constexpr int kQrMaxSteps = 64;

// ||dev A||_F^2 = (d0^2 + d1^2 + d2^2)/3 + sum of the squared off-diagonal
// entries, in the scaled units of v (2^-e A); compared with rho * 2 J2.
__device__ __forceinline__ bool needs_switch(const double (&a)[9], const Inv &v) {
  const double sc = v.e == 0 ? 1.0 : pow2d(-v.e);
  const double d0 = (a[0] - a[4]) * sc, d1 = (a[0] - a[8]) * sc, d2 = (a[4] - a[8]) * sc;
  double off = 0.0;
#pragma unroll
  for (int j = 1; j < 8; ++j) {
    if (j == 4) continue;
    const double x = a[j] * sc;
    off = fma(x, x, off);
  }
  const double nd2 = fma(fma(d0, d0, fma(d1, d1, d2 * d2)), kInv3, off);
  return !(nd2 <= (2.0 * kGuardRho) * v.J2);
}

// Eigenvalues of the 2x2 block [[a, b], [c, d]]: with p = (a - d)/2 they are
// d + t for the roots t of t^2 - 2 p t - b c = 0; the larger-magnitude root
// t1 = p + sign(p) sqrt(p^2 + b c) has no cancellation and t2 = -b c / t1.  A
// negative discriminant (a complex pair, or rounding at a repeated real
// eigenvalue) is clamped to 0.
__device__ __forceinline__ void eig2x2(double a, double b, double c, double d, double &l1,
                                       double &l2) {
  const double p = 0.5 * (a - d);
  const double bc = b * c;
  const double t = p + copysign(sqrt(fmax(fma(p, p, bc), 0.0)), p);
  if (t == 0.0) {
    l1 = l2 = d;
    return;
  }
  l1 = d + t;
  l2 = d - bc / t;
}

// Plane rotation (c, s) with c x + s y = sqrt(x^2 + y^2) and -s x + c y = 0.
// The QR iteration runs on the matrix scaled to entries below 2 in magnitude,
// so x^2 + y^2 cannot overflow; below the normal range it is treated as 0.
__device__ __forceinline__ void rotation(double x, double y, double &c, double &s) {
  const double r2 = fma(x, x, y * y);
  const bool ok = r2 >= 2.2250738585072014e-308;
  const double t = rsqrt(ok ? r2 : 1.0);
  c = ok ? x * t : 1.0;
  s = ok ? y * t : 0.0;
}

// (p, q) <- (c p + s q, -s p + c q): the rotation applied to two entries of a
// column (rows p, q) or, for X G^T, to two entries of a row (columns p, q).
__device__ __forceinline__ void rot(double c, double s, double &p, double &q) {
  const double t = c * p + s * q;
  q = c * q - s * p;
  p = t;
}

__device__ __forceinline__ void sort3(double &x, double &y, double &z) {
  double t;
  if (y < x) { t = x; x = y; y = t; }
  if (z < y) { t = y; y = z; z = t; }
  if (y < x) { t = x; x = y; y = t; }
}

// Ascending eigenvalues by the shifted QR algorithm (see the file comment),
// with the adjoint inputs from the gaps.  At most kQrMaxSteps QR steps;
// non-finite input, or no convergence, gives NaNs.  Not inlined: only the
// switched matrices call it, and the common path keeps its compact code.
__device__ __noinline__ Eig eigvals_qr(const double (&a)[9]) {
  // exact power-of-two scaling: the largest magnitude into [1, 2)
  int hm = hi_abs(a[0]);
#pragma unroll
  for (int j = 1; j < 9; ++j) hm = max(hm, hi_abs(a[j]));
  const int e = min(max(hm >> 20, 1), 2045) - 1023;
  const double sc = pow2d(-e);
  double h00 = a[0] * sc, h01 = a[1] * sc, h02 = a[2] * sc;
  double h10 = a[3] * sc, h11 = a[4] * sc, h12 = a[5] * sc;
  double h20 = a[6] * sc, h21 = a[7] * sc, h22 = a[8] * sc;
  if (h20 != 0.0) {  // Hessenberg form: G H G^T with G acting on rows/columns 1, 2
    double c, s;
    rotation(h10, h20, c, s);
    rot(c, s, h10, h20);
    rot(c, s, h11, h21);
    rot(c, s, h12, h22);
    rot(c, s, h01, h02);
    rot(c, s, h11, h12);
    rot(c, s, h21, h22);
    h20 = 0.0;
  }
  const double u = 1.1102230246251565e-16;  // 2^-53
  double l1 = __longlong_as_double(0x7ff8000000000000ll), l2 = l1, l3 = l1;
  for (int step = 0; step < kQrMaxSteps; ++step) {
    if (fabs(h21) <= u * (fabs(h11) + fabs(h22))) {  // h22 has converged
      l3 = h22;
      eig2x2(h00, h01, h10, h11, l1, l2);
      break;
    }
    if (fabs(h10) <= u * (fabs(h00) + fabs(h11))) {  // h00 has converged
      l1 = h00;
      eig2x2(h11, h12, h21, h22, l2, l3);
      break;
    }
    double m1, m2;
    eig2x2(h11, h12, h21, h22, m1, m2);
    double sg = fabs(m1 - h22) < fabs(m2 - h22) ? m1 : m2;
    if (step > 0 && step % 16 == 0) sg = h22 + fabs(h21);  // breaks a rare cycle
    // H - sg I = Q R with Q^T = G2 G1, then H <- R Q + sg I = R G1^T G2^T + sg I
    double b00 = h00 - sg, b01 = h01, b02 = h02;
    double b10 = h10, b11 = h11 - sg, b12 = h12;
    double b21 = h21, b22 = h22 - sg;
    double c1, s1, c2, s2;
    rotation(b00, b10, c1, s1);
    rot(c1, s1, b00, b10);
    rot(c1, s1, b01, b11);
    rot(c1, s1, b02, b12);
    rotation(b11, b21, c2, s2);
    rot(c2, s2, b11, b21);
    rot(c2, s2, b12, b22);
    // R is upper triangular: b00 b01 b02 / 0 b11 b12 / 0 0 b22
    double r10 = 0.0, r21 = 0.0;
    rot(c1, s1, b00, b01);  // columns 0, 1 of row 0
    rot(c1, s1, r10, b11);  // row 1
    rot(c2, s2, b01, b02);  // columns 1, 2 of row 0
    rot(c2, s2, b11, b12);  // row 1
    rot(c2, s2, r21, b22);  // row 2
    h00 = b00 + sg; h01 = b01; h02 = b02;
    h10 = r10;      h11 = b11 + sg; h12 = b12;
    h21 = r21;      h22 = b22 + sg;
  }
  sort3(l1, l2, l3);
  const double us = pow2d(e);  // back from the scaling
  Eig o;
  o.l1 = l1 * us;
  o.l2 = l2 * us;
  o.l3 = l3 * us;
  // adjoint inputs from the gaps (scale-free sigmas; r scaled back)
  const double g12 = l2 - l1, g23 = l3 - l2;
  const double r = sqrt(fma(g12, g12, fma(g12, g23, g23 * g23)));
  o.r = r * us;
  o.sigma1 = r > 0.0 ? kHalfSqrt3 * g12 / r : 0.0;
  o.sigma2 = r > 0.0 ? kHalfSqrt3 * g23 / r : 0.0;
  o.j2_clamped = false;
  o.d_clamped = false;
  return o;
}

// The binary64 path's eigenvalues, or the QR algorithm's for a strongly
// non-normal matrix.
__device__ __forceinline__ Eig guarded_eigvals(const double (&a)[9], bool &switched) {
  const Inv v = invariants_general(a);
  switched = needs_switch(a, v);
  return switched ? eigvals_qr(a) : eigvals_from_inv(v);
}

// Adds this thread's count to *dst: one atomic per warp.
__device__ __forceinline__ void add_count(unsigned c, unsigned long long *dst) {
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0 && c != 0) atomicAdd(dst, (unsigned long long)c);
}

template <typename T>
__device__ __forceinline__ void load9(const T *row, double (&a)[9]) {
#pragma unroll
  for (int j = 0; j < 9; ++j) a[j] = (double)row[j];
}

template <typename T, bool AUX, bool STATS>
__global__ void __launch_bounds__(kThreads)
    k_eigvals_guarded(const T *__restrict__ A, int64_t n, T *__restrict__ lam,
                      T *__restrict__ aux, eig3_stats *__restrict__ stats) {
  __shared__ __align__(16) T sA[2][kTile * 9];
  StatAcc acc;
  if constexpr (STATS) stat_init(acc);
  unsigned nsw = 0;
  for_each_row<9, T>(A, n, sA, [&](int64_t i, const T *row) {
    double a[9];
    load9(row, a);
    bool switched;
    const Eig e = guarded_eigvals(a, switched);
    nsw += switched ? 1u : 0u;
    lam[3 * i + 0] = (T)e.l1;
    lam[3 * i + 1] = (T)e.l2;
    lam[3 * i + 2] = (T)e.l3;
    if constexpr (AUX) {
      T *q = aux + 4 * i;
      q[0] = (T)e.r;
      q[1] = (T)e.sigma1;
      q[2] = (T)e.sigma2;
      q[3] = (T)((a[0] + a[4]) + a[8]);
    }
    if constexpr (STATS) {
      stat_add(acc, e.d_clamped, e.j2_clamped, __double_as_longlong(e.r) > 0,
               seed_float(min_nonneg(e.sigma1, e.sigma2)), (T)e.l1, (T)e.l2, (T)e.l3);
    }
  });
  if constexpr (STATS) {
    stat_flush(acc, stats);
    add_count(nsw, &stats->n_guarded);
  }
}

// Adjoint with the adjoint inputs recomputed by the guarded forward step.
template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_backward_guarded(const T *__restrict__ A, int64_t n, const T *__restrict__ g,
                       T *__restrict__ gA) {
  __shared__ __align__(16) T sA[2][kTile * 9];
  for_each_row<9, T>(A, n, sA, [&](int64_t i, const T *row) {
    double a[9];
    load9(row, a);
    bool switched;
    const Eig e = guarded_eigvals(a, switched);
    const Adj s = adjoint_scalars(e.r, e.sigma1, e.sigma2, (double)__ldg(g + 3 * i),
                                  (double)__ldg(g + 3 * i + 1), (double)__ldg(g + 3 * i + 2));
    double G[9];
    grad_general(a, s, G);
    T *q = gA + 9 * i;
#pragma unroll
    for (int j = 0; j < 9; ++j) q[j] = (T)G[j];
  });
}

template <typename T, bool AUX, bool STATS>
cudaError_t eig_g(const void *A, int64_t n, void *lam, void *aux, eig3_stats *st,
                  cudaStream_t s) {
  auto k = k_eigvals_guarded<T, AUX, STATS>;
  k<<<grid_for((const void *)k, kThreads, 0, n), kThreads, 0, s>>>((const T *)A, n, (T *)lam,
                                                                    (T *)aux, st);
  return cudaGetLastError();
}

template <typename T>
cudaError_t eig_g(const void *A, int64_t n, void *lam, void *aux, eig3_stats *st,
                  cudaStream_t s) {
  if (aux) return st ? eig_g<T, true, true>(A, n, lam, aux, st, s)
                     : eig_g<T, true, false>(A, n, lam, aux, st, s);
  return st ? eig_g<T, false, true>(A, n, lam, aux, st, s)
            : eig_g<T, false, false>(A, n, lam, aux, st, s);
}

template <typename T>
cudaError_t bwd_g(const void *A, int64_t n, const void *g, void *gA, cudaStream_t s) {
  auto k = k_backward_guarded<T>;
  k<<<grid_for((const void *)k, kThreads, 0, n), kThreads, 0, s>>>((const T *)A, n,
                                                                    (const T *)g, (T *)gA);
  return cudaGetLastError();
}

}  // namespace

// General 9-entry layout only; the symmetric layout is dispatched to the
// binary64 kernels by the caller.
cudaError_t launch_eigvals_guarded(const void *A, int dtype, int64_t n, void *lam, void *aux,
                                   eig3_stats *stats, cudaStream_t s) {
  return dtype == EIG3_F64 ? eig_g<double>(A, n, lam, aux, stats, s)
                           : eig_g<float>(A, n, lam, aux, stats, s);
}

cudaError_t launch_backward_guarded(const void *A, int dtype, int64_t n, const void *grad_lam,
                                    void *grad_A, cudaStream_t s) {
  return dtype == EIG3_F64 ? bwd_g<double>(A, n, grad_lam, grad_A, s)
                           : bwd_g<float>(A, n, grad_lam, grad_A, s);
}

}  // namespace eig3
