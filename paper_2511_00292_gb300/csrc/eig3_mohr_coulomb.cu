// eig3_mohr_coulomb.cu -- fused Mohr-Coulomb yield value and gradient
// (Section "Application") in binary64 (storage binary64 or binary32) and in
// compensated binary32, for both layouts.
//
// f(sigma) = ((m+1)/(2 S_yc)) max_{i<j} (|s_i - s_j| + K (s_i + s_j)) - 1 with
// K = (m-1)/(m+1).  With ascending eigenvalues the pair term of (i, j), i < j,
// is (1+K) s_j - (1-K) s_i; for m > 0 both 1+K and 1-K are positive, so the
// maximum is always taken by the extreme pair and
//   f = (m lambda_3 - lambda_1) / S_yc - 1,
//   df/dsigma = adjoint of the eigenvalues with weights (-1/S_yc, 0, m/S_yc).
// One thread per stress tensor: invariants, Algorithm 6, the value, and the
// adjoint of the same eigenvalues in registers; the input tiles are staged as
// in the other kernels (eig3_tile.cuh); only f and the gradient are written.
#include <cstdint>

#include "eig3_f32c.cuh"
#include "eig3_f64.cuh"
#include "eig3_internal.h"
#include "eig3_tile.cuh"

namespace eig3 {
namespace {

template <int LAYOUT>
struct Rows {
  static constexpr int N = (LAYOUT == EIG3_GENERAL9) ? 9 : 6;
};

// binary64 arithmetic; c1 = 1/S_yc, cm = m/S_yc
template <int LAYOUT, typename T, bool GRAD>
__global__ void __launch_bounds__(kThreads)
    k_mohr_coulomb(const T *__restrict__ A, int64_t n, double c1, double cm, T *__restrict__ f,
                   T *__restrict__ gA) {
  constexpr int N = Rows<LAYOUT>::N;
  __shared__ __align__(16) T sA[2][kTile * N];
  for_each_row<N, T>(A, n, sA, [&](int64_t i, const T *row) {
    double a[N];
#pragma unroll
    for (int j = 0; j < N; ++j) a[j] = (double)row[j];
    Inv v;
    if constexpr (LAYOUT == EIG3_GENERAL9) {
      v = invariants_general(a);
    } else {
      v = invariants_sym(a);
    }
    const Eig e = eigvals_from_inv(v);
    f[i] = (T)fma(cm, e.l3, fma(-c1, e.l1, -1.0));
    if constexpr (GRAD) {
      const Adj s = adjoint_scalars(e.r, e.sigma1, e.sigma2, -c1, 0.0, cm);
      double G[N];
      if constexpr (LAYOUT == EIG3_GENERAL9) {
        grad_general(a, s, G);
      } else {
        grad_sym(a, s, G);
      }
      T *q = gA + N * i;
#pragma unroll
      for (int j = 0; j < N; ++j) q[j] = (T)G[j];
    }
  });
}

// compensated binary32 arithmetic (eig3_f32c.cuh); c1, cm rounded to binary32
template <int LAYOUT, bool GRAD>
__global__ void __launch_bounds__(kThreads)
    k_mohr_coulomb_c(const float *__restrict__ A, int64_t n, float c1, float cm,
                     float *__restrict__ f, float *__restrict__ gA) {
  using namespace c32;
  constexpr int N = Rows<LAYOUT>::N;
  __shared__ __align__(16) float sA[2][kTile * N];
  for_each_row<N, float>(A, n, sA, [&](int64_t i, const float *row) {
    float a[N];
#pragma unroll
    for (int j = 0; j < N; ++j) a[j] = row[j];
    const EigC e = eig_c<N>(a);
    f[i] = fmaf(cm, e.l3, fmaf(-c1, e.l1, -1.0f));
    if constexpr (GRAD) {
      const AdjC s = adjoint_c(e.r, e.sigma1, e.sigma2, -c1, 0.0f, cm);
      float G[N];
      if constexpr (LAYOUT == EIG3_GENERAL9) {
        grad_general_c(a, s, G);
      } else {
        grad_sym_c(a, s, G);
      }
      float *q = gA + N * i;
#pragma unroll
      for (int j = 0; j < N; ++j) q[j] = G[j];
    }
  });
}

template <int LAYOUT, typename T, bool GRAD>
cudaError_t launch64(const void *A, int64_t n, double c1, double cm, void *f, void *gA,
                     cudaStream_t s) {
  auto k = k_mohr_coulomb<LAYOUT, T, GRAD>;
  k<<<grid_for((const void *)k, kThreads, 0, n), kThreads, 0, s>>>((const T *)A, n, c1, cm,
                                                                    (T *)f, (T *)gA);
  return cudaGetLastError();
}

template <int LAYOUT, typename T>
cudaError_t launch64(const void *A, int64_t n, double c1, double cm, void *f, void *gA,
                     cudaStream_t s) {
  return gA ? launch64<LAYOUT, T, true>(A, n, c1, cm, f, gA, s)
            : launch64<LAYOUT, T, false>(A, n, c1, cm, f, gA, s);
}

template <int LAYOUT, bool GRAD>
cudaError_t launch32(const void *A, int64_t n, float c1, float cm, void *f, void *gA,
                     cudaStream_t s) {
  auto k = k_mohr_coulomb_c<LAYOUT, GRAD>;
  k<<<grid_for((const void *)k, kThreads, 0, n), kThreads, 0, s>>>((const float *)A, n, c1, cm,
                                                                    (float *)f, (float *)gA);
  return cudaGetLastError();
}

template <int LAYOUT>
cudaError_t launch32(const void *A, int64_t n, float c1, float cm, void *f, void *gA,
                     cudaStream_t s) {
  return gA ? launch32<LAYOUT, true>(A, n, c1, cm, f, gA, s)
            : launch32<LAYOUT, false>(A, n, c1, cm, f, gA, s);
}

}  // namespace

cudaError_t launch_mohr_coulomb_f64(const void *A, int layout, int dtype, int64_t n, double s_yc,
                                    double m, void *f, void *grad_A, cudaStream_t s) {
  const double c1 = 1.0 / s_yc, cm = m / s_yc;
  if (layout == EIG3_GENERAL9)
    return dtype == EIG3_F64 ? launch64<EIG3_GENERAL9, double>(A, n, c1, cm, f, grad_A, s)
                             : launch64<EIG3_GENERAL9, float>(A, n, c1, cm, f, grad_A, s);
  return dtype == EIG3_F64 ? launch64<EIG3_SYM6, double>(A, n, c1, cm, f, grad_A, s)
                           : launch64<EIG3_SYM6, float>(A, n, c1, cm, f, grad_A, s);
}

cudaError_t launch_mohr_coulomb_f32c(const void *A, int layout, int64_t n, double s_yc, double m,
                                     void *f, void *grad_A, cudaStream_t s) {
  const float c1 = (float)(1.0 / s_yc), cm = (float)(m / s_yc);
  return layout == EIG3_GENERAL9 ? launch32<EIG3_GENERAL9>(A, n, c1, cm, f, grad_A, s)
                                 : launch32<EIG3_SYM6>(A, n, c1, cm, f, grad_A, s);
}

}  // namespace eig3
