// eig3_f64.cu -- binary64 kernels: invariants, eigenvalues (+ adjoint inputs,
// + statistics) and the adjoint, for the general 9-entry and symmetric
// 6-entry layouts with binary64 or binary32 storage.
//
// One thread per matrix, grid-stride over the batch with a grid sized to fill
// every SM once.  The binary64 path is bound by the FP64 pipe (two DFMA per
// SM per clock on GB300, far below what HBM could feed), so the kernels keep
// the memory side simple -- each thread reads its row with read-only loads
// that the L1 merges -- and spend the design effort on the FP64 instruction
// count (see eig3_f64.cuh).
#include <cstdint>

#include "eig3_f64.cuh"
#include "eig3_internal.h"
#include "eig3_stats.cuh"

namespace eig3 {
namespace {

template <int LAYOUT>
struct Width {
  static constexpr int N = (LAYOUT == EIG3_GENERAL9) ? 9 : 6;
};

template <typename T, int N>
__device__ __forceinline__ void load_row(const T *__restrict__ p, int64_t i, double (&a)[N]) {
  const T *q = p + i * N;
#pragma unroll
  for (int j = 0; j < N; ++j) a[j] = (double)__ldg(q + j);
}

template <typename T, int N>
__device__ __forceinline__ void store_row(T *__restrict__ p, int64_t i, const double (&a)[N]) {
  T *q = p + i * N;
#pragma unroll
  for (int j = 0; j < N; ++j) q[j] = (T)a[j];
}

template <int LAYOUT, int N>
__device__ __forceinline__ Inv invariants_of(const double (&a)[N]) {
  if constexpr (LAYOUT == EIG3_GENERAL9) {
    return invariants_general(a);
  } else {
    return invariants_sym(a);
  }
}

template <int LAYOUT, typename T>
__global__ void __launch_bounds__(kThreads) k_invariants(const T *__restrict__ A, int64_t n,
                                                         double *__restrict__ inv) {
  constexpr int N = Width<LAYOUT>::N;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double a[N];
    load_row<T, N>(A, i, a);
    const Inv v = invariants_of<LAYOUT, N>(a);
    double *o = inv + 4 * i;
    o[0] = v.I1;
    if (v.e == 0) {
      o[1] = v.J2;
      o[2] = v.J3;
      o[3] = v.D;
    } else {  // back from 2^-e A
      o[1] = ldexp(v.J2, 2 * v.e);
      o[2] = ldexp(v.J3, 3 * v.e);
      o[3] = ldexp(v.D, 6 * v.e);
    }
  }
}

template <int LAYOUT, typename T, bool AUX, bool STATS>
__global__ void __launch_bounds__(kThreads)
    k_eigvals(const T *__restrict__ A, int64_t n, T *__restrict__ lam, T *__restrict__ aux,
              eig3_stats *__restrict__ stats) {
  constexpr int N = Width<LAYOUT>::N;
  StatAcc acc;
  if constexpr (STATS) stat_init(acc);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double a[N];
    load_row<T, N>(A, i, a);
    const Inv v = invariants_of<LAYOUT, N>(a);
    const Eig e = eigvals_from_inv(v);
    const double l[3] = {e.l1, e.l2, e.l3};
    store_row<T, 3>(lam, i, l);
    if constexpr (AUX) {
      const double x[4] = {e.r, e.sigma1, e.sigma2, v.I1};
      store_row<T, 4>(aux, i, x);
    }
    if constexpr (STATS) {
      stat_add(acc, e.d_clamped, e.j2_clamped, e.r > 0.0,
               (float)fmin(e.sigma1, e.sigma2), (T)e.l1, (T)e.l2, (T)e.l3);
    }
  }
  if constexpr (STATS) stat_flush(acc, stats);
}

template <int LAYOUT, typename T, bool AUX>
__global__ void __launch_bounds__(kThreads)
    k_backward(const T *__restrict__ A, int64_t n, const T *__restrict__ g,
               const T *__restrict__ aux, T *__restrict__ gA) {
  constexpr int N = Width<LAYOUT>::N;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double a[N];
    load_row<T, N>(A, i, a);
    double gb[3];
    load_row<T, 3>(g, i, gb);
    double r, s1, s2;
    if constexpr (AUX) {
      double x[4];
      load_row<T, 4>(aux, i, x);
      r = x[0];
      s1 = x[1];
      s2 = x[2];
    } else {
      const Eig e = eigvals_from_inv(invariants_of<LAYOUT, N>(a));
      r = e.r;
      s1 = e.sigma1;
      s2 = e.sigma2;
    }
    const Adj s = adjoint_scalars(r, s1, s2, gb[0], gb[1], gb[2]);
    double G[N];
    if constexpr (LAYOUT == EIG3_GENERAL9) {
      grad_general(a, s, G);
    } else {
      grad_sym(a, s, G);
    }
    store_row<T, N>(gA, i, G);
  }
}

template <int LAYOUT, typename T>
cudaError_t inv_launch(const void *A, int64_t n, double *inv, cudaStream_t s) {
  auto k = k_invariants<LAYOUT, T>;
  const int grid = grid_for((const void *)k, kThreads, 0, n);
  k<<<grid, kThreads, 0, s>>>((const T *)A, n, inv);
  return cudaGetLastError();
}

template <int LAYOUT, typename T, bool AUX, bool STATS>
cudaError_t eig_launch4(const void *A, int64_t n, void *lam, void *aux, eig3_stats *st,
                        cudaStream_t s) {
  auto k = k_eigvals<LAYOUT, T, AUX, STATS>;
  const int grid = grid_for((const void *)k, kThreads, 0, n);
  k<<<grid, kThreads, 0, s>>>((const T *)A, n, (T *)lam, (T *)aux, st);
  return cudaGetLastError();
}

template <int LAYOUT, typename T>
cudaError_t eig_launch(const void *A, int64_t n, void *lam, void *aux, eig3_stats *st,
                       cudaStream_t s) {
  if (aux) {
    return st ? eig_launch4<LAYOUT, T, true, true>(A, n, lam, aux, st, s)
              : eig_launch4<LAYOUT, T, true, false>(A, n, lam, aux, st, s);
  }
  return st ? eig_launch4<LAYOUT, T, false, true>(A, n, lam, aux, st, s)
            : eig_launch4<LAYOUT, T, false, false>(A, n, lam, aux, st, s);
}

template <int LAYOUT, typename T, bool AUX>
cudaError_t bwd_launch2(const void *A, int64_t n, const void *g, const void *aux, void *gA,
                        cudaStream_t s) {
  auto k = k_backward<LAYOUT, T, AUX>;
  const int grid = grid_for((const void *)k, kThreads, 0, n);
  k<<<grid, kThreads, 0, s>>>((const T *)A, n, (const T *)g, (const T *)aux, (T *)gA);
  return cudaGetLastError();
}

template <int LAYOUT, typename T>
cudaError_t bwd_launch(const void *A, int64_t n, const void *g, const void *aux, void *gA,
                       cudaStream_t s) {
  return aux ? bwd_launch2<LAYOUT, T, true>(A, n, g, aux, gA, s)
             : bwd_launch2<LAYOUT, T, false>(A, n, g, aux, gA, s);
}

}  // namespace

cudaError_t launch_invariants_f64(const void *A, int layout, int dtype, int64_t n, double *inv,
                                  cudaStream_t s) {
  if (layout == EIG3_GENERAL9)
    return dtype == EIG3_F64 ? inv_launch<EIG3_GENERAL9, double>(A, n, inv, s)
                             : inv_launch<EIG3_GENERAL9, float>(A, n, inv, s);
  return dtype == EIG3_F64 ? inv_launch<EIG3_SYM6, double>(A, n, inv, s)
                           : inv_launch<EIG3_SYM6, float>(A, n, inv, s);
}

cudaError_t launch_eigvals_f64(const void *A, int layout, int dtype, int64_t n, void *lam,
                               void *aux, eig3_stats *stats, cudaStream_t s) {
  if (layout == EIG3_GENERAL9)
    return dtype == EIG3_F64 ? eig_launch<EIG3_GENERAL9, double>(A, n, lam, aux, stats, s)
                             : eig_launch<EIG3_GENERAL9, float>(A, n, lam, aux, stats, s);
  return dtype == EIG3_F64 ? eig_launch<EIG3_SYM6, double>(A, n, lam, aux, stats, s)
                           : eig_launch<EIG3_SYM6, float>(A, n, lam, aux, stats, s);
}

cudaError_t launch_backward_f64(const void *A, int layout, int dtype, int64_t n,
                                const void *grad_lam, const void *aux, void *grad_A,
                                cudaStream_t s) {
  if (layout == EIG3_GENERAL9)
    return dtype == EIG3_F64
               ? bwd_launch<EIG3_GENERAL9, double>(A, n, grad_lam, aux, grad_A, s)
               : bwd_launch<EIG3_GENERAL9, float>(A, n, grad_lam, aux, grad_A, s);
  return dtype == EIG3_F64 ? bwd_launch<EIG3_SYM6, double>(A, n, grad_lam, aux, grad_A, s)
                           : bwd_launch<EIG3_SYM6, float>(A, n, grad_lam, aux, grad_A, s);
}

}  // namespace eig3
