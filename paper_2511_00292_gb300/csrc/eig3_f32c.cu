// eig3_f32c.cu -- compensated binary32 kernels (storage and arithmetic in
// binary32, see eig3_f32c.cuh): invariants, eigenvalues (+ adjoint inputs,
// + statistics) and the adjoint, for both layouts.  One thread per matrix,
// grid-stride over the batch.
#include <cstdint>

#include "eig3_f32c.cuh"
#include "eig3_internal.h"
#include "eig3_stats.cuh"

namespace eig3 {
namespace {

using namespace c32;

template <int N>
__device__ __forceinline__ void load_f(const float *__restrict__ p, int64_t i, float (&a)[N]) {
  const float *q = p + i * N;
#pragma unroll
  for (int j = 0; j < N; ++j) a[j] = __ldg(q + j);
}

template <int N>
__device__ __forceinline__ void store_f(float *__restrict__ p, int64_t i, const float (&a)[N]) {
  float *q = p + i * N;
#pragma unroll
  for (int j = 0; j < N; ++j) q[j] = a[j];
}

template <int LAYOUT>
struct WidthC {
  static constexpr int N = (LAYOUT == EIG3_GENERAL9) ? 9 : 6;
};

template <int LAYOUT, int N>
__device__ __forceinline__ InvC invariants_c(const float (&a)[N]) {
  if constexpr (LAYOUT == EIG3_GENERAL9) {
    return invariants_general_c(a);
  } else {
    return invariants_sym_c(a[0], a[1], a[2], a[3], a[4], a[5]);
  }
}

template <int LAYOUT>
__global__ void __launch_bounds__(kThreads)
    k_invariants_c(const float *__restrict__ A, int64_t n, double *__restrict__ inv) {
  constexpr int N = WidthC<LAYOUT>::N;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    float a[N];
    load_f<N>(A, i, a);
    invariants_out(invariants_c<LAYOUT, N>(a), inv + 4 * i);
  }
}

template <int LAYOUT, bool AUX, bool STATS>
__global__ void __launch_bounds__(kThreads)
    k_eigvals_c(const float *__restrict__ A, int64_t n, float *__restrict__ lam,
                float *__restrict__ aux, eig3_stats *__restrict__ stats) {
  constexpr int N = WidthC<LAYOUT>::N;
  StatAcc acc;
  if constexpr (STATS) stat_init(acc);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    float a[N];
    load_f<N>(A, i, a);
    const InvC v = invariants_c<LAYOUT, N>(a);
    const EigC e = eigvals_c(v);
    const float l[3] = {e.l1, e.l2, e.l3};
    store_f<3>(lam, i, l);
    if constexpr (AUX) {
      const float x[4] = {e.r, e.sigma1, e.sigma2, e.I1};
      store_f<4>(aux, i, x);
    }
    if constexpr (STATS) {
      stat_add(acc, e.d_clamped, e.j2_clamped, e.r > 0.0f, fminf(e.sigma1, e.sigma2), e.l1,
               e.l2, e.l3);
    }
  }
  if constexpr (STATS) stat_flush(acc, stats);
}

template <int LAYOUT, bool AUX>
__global__ void __launch_bounds__(kThreads)
    k_backward_c(const float *__restrict__ A, int64_t n, const float *__restrict__ g,
                 const float *__restrict__ aux, float *__restrict__ gA) {
  constexpr int N = WidthC<LAYOUT>::N;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    float a[N];
    load_f<N>(A, i, a);
    float gb[3];
    load_f<3>(g, i, gb);
    float r, s1, s2;
    if constexpr (AUX) {
      float x[4];
      load_f<4>(aux, i, x);
      r = x[0];
      s1 = x[1];
      s2 = x[2];
    } else {
      const EigC e = eigvals_c(invariants_c<LAYOUT, N>(a));
      r = e.r;
      s1 = e.sigma1;
      s2 = e.sigma2;
    }
    const AdjC s = adjoint_c(r, s1, s2, gb[0], gb[1], gb[2]);
    float G[N];
    if constexpr (LAYOUT == EIG3_GENERAL9) {
      grad_general_c(a, s, G);
    } else {
      grad_sym_c(a, s, G);
    }
    store_f<N>(gA, i, G);
  }
}

template <int LAYOUT>
cudaError_t inv_c(const void *A, int64_t n, double *inv, cudaStream_t s) {
  auto k = k_invariants_c<LAYOUT>;
  const int grid = grid_for((const void *)k, kThreads, 0, n);
  k<<<grid, kThreads, 0, s>>>((const float *)A, n, inv);
  return cudaGetLastError();
}

template <int LAYOUT, bool AUX, bool STATS>
cudaError_t eig_c4(const void *A, int64_t n, void *lam, void *aux, eig3_stats *st,
                   cudaStream_t s) {
  auto k = k_eigvals_c<LAYOUT, AUX, STATS>;
  const int grid = grid_for((const void *)k, kThreads, 0, n);
  k<<<grid, kThreads, 0, s>>>((const float *)A, n, (float *)lam, (float *)aux, st);
  return cudaGetLastError();
}

template <int LAYOUT>
cudaError_t eig_c(const void *A, int64_t n, void *lam, void *aux, eig3_stats *st,
                  cudaStream_t s) {
  if (aux)
    return st ? eig_c4<LAYOUT, true, true>(A, n, lam, aux, st, s)
              : eig_c4<LAYOUT, true, false>(A, n, lam, aux, st, s);
  return st ? eig_c4<LAYOUT, false, true>(A, n, lam, aux, st, s)
            : eig_c4<LAYOUT, false, false>(A, n, lam, aux, st, s);
}

template <int LAYOUT, bool AUX>
cudaError_t bwd_c2(const void *A, int64_t n, const void *g, const void *aux, void *gA,
                   cudaStream_t s) {
  auto k = k_backward_c<LAYOUT, AUX>;
  const int grid = grid_for((const void *)k, kThreads, 0, n);
  k<<<grid, kThreads, 0, s>>>((const float *)A, n, (const float *)g, (const float *)aux,
                              (float *)gA);
  return cudaGetLastError();
}

template <int LAYOUT>
cudaError_t bwd_c(const void *A, int64_t n, const void *g, const void *aux, void *gA,
                  cudaStream_t s) {
  return aux ? bwd_c2<LAYOUT, true>(A, n, g, aux, gA, s)
             : bwd_c2<LAYOUT, false>(A, n, g, aux, gA, s);
}

}  // namespace

cudaError_t launch_invariants_f32c(const void *A, int layout, int64_t n, double *inv,
                                   cudaStream_t s) {
  return layout == EIG3_GENERAL9 ? inv_c<EIG3_GENERAL9>(A, n, inv, s)
                                 : inv_c<EIG3_SYM6>(A, n, inv, s);
}

cudaError_t launch_eigvals_f32c(const void *A, int layout, int64_t n, void *lam, void *aux,
                                eig3_stats *stats, cudaStream_t s) {
  return layout == EIG3_GENERAL9 ? eig_c<EIG3_GENERAL9>(A, n, lam, aux, stats, s)
                                 : eig_c<EIG3_SYM6>(A, n, lam, aux, stats, s);
}

cudaError_t launch_backward_f32c(const void *A, int layout, int64_t n, const void *grad_lam,
                                 const void *aux, void *grad_A, cudaStream_t s) {
  return layout == EIG3_GENERAL9 ? bwd_c<EIG3_GENERAL9>(A, n, grad_lam, aux, grad_A, s)
                                 : bwd_c<EIG3_SYM6>(A, n, grad_lam, aux, grad_A, s);
}

}  // namespace eig3
