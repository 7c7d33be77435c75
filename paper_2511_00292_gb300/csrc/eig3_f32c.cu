// eig3_f32c.cu -- compensated binary32 kernels (storage and arithmetic in
// binary32, see eig3_f32c.cuh): invariants, eigenvalues (+ adjoint inputs,
// + statistics), the adjoint, the fused forward + vector-Jacobian product and
// the eigenprojectors, for both layouts.  One thread per matrix; blocks walk
// the batch in tiles of 256 rows (for_each_row / for_each_tile: for these
// issue-bound kernels the block tiles measured 3-9% faster than the warp
// tiles of the binary64 kernels), the inputs copied into shared memory
// asynchronously one tile ahead (eig3_tile.cuh); the 16-byte adjoint-input
// rows move as one float4 each; outputs are stored directly, the projectors
// through shared memory.
#include <cstdint>

#include "eig3_f32c.cuh"
#include "eig3_internal.h"
#include "eig3_stats.cuh"
#include "eig3_tile.cuh"

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

// The compensated invariants (the invariants output, accurate at u32^2).
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

__device__ __forceinline__ bool aligned16c(const void *p) {
  return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

template <int LAYOUT, bool AUX, bool STATS, bool ANGLE64>
__global__ void __launch_bounds__(kThreads)
    k_eigvals_c(const float *__restrict__ A, int64_t n, float *__restrict__ lam,
                float *__restrict__ aux, eig3_stats *__restrict__ stats) {
  constexpr int N = WidthC<LAYOUT>::N;
  __shared__ __align__(16) float sA[2][kTile * N];
  StatAcc acc;
  if constexpr (STATS) stat_init(acc);
  const bool vaux = AUX && aligned16c(aux);
  for_each_row<N, float>(A, n, sA, [&](int64_t i, const float *row) {
    float a[N];
#pragma unroll
    for (int j = 0; j < N; ++j) a[j] = row[j];
    const EigC e = eig_c<N, ANGLE64>(a);
    lam[3 * i + 0] = e.l1;
    lam[3 * i + 1] = e.l2;
    lam[3 * i + 2] = e.l3;
    if constexpr (AUX) {
      if (vaux) {
        *reinterpret_cast<float4 *>(aux + 4 * i) = make_float4(e.r, e.sigma1, e.sigma2, e.I1);
      } else {
        aux[4 * i] = e.r;
        aux[4 * i + 1] = e.sigma1;
        aux[4 * i + 2] = e.sigma2;
        aux[4 * i + 3] = e.I1;
      }
    }
    if constexpr (STATS) {
      stat_add(acc, e.d_clamped, e.j2_clamped, e.r > 0.0f, fminf(e.sigma1, e.sigma2), e.l1,
               e.l2, e.l3);
    }
  });
  if constexpr (STATS) stat_flush(acc, stats);
}

template <int LAYOUT, bool AUX>
__global__ void __launch_bounds__(kThreads)
    k_backward_c(const float *__restrict__ A, int64_t n, const float *__restrict__ g,
                 const float *__restrict__ aux, float *__restrict__ gA) {
  constexpr int N = WidthC<LAYOUT>::N;
  __shared__ __align__(16) float sA[2][kTile * N];
  __shared__ __align__(16) float sG[2][kTile * 3];
  const bool vaux = AUX && aligned16c(aux);
  for_each_tile<N, 3, float, float>(A, g, n, sA, sG, [&](int64_t r0, int rows, const float *tA,
                                                         const float *tG) {
    if ((int)threadIdx.x >= rows) return;
    float a[N];
#pragma unroll
    for (int j = 0; j < N; ++j) a[j] = tA[threadIdx.x * N + j];
    const float g1 = tG[threadIdx.x * 3 + 0];
    const float g2 = tG[threadIdx.x * 3 + 1];
    const float g3 = tG[threadIdx.x * 3 + 2];
    const int64_t i = r0 + threadIdx.x;
    float r, s1, s2;
    if constexpr (AUX) {
      if (vaux) {
        const float4 x = __ldg(reinterpret_cast<const float4 *>(aux + 4 * i));
        r = x.x;
        s1 = x.y;
        s2 = x.z;
      } else {
        r = __ldg(aux + 4 * i);
        s1 = __ldg(aux + 4 * i + 1);
        s2 = __ldg(aux + 4 * i + 2);
      }
    } else {
      const EigC e = eig_c<N>(a);
      r = e.r;
      s1 = e.sigma1;
      s2 = e.sigma2;
    }
    const AdjC s = adjoint_c(r, s1, s2, g1, g2, g3);
    float G[N];
    if constexpr (LAYOUT == EIG3_GENERAL9) {
      grad_general_c(a, s, G);
    } else {
      grad_sym_c(a, s, G);
    }
    float *q = gA + N * i;
#pragma unroll
    for (int j = 0; j < N; ++j) q[j] = G[j];
  });
}

// Fused forward + vector-Jacobian product (eig3_eigvals_vjp): lambda
// (optional) and dL/dA for L = sum_k w_k lambda_k in one pass per matrix,
// the adjoint from the forward's r and sigmas in registers.  Rows of A go
// through the block's shared-memory tiles; the weights are read directly.
template <int LAYOUT, bool LAM, bool STATS>
__global__ void __launch_bounds__(kThreads)
    k_eigvals_vjp_c(const float *__restrict__ A, const float *__restrict__ w, int64_t n,
                    float *__restrict__ lam, float *__restrict__ gA,
                    eig3_stats *__restrict__ stats) {
  constexpr int N = WidthC<LAYOUT>::N;
  __shared__ __align__(16) float sA[2][kTile * N];
  StatAcc acc;
  if constexpr (STATS) stat_init(acc);
  for_each_row<N, float>(A, n, sA, [&](int64_t i, const float *row) {
    float a[N];
#pragma unroll
    for (int j = 0; j < N; ++j) a[j] = row[j];
    const float g1 = __ldg(w + 3 * i + 0);
    const float g2 = __ldg(w + 3 * i + 1);
    const float g3 = __ldg(w + 3 * i + 2);
    const EigC e = eig_c<N>(a);
    if constexpr (LAM) {
      lam[3 * i + 0] = e.l1;
      lam[3 * i + 1] = e.l2;
      lam[3 * i + 2] = e.l3;
    }
    const AdjC s = adjoint_c(e.r, e.sigma1, e.sigma2, g1, g2, g3);
    float G[N];
    if constexpr (LAYOUT == EIG3_GENERAL9) {
      grad_general_c(a, s, G);
    } else {
      grad_sym_c(a, s, G);
    }
    float *q = gA + N * i;
#pragma unroll
    for (int j = 0; j < N; ++j) q[j] = G[j];
    if constexpr (STATS) {
      stat_add(acc, e.d_clamped, e.j2_clamped, e.r > 0.0f, fminf(e.sigma1, e.sigma2), e.l1,
               e.l2, e.l3);
    }
  });
  if constexpr (STATS) stat_flush(acc, stats);
}

template <int LAYOUT, bool LAM, bool STATS>
cudaError_t vjp_c4(const void *A, const void *w, int64_t n, void *lam, void *gA, eig3_stats *st,
                   cudaStream_t s) {
  auto k = k_eigvals_vjp_c<LAYOUT, LAM, STATS>;
  const int grid = grid_for((const void *)k, kThreads, 0, n);
  k<<<grid, kThreads, 0, s>>>((const float *)A, (const float *)w, n, (float *)lam, (float *)gA,
                              st);
  return cudaGetLastError();
}

template <int LAYOUT>
cudaError_t vjp_c(const void *A, const void *w, int64_t n, void *lam, void *gA, eig3_stats *st,
                  cudaStream_t s) {
  if (lam)
    return st ? vjp_c4<LAYOUT, true, true>(A, w, n, lam, gA, st, s)
              : vjp_c4<LAYOUT, true, false>(A, w, n, lam, gA, st, s);
  return st ? vjp_c4<LAYOUT, false, true>(A, w, n, lam, gA, st, s)
            : vjp_c4<LAYOUT, false, false>(A, w, n, lam, gA, st, s);
}

template <int LAYOUT, bool LAM>
__global__ void __launch_bounds__(kThreads)
    k_projectors_c(const float *__restrict__ A, int64_t n, float *__restrict__ lam,
                   float *__restrict__ P) {
  constexpr int N = WidthC<LAYOUT>::N;
  __shared__ __align__(16) float sA[2][kTile * N];
  // the tile's outputs, written back coalesced (27 floats per row: a 108-byte
  // stride between lanes when stored directly)
  __shared__ __align__(16) float sP[kTile * 27];
  __shared__ __align__(16) float sL[LAM ? kTile * 3 : 4];
  for_each_tile<N, 0, float, float>(
      A, (const float *)nullptr, n, sA, (float(*)[kTile])nullptr,
      [&](int64_t r0, int rows, const float *tA, const float *) {
        if ((int)threadIdx.x < rows) {
          float a[N];
#pragma unroll
          for (int j = 0; j < N; ++j) a[j] = tA[threadIdx.x * N + j];
          const EigC e = eig_c<N>(a);
          if constexpr (LAM) {
            sL[3 * threadIdx.x + 0] = e.l1;
            sL[3 * threadIdx.x + 1] = e.l2;
            sL[3 * threadIdx.x + 2] = e.l3;
          }
          float E[27];
          projectors_c<N>(a, adjoint_units_c(e.r, e.sigma1, e.sigma2), E);
          float *q = sP + 27 * threadIdx.x;
#pragma unroll
          for (int j = 0; j < 27; ++j) q[j] = E[j];
        }
        __syncthreads();  // the tile's outputs are staged; the next barrier protects them
        tile_store(sP, rows * 27, P, r0 * 27);
        if constexpr (LAM) tile_store(sL, rows * 3, lam, r0 * 3);
      });
}

template <int LAYOUT>
cudaError_t proj_c(const void *A, int64_t n, void *lam, void *P, cudaStream_t s) {
  if (lam) {
    auto k = k_projectors_c<LAYOUT, true>;
    k<<<grid_for((const void *)k, kThreads, 0, n), kThreads, 0, s>>>((const float *)A, n,
                                                                      (float *)lam, (float *)P);
  } else {
    auto k = k_projectors_c<LAYOUT, false>;
    k<<<grid_for((const void *)k, kThreads, 0, n), kThreads, 0, s>>>((const float *)A, n,
                                                                      (float *)lam, (float *)P);
  }
  return cudaGetLastError();
}

template <int LAYOUT>
cudaError_t inv_c(const void *A, int64_t n, double *inv, cudaStream_t s) {
  auto k = k_invariants_c<LAYOUT>;
  const int grid = grid_for((const void *)k, kThreads, 0, n);
  k<<<grid, kThreads, 0, s>>>((const float *)A, n, inv);
  return cudaGetLastError();
}

template <int LAYOUT, bool AUX, bool STATS, bool ANGLE64>
cudaError_t eig_c4(const void *A, int64_t n, void *lam, void *aux, eig3_stats *st,
                   cudaStream_t s) {
  auto k = k_eigvals_c<LAYOUT, AUX, STATS, ANGLE64>;
  const int grid = grid_for((const void *)k, kThreads, 0, n);
  k<<<grid, kThreads, 0, s>>>((const float *)A, n, (float *)lam, (float *)aux, st);
  return cudaGetLastError();
}

template <int LAYOUT, bool ANGLE64>
cudaError_t eig_c(const void *A, int64_t n, void *lam, void *aux, eig3_stats *st,
                  cudaStream_t s) {
  if (aux)
    return st ? eig_c4<LAYOUT, true, true, ANGLE64>(A, n, lam, aux, st, s)
              : eig_c4<LAYOUT, true, false, ANGLE64>(A, n, lam, aux, st, s);
  return st ? eig_c4<LAYOUT, false, true, ANGLE64>(A, n, lam, aux, st, s)
            : eig_c4<LAYOUT, false, false, ANGLE64>(A, n, lam, aux, st, s);
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
                                eig3_stats *stats, bool angle64, cudaStream_t s) {
  if (angle64)
    return layout == EIG3_GENERAL9 ? eig_c<EIG3_GENERAL9, true>(A, n, lam, aux, stats, s)
                                   : eig_c<EIG3_SYM6, true>(A, n, lam, aux, stats, s);
  return layout == EIG3_GENERAL9 ? eig_c<EIG3_GENERAL9, false>(A, n, lam, aux, stats, s)
                                 : eig_c<EIG3_SYM6, false>(A, n, lam, aux, stats, s);
}

cudaError_t launch_projectors_f32c(const void *A, int layout, int64_t n, void *lam, void *P,
                                   cudaStream_t s) {
  return layout == EIG3_GENERAL9 ? proj_c<EIG3_GENERAL9>(A, n, lam, P, s)
                                 : proj_c<EIG3_SYM6>(A, n, lam, P, s);
}

cudaError_t launch_eigvals_vjp_f32c(const void *A, int layout, int64_t n, const void *w, void *lam,
                                    void *grad_A, eig3_stats *stats, cudaStream_t s) {
  return layout == EIG3_GENERAL9 ? vjp_c<EIG3_GENERAL9>(A, w, n, lam, grad_A, stats, s)
                                 : vjp_c<EIG3_SYM6>(A, w, n, lam, grad_A, stats, s);
}

cudaError_t launch_backward_f32c(const void *A, int layout, int64_t n, const void *grad_lam,
                                 const void *aux, void *grad_A, cudaStream_t s) {
  return layout == EIG3_GENERAL9 ? bwd_c<EIG3_GENERAL9>(A, n, grad_lam, aux, grad_A, s)
                                 : bwd_c<EIG3_SYM6>(A, n, grad_lam, aux, grad_A, s);
}

}  // namespace eig3
