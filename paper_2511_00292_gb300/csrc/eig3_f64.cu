// eig3_f64.cu -- binary64 kernels: invariants, eigenvalues (+ adjoint inputs,
// + statistics), the adjoint, the fused forward + vector-Jacobian product and
// the eigenprojectors, for the general 9-entry and symmetric 6-entry layouts
// with binary64 or binary32 storage.
//
// One thread per matrix.  The eigenvalue and fused kernels' warps walk the
// batch in tiles of 32 rows each (for_each_row_warp: no block barrier); the other
// kernels' blocks of 256 threads in tiles of 256 rows (for_each_row /
// for_each_tile); either way the grid is sized to fill every SM and the input
// rows of the next tile are copied into shared memory with asynchronous
// 16-byte copies while the current tile is computed (eig3_tile.cuh).  The
// adjoint inputs (16- or 32-byte rows) move with direct vector accesses and
// the outputs are stored directly.  The binary64 path is bound by the FP64 pipe
// (two DFMA per SM per clock on GB300, far below what HBM could feed) and, with
// part of its products formed on the integer pipes (dmul), by the latency of
// the two.
#include <atomic>
#include <cstdint>

#include "eig3_f64.cuh"
#include "eig3_internal.h"
#include "eig3_stats.cuh"
#include "eig3_tile.cuh"

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

// aux rows (r, sigma1, sigma2, I1): 32 B (binary64) or 16 B (binary32), so
// 16-byte aligned whenever the base is; one or two vector accesses per row.
template <typename T>
__device__ __forceinline__ void store_aux(T *__restrict__ aux, int64_t i, bool vec,
                                          const double (&x)[4]) {
  if constexpr (sizeof(T) == 8) {
    if (vec) {
      double2 *q = reinterpret_cast<double2 *>(aux + 4 * i);
      q[0] = make_double2(x[0], x[1]);
      q[1] = make_double2(x[2], x[3]);
      return;
    }
  } else {
    if (vec) {
      *reinterpret_cast<float4 *>(aux + 4 * i) =
          make_float4((float)x[0], (float)x[1], (float)x[2], (float)x[3]);
      return;
    }
  }
  T *q = aux + 4 * i;
#pragma unroll
  for (int j = 0; j < 4; ++j) q[j] = (T)x[j];
}

template <typename T>
__device__ __forceinline__ void load_aux(const T *__restrict__ aux, int64_t i, bool vec,
                                         double &r, double &s1, double &s2) {
  if constexpr (sizeof(T) == 8) {
    if (vec) {
      const double2 *q = reinterpret_cast<const double2 *>(aux + 4 * i);
      const double2 a = __ldg(q), b = __ldg(q + 1);
      r = a.x;
      s1 = a.y;
      s2 = b.x;
      return;
    }
  } else {
    if (vec) {
      const float4 a = __ldg(reinterpret_cast<const float4 *>(aux + 4 * i));
      r = a.x;
      s1 = a.y;
      s2 = a.z;
      return;
    }
  }
  r = (double)__ldg(aux + 4 * i);
  s1 = (double)__ldg(aux + 4 * i + 1);
  s2 = (double)__ldg(aux + 4 * i + 2);
}

__device__ __forceinline__ bool aligned16(const void *p) {
  return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

template <int LAYOUT, typename T, bool AUX, bool STATS>
__global__ void __launch_bounds__(kThreads, 2)
    k_eigvals(const T *__restrict__ A, int64_t n, T *__restrict__ lam, T *__restrict__ aux,
              eig3_stats *__restrict__ stats) {
  constexpr int N = Width<LAYOUT>::N;
  __shared__ __align__(16) T sW[kThreads / 32][2][kWarpTile * N];
  StatAcc acc;
  if constexpr (STATS) stat_init(acc);
  const bool vaux = AUX && aligned16(aux);
  for_each_row_warp<N, T>(A, n, sW[threadIdx.x >> 5], [&](int64_t i, const T *row) {
    double a[N];
#pragma unroll
    for (int j = 0; j < N; ++j) a[j] = (double)row[j];
    const Inv v = invariants_of<LAYOUT, N>(a);
    const Eig e = eigvals_from_inv(v);
    lam[3 * i + 0] = (T)e.l1;
    lam[3 * i + 1] = (T)e.l2;
    lam[3 * i + 2] = (T)e.l3;
    if constexpr (AUX) {
      const double x[4] = {e.r, e.sigma1, e.sigma2, v.I1};
      store_aux<T>(aux, i, vaux, x);
    }
    if constexpr (STATS) {
      stat_add(acc, e.d_clamped, e.j2_clamped, __double_as_longlong(e.r) > 0,
               seed_float(min_nonneg(e.sigma1, e.sigma2)), (T)e.l1, (T)e.l2, (T)e.l3);
    }
  });
  if constexpr (STATS) stat_flush(acc, stats);
}

// Fused forward + vector-Jacobian product: lambda (optional) and
// dL/dA for L = sum_k w_k lambda_k, one pass per matrix (eig3_eigvals_vjp).
// The rows of A go through the warp's shared-memory tiles; the three weights
// of a row are read directly (24 or 12 bytes, contiguous across the warp).
template <int LAYOUT, typename T, bool LAM, bool STATS>
__global__ void __launch_bounds__(kThreads, 2)
    k_eigvals_vjp(const T *__restrict__ A, const T *__restrict__ w, int64_t n,
                  T *__restrict__ lam, T *__restrict__ gA, eig3_stats *__restrict__ stats) {
  constexpr int N = Width<LAYOUT>::N;
  __shared__ __align__(16) T sW[kThreads / 32][2][kWarpTile * N];
  StatAcc acc;
  if constexpr (STATS) stat_init(acc);
  for_each_row_warp<N, T>(A, n, sW[threadIdx.x >> 5], [&](int64_t i, const T *row) {
    double a[N];
#pragma unroll
    for (int j = 0; j < N; ++j) a[j] = (double)row[j];
    const double g1 = (double)__ldg(w + 3 * i + 0);
    const double g2 = (double)__ldg(w + 3 * i + 1);
    const double g3 = (double)__ldg(w + 3 * i + 2);
    double G[N];
    EigV f;
    if constexpr (LAYOUT == EIG3_GENERAL9) {
      ShareG x;
      const Inv v = invariants_general(a, &x);
      f = eigvals_vjp_fwd(v);
      grad_general_vjp(x, v.J2, adjoint_vjp(f, g1, g2, g3), G);
    } else {
      ShareS x;
      const Inv v = invariants_sym(a, &x);
      f = eigvals_vjp_fwd(v);
      grad_sym_vjp(x, v.J2, adjoint_vjp(f, g1, g2, g3), G);
    }
    if constexpr (LAM) {
      lam[3 * i + 0] = (T)f.e.l1;
      lam[3 * i + 1] = (T)f.e.l2;
      lam[3 * i + 2] = (T)f.e.l3;
    }
    T *q = gA + N * i;
#pragma unroll
    for (int j = 0; j < N; ++j) q[j] = (T)G[j];
    if constexpr (STATS) {
      stat_add(acc, f.e.d_clamped, f.e.j2_clamped, __double_as_longlong(f.m) > 0,
               seed_float(min_nonneg(f.e.sigma1, f.e.sigma2)), (T)f.e.l1, (T)f.e.l2,
               (T)f.e.l3);
    }
  });
  if constexpr (STATS) stat_flush(acc, stats);
}

template <int LAYOUT, typename T, bool AUX>
__global__ void __launch_bounds__(kThreads)
    k_backward(const T *__restrict__ A, int64_t n, const T *__restrict__ g,
               const T *__restrict__ aux, T *__restrict__ gA) {
  constexpr int N = Width<LAYOUT>::N;
  __shared__ __align__(16) T sA[2][kTile * N];
  __shared__ __align__(16) T sG[2][kTile * 3];
  const bool vaux = AUX && aligned16(aux);
  for_each_tile<N, 3, T, T>(A, g, n, sA, sG, [&](int64_t r0, int rows, const T *tA,
                                                 const T *tG) {
    if ((int)threadIdx.x >= rows) return;
    double a[N];
#pragma unroll
    for (int j = 0; j < N; ++j) a[j] = (double)tA[threadIdx.x * N + j];
    const double g1 = (double)tG[threadIdx.x * 3 + 0];
    const double g2 = (double)tG[threadIdx.x * 3 + 1];
    const double g3 = (double)tG[threadIdx.x * 3 + 2];
    const int64_t i = r0 + threadIdx.x;
    double r, s1, s2;
    if constexpr (AUX) {
      load_aux<T>(aux, i, vaux, r, s1, s2);
    } else {
      const Eig e = eigvals_from_inv(invariants_of<LAYOUT, N>(a));
      r = e.r;
      s1 = e.sigma1;
      s2 = e.sigma2;
    }
    const Adj s = adjoint_scalars(r, s1, s2, g1, g2, g3);
    double G[N];
    if constexpr (LAYOUT == EIG3_GENERAL9) {
      grad_general(a, s, G);
    } else {
      grad_sym(a, s, G);
    }
    T *q = gA + N * i;
#pragma unroll
    for (int j = 0; j < N; ++j) q[j] = (T)G[j];
  });
}

template <int LAYOUT, typename T, bool LAM>
__global__ void __launch_bounds__(kThreads)
    k_projectors(const T *__restrict__ A, int64_t n, T *__restrict__ lam, T *__restrict__ P) {
  constexpr int N = Width<LAYOUT>::N;
  // dynamic shared memory (proj_smem bytes, above the 48 KB of static arrays):
  // two input tiles, then the tile's outputs, written back coalesced (27 values
  // per row: a 27-element stride between lanes when stored directly;
  // conflict-free in shared memory)
  extern __shared__ __align__(16) unsigned char smem[];
  T(*sA)[kTile * N] = reinterpret_cast<T(*)[kTile * N]>(smem);
  T *sP = reinterpret_cast<T *>(smem + sizeof(T) * 2 * kTile * N);
  T *sL = sP + kTile * 27;
  for_each_tile<N, 0, T, T>(
      A, (const T *)nullptr, n, sA, (T(*)[kTile])nullptr,
      [&](int64_t r0, int rows, const T *tA, const T *) {
        if ((int)threadIdx.x < rows) {
          double a[N];
#pragma unroll
          for (int j = 0; j < N; ++j) a[j] = (double)tA[threadIdx.x * N + j];
          const Eig e = eigvals_from_inv(invariants_of<LAYOUT, N>(a));
          if constexpr (LAM) {
            sL[3 * threadIdx.x + 0] = (T)e.l1;
            sL[3 * threadIdx.x + 1] = (T)e.l2;
            sL[3 * threadIdx.x + 2] = (T)e.l3;
          }
          double E[27];
          projectors<N>(a, adjoint_units(e.r, e.sigma1, e.sigma2), E);
          T *q = sP + 27 * threadIdx.x;
#pragma unroll
          for (int j = 0; j < 27; ++j) q[j] = (T)E[j];
        }
        __syncthreads();  // the tile's outputs are staged; the next barrier protects them
        tile_store(sP, rows * 27, P, r0 * 27);
        if constexpr (LAM) tile_store(sL, rows * 3, lam, r0 * 3);
      });
}

template <int LAYOUT, typename T, bool LAM>
constexpr size_t proj_smem() {
  return sizeof(T) * (2 * kTile * Width<LAYOUT>::N + kTile * 27 + (LAM ? kTile * 3 : 0));
}

// Launch with the dynamic shared memory the kernel stages through.  The
// opt-in above 48 KB is a per-device function attribute, set on the first
// launch on each device (a host call outside any stream, so later launches can
// be captured into CUDA graphs).
template <int LAYOUT, typename T, bool LAM>
cudaError_t proj_launch2(const void *A, int64_t n, void *lam, void *P, cudaStream_t s) {
  auto k = k_projectors<LAYOUT, T, LAM>;
  constexpr size_t bytes = proj_smem<LAYOUT, T, LAM>();
  // one flag per device; host threads may race to set it, which only repeats
  // the (idempotent) attribute call
  static std::atomic<bool> opted[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !opted[dev].load(std::memory_order_acquire)) {
    const cudaError_t e = cudaFuncSetAttribute(
        (const void *)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) opted[dev].store(true, std::memory_order_release);
  }
  k<<<grid_for((const void *)k, kThreads, bytes, n), kThreads, bytes, s>>>((const T *)A, n,
                                                                          (T *)lam, (T *)P);
  return cudaGetLastError();
}

template <int LAYOUT, typename T>
cudaError_t proj_launch(const void *A, int64_t n, void *lam, void *P, cudaStream_t s) {
  return lam ? proj_launch2<LAYOUT, T, true>(A, n, lam, P, s)
             : proj_launch2<LAYOUT, T, false>(A, n, lam, P, s);
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

template <int LAYOUT, typename T, bool LAM, bool STATS>
cudaError_t vjp_launch4(const void *A, const void *w, int64_t n, void *lam, void *gA,
                        eig3_stats *st, cudaStream_t s) {
  auto k = k_eigvals_vjp<LAYOUT, T, LAM, STATS>;
  const int grid = grid_for((const void *)k, kThreads, 0, n);
  k<<<grid, kThreads, 0, s>>>((const T *)A, (const T *)w, n, (T *)lam, (T *)gA, st);
  return cudaGetLastError();
}

template <int LAYOUT, typename T>
cudaError_t vjp_launch(const void *A, const void *w, int64_t n, void *lam, void *gA,
                       eig3_stats *st, cudaStream_t s) {
  if (lam) {
    return st ? vjp_launch4<LAYOUT, T, true, true>(A, w, n, lam, gA, st, s)
              : vjp_launch4<LAYOUT, T, true, false>(A, w, n, lam, gA, st, s);
  }
  return st ? vjp_launch4<LAYOUT, T, false, true>(A, w, n, lam, gA, st, s)
            : vjp_launch4<LAYOUT, T, false, false>(A, w, n, lam, gA, st, s);
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

cudaError_t launch_projectors_f64(const void *A, int layout, int dtype, int64_t n, void *lam,
                                  void *P, cudaStream_t s) {
  if (layout == EIG3_GENERAL9)
    return dtype == EIG3_F64 ? proj_launch<EIG3_GENERAL9, double>(A, n, lam, P, s)
                             : proj_launch<EIG3_GENERAL9, float>(A, n, lam, P, s);
  return dtype == EIG3_F64 ? proj_launch<EIG3_SYM6, double>(A, n, lam, P, s)
                           : proj_launch<EIG3_SYM6, float>(A, n, lam, P, s);
}

cudaError_t launch_eigvals_vjp_f64(const void *A, int layout, int dtype, int64_t n, const void *w,
                                   void *lam, void *grad_A, eig3_stats *stats, cudaStream_t s) {
  if (layout == EIG3_GENERAL9)
    return dtype == EIG3_F64
               ? vjp_launch<EIG3_GENERAL9, double>(A, w, n, lam, grad_A, stats, s)
               : vjp_launch<EIG3_GENERAL9, float>(A, w, n, lam, grad_A, stats, s);
  return dtype == EIG3_F64 ? vjp_launch<EIG3_SYM6, double>(A, w, n, lam, grad_A, stats, s)
                           : vjp_launch<EIG3_SYM6, float>(A, w, n, lam, grad_A, stats, s);
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
