// eig3_internal.h -- launchers shared between the library's translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "eig3.h"

namespace eig3 {

constexpr int kThreads = 256;

// Number of SMs of the current device (cached per device).
int sm_count();

// Grid for a grid-stride kernel: enough blocks to fill every SM at the
// kernel's occupancy, never more than the work needs.
int grid_for(const void *kernel, int threads, size_t smem, int64_t work_items);

// binary64 arithmetic (storage dtype EIG3_F64 or EIG3_F32)
cudaError_t launch_invariants_f64(const void *A, int layout, int dtype, int64_t n, double *inv,
                                  cudaStream_t s);
cudaError_t launch_eigvals_f64(const void *A, int layout, int dtype, int64_t n, void *lam,
                               void *aux, eig3_stats *stats, cudaStream_t s);
cudaError_t launch_projectors_f64(const void *A, int layout, int dtype, int64_t n, void *lam,
                                  void *P, cudaStream_t s);
cudaError_t launch_mohr_coulomb_f64(const void *A, int layout, int dtype, int64_t n, double s_yc,
                                    double m, void *f, void *grad_A, cudaStream_t s);
cudaError_t launch_variant_f64(const void *A, int layout, int dtype, int variant, int64_t n,
                               double *inv, void *lam, cudaStream_t s);
cudaError_t launch_eigvals_vjp_f64(const void *A, int layout, int dtype, int64_t n, const void *w,
                                   void *lam, void *grad_A, eig3_stats *stats, cudaStream_t s);
cudaError_t launch_backward_f64(const void *A, int layout, int dtype, int64_t n,
                                const void *grad_lam, const void *aux, void *grad_A,
                                cudaStream_t s);

// binary32 compensated arithmetic (storage dtype EIG3_F32)
cudaError_t launch_invariants_f32c(const void *A, int layout, int64_t n, double *inv,
                                   cudaStream_t s);
cudaError_t launch_eigvals_f32c(const void *A, int layout, int64_t n, void *lam, void *aux,
                                eig3_stats *stats, bool angle64, cudaStream_t s);
cudaError_t launch_projectors_f32c(const void *A, int layout, int64_t n, void *lam, void *P,
                                   cudaStream_t s);
cudaError_t launch_mohr_coulomb_f32c(const void *A, int layout, int64_t n, double s_yc, double m,
                                     void *f, void *grad_A, cudaStream_t s);
cudaError_t launch_eigvals_vjp_f32c(const void *A, int layout, int64_t n, const void *w, void *lam,
                                    void *grad_A, eig3_stats *stats, cudaStream_t s);
cudaError_t launch_backward_f32c(const void *A, int layout, int64_t n, const void *grad_lam,
                                 const void *aux, void *grad_A, cudaStream_t s);

// binary64 with the guard for ill-conditioned eigenbases, general 9-entry layout
cudaError_t launch_eigvals_guarded(const void *A, int dtype, int64_t n, void *lam, void *aux,
                                   eig3_stats *stats, cudaStream_t s);
cudaError_t launch_backward_guarded(const void *A, int dtype, int64_t n, const void *grad_lam,
                                    void *grad_A, cudaStream_t s);

cudaError_t launch_stats_reset(eig3_stats *stats, cudaStream_t s);

}  // namespace eig3
