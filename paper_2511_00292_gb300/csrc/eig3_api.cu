// eig3_api.cu -- the library's C ABI (include/eig3.h): host-side argument
// checks, dispatch to the binary64 or compensated binary32 kernels, launch
// error reporting, and launch-geometry helpers.
#include <atomic>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "eig3.h"
#include "eig3_internal.h"

namespace eig3 {

int sm_count() {
  // per-device cache; concurrent first calls may both query, then store the same value
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (dev >= 0 && dev < 64) {
    const int c = cache[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 1;
  if (dev >= 0 && dev < 64) cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

int grid_for(const void *kernel, int threads, size_t smem, int64_t work_items) {
  // occupancy per (kernel, device), cached after the first query
  struct Entry {
    const void *k;
    int dev;
    size_t smem;
    int per_sm;
  };
  static Entry table[256];
  static int used = 0;
  static std::mutex mu;
  int dev = 0;
  cudaGetDevice(&dev);
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> g(mu);
    for (int i = 0; i < used; ++i)
      if (table[i].k == kernel && table[i].dev == dev && table[i].smem == smem) {
        per_sm = table[i].per_sm;
        break;
      }
  }
  if (per_sm == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) !=
            cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    std::lock_guard<std::mutex> g(mu);
    if (used < 256) table[used++] = Entry{kernel, dev, smem, per_sm};
  }
  const int64_t need = (work_items + threads - 1) / threads;
  const int64_t cap = (int64_t)sm_count() * per_sm;
  int64_t grid = need < cap ? need : cap;
  if (grid < 1) grid = 1;
  return (int)grid;
}

namespace {

__global__ void k_stats_reset(eig3_stats *s) {
  s->n_delta_clamped = 0ull;
  s->n_j2_clamped = 0ull;
  s->n_nonfinite = 0ull;
  s->min_disc_ratio = __longlong_as_double(0x7ff0000000000000ll);
  s->max_abs_lambda = 0.0;
  s->n_guarded = 0ull;
}

}  // namespace

cudaError_t launch_stats_reset(eig3_stats *stats, cudaStream_t s) {
  k_stats_reset<<<1, 1, 0, s>>>(stats);
  return cudaGetLastError();
}

}  // namespace eig3

namespace {

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

size_t elem_size(int dtype) { return dtype == EIG3_F64 ? 8 : 4; }

eig3_status check_modes(int layout, int dtype, int precision, int64_t n) {
  if (layout != EIG3_GENERAL9 && layout != EIG3_SYM6) return EIG3_ERR_LAYOUT;
  if (dtype != EIG3_F64 && dtype != EIG3_F32) return EIG3_ERR_DTYPE;
  if (precision != EIG3_PREC_F64 && precision != EIG3_PREC_F32_COMP &&
      precision != EIG3_PREC_F64_GUARDED && precision != EIG3_PREC_F32_COMP_A64)
    return EIG3_ERR_DTYPE;
  if ((precision == EIG3_PREC_F32_COMP || precision == EIG3_PREC_F32_COMP_A64) &&
      dtype != EIG3_F32)
    return EIG3_ERR_DTYPE;
  // n * 9 elements must be addressable with 64-bit offsets
  if (n < 0 || n > (INT64_MAX / 64)) return EIG3_ERR_ARG;
  return EIG3_OK;
}

eig3_status from_cuda(cudaError_t e) { return e == cudaSuccess ? EIG3_OK : EIG3_ERR_CUDA; }

}  // namespace

extern "C" {

eig3_status eig3_invariants(const void *A, int layout, int dtype, int precision, int64_t n,
                            double *inv, void *stream) {
  eig3_status st = check_modes(layout, dtype, precision, n);
  if (st != EIG3_OK) return st;
  if (precision == EIG3_PREC_F64_GUARDED || precision == EIG3_PREC_F32_COMP_A64)
    return EIG3_ERR_DTYPE;
  if (n == 0) return EIG3_OK;
  if (!A || !inv) return EIG3_ERR_ARG;
  if (!aligned(A, elem_size(dtype)) || !aligned(inv, 8)) return EIG3_ERR_ALIGN;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == EIG3_PREC_F32_COMP)
    return from_cuda(eig3::launch_invariants_f32c(A, layout, n, inv, s));
  return from_cuda(eig3::launch_invariants_f64(A, layout, dtype, n, inv, s));
}

eig3_status eig3_eigvals(const void *A, int layout, int dtype, int precision, int64_t n,
                         void *lam, void *aux, eig3_stats *stats, void *stream) {
  eig3_status st = check_modes(layout, dtype, precision, n);
  if (st != EIG3_OK) return st;
  if (n == 0) return EIG3_OK;
  if (!A || !lam) return EIG3_ERR_ARG;
  const size_t es = elem_size(dtype);
  if (!aligned(A, es) || !aligned(lam, es) || (aux && !aligned(aux, es)) ||
      (stats && !aligned(stats, 8)))
    return EIG3_ERR_ALIGN;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == EIG3_PREC_F32_COMP || precision == EIG3_PREC_F32_COMP_A64)
    return from_cuda(eig3::launch_eigvals_f32c(A, layout, n, lam, aux, stats,
                                               precision == EIG3_PREC_F32_COMP_A64, s));
  if (precision == EIG3_PREC_F64_GUARDED && layout == EIG3_GENERAL9)
    return from_cuda(eig3::launch_eigvals_guarded(A, dtype, n, lam, aux, stats, s));
  return from_cuda(eig3::launch_eigvals_f64(A, layout, dtype, n, lam, aux, stats, s));
}

eig3_status eig3_eigvals_backward(const void *A, int layout, int dtype, int precision, int64_t n,
                                  const void *grad_lam, const void *aux, void *grad_A,
                                  void *stream) {
  eig3_status st = check_modes(layout, dtype, precision, n);
  if (st != EIG3_OK) return st;
  if (n == 0) return EIG3_OK;
  if (!A || !grad_lam || !grad_A) return EIG3_ERR_ARG;
  const size_t es = elem_size(dtype);
  if (!aligned(A, es) || !aligned(grad_lam, es) || !aligned(grad_A, es) ||
      (aux && !aligned(aux, es)))
    return EIG3_ERR_ALIGN;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == EIG3_PREC_F32_COMP || precision == EIG3_PREC_F32_COMP_A64)
    return from_cuda(eig3::launch_backward_f32c(A, layout, n, grad_lam, aux, grad_A, s));
  // the guarded forward step only changes the adjoint inputs (r, sigma1,
  // sigma2): with aux given the binary64 adjoint is the same computation
  if (precision == EIG3_PREC_F64_GUARDED && layout == EIG3_GENERAL9 && !aux)
    return from_cuda(eig3::launch_backward_guarded(A, dtype, n, grad_lam, grad_A, s));
  return from_cuda(eig3::launch_backward_f64(A, layout, dtype, n, grad_lam, aux, grad_A, s));
}

eig3_status eig3_eigvals_vjp(const void *A, int layout, int dtype, int precision, int64_t n,
                             const void *w, void *lam, void *grad_A, eig3_stats *stats,
                             void *stream) {
  eig3_status st = check_modes(layout, dtype, precision, n);
  if (st != EIG3_OK) return st;
  if (precision == EIG3_PREC_F64_GUARDED || precision == EIG3_PREC_F32_COMP_A64)
    return EIG3_ERR_DTYPE;
  if (n == 0) return EIG3_OK;
  if (!A || !w || !grad_A) return EIG3_ERR_ARG;
  const size_t es = elem_size(dtype);
  if (!aligned(A, es) || !aligned(w, es) || !aligned(grad_A, es) || (lam && !aligned(lam, es)) ||
      (stats && !aligned(stats, 8)))
    return EIG3_ERR_ALIGN;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == EIG3_PREC_F32_COMP)
    return from_cuda(eig3::launch_eigvals_vjp_f32c(A, layout, n, w, lam, grad_A, stats, s));
  return from_cuda(eig3::launch_eigvals_vjp_f64(A, layout, dtype, n, w, lam, grad_A, stats, s));
}

eig3_status eig3_eigprojectors(const void *A, int layout, int dtype, int precision, int64_t n,
                               void *lam, void *P, void *stream) {
  eig3_status st = check_modes(layout, dtype, precision, n);
  if (st != EIG3_OK) return st;
  if (precision == EIG3_PREC_F64_GUARDED || precision == EIG3_PREC_F32_COMP_A64)
    return EIG3_ERR_DTYPE;
  if (n == 0) return EIG3_OK;
  if (!A || !P) return EIG3_ERR_ARG;
  const size_t es = elem_size(dtype);
  if (!aligned(A, es) || !aligned(P, es) || (lam && !aligned(lam, es))) return EIG3_ERR_ALIGN;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == EIG3_PREC_F32_COMP)
    return from_cuda(eig3::launch_projectors_f32c(A, layout, n, lam, P, s));
  return from_cuda(eig3::launch_projectors_f64(A, layout, dtype, n, lam, P, s));
}

eig3_status eig3_mohr_coulomb(const void *sigma, int layout, int dtype, int precision, int64_t n,
                              double s_yc, double m, void *f, void *grad_sigma, void *stream) {
  eig3_status st = check_modes(layout, dtype, precision, n);
  if (st != EIG3_OK) return st;
  if (precision == EIG3_PREC_F64_GUARDED || precision == EIG3_PREC_F32_COMP_A64)
    return EIG3_ERR_DTYPE;
  // S_yc and m are positive finite material constants (1/S_yc and m/S_yc
  // must be finite); checked before anything else is looked at.
  if (!(s_yc > 0.0) || !(m > 0.0) || !std::isfinite(s_yc) || !std::isfinite(m) ||
      !std::isfinite(1.0 / s_yc) || !std::isfinite(m / s_yc))
    return EIG3_ERR_ARG;
  if (n == 0) return EIG3_OK;
  if (!sigma || !f) return EIG3_ERR_ARG;
  const size_t es = elem_size(dtype);
  if (!aligned(sigma, es) || !aligned(f, es) || (grad_sigma && !aligned(grad_sigma, es)))
    return EIG3_ERR_ALIGN;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == EIG3_PREC_F32_COMP)
    return from_cuda(eig3::launch_mohr_coulomb_f32c(sigma, layout, n, s_yc, m, f, grad_sigma, s));
  return from_cuda(
      eig3::launch_mohr_coulomb_f64(sigma, layout, dtype, n, s_yc, m, f, grad_sigma, s));
}

eig3_status eig3_eigvals_variant(const void *A, int layout, int dtype, int variant, int64_t n,
                                 double *inv, void *lam, void *stream) {
  eig3_status st = check_modes(layout, dtype, EIG3_PREC_F64, n);
  if (st != EIG3_OK) return st;
  if (variant != EIG3_VARIANT_PRESENT && variant != EIG3_VARIANT_NAIVE &&
      variant != EIG3_VARIANT_NAIVE_TENSOR)
    return EIG3_ERR_ARG;
  if (n == 0) return EIG3_OK;
  if (!A || (!inv && !lam)) return EIG3_ERR_ARG;
  const size_t es = elem_size(dtype);
  if (!aligned(A, es) || (inv && !aligned(inv, 8)) || (lam && !aligned(lam, es)))
    return EIG3_ERR_ALIGN;
  return from_cuda(
      eig3::launch_variant_f64(A, layout, dtype, variant, n, inv, lam, (cudaStream_t)stream));
}

eig3_status eig3_stats_reset(eig3_stats *stats, void *stream) {
  if (!stats) return EIG3_ERR_ARG;
  if (!aligned(stats, 8)) return EIG3_ERR_ALIGN;
  return from_cuda(eig3::launch_stats_reset(stats, (cudaStream_t)stream));
}

const char *eig3_status_string(int status) {
  switch (status) {
    case EIG3_OK: return "EIG3_OK";
    case EIG3_ERR_ARG:
      return "EIG3_ERR_ARG: n < 0, a required pointer is NULL, or a scalar argument is out of range";
    case EIG3_ERR_LAYOUT: return "EIG3_ERR_LAYOUT: layout must be EIG3_GENERAL9 or EIG3_SYM6";
    case EIG3_ERR_DTYPE: return "EIG3_ERR_DTYPE: unsupported dtype/precision combination";
    case EIG3_ERR_ALIGN: return "EIG3_ERR_ALIGN: pointer not aligned to its element size";
    case EIG3_ERR_CUDA: return "EIG3_ERR_CUDA: kernel launch failed";
    default: return "EIG3 unknown status";
  }
}

int eig3_version(void) { return 10300; }

}  // extern "C"
