// eig3_stats.cuh -- per-launch numerical statistics: each thread accumulates
// in registers over its grid-stride loop, the block reduces with warp
// shuffles and shared memory, and one thread per block commits with atomics
// (a few hundred atomics per launch, whatever n is).
#pragma once

#include <cuda_runtime.h>

#include "eig3.h"

namespace eig3 {

// max |lambda| is kept as bit patterns (non-negative doubles and floats order
// like their bits), so the per-matrix work runs on the integer pipe, not the
// FP64 pipe: max_bits for binary64 results, max_bits32 for binary32 ones.
struct StatAcc {
  unsigned long long n_d, n_j2, n_nf;
  unsigned long long max_bits;
  unsigned max_bits32;
  float min_ratio_f;
};

__device__ __forceinline__ void stat_init(StatAcc &a) {
  a.n_d = a.n_j2 = a.n_nf = 0ull;
  a.min_ratio_f = __int_as_float(0x7f800000);  // +inf
  a.max_bits = 0ull;
  a.max_bits32 = 0u;
}

// Bit pattern of |x|: the sign bit cleared in PTX, so that the compiler does
// not turn the integer mask back into a floating-point absolute value (which
// it would issue on the FP64 pipe).
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  unsigned long long r;
  asm("{\n\t.reg .b32 lo, hi;\n\tmov.b64 {lo, hi}, %1;\n\tand.b32 hi, hi, 0x7fffffff;\n\t"
      "mov.b64 %0, {lo, hi};\n\t}"
      : "=l"(r)
      : "d"(x));
  return r;
}

__device__ __forceinline__ unsigned abs_bits(float x) {
  unsigned r;
  asm("and.b32 %0, %1, 0x7fffffff;" : "=r"(r) : "r"(__float_as_uint(x)));
  return r;
}

// One matrix: clamps, finiteness, Delta+/J2+^3 and max |lambda|.  The ratio
// comes from the computed triple angle instead of a binary64 division:
// Delta = 4 J2^3 sin^2(phi), and with s = sin(psi~) (the smaller of the two
// sigmas) sin(phi) = sin(3 psi~) = s (3 - 4 s^2), so the ratio is
// 4 (s (3 - 4 s^2))^2, evaluated in binary32 (a diagnostic, not a result).
// The eigenvalues are finite exactly when the largest absolute bit pattern
// lies below that of infinity.
__device__ __forceinline__ void stat_common(StatAcc &a, bool d_clamped, bool j2_clamped,
                                            bool has_angle, float s_small, bool finite) {
  a.n_d += d_clamped ? 1ull : 0ull;
  a.n_j2 += j2_clamped ? 1ull : 0ull;
  a.n_nf += finite ? 0ull : 1ull;
  if (has_angle && finite) {
    const float sp = s_small * fmaf(-4.0f * s_small, s_small, 3.0f);
    a.min_ratio_f = fminf(a.min_ratio_f, 4.0f * sp * sp);
  }
}

__device__ __forceinline__ void stat_add(StatAcc &a, bool d_clamped, bool j2_clamped,
                                         bool has_angle, float s_small, double l1, double l2,
                                         double l3) {
  const unsigned long long m = max(abs_bits(l1), max(abs_bits(l2), abs_bits(l3)));
  const bool finite = m < 0x7ff0000000000000ull;
  if (finite) a.max_bits = max(a.max_bits, m);
  stat_common(a, d_clamped, j2_clamped, has_angle, s_small, finite);
}

__device__ __forceinline__ void stat_add(StatAcc &a, bool d_clamped, bool j2_clamped,
                                         bool has_angle, float s_small, float l1, float l2,
                                         float l3) {
  const unsigned m = max(abs_bits(l1), max(abs_bits(l2), abs_bits(l3)));
  const bool finite = m < 0x7f800000u;
  if (finite) a.max_bits32 = max(a.max_bits32, m);
  stat_common(a, d_clamped, j2_clamped, has_angle, s_small, finite);
}

// Block-wide reduction and commit.  Every thread of the block must call it.
__device__ __forceinline__ void stat_flush(StatAcc a, eig3_stats *s) {
  const unsigned full = 0xffffffffu;
  // the binary32 maximum joins the binary64 one (one conversion per thread)
  a.max_bits = max(a.max_bits, (unsigned long long)__double_as_longlong(
                                   (double)__uint_as_float(a.max_bits32)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a.n_d += __shfl_xor_sync(full, a.n_d, o);
    a.n_j2 += __shfl_xor_sync(full, a.n_j2, o);
    a.n_nf += __shfl_xor_sync(full, a.n_nf, o);
    a.min_ratio_f = fminf(a.min_ratio_f, __shfl_xor_sync(full, a.min_ratio_f, o));
    a.max_bits = max(a.max_bits, __shfl_xor_sync(full, a.max_bits, o));
  }
  __shared__ StatAcc part[32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = (blockDim.x + 31) >> 5;
  if (lane == 0) part[warp] = a;
  __syncthreads();
  if (warp == 0) {
    StatAcc b;
    if (lane < nwarps) {
      b = part[lane];
    } else {
      stat_init(b);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      b.n_d += __shfl_xor_sync(full, b.n_d, o);
      b.n_j2 += __shfl_xor_sync(full, b.n_j2, o);
      b.n_nf += __shfl_xor_sync(full, b.n_nf, o);
      b.min_ratio_f = fminf(b.min_ratio_f, __shfl_xor_sync(full, b.min_ratio_f, o));
      b.max_bits = max(b.max_bits, __shfl_xor_sync(full, b.max_bits, o));
    }
    if (lane == 0) {
      if (b.n_d) atomicAdd(&s->n_delta_clamped, b.n_d);
      if (b.n_j2) atomicAdd(&s->n_j2_clamped, b.n_j2);
      if (b.n_nf) atomicAdd(&s->n_nonfinite, b.n_nf);
      // non-negative doubles order like their bit patterns
      atomicMin(reinterpret_cast<unsigned long long *>(&s->min_disc_ratio),
                (unsigned long long)__double_as_longlong((double)b.min_ratio_f));
      atomicMax(reinterpret_cast<unsigned long long *>(&s->max_abs_lambda), b.max_bits);
    }
  }
}

}  // namespace eig3
