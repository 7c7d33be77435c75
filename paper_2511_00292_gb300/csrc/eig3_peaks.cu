// eig3_peaks.cu -- throughput loops for the roofline denominators of the
// benchmark: binary64 FMA, multiply and add, and binary32 FMA, each as a
// dependency-free unrolled body of C independent chains per thread.  The
// benchmark runs every loop over a few launch shapes and chain counts and
// takes the fastest as the pipe's measured peak.  Built as its own small
// library (libeig3_peaks.so), loaded only by the benchmark; not part of the
// eig3 ABI.
//
//   int eig3_peak_loop(int kind, int chains, int blocks, int threads, int iters,
//                      void *out, void *stream)
//     kind     0 DFMA, 1 DMUL, 2 DADD, 3 FFMA; 4 DFMA with two integer
//              operations per DFMA, 5 DFMA with two FFMA per DFMA (the binary64
//              pipe fed between other instructions, as in a real kernel; only
//              the DFMA are counted); 6 FFMA2 (the packed two-lane binary32
//              FMA, __ffma2_rn: one instruction, two FMAs), 7 FFMA2 with one
//              integer operation per FFMA2 (whether the packed form leaves
//              issue slots free for other work; only the FFMA2 are counted),
//              8 binary64 multiplications on the integer pipes
//              (softfp::mul_rn_int, the kernels' dmul)
//     chains   independent chains per thread: 2, 4, 8 or 16
//     blocks, threads   launch shape (threads <= 1024)
//     iters    loop trips; every trip issues `chains` instructions of `kind`
//              per thread
//     out      device buffer of blocks * threads elements (double for kinds
//              0-2, 4, 5, 8, float for 3, 6, 7): each thread's result, so that
//              nothing is optimised away
//   Returns the cudaError_t of the launch (0 on success); asynchronous on
//   `stream`.  Instructions executed = blocks * threads * iters * chains.
#include <cuda_runtime.h>

#include "eig3_dmul.cuh"

namespace {

template <int KIND, int C>
__global__ void __launch_bounds__(1024) k_peak64(int iters, double a, double b,
                                                 double *__restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double x[C], y[C];
#pragma unroll
  for (int j = 0; j < C; ++j) {
    x[j] = 1.0 + 1e-3 * (double)((t + j) & 255);
    y[j] = a + 1e-12 * (double)j;  // a separate multiplier per chain
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < C; ++j) {
      if constexpr (KIND == 0) x[j] = fma(x[j], y[j], b);
      if constexpr (KIND == 1) x[j] = x[j] * y[j];
      if constexpr (KIND == 2) x[j] = x[j] + b;
      if constexpr (KIND == 8) x[j] = eig3::softfp::mul_rn_int(x[j], y[j]);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < C; ++j) s += x[j];
  out[t] = s;
}

// DFMA chains with independent integer (MIX = 0) or binary32 FMA (MIX = 1)
// work between them, two such instructions per DFMA.
template <int MIX, int C>
__global__ void __launch_bounds__(1024) k_peak64_mixed(int iters, double a, double b,
                                                       double *__restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double x[C], y[C];
  unsigned k[C];
  float f[C];
#pragma unroll
  for (int j = 0; j < C; ++j) {
    x[j] = 1.0 + 1e-3 * (double)((t + j) & 255);
    y[j] = a + 1e-12 * (double)j;
    k[j] = (unsigned)(t * 2654435761u + j);
    f[j] = 1.0f + 1e-3f * (float)j;
  }
  const float fa = (float)a, fb = (float)b;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < C; ++j) {
      x[j] = fma(x[j], y[j], b);
      if constexpr (MIX == 0) {
        k[j] = (k[j] ^ (k[j] >> 7)) + (unsigned)i;
      } else {
        f[j] = fmaf(f[j], fa, fb);
        f[j] = fmaf(f[j], fa, fb);
      }
    }
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < C; ++j) s += x[j] + (double)(k[j] & 1u) * 1e-30 + (double)f[j] * 1e-30;
  out[t] = s;
}

template <int C>
__global__ void __launch_bounds__(1024) k_peak32(int iters, float a, float b,
                                                 float *__restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  float x[C];
#pragma unroll
  for (int j = 0; j < C; ++j) x[j] = 1.0f + 1e-3f * (float)((t + j) & 255);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < C; ++j) x[j] = fmaf(x[j], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < C; ++j) s += x[j];
  out[t] = s;
}

// Packed binary32 FMA chains (MIX = 1: one integer operation per FFMA2).
template <int MIX, int C>
__global__ void __launch_bounds__(1024) k_peak32x2(int iters, float a, float b,
                                                   float *__restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  float2 x[C];
  unsigned k[C];
#pragma unroll
  for (int j = 0; j < C; ++j) {
    x[j] = make_float2(1.0f + 1e-3f * (float)((t + j) & 255), 1.0f - 1e-3f * (float)j);
    k[j] = (unsigned)(t * 2654435761u + j);
  }
  const float2 va = make_float2(a, a), vb = make_float2(b, b);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < C; ++j) {
      x[j] = __ffma2_rn(x[j], va, vb);
      if constexpr (MIX == 1) k[j] ^= (unsigned)i;
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < C; ++j) s += x[j].x + x[j].y + (float)(k[j] & 1u) * 1e-30f;
  out[t] = s;
}

template <int C>
int launch(int kind, int blocks, int threads, int iters, void *out, cudaStream_t s) {
  // a, b chosen so that the chains neither overflow nor flush to zero over
  // any realistic trip count; passed at run time so nothing folds
  const double a = 0.99999999, b = 1e-9;
  double *o64 = static_cast<double *>(out);
  switch (kind) {
    case 0: k_peak64<0, C><<<blocks, threads, 0, s>>>(iters, a, b, o64); break;
    case 1: k_peak64<1, C><<<blocks, threads, 0, s>>>(iters, a, b, o64); break;
    case 2: k_peak64<2, C><<<blocks, threads, 0, s>>>(iters, a, b, o64); break;
    case 3:
      k_peak32<C><<<blocks, threads, 0, s>>>(iters, (float)a, (float)b, static_cast<float *>(out));
      break;
    case 4: k_peak64_mixed<0, C><<<blocks, threads, 0, s>>>(iters, a, b, o64); break;
    case 5: k_peak64_mixed<1, C><<<blocks, threads, 0, s>>>(iters, a, b, o64); break;
    case 6:
      k_peak32x2<0, C><<<blocks, threads, 0, s>>>(iters, (float)a, (float)b,
                                                  static_cast<float *>(out));
      break;
    case 8: k_peak64<8, C><<<blocks, threads, 0, s>>>(iters, a, b, o64); break;
    case 7:
      k_peak32x2<1, C><<<blocks, threads, 0, s>>>(iters, (float)a, (float)b,
                                                  static_cast<float *>(out));
      break;
    default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

}  // namespace

extern "C" int eig3_peak_loop(int kind, int chains, int blocks, int threads, int iters,
                              void *out, void *stream) {
  if (blocks < 1 || threads < 1 || threads > 1024 || iters < 0 || out == nullptr)
    return (int)cudaErrorInvalidValue;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (chains) {
    case 2: return launch<2>(kind, blocks, threads, iters, out, s);
    case 4: return launch<4>(kind, blocks, threads, iters, out, s);
    case 8: return launch<8>(kind, blocks, threads, iters, out, s);
    case 16: return launch<16>(kind, blocks, threads, iters, out, s);
    default: return (int)cudaErrorInvalidValue;
  }
}
