// eig3_f64.cuh -- binary64 device arithmetic of the closed-form 3x3 eigenvalue
// method (Habera & Zilian, arXiv 2511.00292), one matrix per thread.
//
// Everything here is written for the GB300 FP64 pipe, which issues about two
// DFMA per SM per clock (64x below FP32): every DADD/DMUL/DFMA counts, so the
// algorithms are evaluated with fused multiply-adds and with products shared
// between the invariants, between dx(A) and dx(A^T), and between the terms of
// Algorithm 5, and many of the plain products are formed on the integer pipes
// (dmul, bit-identical to the FP64 multiplication) to share the work.  The numerical structure of the paper is kept: the diagonal
// enters only through the differences d0, d1, d2, every r_i of Algorithm 5
// is a sum of products of small factors, and the discriminant is the weighted
// sum of products u_i v_i.  Only the grouping of the products changes (and
// three r_i of dx(M) come from exact identities between the others), which
// moves rounding errors by a few units in the last place.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "eig3_dmul.cuh"

namespace eig3 {

// A binary64 product on the integer pipes (softfp::mul_rn_int: the same bits
// as x * y).  With every operation on the FP64 pipe the kernels were bound by
// it while their integer pipes sat nearly idle, so the plain products of the
// invariants (Algorithms 2, 4 and 5), of the triple angle and of the adjoint
// are formed here and the FP64 pipe keeps the FMAs, the additions and the rest.
__device__ __forceinline__ double dmul(double x, double y) { return softfp::mul_rn_int(x, y); }

// Constants (binary64 nearest values).
constexpr double kInv3 = 0.333333333333333314829616256247390992939472198486328125;
constexpr double kInv6 = 0.1666666666666666574148081281236954964697360992431640625;
constexpr double kInv9 = 0.111111111111111104943205418749130330979824066162109375;
constexpr double kInv27 = 0.037037037037037034981127388472299207933247089385986328125;
constexpr double kHalfSqrt3 = 0.86602540378443859658830206171842291951179504394531250;
constexpr double kTwoOverSqrt3 = 1.1547005383792514621144972236652486026287078857421875;
// 2 / (3 sqrt 3): eigenvalue offsets are k * (...) with k = r * kK
constexpr double kK = 0.38490017945975052082056230772286653518676757812500;

// Invariants of one matrix.  J2, J3 and D are those of 2^-e A (e = 0 unless
// the deviatoric data was out of the safe exponent range, see dev_scale).
struct Inv {
  double I1, J2, J3, D;
  int e;
};

// Power-of-two scaling of the deviatoric data (the diagonal differences and
// the off-diagonal entries).  Delta is of degree 6 in these, so without it
// Delta underflows once their magnitude m drops below about 1e-51 (and
// overflows above 1e51), and the triple angle is lost.  When the largest
// exponent lies outside [2^-150, 2^150) the data is multiplied by 2^-e so that
// m lies in [1, 2); the angle does not depend on the scale and r is scaled
// back exactly.  The test is a few integer operations on the high words; the
// nine multiplications only run for matrices that need them.
__device__ __forceinline__ int hi_abs(double x) { return __double2hiint(x) & 0x7fffffff; }

__device__ __forceinline__ double pow2d(int k) {  // 2^k for -1022 <= k <= 1023
  return __hiloint2double((k + 1023) << 20, 0);
}

// max(x, 0) by the sign bit (integer pipe, not the FP64 pipe); -0 and NaNs
// with the sign bit set give +0, like fmax(x, 0).
__device__ __forceinline__ double nonneg(double x) { return __double2hiint(x) < 0 ? 0.0 : x; }

// Conversions for the binary32 seed, done with integer operations: on GB300
// the float<->double conversion instructions occupy the FP64 pipe, the
// integer pipe is idle.
// Non-negative double -> float, mantissa truncated (relative error < 2^-23);
// values below the binary32 normal range give 0.
__device__ __forceinline__ float seed_float(double x) {
  const int hi = __double2hiint(x);
  const int e = (hi >> 20) & 0x7ff;
  const int f = ((e - 896) << 23) | ((hi & 0xfffff) << 3) | (int)((unsigned)__double2loint(x) >> 29);
  return (e < 897) ? 0.0f : __int_as_float(f);
}

// Non-negative normal float -> double, exactly (0 for zero and subnormals).
__device__ __forceinline__ double widen(float f) {
  const int b = __float_as_int(f);
  return ((b & 0x7f800000) == 0) ? 0.0 : __hiloint2double((b >> 3) + (896 << 20), b << 29);
}

// Binary32 reciprocal and reciprocal square root of a normal seed: one MUFU
// instruction each (PTX rcp.approx / rsqrt.approx, relative error below
// 2^-22), without the subnormal and special-value paths of the IEEE forms.
__device__ __forceinline__ float rcp_seed(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float rsqrt_seed(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// seed_float(x 2^-s) and widen(f) 2^s for values outside the binary32 range:
// the exponent is moved by integer arithmetic on the high word.  The caller
// picks s so that the results stay in range; zero and subnormal x give 0.
__device__ __forceinline__ float seed_float_scaled(double x, int s) {
  const int hi = __double2hiint(x);
  const int E = (hi >> 20) & 0x7ff;
  const int e = E - s;
  const int f = ((e - 896) << 23) | ((hi & 0xfffff) << 3) | (int)((unsigned)__double2loint(x) >> 29);
  return (E == 0 || e < 897) ? 0.0f : __int_as_float(f);
}

__device__ __forceinline__ double widen_scaled(float f, int s) {
  const int b = __float_as_int(f);
  return ((b & 0x7f800000) == 0) ? 0.0 : __hiloint2double((b >> 3) + ((896 + s) << 20), b << 29);
}

// A double from its two 32-bit words through an opaque move.  Exponent
// arithmetic done on the words (x 2^k for a k the code knows is in range)
// would otherwise be recognised by the compiler as a multiplication by a
// power of two and issued on the FP64 pipe, in some kernels and not others.
__device__ __forceinline__ double from_words(int hi, int lo) {
  double r;
  asm("mov.b64 %0, {%1, %2};" : "=d"(r) : "r"(lo), "r"(hi));
  return r;
}

// Square root and reciprocal from binary32 seeds, corrected by a truncated
// binomial series in binary64.  The correction is a handful of FMAs on the
// FP64 pipe; the seed, the exponent handling and the special cases run on the
// FP32, MUFU and integer pipes.  Both are faithful (error below one unit in
// the last place), not correctly rounded.
//
// sqrt(c x), x >= 0, c = 1 or 3: with x = 2^(2k) x', x' in [1, 4), and a
// binary32 seed y0 ~ (c x')^(-1/2) (rsqrt_seed of the truncated c x': relative
// error below 2^-21; for c = 3 rounded down to 22 significant bits, below
// 2^-20, so that c y0 is exact in binary32),
//   sqrt(c x') = g (1 - t)^(-1/2) = g (1 + t/2 + (3/8) t^2 + ...),  g = x' (c y0),  t = 1 - g y0,
// truncated after t^2 (the next term is below 2^-60 g).  Forming t from the
// rounded g cancels half of g's rounding error.  Zero and subnormal x give 0;
// infinity and NaN pass through.
//
// sqrt_nonneg_split returns the same root as a product sqrt(C x) = s 2^k with
// s = sqrt(C x') in [1, 2 sqrt3) (k set; s = 0, k = 0 for zero and subnormal
// x; s = x, k = 0 for infinity and NaN), for callers that want the scale of
// the root apart from it.
template <int C = 1>
__device__ __forceinline__ double sqrt_nonneg_split(double x, int &k) {
  static_assert(C == 1 || C == 3, "factor 1 or 3");
  const int hi = __double2hiint(x);
  const int E = (hi >> 20) & 0x7ff;
  const int kk = (E - 1023) >> 1;
  const double xs = from_words(hi - (kk << 21), __double2loint(x));
  float y0 = rsqrt_seed((float)C * seed_float(xs));
  if (C == 3) y0 = __int_as_float(__float_as_int(y0) & ~3);
  const double g = xs * widen((float)C * y0);
  const double h = fma(-g, widen(0.5f * y0), 0.5);  // t / 2
  const double s = fma(g * h, fma(1.5, h, 1.0), g);
  const bool special = (E == 0) || (E == 0x7ff);
  k = special ? 0 : kk;
  return (E == 0) ? 0.0 : ((E == 0x7ff) ? x : s);
}

template <int C = 1>
__device__ __forceinline__ double sqrt_nonneg(double x) {
  int k;
  const double s = sqrt_nonneg_split<C>(x, k);
  return from_words(__double2hiint(s) + (k << 20), __double2loint(s));
}

// 1/x for positive normal x: with x = 2^k x', x' in [1, 2), the binary32
// reciprocal c0 of the truncated x' (rcp_seed; e = 1 - x' c0 is below 2^-21)
// and 1/x' = c0 / (1 - e) = c0 (1 + e + e^2 + ...), truncated after e^2.
__device__ __forceinline__ double recip_pos(double x) {
  const int hi = __double2hiint(x);
  const int k = ((hi >> 20) & 0x7ff) - 1023;
  const double xs = from_words(hi - (k << 20), __double2loint(x));
  const double c0 = widen(rcp_seed(seed_float(xs)));
  const double e = fma(-xs, c0, 1.0);
  const double c = fma(c0, fma(e, e, e), c0);
  return from_words(__double2hiint(c) - (k << 20), __double2loint(c));
}

// 1/(3x) for a positive normal x, as recip_pos: the binary32 seed of
// 1/(3x') is cut to 22 significant bits so that its triple is exact in
// binary32, and e = 1 - x' (3 c0) is one FMA; three FP64-pipe instructions,
// the factor 1/3 costing none.
__device__ __forceinline__ double recip3_pos(double x) {
  const int hi = __double2hiint(x);
  const int k = ((hi >> 20) & 0x7ff) - 1023;
  const double xs = from_words(hi - (k << 20), __double2loint(x));
  const float cf =
      __int_as_float(__float_as_int(rcp_seed(seed_float(xs)) * (1.0f / 3.0f)) & ~3);
  const double c0 = widen(cf);
  const double e = fma(-xs, widen(3.0f * cf), 1.0);
  const double c = fma(c0, fma(e, e, e), c0);
  return from_words(__double2hiint(c) - (k << 20), __double2loint(c));
}

// x 2^k by adding k to the exponent field (integer pipe): exact for normal x
// whose result stays below the overflow threshold, which the caller ensures
// (|k| small, |x| far from it).  Zero, subnormal and non-finite x are
// returned unchanged, so zeros stay exact; a subnormal x enters its
// product without the factor, an error below 2^-1019 |y| for x y that the
// callers' magnitudes (deviatoric data scaled into [2^-150, 2^150]) keep far
// under every rounding error of the sums it enters.
// Written in PTX: from the same steps in C the compiler may recognise a
// multiplication by 2^k and issue it on the FP64 pipe.
__device__ __forceinline__ double times_pow2(double x, int k) {
  double r;
  asm("{\n\t.reg .b32 lo, hi, f, t;\n\t.reg .pred p, q;\n\t"
      "mov.b64 {lo, hi}, %1;\n\tand.b32 f, hi, 0x7ff00000;\n\t"
      "setp.ne.u32 p, f, 0;\n\tsetp.ne.u32 q, f, 0x7ff00000;\n\tand.pred p, p, q;\n\t"
      "add.s32 t, hi, %2;\n\tselp.b32 hi, t, hi, p;\n\tmov.b64 %0, {lo, hi};\n\t}"
      : "=d"(r)
      : "d"(x), "r"(k << 20));
  return r;
}

// x 2^k for any x and |k| < 2^11 by exponent arithmetic, saturating: a
// result beyond the binary64 range becomes +-infinity, one below the normal
// range +-0 (no subnormal results); zero, subnormal and non-finite x are
// returned unchanged.  For rarely taken rescalings that must not touch the
// FP64 pipe.
__device__ __forceinline__ double times_pow2_sat(double x, int k) {
  double r;
  asm("{\n\t.reg .b32 lo, hi, e, ne, sg, t, l2;\n\t.reg .pred pk, po, pu;\n\t"
      "mov.b64 {lo, hi}, %1;\n\tbfe.u32 e, hi, 20, 11;\n\tadd.s32 ne, e, %2;\n\t"
      "and.b32 sg, hi, 0x80000000;\n\tsetp.ne.u32 pk, e, 0;\n\t"
      "setp.ne.and.u32 pk, e, 2047, pk;\n\tsetp.ge.s32 po, ne, 2047;\n\t"
      "setp.le.s32 pu, ne, 0;\n\tshl.b32 t, %2, 20;\n\tadd.s32 t, hi, t;\n\t"
      "mov.b32 l2, lo;\n\t@po or.b32 t, sg, 0x7ff00000;\n\t@po mov.b32 l2, 0;\n\t"
      "@pu mov.b32 t, sg;\n\t@pu mov.b32 l2, 0;\n\tselp.b32 hi, t, hi, pk;\n\t"
      "selp.b32 lo, l2, lo, pk;\n\tmov.b64 %0, {lo, hi};\n\t}"
      : "=d"(r)
      : "d"(x), "r"(k));
  return r;
}

// x 2^k exactly as the binary64 product x * 2^k rounds it, for any x and
// |k| < 2^11, by integer operations on the bits (no FP64-pipe instruction):
// a subnormal x is normalised first, a result below the normal range is
// rounded to nearest even into the subnormals, one beyond it is +-infinity,
// zero and non-finite x are returned unchanged.  For the rescalings of the
// rare out-of-range data (whose FP64 multiplications were issued, predicated
// off, by every warp) and for the powers of two of the fused adjoint.
__device__ __forceinline__ double scale2k(double x, int k) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned long long sign = b & 0x8000000000000000ull;
  const unsigned long long mag = b ^ sign;
  int E = (int)(mag >> 52);
  if (E == 0x7ff || mag == 0) return x;
  unsigned long long m;
  if (E == 0) {
    const int s = __clzll((long long)mag) - 11;
    m = mag << s;
    E = 1 - s;
  } else {
    m = (mag & 0xfffffffffffffull) | 0x10000000000000ull;
  }
  const int ne = E + k;
  if (ne >= 0x7ff) return from_words((int)((sign | 0x7ff0000000000000ull) >> 32), 0);
  if (ne >= 1) {
    const unsigned long long r = sign | ((unsigned long long)ne << 52) | (m & 0xfffffffffffffull);
    return from_words((int)(r >> 32), (int)(unsigned)r);
  }
  const int sh = 1 - ne;  // >= 1: the result is subnormal (or rounds up to 2^-1022)
  if (sh > 54) return from_words((int)(sign >> 32), 0);
  const unsigned long long q = m >> sh, rem = m & ((1ull << sh) - 1), half = 1ull << (sh - 1);
  const unsigned long long r = q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
  return from_words((int)((sign | r) >> 32), (int)(unsigned)(sign | r));
}

// |x| by clearing the sign bit (integer pipe, in PTX for the same reason: a
// floating-point absolute value would take an FP64-pipe slot).
__device__ __forceinline__ double abs_bits64(double x) {
  double r;
  asm("{\n\t.reg .b32 lo, hi;\n\tmov.b64 {lo, hi}, %1;\n\tand.b32 hi, hi, 0x7fffffff;\n\t"
      "mov.b64 %0, {lo, hi};\n\t}"
      : "=d"(r)
      : "d"(x));
  return r;
}

// min of two non-negative doubles: their bit patterns order like their values.
__device__ __forceinline__ double min_nonneg(double a, double b) {
  return __double_as_longlong(a) < __double_as_longlong(b) ? a : b;
}

// x < 0 (excluding -0) by the bits.
__device__ __forceinline__ bool negative(double x) {
  const int hi = __double2hiint(x);
  return hi < 0 && ((hi & 0x7fffffff) | __double2loint(x)) != 0;
}

template <int N>
__device__ __forceinline__ int dev_scale(double (&v)[N]) {
  int h = hi_abs(v[0]);
#pragma unroll
  for (int j = 1; j < N; ++j) h = max(h, hi_abs(v[j]));
  const int E = h >> 20;  // biased exponent of the largest magnitude
  int e = 0;
  if (E < 1023 - 150 || E >= 1023 + 150) {
    e = min(max(E, 1), 2045) - 1023;  // zero / subnormal data: scale by 2^1022
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = scale2k(v[j], -e);
  }
  return e;
}

// What the invariants hand on to the fused vector-Jacobian product, all of
// the scaled data 2^-e A: the sums that give dev(A)'s diagonal,
// 3 (S00, S11, S22) = (tn, -t2, -t1), the off-diagonal entries, and the pair
// products that the cofactors of S = dev(A) are made of.  Filled only when
// the caller asks for it (a null pointer otherwise; nothing is then kept).
struct ShareG {
  double t1, t2, tn;
  double a01, a02, a10, a12, a20, a21;
  double p01, p02, p12;                              // A01 A10, A02 A20, A12 A21
  double m0112, m0210, m0221, m2001, m1021, m2012;   // A01 A12, A02 A10, A02 A21,
                                                     // A20 A01, A10 A21, A20 A12
};

struct ShareS {
  double t1, t2, tn;
  double a, b, c;                 // A01, A02, A12
  double aa, bb, cc, ab, ac, bc;  // their products
};

// --------------------------------------------------------------------------
// General 9-entry matrix: Algorithms 1, 2, 4, 5.
// --------------------------------------------------------------------------
//
// dx(M) of Algorithm 5 for M = A and M = A^T.  Products that are the same for
// A and A^T (A01 A10, A02 A20, A12 A21, products of the d's) are formed once.
// Reading R1 (r10 = M01 d1 d2 + M02 M21 d2 + M01 M02 M20 - M01^2 M10) applies.
//
// Factored forms used below (each is the paper's r_i regrouped, no terms
// dropped; the diagonal still enters only through d0, d1, d2):
//   r1  = (M01 M12) M20 - (M02 M10) M21      (for A^T: -r1 of A)
//   r2  = M01 X - M02 (M02 M21),              X = M01 M12 - M02 d2
//   r3  = M01 (M21 d1 - M01 M20) + M21 (M02 M21)
//   r4  = M12 (M02 d0 + M01 M12) - M02 (M02 M10)
//   r5  = r12 + r13,  r6 = r11 - r10,  r7 = r8 - r9   (identities for any M:
//         the d0 d2, d1 d2 and d0 d1 terms cancel, d0 + d2 = d1, d1 - d2 = d0,
//         d1 - d0 = d2; each is one addition of two computed r's, whose
//         rounding errors, like those of the direct sums, are units of u on
//         terms of size |M|^3)
//   r8  = d1 (M12 d0 - M02 M10) + M12 (M01 M10 - M12 M21)
//   r9  = d0 Y + M12 (M02 M20 - M12 M21),     Y = M12 d1 - M02 M10
//   r10 = M01 (d1 d2 + M02 M20 - M01 M10) + d2 (M02 M21)
//   r11 = M01 (d1 d2 + M12 M21 - M01 M10) + d1 (M02 M21)
//   r12 = M02 (M12 M21 - M02 M20 - d0 d2) + d0 (M01 M12)
//   r13 = M02 (d0 d2 + M02 M20 - M01 M10) + d2 (M01 M12)
//   r14 = d0 (d1 d2 - M01 M10) + d1 (M02 M20) - d2 (M12 M21)   (same for A^T)
struct DxShared {
  double d0, d1, d2;
  double p01, p02, p12;  // A01 A10, A02 A20, A12 A21
  double e8, e9;         // p01 - p12, p02 - p12
  double q10, q11, q12, q13;
};

struct Dx {
  double r2, r3, r4, r5, r6, r7, r8, r9, r10, r11, r12, r13;  // r1 is formed by the caller
  double m0221;                                               // M02 M21
};

// r2 .. r13 of dx(M); m0112 = M01 M12 and m0210 = M02 M10 come from the caller
// (for M = A they are shared with J3 and r1).
__device__ __forceinline__ Dx dx13(double M01, double M02, double M10, double M12, double M20,
                                   double M21, double m0112, double m0210, const DxShared &s) {
  Dx r;
  const double m0221 = dmul(M02, M21);
  const double m0120 = dmul(M01, M20);
  const double X = fma(-M02, s.d2, m0112);
  const double Y = fma(M12, s.d1, -m0210);
  r.r2 = fma(M01, X, -dmul(M02, m0221));
  r.r3 = fma(M01, fma(M21, s.d1, -m0120), dmul(M21, m0221));
  r.r4 = fma(M12, fma(M02, s.d0, m0112), -dmul(M02, m0210));
  r.r8 = fma(s.d1, fma(M12, s.d0, -m0210), dmul(M12, s.e8));
  r.r9 = fma(s.d0, Y, dmul(M12, s.e9));
  r.r10 = fma(M01, s.q10, dmul(s.d2, m0221));
  r.r11 = fma(M01, s.q11, dmul(s.d1, m0221));
  r.r12 = fma(M02, s.q12, dmul(s.d0, m0112));
  r.r13 = fma(M02, s.q13, dmul(s.d2, m0112));
  // r5 = r12 + r13, r6 = r11 - r10, r7 = r8 - r9 for any M: the terms with
  // d0 d2, d1 d2 and d0 d1 cancel, and the diagonal differences satisfy
  // d0 + d2 = d1, d1 - d2 = d0, d1 - d0 = d2
  r.r5 = r.r12 + r.r13;
  r.r6 = r.r11 - r.r10;
  r.r7 = r.r8 - r.r9;
  r.m0221 = m0221;
  return r;
}

// a[0..8] row-major.  Returns the four invariants (unclamped); fills *x when
// given (see ShareG).
__device__ __forceinline__ Inv invariants_general(const double (&a)[9], ShareG *x = nullptr) {
  const double a00 = a[0], a11 = a[4], a22 = a[8];
  Inv o;
  // Algorithm 1
  o.I1 = (a00 + a11) + a22;
  // diagonal differences (shared by Algorithms 2, 4, 5), then the scaling
  double sv[9] = {a00 - a11, a00 - a22, a11 - a22, a[1], a[2], a[3], a[5], a[6], a[7]};
  o.e = dev_scale<9>(sv);
  DxShared s;
  s.d0 = sv[0];
  s.d1 = sv[1];
  s.d2 = sv[2];
  const double a01 = sv[3], a02 = sv[4], a10 = sv[5], a12 = sv[6], a20 = sv[7], a21 = sv[8];
  s.p01 = dmul(a01, a10);
  s.p02 = dmul(a02, a20);
  s.p12 = dmul(a12, a21);
  // Algorithm 2: diag/6 + offdiag
  o.J2 = fma(fma(s.d0, s.d0, fma(s.d1, s.d1, dmul(s.d2, s.d2))), kInv6, (s.p01 + s.p02) + s.p12);
  // Algorithm 5's differences of the paired products, shared with J3:
  // e8 = A01 A10 - A12 A21, e9 = A02 A20 - A12 A21
  s.e8 = s.p01 - s.p12;
  s.e9 = s.p02 - s.p12;
  // Algorithm 4: offdiag + mixed/3 - t1 t2 t3 / 27 with t1 = d1 + d2,
  // t2 = d0 - d2, t3 = -(d0 + d1) = -tn.  As t1 + t2 + t3 = 0,
  // mixed = A01 A10 t1 + A02 A20 t2 + A12 A21 t3 = t1 e8 + t2 e9, so
  //   mixed/3 - t1 t2 t3/27 = (1/3) [t1 (e8 + t2 tn / 9) + t2 e9]
  const double t1 = s.d1 + s.d2;
  const double t2 = s.d0 - s.d2;
  const double tn = s.d0 + s.d1;
  // A01 A12 A20 + A02 A10 A21; the same two triple products give r1 of
  // Algorithm 5 for A, and r1 for A^T is its negative (A10 A21 A02 - A20 A01 A12)
  const double m0112 = dmul(a01, a12), m0210 = dmul(a02, a10);
  const double q = dmul(m0210, a21);
  const double offdiag = fma(m0112, a20, q);
  o.J3 = fma(fma(t1, fma(t2, dmul(tn, kInv9), s.e8), dmul(t2, s.e9)), kInv3, offdiag);
  // Algorithm 5 (reading R1 for r10).  The bracketed sums of r10 .. r14 are
  // single FMAs (d1 d2 + (A02 A20 - A01 A10) and so on); p12 - p01 = -e8 and
  // p12 - p02 = -e9 exactly.
  const double f0201 = s.p02 - s.p01;
  s.q10 = fma(s.d1, s.d2, f0201);
  s.q11 = fma(s.d1, s.d2, -s.e8);
  s.q12 = fma(-s.d0, s.d2, -s.e9);
  s.q13 = fma(s.d0, s.d2, f0201);
  const double r14 = fma(s.d0, fma(s.d1, s.d2, -s.p01), fma(s.d1, s.p02, -dmul(s.d2, s.p12)));
  const double r1 = fma(m0112, a20, -q);
  const double m1021 = dmul(a10, a21), m2001 = dmul(a20, a01);
  const Dx u = dx13(a01, a02, a10, a12, a20, a21, m0112, m0210, s);
  const Dx v = dx13(a10, a20, a01, a21, a02, a12, m1021, m2001, s);
  if (x) {
    *x = ShareG{t1,    t2,    tn,    a01,   a02,     a10,   a12,  a20,     a21,
                s.p01, s.p02, s.p12, m0112, m0210, u.m0221, m2001, m1021, v.m0221};
  }
  // sum_i w_i u_i v_i, w = (9, 6, 6, 6, 8, 8, 8, 2, 2, 2, 2, 2, 2, 1), as one FMA
  // chain: w1 u1 v1 = 9 r1 (-r1), the power-of-two weights 2 and 8 applied to
  // u_i exactly on the integer pipe (times_pow2), the weight-6 group last
  double acc = fma(dmul(-9.0, r1), r1, dmul(r14, r14));
  acc = fma(times_pow2(u.r13, 1), v.r13, acc);
  acc = fma(times_pow2(u.r12, 1), v.r12, acc);
  acc = fma(times_pow2(u.r11, 1), v.r11, acc);
  acc = fma(times_pow2(u.r10, 1), v.r10, acc);
  acc = fma(times_pow2(u.r9, 1), v.r9, acc);
  acc = fma(times_pow2(u.r8, 1), v.r8, acc);
  acc = fma(times_pow2(u.r7, 3), v.r7, acc);
  acc = fma(times_pow2(u.r6, 3), v.r6, acc);
  acc = fma(times_pow2(u.r5, 3), v.r5, acc);
  o.D = fma(6.0, fma(u.r2, v.r2, fma(u.r3, v.r3, dmul(u.r4, v.r4))), acc);
  return o;
}

// --------------------------------------------------------------------------
// Symmetric matrix, stored (A00, A11, A22, A12, A02, A01).
// With A = A^T, dx(A) = dx(A^T), r1 = 0, r2 = r7, r3 = r5, r4 = r6, so
// Delta = 14 (r2^2 + r3^2 + r4^2) + 2 (r8^2 + ... + r13^2) + r14^2.
// --------------------------------------------------------------------------
__device__ __forceinline__ Inv invariants_sym(const double (&s6)[6], ShareS *x = nullptr) {
  const double a00 = s6[0], a11 = s6[1], a22 = s6[2];
  Inv o;
  o.I1 = (a00 + a11) + a22;
  double sv[6] = {a00 - a11, a00 - a22, a11 - a22, s6[3], s6[4], s6[5]};
  o.e = dev_scale<6>(sv);
  const double d0 = sv[0], d1 = sv[1], d2 = sv[2];
  const double c = sv[3];  // A12
  const double b = sv[4];  // A02
  const double a = sv[5];  // A01
  const double aa = dmul(a, a), bb = dmul(b, b), cc = dmul(c, c);
  const double ab = dmul(a, b), ac = dmul(a, c), bc = dmul(b, c);
  o.J2 = fma(fma(d0, d0, fma(d1, d1, dmul(d2, d2))), kInv6, (aa + bb) + cc);
  // Algorithm 4 as in the general case, (1/3) [t1 (e8 + t2 tn / 9) + t2 e9]
  // with e8 = aa - cc, e9 = bb - cc
  const double fba = bb - aa, fac = aa - cc, fbc = bb - cc;
  const double t1 = d1 + d2, t2 = d0 - d2, tn = d0 + d1;
  const double offdiag = scale2k(dmul(ab, c), 1);
  o.J3 = fma(fma(t1, fma(t2, dmul(tn, kInv9), fac), dmul(t2, fbc)), kInv3, offdiag);
  if (x) *x = ShareS{t1, t2, tn, a, b, c, aa, bb, cc, ab, ac, bc};
  const double r8 = fma(d1, fma(c, d0, -ab), dmul(c, fac));
  const double r9 = fma(d0, fma(c, d1, -ab), dmul(c, fbc));
  const double r10 = fma(a, fma(d1, d2, fba), dmul(d2, bc));
  const double r11 = fma(a, fma(d1, d2, -fac), dmul(d1, bc));
  const double r12 = fma(b, fma(-d0, d2, -fbc), dmul(d0, ac));
  const double r13 = fma(b, fma(d0, d2, fba), dmul(d2, ac));
  // r2 = r8 - r9, r3 = r12 + r13, r4 = r11 - r10: the identities of dx13 (the
  // diagonal differences satisfy d1 - d0 = d2, d0 + d2 = d1, d1 - d2 = d0)
  const double r2 = r8 - r9;
  const double r3 = r12 + r13;
  const double r4 = r11 - r10;
  const double r14 = fma(d0, fma(d1, d2, -aa), fma(d1, bb, -dmul(d2, cc)));
  // 14 (r2^2 + r3^2 + r4^2) + 2 (r8^2 + ... + r13^2) + r14^2 as one FMA chain, the
  // weight 2 applied on the integer pipe (times_pow2)
  double acc = dmul(r14, r14);
  acc = fma(times_pow2(r13, 1), r13, acc);
  acc = fma(times_pow2(r12, 1), r12, acc);
  acc = fma(times_pow2(r11, 1), r11, acc);
  acc = fma(times_pow2(r10, 1), r10, acc);
  acc = fma(times_pow2(r9, 1), r9, acc);
  acc = fma(times_pow2(r8, 1), r8, acc);
  o.D = fma(14.0, fma(r2, r2, fma(r3, r3, dmul(r4, r4))), acc);
  return o;
}

// --------------------------------------------------------------------------
// Algorithm 6, angle part.  With x = 27 J3 and y = sqrt(27 Delta+) the triple
// angle is phi = atan2(y, x) in [0, pi] (reading R2); any positive multiple
// of (x, y) gives the same angle, and the caller passes (J3, sqrt(Delta+/27)).  The kernel needs
//   sigma1 = sin(phi / 3)          and   sigma2 = sin((pi - phi) / 3),
// from which cos(phi/3) = (2 sigma2 + sigma1) / sqrt 3 and the three
// eigenvalues follow without cancellation, and which are also the adjoint's
// eigenvalue gaps (lambda2 - lambda1 and lambda3 - lambda2, up to 2r/sqrt3).
//
// The folded angle phi~ = atan2(y, |x|) in [0, pi/2] is phi when x >= 0 and
// pi - phi when x < 0, so both sigmas come from psi~ = phi~/3 in [0, pi/6]:
// the small one is sin(psi~) and the other sin(pi/3 - psi~).
//
// cos(psi~) + i sin(psi~) is the principal cube root of z / |z| with
// z = |x| + i y.  It is obtained without a binary64 arctangent or sine: a
// binary32 seed w0 = e^{i psi0} (atan2f and __sincosf on the power-of-two
// scaled z) is rotated by eps = arg(z conj(w0)^3) / 3, the Newton correction
// of the cube root on the unit circle, and renormalised.  With |3 eps| below
// about 1e-5 the neglected terms (eps^3, and t^3 in arg = t - t^3/3) are
// below 1e-17, so the result carries binary64 accuracy; the conditioning is
// that of phi itself (the three cube roots are 120 degrees apart).
// --------------------------------------------------------------------------
__device__ __forceinline__ void triple_angle_sines(double x, double y, double &sigma1,
                                                   double &sigma2) {
  const double ax = abs_bits64(x);
  // the seeds are taken from 2^-s |x| and 2^-s y, s the exponent of max(|x|, y),
  // so that their maximum lies in [1, 2); the binary64 steps below use |x| and y
  // themselves (|z| < 2^460 for the scaled deviatoric data)
  const int h = max(__double2hiint(ax), __double2hiint(y));
  const int s = min((h >> 20) & 0x7ff, 2045) - 1023;
  // binary32 seed w0 = c0 + i s0 (pf in [0, pi/6], so c0, s0 >= 0)
  const float pf = atan2f(seed_float_scaled(y, s), seed_float_scaled(ax, s)) * (1.0f / 3.0f);
  float sf, cf;
  __sincosf(pf, &sf, &cf);
  const double c0 = widen(cf), s0 = widen(fmaxf(sf, 0.0f));
  const double cc = dmul(c0, c0), ss = dmul(s0, s0);  // exact: 24-bit factors
  // w0^3 = c0 (c0^2 - 3 s0^2) + i s0 (3 c0^2 - s0^2)
  const double a3 = dmul(c0, fma(-3.0, ss, cc));
  const double b3 = dmul(s0, fma(3.0, cc, -ss));
  // rho = z conj(w0^3); its argument is 3 eps (|3 eps| ~ 1e-6: arg = Im/Re to 1e-18)
  const double re = fma(ax, a3, dmul(y, b3));
  const double im = fma(y, a3, -dmul(ax, b3));
  // eps = im / (3 re): a binary32 seed rc0 of 1/(3 re) with 22 significant bits
  // (so that 3 rc0 is exact) and one Newton step, rc0 (1 + e), e = 1 - 3 re rc0
  const float rcf =
      __int_as_float(__float_as_int(rcp_seed(seed_float_scaled(re, s)) * (1.0f / 3.0f)) & ~3);
  const double rc0 = widen_scaled(rcf, -s);
  const double e = fma(-re, widen_scaled(3.0f * rcf, -s), 1.0);
  // z = 0 (or both |x| and y subnormal): the angle is undetermined, keep phi = 0
  const double eps = (h >= (1 << 20)) ? dmul(im, fma(rc0, e, rc0)) : 0.0;
  // 1/|w0| to second order in eta0 = |w0|^2 - 1 (|eta0| ~ 1e-7), folded into
  // the rotation w~ = w0 e^{i eps} / |w0| with e^{i eps} = 1 - eps^2/2 + i eps
  const double eta0 = (cc - 1.0) + ss;
  const double f0 = fma(eta0, fma(eta0, 0.375, -0.5), 1.0);
  const double ef = dmul(f0, eps);
  const double cef = fma(-times_pow2(eps, -1), ef, f0);  // eps/2 on the integer pipe
  const double ct = fma(c0, cef, -dmul(s0, ef));
  const double st = nonneg(fma(s0, cef, dmul(c0, ef)));
  const double other = fma(kHalfSqrt3, ct, -times_pow2(st, -1));  // sin(pi/3 - psi~)
  // sign test on the bits: x = -0 goes with x < 0, as atan2(0, -0) = pi does
  const bool pos = __double2hiint(x) >= 0;
  sigma1 = pos ? st : other;
  sigma2 = pos ? other : st;
}

// Algorithm 6, eigenvalues: lambda_k = I1/3 + (2/3) r cos((phi + 2 pi k)/3),
// r = sqrt(3 J2+), written with the sigmas:
//   lambda_1 = I1/3 - k (sigma2 + 2 sigma1)
//   lambda_2 = I1/3 + k (sigma1 - sigma2)
//   lambda_3 = I1/3 + k (2 sigma2 + sigma1),     k = 2 r / (3 sqrt 3).
// With sigma1, sigma2 >= 0 and monotone rounding the order
// lambda_1 <= lambda_2 <= lambda_3 holds exactly.
struct Eig {
  double l1, l2, l3;  // ascending
  double r, sigma1, sigma2;
  bool j2_clamped, d_clamped;
};

__device__ __forceinline__ Eig eigvals_from_inv(const Inv &v) {
  Eig o;
  o.j2_clamped = negative(v.J2);
  o.d_clamped = negative(v.D);
  const double J2p = nonneg(v.J2);
  const double Dp = nonneg(v.D);
  o.r = sqrt_nonneg<3>(J2p);
  if (v.e != 0) o.r = scale2k(o.r, v.e);
  // (J3, sqrt(Delta/27)) has the direction of (27 J3, sqrt(27 Delta))
  triple_angle_sines(v.J3, sqrt_nonneg(Dp * kInv27), o.sigma1, o.sigma2);
  const double k = o.r * kK;
  const double i3 = v.I1 * kInv3;
  o.l1 = fma(-k, fma(2.0, o.sigma1, o.sigma2), i3);
  o.l2 = fma(k, o.sigma1 - o.sigma2, i3);
  o.l3 = fma(k, fma(2.0, o.sigma2, o.sigma1), i3);
  return o;
}

// --------------------------------------------------------------------------
// Adjoint.  lambda_k = I1/3 + mu_k with mu_k the roots of mu^3 - J2 mu - J3
// (the trigonometric formula solves exactly this depressed cubic).  The chain
// rule through I1, J2, J3 gives
//   dL/dA = a_I1 I + a_J2 dev(A)^T + a_J3 dev(cof(dev A))
// (Jacobians of J2 and J3 from the Lemmas of Sections J2 and J3) with
//   a_I1 = sum_k g_k / 3,
//   a_J2 = sum_k g_k mu_k / p'(mu_k),   a_J3 = sum_k g_k / p'(mu_k),
// p'(mu_k) = prod_{j != k} (mu_k - mu_j).  These are divided differences of
// the weights over the nodes mu_1 <= mu_2 <= mu_3:
//   a_J3 = g[mu1, mu2, mu3] = (D23 - D12) / (mu3 - mu1),
//   a_J2 = mu1 a_J3 + D23,   D12 = (g2 - g1)/(mu2 - mu1), D23 = (g3 - g2)/(mu3 - mu2).
// The gaps come straight from the angle: mu2 - mu1 = (2r/sqrt3) sigma1,
// mu3 - mu2 = (2r/sqrt3) sigma2, mu3 - mu1 = (2r/sqrt3)(sigma1 + sigma2), so
// a coalescing pair enters only through the difference of its weights.
// Where a computed gap is exactly 0 the pair's divided difference is taken as
// 0, i.e. the cluster's weights are replaced by their mean; r = 0 (a triple
// eigenvalue) leaves a_I1 I.
//
// With r = m 2^k (m in [1, 2)) the scalars are carried as a_J2 2^k and
// a_J3 2^2k: these depend only on m, the sigmas and the weights, so they
// neither over- nor underflow for matrices of any scale, and the gradient
// routines apply 2^-k and 2^-2k exactly (or, out of range, 2^-k to dev(A)).
// One reciprocal R = 1/(m P), P = s1 s2 s3, serves every divided difference.
// --------------------------------------------------------------------------
struct Adj {
  double aI1, aJ2s, aJ3s;  // a_I1, a_J2 2^k, a_J3 2^2k
  double n2, g2;           // adjoint_vjp: a_I1 = g2 + n2 / 3, finished in the gradient
  int k;                   // r = m 2^k; 0 when r = 0
  bool rz;                 // r = 0 (or subnormal): a triple eigenvalue, a_J2 = a_J3 = 0
};

__device__ __forceinline__ Adj adjoint_scalars(double r, double sigma1, double sigma2, double g1,
                                               double g2, double g3) {
  // Sigmas below 2^-960 count as exact coalescence (divided difference 0).
  const bool z1 = hi_abs(sigma1) < (63 << 20);
  const bool z2 = hi_abs(sigma2) < (63 << 20);
  const double s1 = z1 ? 1.0 : sigma1, s2 = z2 ? 1.0 : sigma2;
  const double s3 = sigma1 + sigma2;  // >= sin(pi/6) cos(pi/6): never 0
  // The gaps are (2r/sqrt3) sigma1, (2r/sqrt3) sigma2 and (2r/sqrt3)(sigma1 +
  // sigma2); with Rh = (sqrt3/2) / (P m), P = s1 s2 s3, their reciprocals
  // times 2^k are (s2 s3) Rh, (s1 s3) Rh and (s1 s2) Rh.
  const int hr = hi_abs(r);
  const bool rz = hr < (1 << 20);  // r = 0 or subnormal: a triple eigenvalue
  const int kr = min((hr >> 20) - 1023, 1022);
  const double m = rz ? 1.0 : scale2k(r, -kr);  // r 2^-kr on the integer pipe
  const double s12 = dmul(s1, s2);
  const double P = dmul(s12, s3);
  const double R = recip_pos(m * P);
  const double Rh = kHalfSqrt3 * R;
  double n12 = g2 - g1, n23 = g3 - g2;
  if (z1 || z2) {  // an exactly coalesced pair takes the mean of its two weights
    n12 = z1 ? 0.0 : 0.5 * (g2 + g3) - g1;
    n23 = z2 ? 0.0 : g3 - 0.5 * (g1 + g2);
  }
  const double D12 = n12 * ((s2 * s3) * Rh);
  const double D23 = n23 * ((s1 * s3) * Rh);
  const double aJ3s = (D23 - D12) * (s12 * Rh);
  // mu1 2^-k = -kK m (2 sigma1 + sigma2)
  const double aJ2s = fma((-kK * m) * fma(2.0, sigma1, sigma2), aJ3s, D23);
  Adj o;
  o.aI1 = ((g1 + g2) + g3) * kInv3;
  o.aJ2s = rz ? 0.0 : aJ2s;
  o.aJ3s = rz ? 0.0 : aJ3s;
  o.k = rz ? 0 : kr;
  o.rz = rz;
  return o;
}

// The adjoint scalars for the three unit weights e_1, e_2, e_3 at once (the
// eigenprojectors), from the same single reciprocal: with X12 = (sqrt3/2)/s1,
// X23 = (sqrt3/2)/s2, X13 = (sqrt3/2)/s3 and c = -kK (2 sigma1 + sigma2), for
// distinct eigenvalues
//   e_1: r^2 a_J3 =  X12 X13,          r a_J2 = c (r^2 a_J3)
//   e_2: r^2 a_J3 = -(X12 + X23) X13,  r a_J2 = c (r^2 a_J3) - X23
//   e_3: r^2 a_J3 =  X23 X13,          r a_J2 = c (r^2 a_J3) + X23
// (each sums to 0 over k, so sum_k E_k = I exactly in real arithmetic); an
// exactly coalesced pair shares the mean of its two weights.
struct Adj3 {
  double b2[3], b3[3], inv_r;
};

__device__ __forceinline__ Adj3 adjoint_units(double r, double sigma1, double sigma2) {
  const bool z1 = hi_abs(sigma1) < (63 << 20);
  const bool z2 = hi_abs(sigma2) < (63 << 20);
  const double s1 = z1 ? 1.0 : sigma1, s2 = z2 ? 1.0 : sigma2;
  const double s3 = sigma1 + sigma2;
  const int hr = hi_abs(r);
  const bool rz = hr < (1 << 20);
  const int kr = min((hr >> 20) - 1023, 1022);
  const double m = rz ? 1.0 : scale2k(r, -kr);  // r 2^-kr on the integer pipe
  const double s12 = dmul(s1, s2);
  const double P = dmul(s12, s3);
  const double R = recip_pos(m * P);
  const double Rh = kHalfSqrt3 * (m * R);
  const double X12 = (s2 * s3) * Rh;
  const double X23 = (s1 * s3) * Rh;
  const double X13 = s12 * Rh;
  const double c = -kK * fma(2.0, sigma1, sigma2);
  Adj3 o;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    // weights e_k, with an exactly coalesced pair taking the mean of its two
    const double g1 = k == 0 ? 1.0 : 0.0, g2 = k == 1 ? 1.0 : 0.0, g3 = k == 2 ? 1.0 : 0.0;
    const double D12 = z1 ? 0.0 : ((z2 ? 0.5 * (g2 + g3) : g2) - g1) * X12;
    const double D23 = z2 ? 0.0 : (g3 - (z1 ? 0.5 * (g1 + g2) : g2)) * X23;
    o.b3[k] = (D23 - D12) * X13;
    o.b2[k] = fma(c, o.b3[k], D23);
  }
  o.inv_r = rz ? 0.0 : scale2k(P * R, -kr);
  return o;
}

// Eigenprojectors E_k = d lambda_k/dA ^T = I/3 + (r a_J2) S^ + (r^2 a_J3) dev(cof S^)^T
// with S^ = dev(A)/r, written as 27 values (k-major, row-major 3 x 3).
// Input: the 9 entries of a general matrix, or the 6 of a symmetric one.
template <int N>
__device__ __forceinline__ void projectors(const double (&a)[N], const Adj3 &s, double (&E)[27]) {
  const double ir = s.inv_r;
  double d0, d1, d2, S01, S02, S10, S12, S20, S21;
  if constexpr (N == 9) {
    d0 = a[0] - a[4];
    d1 = a[0] - a[8];
    d2 = a[4] - a[8];
    S01 = a[1] * ir;
    S02 = a[2] * ir;
    S10 = a[3] * ir;
    S12 = a[5] * ir;
    S20 = a[6] * ir;
    S21 = a[7] * ir;
  } else {
    d0 = a[0] - a[1];
    d1 = a[0] - a[2];
    d2 = a[1] - a[2];
    S12 = S21 = a[3] * ir;
    S02 = S20 = a[4] * ir;
    S01 = S10 = a[5] * ir;
  }
  const double ir3 = ir * kInv3;
  const double S00 = (d0 + d1) * ir3;
  const double S11 = (d2 - d0) * ir3;
  const double S22 = -(d1 + d2) * ir3;
  const double S[9] = {S00, S01, S02, S10, S11, S12, S20, S21, S22};
  // Ct = cof(S^)^T = adj(S^), row-major
  const double Ct[9] = {fma(S11, S22, -(S12 * S21)), fma(S02, S21, -(S01 * S22)),
                        fma(S01, S12, -(S02 * S11)), fma(S12, S20, -(S10 * S22)),
                        fma(S00, S22, -(S02 * S20)), fma(S02, S10, -(S00 * S12)),
                        fma(S10, S21, -(S11 * S20)), fma(S01, S20, -(S00 * S21)),
                        fma(S00, S11, -(S01 * S10))};
  const double tc = ((Ct[0] + Ct[4]) + Ct[8]) * kInv3;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      const bool diag = (j == 0 || j == 4 || j == 8);
      const double cj = diag ? Ct[j] - tc : Ct[j];
      E[9 * k + j] = fma(s.b2[k], S[j], fma(s.b3[k], cj, diag ? kInv3 : 0.0));
    }
  }
}

// The gradient weights from b2 = a_J2 2^k and b3 = a_J3 2^2k (in place):
// while r and the entries of dev(A) lie in [2^-448, 2^448], b2 *= 2^-k and
// b3 *= 2^-2k (exact) and dev(A) is used as it is; otherwise dev(A) is
// multiplied by 2^-k instead (exact; zero for r = 0, where b2 = b3 = 0), so
// that its products stay in range.  Every term of the gradient is the same
// either way.
template <int N>
__device__ __forceinline__ void grad_units(double (&D)[N], const Adj &s, double &b2, double &b3) {
  int h = hi_abs(D[0]);
#pragma unroll
  for (int j = 1; j < N; ++j) h = max(h, hi_abs(D[j]));
  const int E = h >> 20;
  // the powers of two by exponent arithmetic (scale2k, rounding as the
  // products would): the rare branch's N multiplications were issued by every
  // warp with its lanes predicated off
  if (E >= 1023 - 448 && E <= 1023 + 448 && s.k >= -448 && s.k <= 448) {
    b2 = scale2k(b2, -s.k);
    b3 = scale2k(b3, -2 * s.k);
  } else {
    // r = 0 (whose data are finite) takes D * 0: zeros of D's sign
#pragma unroll
    for (int j = 0; j < N; ++j)
      D[j] = s.rz ? __hiloint2double(__double2hiint(D[j]) & (int)0x80000000, 0)
                  : scale2k(D[j], -s.k);
  }
}

// Gradient of a general matrix from the adjoint scalars, G[0..8] row-major:
//   G = a_I1 I + a_J2 dev(A)^T + a_J3 (C - tr(C)/3 I),  C = cof(dev A),
// the diagonal written as (a_I1 - a_J3 tr(C)/3) + a_J2 dev(A)_ii + a_J3 C_ii.
__device__ __forceinline__ void grad_general(const double (&a)[9], const Adj &s, double (&G)[9]) {
  const double d0 = a[0] - a[4], d1 = a[0] - a[8], d2 = a[4] - a[8];
  // dev(A): diagonal from the differences, exact for A = alpha I
  double D[9] = {(d0 + d1) * kInv3, a[1], a[2], a[3], (d2 - d0) * kInv3, a[5], a[6], a[7],
                 -(d1 + d2) * kInv3};
  double b2 = s.aJ2s, b3 = s.aJ3s;
  grad_units<9>(D, s, b2, b3);
  const double S00 = D[0], S01 = D[1], S02 = D[2], S10 = D[3], S11 = D[4], S12 = D[5];
  const double S20 = D[6], S21 = D[7], S22 = D[8];
  const double C00 = fma(S11, S22, -(S12 * S21));
  const double C01 = fma(S12, S20, -(S10 * S22));
  const double C02 = fma(S10, S21, -(S11 * S20));
  const double C10 = fma(S02, S21, -(S01 * S22));
  const double C11 = fma(S00, S22, -(S02 * S20));
  const double C12 = fma(S01, S20, -(S00 * S21));
  const double C20 = fma(S01, S12, -(S02 * S11));
  const double C21 = fma(S02, S10, -(S00 * S12));
  const double C22 = fma(S00, S11, -(S01 * S10));
  const double base = fma(-b3, ((C00 + C11) + C22) * kInv3, s.aI1);
  G[0] = fma(b2, S00, fma(b3, C00, base));
  G[1] = fma(b2, S10, b3 * C01);
  G[2] = fma(b2, S20, b3 * C02);
  G[3] = fma(b2, S01, b3 * C10);
  G[4] = fma(b2, S11, fma(b3, C11, base));
  G[5] = fma(b2, S21, b3 * C12);
  G[6] = fma(b2, S02, b3 * C20);
  G[7] = fma(b2, S12, b3 * C21);
  G[8] = fma(b2, S22, fma(b3, C22, base));
}

// Gradient with respect to the six stored entries of a symmetric matrix:
// diagonal G_ii, off-diagonal G_ij + G_ji = 2 (a_J2 S_ij + a_J3 C_ij) (S =
// dev(A) and cof(S) are symmetric).  Output order (A00, A11, A22, A12, A02, A01).
__device__ __forceinline__ void grad_sym(const double (&s6)[6], const Adj &s, double (&G)[6]) {
  const double d0 = s6[0] - s6[1], d1 = s6[0] - s6[2], d2 = s6[1] - s6[2];
  double D[6] = {(d0 + d1) * kInv3, (d2 - d0) * kInv3, -(d1 + d2) * kInv3, s6[3], s6[4], s6[5]};
  double b2 = s.aJ2s, b3 = s.aJ3s;
  grad_units<6>(D, s, b2, b3);
  const double S00 = D[0], S11 = D[1], S22 = D[2], S12 = D[3], S02 = D[4], S01 = D[5];
  const double C00 = fma(S11, S22, -(S12 * S12));
  const double C11 = fma(S00, S22, -(S02 * S02));
  const double C22 = fma(S00, S11, -(S01 * S01));
  const double C12 = fma(S01, S02, -(S00 * S12));
  const double C02 = fma(S01, S12, -(S02 * S11));
  const double C01 = fma(S12, S02, -(S01 * S22));
  const double base = fma(-b3, ((C00 + C11) + C22) * kInv3, s.aI1);
  const double b2x2 = 2.0 * b2, b3x2 = 2.0 * b3;
  G[0] = fma(b2, S00, fma(b3, C00, base));
  G[1] = fma(b2, S11, fma(b3, C11, base));
  G[2] = fma(b2, S22, fma(b3, C22, base));
  G[3] = fma(b2x2, S12, b3x2 * C12);
  G[4] = fma(b2x2, S02, b3x2 * C02);
  G[5] = fma(b2x2, S01, b3x2 * C01);
}

// --------------------------------------------------------------------------
// Fused forward + vector-Jacobian product (eig3_eigvals_vjp): the eigenvalues
// and the gradient of L = sum_k w_k lambda_k in one pass per matrix.  The
// adjoint is taken in the frame of the scaled data 2^-e A: the part
// a_J2 dev(A)^T + a_J3 dev(cof dev A) of the gradient is homogeneous of degree
// 0 in dev(A), and the scaling is by a power of two, so the scaled data give
// it exactly; and the quantities the invariants formed are reused:
//   * dev(A)'s diagonal from the sums t1, t2, tn of Algorithm 4,
//     3 (S00, S11, S22) = (tn, -t2, -t1);
//   * every cofactor of S = dev(A) is one FMA on a pair product of Algorithms
//     2, 4 and 5: C00 = S11 S22 - A12 A21, C01 = A12 A20 - S10 S22, and so on;
//   * tr(cof S) = ((tr S)^2 - tr(S^2)) / 2 = -J2 for the trace-free S, so the
//     diagonal shift of dev(cof S) is the computed J2 / 3;
//   * r = m 2^kr from the square root's own split, and kK m serves both the
//     eigenvalue offsets and the adjoint.
// --------------------------------------------------------------------------
struct EigV {
  Eig e;       // eigenvalues of A (l1, l2, l3), the sigmas and the clamp flags
  double m;    // r of 2^-e A = m 2^kr, m in [1, 2 sqrt3); 0 for r = 0
  int kr;
  double kKm;  // kK m
  double c12;  // 2 sigma1 + sigma2
};

// Algorithm 6 as in eigvals_from_inv (the same eigenvalues bit for bit), with
// the scale of r kept apart.
__device__ __forceinline__ EigV eigvals_vjp_fwd(const Inv &v) {
  EigV o;
  o.e.j2_clamped = negative(v.J2);
  o.e.d_clamped = negative(v.D);
  const double J2p = nonneg(v.J2);
  const double Dp = nonneg(v.D);
  o.m = sqrt_nonneg_split<3>(J2p, o.kr);
  triple_angle_sines(v.J3, sqrt_nonneg(Dp * kInv27), o.e.sigma1, o.e.sigma2);
  o.kKm = dmul(kK, o.m);
  // k = kK r of A itself = kK m 2^(kr + e): for unscaled data (e = 0) the
  // exponent is added on the integer pipe (kK m 2^kr is a normal number:
  // J2+ >= 2^-1074 keeps r above 2^-537), otherwise by two exact scalings
  // (scale2k) that round, over- and underflow like the products themselves
  const double k =
      (v.e == 0) ? times_pow2(o.kKm, o.kr) : scale2k(scale2k(o.kKm, o.kr), v.e);
  o.e.r = o.m;  // r of the scaled data up to 2^kr (the fused kernel stores no r)
  const double i3 = dmul(v.I1, kInv3);
  o.c12 = fma(2.0, o.e.sigma1, o.e.sigma2);
  o.e.l1 = fma(-k, o.c12, i3);
  o.e.l2 = fma(k, o.e.sigma1 - o.e.sigma2, i3);
  o.e.l3 = fma(k, fma(2.0, o.e.sigma2, o.e.sigma1), i3);
  return o;
}

// The adjoint scalars of adjoint_scalars (a_I1, a_J2 2^kr, a_J3 2^2kr, in
// the scaled frame) from the forward's m, kr, kK m and 2 sigma1 + sigma2:
//   D23 = n23 s1 (s3 Rh),  D23 - D12 = D23 - n12 s2 (s3 Rh),
//   a_J3 2^2k = (D23 - D12) s1 s2 Rh,  a_J2 2^k = D23 - kK m (2 s1 + s2) a_J3 2^2k,
// with Rh = (sqrt3/2) / (m s1 s2 s3), and a_I1 = g2 + (n23 - n12)/3 (the
// last step in the gradient).
__device__ __forceinline__ Adj adjoint_vjp(const EigV &f, double g1, double g2, double g3) {
  const double sigma1 = f.e.sigma1, sigma2 = f.e.sigma2;
  const bool z1 = hi_abs(sigma1) < (63 << 20);
  const bool z2 = hi_abs(sigma2) < (63 << 20);
  const double s1 = z1 ? 1.0 : sigma1, s2 = z2 ? 1.0 : sigma2;
  const double s3 = sigma1 + sigma2;
  const bool rz = hi_abs(f.m) < (1 << 20);  // r = 0: a triple eigenvalue
  const double km = rz ? kK : f.kKm;         // kK m, m = 1 for r = 0
  const double s12 = dmul(s1, s2);
  const double P = dmul(s12, s3);
  // Rh = (sqrt3/2) / (m P) = 1 / (3 kK m P): the factor in the seed (recip3_pos)
  const double Rh = recip3_pos(dmul(km, P));
  double n12 = g2 - g1, n23 = g3 - g2;
  Adj o;
  // a_I1 = (g1 + g2 + g3)/3 = g2 + (n23 - n12)/3, finished in the gradient's
  // diagonal constant (grad_*_vjp)
  o.n2 = n23 - n12;
  o.g2 = g2;
  if (z1 || z2) {  // an exactly coalesced pair takes the mean of its two weights
    n12 = z1 ? 0.0 : 0.5 * (g2 + g3) - g1;
    n23 = z2 ? 0.0 : g3 - 0.5 * (g1 + g2);
  }
  const double s3Rh = dmul(s3, Rh);
  const double D23 = dmul(n23, dmul(s1, s3Rh));
  const double aJ3s = dmul(fma(-dmul(n12, s2), s3Rh, D23), dmul(s12, Rh));
  const double aJ2s = fma(-dmul(f.kKm, f.c12), aJ3s, D23);
  o.aJ2s = rz ? 0.0 : aJ2s;
  o.aJ3s = rz ? 0.0 : aJ3s;
  o.k = rz ? 0 : f.kr;
  o.rz = rz;
  return o;
}

// b2 = a_J2, b3 = a_J3 of the scaled frame from the carried a_J2 2^k and
// a_J3 2^2k, as grad_units does it but without a branch: while they and the
// scaled deviatoric data stay inside 2^+-448 (always, but for J2 tiny against
// the data of a nearly defective matrix), b2 = a_J2 2^k 2^-k and b3 = a_J3
// 2^2k 2^-2k; otherwise b2, b3 stay as carried and the data and products are
// shifted by 2^-k and 2^-2k instead.  The scalings of b2, b3 (exact, as the
// products by 2^-k and 2^-2k would round) and the shift returned (0 in
// range, applied by times_pow2_sat) are integer operations, so neither case
// takes an FP64-pipe slot.
__device__ __forceinline__ int vjp_units(const Adj &s, int hmax, double &b2, double &b3) {
  const int E = hmax >> 20;
  const bool in_range = E >= 1023 - 448 && E <= 1023 + 448 && s.k >= -448 && s.k <= 448;
  const double u2 = scale2k(s.aJ2s, in_range ? -s.k : 0);
  const double u3 = scale2k(s.aJ3s, in_range ? -2 * s.k : 0);
  b2 = u2;
  b3 = u3;
  return in_range ? 0 : -s.k;
}

// Gradient of a general matrix from the fused adjoint, G[0..8] row-major
// (as grad_general: a_I1 I + a_J2 dev(A)^T + a_J3 dev(cof dev A)).
__device__ __forceinline__ void grad_general_vjp(const ShareG &x, double J2, const Adj &s,
                                                 double (&G)[9]) {
  double D[9] = {dmul(x.tn, kInv3), x.a01, x.a02, x.a10, -dmul(x.t2, kInv3), x.a12, x.a20, x.a21,
                 -dmul(x.t1, kInv3)};
  int h = hi_abs(D[0]);
#pragma unroll
  for (int j = 1; j < 9; ++j) h = max(h, hi_abs(D[j]));
  double b2, b3;
  const int sh = vjp_units(s, h, b2, b3);
  double P[10] = {x.p12, x.m2012, x.m1021, x.m0221, x.p02, x.m2001, x.m0112, x.m0210, x.p01, J2};
  if (sh != 0) {
#pragma unroll
    for (int j = 0; j < 9; ++j) D[j] = times_pow2_sat(D[j], sh);
#pragma unroll
    for (int j = 0; j < 10; ++j) P[j] = times_pow2_sat(P[j], 2 * sh);
  }
  // diagonal: b2 S_ii + b3 C_ii + base, C_ii the 2x2 minors
  const double C0 = fma(D[4], D[8], -P[0]);
  const double C4 = fma(D[0], D[8], -P[4]);
  const double C8 = fma(D[0], D[4], -P[8]);
  // a_I1 - a_J3 tr(cof S) / 3 = g2 + (n23 - n12 + a_J3 J2) / 3
  const double base = fma(fma(b3, P[9], s.n2), kInv3, s.g2);
  G[0] = fma(b2, D[0], fma(b3, C0, base));
  G[4] = fma(b2, D[4], fma(b3, C4, base));
  G[8] = fma(b2, D[8], fma(b3, C8, base));
  // off-diagonal: b2 S_ji + b3 (P - S_ji S_kk) = S_ji (b2 - b3 S_kk) + b3 P, the
  // bracket shared by the two entries with the same S_kk
  const double q0 = fma(-b3, D[0], b2), q4 = fma(-b3, D[4], b2), q8 = fma(-b3, D[8], b2);
  G[1] = fma(D[3], q8, dmul(b3, P[1]));
  G[3] = fma(D[1], q8, dmul(b3, P[3]));
  G[2] = fma(D[6], q4, dmul(b3, P[2]));
  G[6] = fma(D[2], q4, dmul(b3, P[6]));
  G[5] = fma(D[7], q0, dmul(b3, P[5]));
  G[7] = fma(D[5], q0, dmul(b3, P[7]));
}

// The symmetric form (gradient with respect to the six stored entries, as
// grad_sym), cofactors C00 = S11 S22 - c^2, C12 = ab - S00 c, ... on the
// products of invariants_sym.
__device__ __forceinline__ void grad_sym_vjp(const ShareS &x, double J2, const Adj &s,
                                             double (&G)[6]) {
  double D[6] = {x.tn * kInv3, -(x.t2 * kInv3), -(x.t1 * kInv3), x.c, x.b, x.a};
  int h = hi_abs(D[0]);
#pragma unroll
  for (int j = 1; j < 6; ++j) h = max(h, hi_abs(D[j]));
  double b2, b3;
  const int sh = vjp_units(s, h, b2, b3);
  double P[7] = {x.cc, x.bb, x.aa, x.ab, x.ac, x.bc, J2};
  if (sh != 0) {
#pragma unroll
    for (int j = 0; j < 6; ++j) D[j] = times_pow2_sat(D[j], sh);
#pragma unroll
    for (int j = 0; j < 7; ++j) P[j] = times_pow2_sat(P[j], 2 * sh);
  }
  const double S00 = D[0], S11 = D[1], S22 = D[2];
  const double C00 = fma(S11, S22, -P[0]);
  const double C11 = fma(S00, S22, -P[1]);
  const double C22 = fma(S00, S11, -P[2]);
  const double C12 = fma(-S00, D[3], P[3]);
  const double C02 = fma(-S11, D[4], P[4]);
  const double C01 = fma(-S22, D[5], P[5]);
  const double base = fma(fma(b3, P[6], s.n2), kInv3, s.g2);
  const double b2x2 = 2.0 * b2, b3x2 = 2.0 * b3;
  G[0] = fma(b2, D[0], fma(b3, C00, base));
  G[1] = fma(b2, D[1], fma(b3, C11, base));
  G[2] = fma(b2, D[2], fma(b3, C22, base));
  G[3] = fma(b2x2, D[3], b3x2 * C12);
  G[4] = fma(b2x2, D[4], b3x2 * C02);
  G[5] = fma(b2x2, D[5], b3x2 * C01);
}

}  // namespace eig3
