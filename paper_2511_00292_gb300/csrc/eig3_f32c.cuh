// eig3_f32c.cuh -- compensated binary32 evaluation of the invariants (I1, J2,
// J3, Delta of Algorithms 1, 2, 4, 5) and of the eigenvalues (Algorithm 6),
// one matrix per thread, with no binary64 arithmetic except in the optional
// ANGLE64 form of eigvals_c (precision EIG3_PREC_F32_COMP_A64), which takes the
// final combination of Delta and the triple angle in binary64.
//
// GB300 issues binary32 FMAs 64 times faster than binary64 ones, so this path
// buys accuracy with extra binary32 operations instead:
//   * error-free transformations: TwoSum (Knuth) and TwoProduct through the
//     fused multiply-add; sums of products are accumulated in the manner of
//     Ogita, Rump and Oishi, "Accurate sum and dot product", SIAM J. Sci.
//     Comput. 26 (2005) (Sum2 / Dot2: the result is as accurate as if computed
//     in twice the working precision and then rounded);
//   * the diagonal differences d0, d1, d2 are exact as (hi, lo) pairs;
//   * per-matrix power-of-two scaling of the deviatoric data (the d's and the
//     off-diagonal entries) so that its largest magnitude lies in [1, 2): no
//     overflow or underflow in the degree-6 discriminant for any binary32 input
//     scale, and the scaling itself is exact.  The triple angle does not depend
//     on the scale; r = sqrt(3 J2) is scaled back exactly.
// All arithmetic in the error-free parts uses the __f*_rn intrinsics so that
// the compiler cannot contract it into FMAs (which would break exactness).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "eig3_f64.cuh"  // triple_angle_sines, sqrt_nonneg (ANGLE64 only)

namespace eig3 {
namespace c32 {

struct F2 {
  float h, l;  // unevaluated sum h + l
};

__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ F2 two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

// (x.h + x.l) * z to first order: the product x.h z is split exactly, x.l z
// is added to the low part.
__device__ __forceinline__ F2 mul(F2 x, float z) {
  const float p = __fmul_rn(x.h, z);
  return {p, __fmaf_rn(x.l, z, __fmaf_rn(x.h, z, -p))};
}

// (x.h + x.l)(y.h + y.l) to first order (x.l y.l is below the working
// precision squared).
__device__ __forceinline__ F2 mul(F2 x, F2 y) {
  const float p = __fmul_rn(x.h, y.h);
  const float e = __fmaf_rn(x.h, y.h, -p);
  return {p, __fmaf_rn(x.h, y.l, __fmaf_rn(x.l, y.h, e))};
}

__device__ __forceinline__ F2 neg(F2 x) { return {-x.h, -x.l}; }

__device__ __forceinline__ F2 scale2(F2 x, float p2) {  // exact: p2 is a power of two
  return {__fmul_rn(x.h, p2), __fmul_rn(x.l, p2)};
}

// Sum2 accumulator: s holds the rounded running sum, c the exact rounding
// errors of the additions plus the low parts of the terms.
struct Sum {
  float s, c;
};

__device__ __forceinline__ Sum start(F2 x) { return {x.h, x.l}; }

__device__ __forceinline__ Sum operator+(Sum a, F2 x) {
  const F2 t = two_sum(a.s, x.h);
  return {t.h, __fadd_rn(a.c, __fadd_rn(t.l, x.l))};
}

__device__ __forceinline__ Sum operator-(Sum a, F2 x) { return a + neg(x); }

__device__ __forceinline__ Sum operator-(Sum a) { return {-a.s, -a.c}; }

__device__ __forceinline__ Sum operator+(Sum a, Sum b) {
  const F2 t = two_sum(a.s, b.s);
  return {t.h, __fadd_rn(__fadd_rn(a.c, b.c), t.l)};
}

__device__ __forceinline__ F2 done(Sum a) { return two_sum(a.s, a.c); }

// A Sum state is itself an unevaluated pair s + c (not normalised: after
// cancellation |c| may approach |s|).  It enters products and squares as it
// is; the dropped low-by-low terms stay at the working precision squared
// relative to the summed terms, which is the accuracy of Sum2 itself.
__device__ __forceinline__ F2 pair(Sum a) { return {a.s, a.c}; }

// (s + c)^2 = s^2 + c (2 s + c), keeping the c^2 term.
__device__ __forceinline__ F2 sq(Sum a) {
  const float p = __fmul_rn(a.s, a.s);
  const float e = __fmaf_rn(a.s, a.s, -p);
  return {p, __fmaf_rn(a.c, __fmaf_rn(2.0f, a.s, a.c), e)};
}

__device__ __forceinline__ float round1(F2 x) { return __fadd_rn(x.h, x.l); }

__device__ __forceinline__ float round1(Sum x) { return __fadd_rn(x.s, x.c); }

// (x.h + x.l)^2 to first order, as a pair.
__device__ __forceinline__ F2 sq(F2 x) {
  const float p = __fmul_rn(x.h, x.h);
  const float e = __fmaf_rn(x.h, x.h, -p);
  return {p, __fmaf_rn(__fadd_rn(x.h, x.h), x.l, e)};
}

// Invariants in scaled form (Sum2 states).  With s = 2^-e the scale:
//   J2x6 = 6 J2 s^2, J3x27 = 27 J3 s^3, D = Delta s^6, I1 unscaled.
struct InvC {
  Sum I1, J2x6, J3x27, D;
  int e;  // the scale exponent
};

// Exponent field of the largest magnitude among the deviatoric data; the
// scale 2^(127 - E) maps it into [1, 2) (E clamped so the scale is normal).
__device__ __forceinline__ int scale_exponent(float m0, float m1, float m2, float m3, float m4,
                                              float m5, float m6, float m7, float m8) {
  int b = __float_as_int(m0) & 0x7fffffff;
  b = max(b, __float_as_int(m1) & 0x7fffffff);
  b = max(b, __float_as_int(m2) & 0x7fffffff);
  b = max(b, __float_as_int(m3) & 0x7fffffff);
  b = max(b, __float_as_int(m4) & 0x7fffffff);
  b = max(b, __float_as_int(m5) & 0x7fffffff);
  b = max(b, __float_as_int(m6) & 0x7fffffff);
  b = max(b, __float_as_int(m7) & 0x7fffffff);
  b = max(b, __float_as_int(m8) & 0x7fffffff);
  return min(b >> 23, 253);
}

__device__ __forceinline__ float pow2_from_field(int field) { return __int_as_float(field << 23); }

// 2^e for the unscaling, e = E - 127 with E in [0, 253]; E = 0 (all data zero
// or subnormal, scaled by 2^127) needs the subnormal 2^-127.
__device__ __forceinline__ float unscale_pow2(int e) {
  return e > -127 ? __int_as_float((e + 127) << 23) : __int_as_float(0x00400000);
}

// Diagonal differences as exact pairs, the trace as an exact pair.
struct Diag {
  F2 d0, d1, d2;
  Sum I1;
};

__device__ __forceinline__ Diag diag_parts(float a00, float a11, float a22) {
  Diag g;
  g.d0 = two_sum(a00, -a11);
  g.d1 = two_sum(a00, -a22);
  g.d2 = two_sum(a11, -a22);
  const F2 t = two_sum(a00, a11);
  const F2 u = two_sum(t.h, a22);
  g.I1 = {u.h, __fadd_rn(t.l, u.l)};
  return g;
}

// The discriminant of a symmetric matrix from its r_i (Sum2 states),
//   Delta = 14 (r2^2 + r3^2 + r4^2) + 2 (r8^2 + ... + r13^2) + r14^2,
// two ways.  disc_sym_compensated keeps it a Sum2 state (the invariants
// output, accurate at u32^2).  disc_sym_rounded serves the eigenvalue
// kernels of precision EIG3_PREC_F32_COMP_A64 (the default compensated
// eigenvalues take invariants_sym_eig below): every term is
// non-negative, so nothing cancels and no compensation is needed -- each
// (s + c)^2 is rounded once (sq1) and the terms are summed in a tree, a
// relative error of a few units of binary32 against the 14 compensated
// additions of the other form.  The r_i themselves, where the cancellation
// is, stay compensated either way.
__device__ __forceinline__ float sq1(Sum r) {
  return __fmaf_rn(r.s, r.s, __fmul_rn(r.c, __fmaf_rn(2.0f, r.s, r.c)));
}

__device__ __forceinline__ Sum disc_sym_compensated(Sum r2, Sum r3, Sum r4, Sum r8, Sum r9,
                                                    Sum r10, Sum r11, Sum r12, Sum r13,
                                                    Sum r14) {
  const Sum g14 = start(sq(r2)) + sq(r3) + sq(r4);
  const Sum g2 = start(sq(r8)) + sq(r9) + sq(r10) + sq(r11) + sq(r12) + sq(r13);
  return start(mul(pair(g14), 14.0f)) + scale2(pair(g2), 2.0f) + sq(r14);
}

__device__ __forceinline__ Sum disc_sym_rounded(Sum r2, Sum r3, Sum r4, Sum r8, Sum r9, Sum r10,
                                                Sum r11, Sum r12, Sum r13, Sum r14) {
  const float g14 = __fadd_rn(__fadd_rn(sq1(r2), sq1(r3)), sq1(r4));
  const float g2 = __fadd_rn(__fadd_rn(__fadd_rn(sq1(r8), sq1(r9)), __fadd_rn(sq1(r10), sq1(r11))),
                             __fadd_rn(sq1(r12), sq1(r13)));
  return {__fmaf_rn(14.0f, g14, __fmaf_rn(2.0f, g2, sq1(r14))), 0.0f};
}

// ---------------------------------------------------------------------------
// Symmetric matrix (A00, A11, A22, A12, A02, A01) with a = A01, b = A02,
// c = A12.  The r_i of Algorithm 5 are summed term by term as the paper
// writes them (every term a product of three factors), with the symmetric
// identities r1 = 0, r2 = r7, r3 = r5, r4 = r6 and reading R1 for r10:
//   r2  = -ab d2 + aa c - bb c         r3  = ac d1 - aa b + cc b
//   r4  =  bc d0 + cc a - bb a
//   r8  = (d0d1 c - cc c) + aa c - ab d1
//   r9  = (d0d1 c - cc c) + bb c - ab d0
//   r10 = (d1d2 a - aa a) + bc d2 + bb a
//   r11 = (d1d2 a - aa a) + bc d1 + cc a
//   r13 =  (d0d2 b + bb b) + ac d2 - aa b
//   r12 = -(d0d2 b + bb b) + ac d0 + cc b
//   r14 = d0d1d2 - aa d0 + bb d1 - cc d2
//   Delta = 14 (r2^2 + r3^2 + r4^2) + 2 (r8^2 + ... + r13^2) + r14^2.
// ---------------------------------------------------------------------------
// EIG: for the EIG3_PREC_F32_COMP_A64 eigenvalues (Delta by disc_sym_rounded);
// otherwise the invariants output (disc_sym_compensated).
template <bool EIG = false>
__device__ __forceinline__ InvC invariants_sym_c(float a00, float a11, float a22, float c0,
                                                 float b0, float a0) {
  const Diag g = diag_parts(a00, a11, a22);
  InvC o;
  o.I1 = g.I1;
  const int E = scale_exponent(g.d0.h, g.d1.h, g.d2.h, a0, b0, c0, 0.f, 0.f, 0.f);
  o.e = E - 127;
  const float sc = pow2_from_field(254 - E);
  const F2 d0 = scale2(g.d0, sc), d1 = scale2(g.d1, sc), d2 = scale2(g.d2, sc);
  const float a = __fmul_rn(a0, sc), b = __fmul_rn(b0, sc), c = __fmul_rn(c0, sc);
  const F2 aa = two_prod(a, a), bb = two_prod(b, b), cc = two_prod(c, c);
  const F2 ab = two_prod(a, b), ac = two_prod(a, c), bc = two_prod(b, c);
  // Algorithm 2, times 6: (d0^2 + d1^2 + d2^2) + 6 (aa + bb + cc)
  const Sum off = start(aa) + bb + cc;
  o.J2x6 = start(sq(d0)) + sq(d1) + sq(d2) + mul(pair(off), 6.0f);
  // Algorithm 4, times 27: 27 * 2abc + 9 (aa t1 + bb t2 + cc t3) - t1 t2 t3
  const F2 t1 = pair(start(d1) + d2);
  const F2 t2 = pair(start(d0) - d2);
  const F2 t3 = pair(start(neg(d0)) - d1);
  const F2 abc = mul(ab, c);
  const Sum mixed = start(mul(aa, t1)) + mul(bb, t2) + mul(cc, t3);
  o.J3x27 = start(mul(abc, 54.0f)) + mul(pair(mixed), 9.0f) - mul(mul(t1, t2), t3);
  // Algorithm 5
  const F2 d0d1 = mul(d0, d1), d0d2 = mul(d0, d2), d1d2 = mul(d1, d2);
  const F2 aac = mul(aa, c), bbc = mul(bb, c), aab = mul(aa, b), ccb = mul(cc, b);
  const F2 cca = mul(cc, a), bba = mul(bb, a);
  const Sum r2 = start(neg(mul(ab, d2))) + aac - bbc;
  const Sum r3 = start(mul(ac, d1)) - aab + ccb;
  const Sum r4 = start(mul(bc, d0)) + cca - bba;
  const Sum s89 = start(mul(d0d1, c)) - mul(cc, c);
  const Sum r8 = s89 + aac - mul(ab, d1);
  const Sum r9 = s89 + bbc - mul(ab, d0);
  const Sum s1011 = start(mul(d1d2, a)) - mul(aa, a);
  const Sum r10 = s1011 + mul(bc, d2) + bba;
  const Sum r11 = s1011 + mul(bc, d1) + cca;
  const Sum s1213 = start(mul(d0d2, b)) + mul(bb, b);
  const Sum r13 = s1213 + mul(ac, d2) - aab;
  const Sum r12 = -s1213 + mul(ac, d0) + ccb;
  const Sum r14 = start(mul(d0d1, d2)) - mul(aa, d0) + mul(bb, d1) - mul(cc, d2);
  o.D = EIG ? disc_sym_rounded(r2, r3, r4, r8, r9, r10, r11, r12, r13, r14)
            : disc_sym_compensated(r2, r3, r4, r8, r9, r10, r11, r12, r13, r14);
  return o;
}

// ---------------------------------------------------------------------------
// Sums of products on a fixed grid, for the eigenvalue kernels.
//
// The eigenvalues do not need the scaled 6 J2, 27 J3 and r_i of Algorithm 5
// at the u32^2 relative accuracy of Sum2: 6 J2 enters through its binary32
// rounding, and 27 J3 and the r_i through the angle, whose error is their
// ABSOLUTE error over sqrt(x^2 + y^2) = sqrt(108 J2^3), at least 1/sqrt(2)
// once the scaling puts the largest deviatoric datum in [1, 2) (so 6 J2 >= 1).
// A sum whose terms are bounded by the scaling is therefore accumulated on a
// fixed grid (the extraction of Rump, Ogita and Oishi, "Accurate
// floating-point summation part I: faithful rounding", SIAM J. Sci. Comput.
// 31 (2008)):
//   B = bias + S,  bias = 1.5 * 2^K at least twice every partial sum |S|,
// so B stays in [bias/2, 3 bias/2]; two successive B then differ exactly
// (Sterbenz) and S = B - bias is exact.  Adding a product x y is one FMA into
// B, the exact difference of the old and new B, and one FMA giving the
// rounding residual x y - (B' - B) (|residual| <= ulp(B)/2, itself rounded
// once), which goes into the binary32 low part C; the low parts of pair
// operands enter C by FMA.  4 instructions for x y, 5 for a pair times a
// value, 6 for a pair times a pair, against 11 for a TwoSum-based Sum2 step;
// the error is a few units of u32 * ulp(bias) instead of u32^2 relative.
// The bounds on |S| below take the largest scaled datum below 4: it lies in
// [1, 2) except for data beyond 2^127, where the clamped scale leaves [2, 4).
// ---------------------------------------------------------------------------
struct Grid {
  float B, C;
};

template <int K>
struct GridBias {
  static constexpr float value = 1.5f * (float)(1 << K);
};

template <int K>
__device__ __forceinline__ Grid gstart(float x, float y) {
  const float b = __fmaf_rn(x, y, GridBias<K>::value);
  return {b, __fmaf_rn(x, y, __fsub_rn(GridBias<K>::value, b))};
}

template <int K>
__device__ __forceinline__ Grid gstart(F2 x, float y) {
  const Grid g = gstart<K>(x.h, y);
  return {g.B, __fmaf_rn(x.l, y, g.C)};
}

template <int K>
__device__ __forceinline__ Grid gstart(F2 x, F2 y) {
  const Grid g = gstart<K>(x.h, y.h);
  return {g.B, __fmaf_rn(x.l, y.h, __fmaf_rn(x.h, y.l, g.C))};
}

__device__ __forceinline__ Grid gadd(Grid g, float x, float y) {
  const float b = __fmaf_rn(x, y, g.B);
  return {b, __fadd_rn(g.C, __fmaf_rn(x, y, __fsub_rn(g.B, b)))};
}

__device__ __forceinline__ Grid gadd(Grid g, F2 x, float y) {
  const Grid t = gadd(g, x.h, y);
  return {t.B, __fmaf_rn(x.l, y, t.C)};
}

__device__ __forceinline__ Grid gadd(Grid g, F2 x, F2 y) {
  const Grid t = gadd(g, x.h, y.h);
  return {t.B, __fmaf_rn(x.l, y.h, __fmaf_rn(x.h, y.l, t.C))};
}

// The sum, rounded to binary32: (B - bias) exactly, plus C.
template <int K>
__device__ __forceinline__ float gsum(Grid g) {
  return __fadd_rn(__fsub_rn(g.B, GridBias<K>::value), g.C);
}

// The difference of two sums on the same grid, rounded to binary32: B - B' is
// exact (both lie in [bias/2, 3 bias/2] on the grid of that binade).
__device__ __forceinline__ float gdiff(Grid x, Grid y) {
  return __fadd_rn(__fsub_rn(x.B, y.B), __fsub_rn(x.C, y.C));
}

// The scaled invariants rounded to binary32 (the eigenvalue kernels' input).
struct InvR {
  float I1, J2x6, J3x27, D;
  int e;  // the scale exponent
};

// Symmetric invariants for the eigenvalue kernels: the terms of
// invariants_sym_c, each sum on its grid (K = 9 for 6 J2 < 336 and for the
// r_i, four terms below 64 each; K = 14 for 27 J3 < 7424), the differences
// d_i and t_i and the trace still exact pairs.  Delta is the weighted sum of
// the squares of the rounded r_i, non-negative terms with nothing left to
// cancel (disc_sym_rounded).  -r12 takes the place of r12: only its square
// enters.  With r2, r3, r4 from differences of r8 .. r13 the symmetric Delta
// takes 7 sums of products instead of 10.
__device__ __forceinline__ InvR invariants_sym_eig(float a00, float a11, float a22, float c0,
                                                   float b0, float a0) {
  const Diag g = diag_parts(a00, a11, a22);
  InvR o;
  o.I1 = round1(g.I1);
  const int E = scale_exponent(g.d0.h, g.d1.h, g.d2.h, a0, b0, c0, 0.f, 0.f, 0.f);
  o.e = E - 127;
  const float sc = pow2_from_field(254 - E);
  const F2 d0 = scale2(g.d0, sc), d1 = scale2(g.d1, sc), d2 = scale2(g.d2, sc);
  const float a = __fmul_rn(a0, sc), b = __fmul_rn(b0, sc), c = __fmul_rn(c0, sc);
  const F2 aa = two_prod(a, a), bb = two_prod(b, b), cc = two_prod(c, c);
  const F2 ab = two_prod(a, b), ac = two_prod(a, c), bc = two_prod(b, c);
  // Algorithm 2, times 6: (d0^2 + d1^2 + d2^2) + 6 (aa + bb + cc)
  Grid j2 = gstart<9>(d0, d0);
  j2 = gadd(j2, d1, d1);
  j2 = gadd(j2, d2, d2);
  j2 = gadd(j2, aa, 6.0f);
  j2 = gadd(j2, bb, 6.0f);
  j2 = gadd(j2, cc, 6.0f);
  o.J2x6 = gsum<9>(j2);
  // Algorithm 4, times 27: 54 abc + 9 (aa t1 + bb t2 + cc t3) - t1 t2 t3
  const F2 t1 = pair(start(d1) + d2);
  const F2 t2 = pair(start(d0) - d2);
  const F2 t3 = pair(start(neg(d0)) - d1);
  Grid j3 = gstart<14>(mul(ab, c), 54.0f);
  j3 = gadd(j3, mul(aa, t1), 9.0f);
  j3 = gadd(j3, mul(bb, t2), 9.0f);
  j3 = gadd(j3, mul(cc, t3), 9.0f);
  j3 = gadd(j3, neg(mul(t1, t2)), t3);
  o.J3x27 = gsum<14>(j3);
  // Algorithm 5: r8 .. r14 on their grids; r2, r3, r4 from the symmetric
  // identities r2 = r8 - r9, r3 = r12 + r13, r4 = r11 - r10 (d0 - d1 = -d2,
  // d0 + d2 = d1, d1 - d2 = d0 for the exact pairs), the grid states
  // subtracting exactly (gdiff)
  const F2 d0d1 = mul(d0, d1), d0d2 = mul(d0, d2), d1d2 = mul(d1, d2);
  const Grid s89 = gadd(gstart<9>(d0d1, c), neg(cc), c);
  const Grid g8 = gadd(gadd(s89, aa, c), neg(ab), d1);
  const Grid g9 = gadd(gadd(s89, bb, c), neg(ab), d0);
  const Grid s1011 = gadd(gstart<9>(d1d2, a), neg(aa), a);
  const Grid g10 = gadd(gadd(s1011, bc, d2), bb, a);
  const Grid g11 = gadd(gadd(s1011, bc, d1), cc, a);
  const Grid s1213 = gadd(gstart<9>(d0d2, b), bb, b);
  const Grid g13 = gadd(gadd(s1213, ac, d2), neg(aa), b);
  const Grid g12n = gadd(gadd(s1213, neg(ac), d0), neg(cc), b);
  const float r8 = gsum<9>(g8), r9 = gsum<9>(g9), r10 = gsum<9>(g10), r11 = gsum<9>(g11);
  const float r12n = gsum<9>(g12n), r13 = gsum<9>(g13);
  const float r2 = gdiff(g8, g9), r3 = gdiff(g13, g12n), r4 = gdiff(g11, g10);
  const float r14 =
      gsum<9>(gadd(gadd(gadd(gstart<9>(d0d1, d2), neg(aa), d0), bb, d1), neg(cc), d2));
  // Delta = 14 (r2^2 + r3^2 + r4^2) + 2 (r8^2 + ... + r13^2) + r14^2
  const float g14 = __fmaf_rn(r2, r2, __fmaf_rn(r3, r3, __fmul_rn(r4, r4)));
  const float g2 = __fmaf_rn(
      r8, r8,
      __fmaf_rn(r9, r9,
                __fmaf_rn(r10, r10,
                          __fmaf_rn(r11, r11, __fmaf_rn(r12n, r12n, __fmul_rn(r13, r13))))));
  o.D = __fmaf_rn(14.0f, g14, __fmaf_rn(2.0f, g2, __fmul_rn(r14, r14)));
  return o;
}

// ---------------------------------------------------------------------------
// General matrix.  dx(M) of Algorithm 5 term by term (reading R1 for r10).
// The products M01 M10, M02 M20, M12 M21 and the d-products are the same for
// M = A and M = A^T and are formed once by the caller.
// ---------------------------------------------------------------------------
struct Shared {
  F2 d0, d1, d2, d0d1, d0d2, d1d2, d0d1d2, p01, p02, p12;
};

struct R13 {
  Sum r[13];  // r1 .. r13
};

__device__ __forceinline__ R13 dx_c(float M01, float M02, float M10, float M12, float M20,
                                    float M21, const Shared &s) {
  R13 o;
  const F2 m0112 = two_prod(M01, M12), m0210 = two_prod(M02, M10);
  const F2 m0102 = two_prod(M01, M02), m0101 = two_prod(M01, M01);
  const F2 m0202 = two_prod(M02, M02), m0121 = two_prod(M01, M21);
  const F2 m0221 = two_prod(M02, M21), m0212 = two_prod(M02, M12);
  const F2 m1212 = two_prod(M12, M12);
  // r1 = M01 M12 M20 - M02 M10 M21
  o.r[0] = start(mul(m0112, M20)) - mul(m0210, M21);
  // r2 = -M01 M02 d2 + M01^2 M12 - M02^2 M21
  o.r[1] = start(neg(mul(m0102, s.d2))) + mul(m0101, M12) - mul(m0202, M21);
  // r3 = M01 M21 d1 - M01^2 M20 + M02 M21^2
  o.r[2] = start(mul(m0121, s.d1)) - mul(m0101, M20) + mul(m0221, M21);
  // r4 = M02 M12 d0 + M01 M12^2 - M02^2 M10
  o.r[3] = start(mul(m0212, s.d0)) + mul(m0112, M12) - mul(m0202, M10);
  // r5 = M01 M12 d1 - M01 M02 M10 + M02 M12 M21
  o.r[4] = start(mul(m0112, s.d1)) - mul(m0102, M10) + mul(m0212, M21);
  // r6 = M02 M21 d0 - M01 M02 M20 + M01 M12 M21
  o.r[5] = start(mul(m0221, s.d0)) - mul(m0102, M20) + mul(m0112, M21);
  // r7 = -M02 M10 d2 + M01 M10 M12 - M02 M12 M20
  o.r[6] = start(neg(mul(m0210, s.d2))) + mul(s.p01, M12) - mul(m0212, M20);
  // r8 = M12 d0 d1 - M02 M10 d1 + M01 M10 M12 - M12^2 M21
  // r9 = M12 d0 d1 - M02 M10 d0 + M02 M12 M20 - M12^2 M21
  const Sum s89 = start(mul(s.d0d1, M12)) - mul(m1212, M21);
  o.r[7] = s89 - mul(m0210, s.d1) + mul(s.p01, M12);
  o.r[8] = s89 - mul(m0210, s.d0) + mul(m0212, M20);
  // r10 = M01 d1 d2 + M02 M21 d2 + M01 M02 M20 - M01^2 M10
  // r11 = M01 d1 d2 + M02 M21 d1 + M01 M12 M21 - M01^2 M10
  const Sum s1011 = start(mul(s.d1d2, M01)) - mul(m0101, M10);
  o.r[9] = s1011 + mul(m0221, s.d2) + mul(m0102, M20);
  o.r[10] = s1011 + mul(m0221, s.d1) + mul(m0112, M21);
  // r12 = -M02 d0 d2 + M01 M12 d0 + M02 M12 M21 - M02^2 M20
  // r13 =  M02 d0 d2 + M01 M12 d2 - M01 M02 M10 + M02^2 M20
  const Sum s1213 = start(mul(s.d0d2, M02)) + mul(m0202, M20);
  o.r[11] = -s1213 + mul(m0112, s.d0) + mul(m0212, M21);
  o.r[12] = s1213 + mul(m0112, s.d2) - mul(m0102, M10);
  return o;
}

__device__ __forceinline__ InvC invariants_general_c(const float (&a)[9]) {
  const Diag g = diag_parts(a[0], a[4], a[8]);
  InvC o;
  o.I1 = g.I1;
  const int E = scale_exponent(g.d0.h, g.d1.h, g.d2.h, a[1], a[2], a[3], a[5], a[6], a[7]);
  o.e = E - 127;
  const float sc = pow2_from_field(254 - E);
  Shared s;
  s.d0 = scale2(g.d0, sc);
  s.d1 = scale2(g.d1, sc);
  s.d2 = scale2(g.d2, sc);
  const float A01 = __fmul_rn(a[1], sc), A02 = __fmul_rn(a[2], sc), A10 = __fmul_rn(a[3], sc);
  const float A12 = __fmul_rn(a[5], sc), A20 = __fmul_rn(a[6], sc), A21 = __fmul_rn(a[7], sc);
  s.p01 = two_prod(A01, A10);
  s.p02 = two_prod(A02, A20);
  s.p12 = two_prod(A12, A21);
  // Algorithm 2, times 6
  const Sum off = start(s.p01) + s.p02 + s.p12;
  o.J2x6 = start(sq(s.d0)) + sq(s.d1) + sq(s.d2) + mul(pair(off), 6.0f);
  // Algorithm 4, times 27
  const F2 t1 = pair(start(s.d1) + s.d2);
  const F2 t2 = pair(start(s.d0) - s.d2);
  const F2 t3 = pair(start(neg(s.d0)) - s.d1);
  const Sum offd = start(mul(two_prod(A01, A12), A20)) + mul(two_prod(A02, A10), A21);
  const Sum mixed = start(mul(s.p01, t1)) + mul(s.p02, t2) + mul(s.p12, t3);
  o.J3x27 = start(mul(pair(offd), 27.0f)) + mul(pair(mixed), 9.0f) - mul(mul(t1, t2), t3);
  // Algorithm 5
  s.d0d1 = mul(s.d0, s.d1);
  s.d0d2 = mul(s.d0, s.d2);
  s.d1d2 = mul(s.d1, s.d2);
  // r14 = d0 d1 d2 - M01 M10 d0 + M02 M20 d1 - M12 M21 d2 (same for A and A^T)
  const Sum r14 =
      start(mul(s.d0d1, s.d2)) - mul(s.p01, s.d0) + mul(s.p02, s.d1) - mul(s.p12, s.d2);
  const R13 u = dx_c(A01, A02, A10, A12, A20, A21, s);
  const R13 v = dx_c(A10, A20, A01, A21, A02, A12, s);
  // sum_i w_i u_i v_i, w = (9, 6, 6, 6, 8, 8, 8, 2, 2, 2, 2, 2, 2, 1)
#define UV(k) mul(pair(u.r[k]), pair(v.r[k]))
  const Sum g6 = start(UV(1)) + UV(2) + UV(3);
  const Sum g8 = start(UV(4)) + UV(5) + UV(6);
  const Sum g2 = start(UV(7)) + UV(8) + UV(9) + UV(10) + UV(11) + UV(12);
  o.D = start(mul(UV(0), 9.0f)) + mul(pair(g6), 6.0f) + scale2(pair(g8), 8.0f) +
        scale2(pair(g2), 2.0f) + sq(r14);
#undef UV
  return o;
}

// ---------------------------------------------------------------------------
// Algorithm 6 in binary32 from the compensated invariants.  The folded
// triple angle phi~ = atan2(y, |x|) in [0, pi/2] (x = 27 J3, y = sqrt(27
// Delta+), reading R2) gives sigma1 = sin(phi/3) and sigma2 = sin((pi-phi)/3)
// without cancellation; the eigenvalues follow as in the binary64 path:
//   lambda_1 = I1/3 - k (sigma2 + 2 sigma1), lambda_2 = I1/3 + k (sigma1 - sigma2),
//   lambda_3 = I1/3 + k (2 sigma2 + sigma1),  k = 2 r / (3 sqrt 3).
// ---------------------------------------------------------------------------
// sin and cos on [0, pi/6] from their Taylor series about 0 (Horner in x^2):
// the first omitted terms, x^11/11! and x^10/10!, are below 1e-10 there, far
// under half a binary32 ulp of the results; only rounding (about 1 ulp) is
// left.  Replaces the library sincosf, whose general argument reduction is
// never needed for this range.
__device__ __forceinline__ void sincos_small(float x, float &sn, float &cs) {
  const float z = x * x;
  float ps = fmaf(z, 2.7557319e-6f, -1.9841270e-4f);     // 1/9!, -1/7!
  ps = fmaf(z, ps, 8.3333333e-3f);                       // 1/5!
  ps = fmaf(z, ps, -1.6666667e-1f);                      // -1/3!
  sn = fmaf(x * z, ps, x);
  float pc = fmaf(z, 2.4801587e-5f, -1.3888889e-3f);     // 1/8!, -1/6!
  pc = fmaf(z, pc, 4.1666667e-2f);                       // 1/4!
  pc = fmaf(z, pc, -0.5f);                               // -1/2!
  cs = fmaf(z, pc, 1.0f);
}

struct EigC {
  float l1, l2, l3, r, sigma1, sigma2, I1;
  bool j2_clamped, d_clamped;
};

// I1 / 3 correctly rounded and the three roots from k = 2 r / (3 sqrt 3)
// and the sines.  The quotient is the product with the binary32 reciprocal
// of 3 and one FMA correction (q0 + (I1 - 3 q0)/3; exhaustively checked over a
// binade, so for every normal I1), instead of an IEEE division.
__device__ __forceinline__ void eig_roots(EigC &o) {
  const float k = o.r * 0.38490017945975050967f;
  const float q0 = __fmul_rn(o.I1, 0.333333343267f);
  const float i3 = __fmaf_rn(__fmaf_rn(-3.0f, q0, o.I1), 0.333333343267f, q0);
  o.l1 = fmaf(-k, fmaf(2.0f, o.sigma1, o.sigma2), i3);
  o.l2 = fmaf(k, o.sigma1 - o.sigma2, i3);
  o.l3 = fmaf(k, fmaf(2.0f, o.sigma2, o.sigma1), i3);
}

// Algorithm 6 in binary32 from the rounded scaled invariants.
__device__ __forceinline__ EigC eigvals_r(const InvR &v) {
  EigC o;
  o.j2_clamped = v.J2x6 < 0.0f;
  o.d_clamped = v.D < 0.0f;
  // r = sqrt(3 J2) = sqrt(J2x6 / 2) * 2^e
  o.r = __fmul_rn(sqrtf(0.5f * fmaxf(v.J2x6, 0.0f)), unscale_pow2(v.e));
  const float x = v.J3x27;
  const float y = sqrtf(27.0f * fmaxf(v.D, 0.0f));
  const float pt = atan2f(y, fabsf(x)) * (1.0f / 3.0f);
  float st, ct;
  sincos_small(pt, st, ct);
  st = fmaxf(st, 0.0f);
  const float other = fmaf(0.86602540378443864676f, ct, -0.5f * st);
  const bool pos = !(x < 0.0f);
  o.sigma1 = pos ? st : other;
  o.sigma2 = pos ? other : st;
  o.I1 = v.I1;
  eig_roots(o);
  return o;
}

// From the compensated invariants: rounded to binary32 (eigvals_r), or with
// ANGLE64 (precision EIG3_PREC_F32_COMP_A64) the final combination of
// Delta's and 27 J3's compensated pairs and the triple angle in binary64
// (triple_angle_sines of the binary64 path, which needs the binary64 header),
// rounded back to binary32 sines; everything else as in the binary32 path.
template <bool ANGLE64 = false>
__device__ __forceinline__ EigC eigvals_c(const InvC &v) {
  if constexpr (!ANGLE64) {
    return eigvals_r({round1(v.I1), round1(v.J2x6), round1(v.J3x27), round1(v.D), v.e});
  } else {
    EigC o;
    const float j2x6 = round1(v.J2x6);
    o.j2_clamped = j2x6 < 0.0f;
    o.r = __fmul_rn(sqrtf(0.5f * fmaxf(j2x6, 0.0f)), unscale_pow2(v.e));
    const double x = (double)v.J3x27.s + (double)v.J3x27.c;
    const double d = (double)v.D.s + (double)v.D.c;
    o.d_clamped = d < 0.0;
    double s1, s2;
    // (27 J3, sqrt(27 Delta)) in the common scale of the compensated invariants
    triple_angle_sines(x, sqrt_nonneg<3>(9.0 * nonneg(d)), s1, s2);
    o.sigma1 = __double2float_rn(s1);
    o.sigma2 = __double2float_rn(s2);
    o.I1 = round1(v.I1);
    eig_roots(o);
    return o;
  }
}

// The eigenvalues of one matrix as the eigenvalue, adjoint, projector and
// Mohr-Coulomb kernels compute them: N = 6 (symmetric layout) through the
// grid-accumulated invariants_sym_eig (with ANGLE64 through the compensated
// invariants and the binary64 angle), N = 9 through the compensated general
// invariants.
template <int N, bool ANGLE64 = false>
__device__ __forceinline__ EigC eig_c(const float (&a)[N]) {
  if constexpr (N == 9) {
    return eigvals_c<ANGLE64>(invariants_general_c(a));
  } else if constexpr (ANGLE64) {
    return eigvals_c<true>(invariants_sym_c<true>(a[0], a[1], a[2], a[3], a[4], a[5]));
  } else {
    return eigvals_r(invariants_sym_eig(a[0], a[1], a[2], a[3], a[4], a[5]));
  }
}

// Unscaled binary64 invariants (I1, J2, J3, Delta) from the compensated pairs.
__device__ __forceinline__ void invariants_out(const InvC &v, double *o) {
  const double s = ldexp(1.0, v.e);
  o[0] = (double)v.I1.s + (double)v.I1.c;
  o[1] = ((double)v.J2x6.s + (double)v.J2x6.c) / 6.0 * (s * s);
  o[2] = ((double)v.J3x27.s + (double)v.J3x27.c) / 27.0 * (s * s * s);
  const double s3 = s * s * s;
  o[3] = ((double)v.D.s + (double)v.D.c) * s3 * s3;
}

// ---------------------------------------------------------------------------
// Adjoint in binary32 (same divided-difference form as the binary64 path).
// The cofactors of dev(A) are 2x2 determinants, evaluated with Kahan's
// FMA scheme (w = b c; e = fma(-b, c, w); det = fma(a, d, -w) + e), which is
// accurate to a few ulps even under cancellation.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float det2(float a, float d, float b, float c) {
  const float w = __fmul_rn(b, c);
  const float e = __fmaf_rn(-b, c, w);
  return __fadd_rn(__fmaf_rn(a, d, -w), e);
}

struct AdjC {
  float aI1, aJ2r, aJ3r2, inv_r;  // a_I1, r a_J2, r^2 a_J3, 1/r
};

// Divided-difference adjoint in units of r (see the binary64 path): no
// intermediate over- or underflows whatever the scale of the matrix.
__device__ __forceinline__ AdjC adjoint_c(float r, float sigma1, float sigma2, float g1, float g2,
                                          float g3) {
  const float k2 = 1.15470053837925152902f;  // 2 / sqrt 3
  const float g12 = k2 * sigma1;
  const float g23 = k2 * sigma2;
  const float g13 = k2 * (sigma1 + sigma2);
  const bool z1 = g12 == 0.0f, z2 = g23 == 0.0f;
  // an exactly coalesced pair takes the mean of its two weights.  The
  // divisions are the two-instruction approximate quotient (within 2 ulp):
  // g13 = (2/sqrt3) cos(psi - pi/6) >= 1, and g12, g23 are either exactly 0
  // (guarded) or above 2^-75 (the scaled Delta's smallest positive value
  // gives an angle of that order), so every divisor is a normal number
  const float D12 = z1 ? 0.0f : __fdividef((z2 ? 0.5f * (g2 + g3) : g2) - g1, g12);
  const float D23 = z2 ? 0.0f : __fdividef(g3 - (z1 ? 0.5f * (g1 + g2) : g2), g23);
  AdjC o;
  o.aJ3r2 = (g13 != 0.0f) ? __fdividef(D23 - D12, g13) : 0.0f;
  o.aJ2r = fmaf(-0.38490017945975050967f * fmaf(2.0f, sigma1, sigma2), o.aJ3r2, D23);
  o.aI1 = ((g1 + g2) + g3) * (1.0f / 3.0f);
  // r below the normal range counts as a triple eigenvalue
  o.inv_r = (r >= 1.17549435e-38f) ? 1.0f / r : 0.0f;
  return o;
}

// Adjoint scalars for the unit weights e_1, e_2, e_3 (eigenprojectors), as in
// the binary64 path.
struct Adj3C {
  float b2[3], b3[3], inv_r;
};

__device__ __forceinline__ Adj3C adjoint_units_c(float r, float sigma1, float sigma2) {
  const float h = 0.86602540378443864676f;  // sqrt3 / 2
  const bool z1 = sigma1 == 0.0f, z2 = sigma2 == 0.0f;
  // approximate quotients as in adjoint_c: every divisor is a normal number
  const float X12 = z1 ? 0.0f : __fdividef(h, sigma1);
  const float X23 = z2 ? 0.0f : __fdividef(h, sigma2);
  const float X13 = __fdividef(h, sigma1 + sigma2);
  const float c = -0.38490017945975050967f * fmaf(2.0f, sigma1, sigma2);
  Adj3C o;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float g1 = k == 0 ? 1.0f : 0.0f, g2 = k == 1 ? 1.0f : 0.0f, g3 = k == 2 ? 1.0f : 0.0f;
    const float D12 = z1 ? 0.0f : ((z2 ? 0.5f * (g2 + g3) : g2) - g1) * X12;
    const float D23 = z2 ? 0.0f : (g3 - (z1 ? 0.5f * (g1 + g2) : g2)) * X23;
    o.b3[k] = (D23 - D12) * X13;
    o.b2[k] = fmaf(c, o.b3[k], D23);
  }
  o.inv_r = (r >= 1.17549435e-38f) ? 1.0f / r : 0.0f;
  return o;
}

// E_k = I/3 + (r a_J2) S^ + (r^2 a_J3) dev(cof S^)^T, S^ = dev(A)/r, 27 values.
template <int N>
__device__ __forceinline__ void projectors_c(const float (&a)[N], const Adj3C &s, float (&E)[27]) {
  const float ir = s.inv_r;
  F2 d0, d1, d2;
  float S01, S02, S10, S12, S20, S21;
  if constexpr (N == 9) {
    d0 = two_sum(a[0], -a[4]);
    d1 = two_sum(a[0], -a[8]);
    d2 = two_sum(a[4], -a[8]);
    S01 = a[1] * ir;
    S02 = a[2] * ir;
    S10 = a[3] * ir;
    S12 = a[5] * ir;
    S20 = a[6] * ir;
    S21 = a[7] * ir;
  } else {
    d0 = two_sum(a[0], -a[1]);
    d1 = two_sum(a[0], -a[2]);
    d2 = two_sum(a[1], -a[2]);
    S12 = S21 = a[3] * ir;
    S02 = S20 = a[4] * ir;
    S01 = S10 = a[5] * ir;
  }
  const float ir3 = ir * (1.0f / 3.0f);
  const float S00 = round1(start(d0) + d1) * ir3;
  const float S11 = round1(start(d2) - d0) * ir3;
  const float S22 = -round1(start(d1) + d2) * ir3;
  const float S[9] = {S00, S01, S02, S10, S11, S12, S20, S21, S22};
  const float Ct[9] = {det2(S11, S22, S12, S21), det2(S02, S21, S01, S22), det2(S01, S12, S02, S11),
                       det2(S12, S20, S10, S22), det2(S00, S22, S02, S20), det2(S02, S10, S00, S12),
                       det2(S10, S21, S11, S20), det2(S01, S20, S00, S21), det2(S00, S11, S01, S10)};
  const float tc = ((Ct[0] + Ct[4]) + Ct[8]) * (1.0f / 3.0f);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      const bool diag = (j == 0 || j == 4 || j == 8);
      const float cj = diag ? Ct[j] - tc : Ct[j];
      E[9 * k + j] = fmaf(s.b2[k], S[j], fmaf(s.b3[k], cj, diag ? (1.0f / 3.0f) : 0.0f));
    }
  }
}

__device__ __forceinline__ void grad_general_c(const float (&a)[9], const AdjC &s, float (&G)[9]) {
  const float ir = s.inv_r;
  const F2 d0 = two_sum(a[0], -a[4]), d1 = two_sum(a[0], -a[8]), d2 = two_sum(a[4], -a[8]);
  const float ir3 = ir * (1.0f / 3.0f);
  const float S00 = round1(start(d0) + d1) * ir3;
  const float S11 = round1(start(d2) - d0) * ir3;
  const float S22 = -round1(start(d1) + d2) * ir3;
  const float S01 = a[1] * ir, S02 = a[2] * ir, S10 = a[3] * ir;
  const float S12 = a[5] * ir, S20 = a[6] * ir, S21 = a[7] * ir;
  const float C00 = det2(S11, S22, S12, S21);
  const float C01 = det2(S12, S20, S10, S22);
  const float C02 = det2(S10, S21, S11, S20);
  const float C10 = det2(S02, S21, S01, S22);
  const float C11 = det2(S00, S22, S02, S20);
  const float C12 = det2(S01, S20, S00, S21);
  const float C20 = det2(S01, S12, S02, S11);
  const float C21 = det2(S02, S10, S00, S12);
  const float C22 = det2(S00, S11, S01, S10);
  const float tc = ((C00 + C11) + C22) * (1.0f / 3.0f);
  const float b2 = s.aJ2r, b3 = s.aJ3r2;
  G[0] = fmaf(b2, S00, fmaf(b3, C00 - tc, s.aI1));
  G[1] = fmaf(b2, S10, b3 * C01);
  G[2] = fmaf(b2, S20, b3 * C02);
  G[3] = fmaf(b2, S01, b3 * C10);
  G[4] = fmaf(b2, S11, fmaf(b3, C11 - tc, s.aI1));
  G[5] = fmaf(b2, S21, b3 * C12);
  G[6] = fmaf(b2, S02, b3 * C20);
  G[7] = fmaf(b2, S12, b3 * C21);
  G[8] = fmaf(b2, S22, fmaf(b3, C22 - tc, s.aI1));
}

__device__ __forceinline__ void grad_sym_c(const float (&s6)[6], const AdjC &s, float (&G)[6]) {
  const float ir = s.inv_r;
  const F2 d0 = two_sum(s6[0], -s6[1]), d1 = two_sum(s6[0], -s6[2]), d2 = two_sum(s6[1], -s6[2]);
  const float ir3 = ir * (1.0f / 3.0f);
  const float S00 = round1(start(d0) + d1) * ir3;
  const float S11 = round1(start(d2) - d0) * ir3;
  const float S22 = -round1(start(d1) + d2) * ir3;
  const float S12 = s6[3] * ir, S02 = s6[4] * ir, S01 = s6[5] * ir;
  const float C00 = det2(S11, S22, S12, S12);
  const float C11 = det2(S00, S22, S02, S02);
  const float C22 = det2(S00, S11, S01, S01);
  const float C12 = det2(S01, S02, S00, S12);
  const float C02 = det2(S01, S12, S02, S11);
  const float C01 = det2(S12, S02, S01, S22);
  const float tc = ((C00 + C11) + C22) * (1.0f / 3.0f);
  const float b2 = s.aJ2r, b3 = s.aJ3r2;
  const float b2x2 = 2.0f * b2, b3x2 = 2.0f * b3;
  G[0] = fmaf(b2, S00, fmaf(b3, C00 - tc, s.aI1));
  G[1] = fmaf(b2, S11, fmaf(b3, C11 - tc, s.aI1));
  G[2] = fmaf(b2, S22, fmaf(b3, C22 - tc, s.aI1));
  G[3] = fmaf(b2x2, S12, b3x2 * C12);
  G[4] = fmaf(b2x2, S02, b3x2 * C02);
  G[5] = fmaf(b2x2, S01, b3x2 * C01);
}

}  // namespace c32
}  // namespace eig3
