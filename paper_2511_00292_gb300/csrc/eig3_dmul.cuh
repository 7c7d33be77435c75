// Binary64 multiplication on the integer pipes.
//
// On GB300 the FP64 unit issues two lanes per SM per clock, a 64th of the
// FP32 rate, while the integer units sit nearly idle in the binary64 kernels.
// mul_rn_int computes the IEEE 754 binary64 product rounded to nearest, ties
// to even, with 32-bit integer operations only: the same bits as the hardware
// multiplication for every pair of operands with a non-NaN product (zeros,
// subnormals, infinities, overflow and gradual underflow included); a NaN
// product is the quiet NaN 0x7ff8000000000000 with the product's sign, as the
// payload of a NaN result is not fixed by IEEE 754.  Kernels move some of
// their multiplications here to share the work between the FP64 pipe and the
// integer pipes.
//
// Method (the textbook significand product, e.g. Muller et al., Handbook of
// Floating-Point Arithmetic, 2nd ed., section 7.5): with both significands as
// 64-bit integers in [2^63, 2^64) (the 53-bit significand shifted left by 11),
// their product P lies in [2^126, 2^128).  Its upper 64 bits, shifted left by
// one when P < 2^127, carry the 53-bit result in bits 63..11, the rounding bit
// in bit 10, and the bits below it together with the lower 64 bits of P form
// the sticky bit.  Rounding adds 1 at bit 11 when the rounding bit is set and
// the sticky bit or the last kept bit is; the carry of that addition runs into
// the exponent field of the packed result, which is exactly the rounding's
// renormalisation (and gives infinity from the largest exponent).
//
// The header compiles for the host as well, so that the same code is tested
// bit for bit against the host's IEEE multiplication.
#pragma once

#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define EIG3_HD __host__ __device__ __forceinline__
#else
#define EIG3_HD inline
#endif

namespace eig3 {
namespace softfp {

EIG3_HD uint64_t to_bits(double x) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t u;
  memcpy(&u, &x, sizeof u);
  return u;
#endif
}

EIG3_HD double from_bits(uint32_t hi, uint32_t lo) {
#if defined(__CUDA_ARCH__)
  double r;
  asm("mov.b64 %0, {%1, %2};" : "=d"(r) : "r"(lo), "r"(hi));
  return r;
#else
  const uint64_t u = ((uint64_t)hi << 32) | lo;
  double r;
  memcpy(&r, &u, sizeof r);
  return r;
#endif
}

EIG3_HD int clz32(uint32_t x) {  // x != 0
#if defined(__CUDA_ARCH__)
  return __clz((int)x);
#else
  return __builtin_clz(x);
#endif
}

// The upper 64 bits (h, l) of the 128-bit product of two 64-bit integers
// (ah, al) and (bh, bl), and whether its lower 64 bits are nonzero.
EIG3_HD void mul_hi128(uint32_t ah, uint32_t al, uint32_t bh, uint32_t bl, uint32_t &h,
                       uint32_t &l, bool &low_nz) {
  const uint64_t t0 = (uint64_t)al * bl;
  const uint64_t t1 = (uint64_t)ah * bl + (t0 >> 32);
  const uint64_t t2 = (uint64_t)al * bh + (uint32_t)t1;
  const uint64_t t3 = (uint64_t)ah * bh + (t1 >> 32) + (t2 >> 32);
  h = (uint32_t)(t3 >> 32);
  l = (uint32_t)t3;
  low_nz = ((uint32_t)t2 | (uint32_t)t0) != 0;
}

// Round the significand (h, l) (bit 63 set; sticky already folded into bit 0)
// to 53 bits and pack it with the sign and the biased exponent E - 1 added to
// the field (the significand's leading bit adds the last 1).  E must lie in
// [1, 2046]; a rounding carry out of E = 2046 gives infinity.
EIG3_HD double round_pack(uint32_t sign, int E, uint32_t h, uint32_t l) {
  const uint32_t up = ((l & 0x7ffu) + 0x3ffu + ((l >> 11) & 1u)) >> 11;
  const uint32_t mh = h >> 11;
  const uint32_t ml = (l >> 11) | (h << 21);
  const uint32_t lo = ml + up;
  const uint32_t hi = sign + ((uint32_t)(E - 1) << 20) + mh + (lo < up ? 1u : 0u);
  return from_bits(hi, lo);
}

// Significand of a finite nonzero operand as (h, l) in [2^63, 2^64) and its
// exponent E (value = (h, l) 2^(E - 1086)); subnormals are normalised.
EIG3_HD void unpack(uint32_t hi, uint32_t lo, uint32_t &h, uint32_t &l, int &E) {
  const int e = (int)((hi >> 20) & 0x7ffu);
  uint32_t fh = hi & 0xfffffu, fl = lo;
  if (e != 0) {
    E = e;
    fh |= 0x100000u;
  } else {  // subnormal: shift the fraction up to the hidden bit's place
    // shift left by s puts the leading one of the fraction at bit 52
    const int s = (fh != 0) ? clz32(fh) - 11 : 21 + clz32(fl);
    if (s >= 32) {
      fh = fl << (s - 32);
      fl = 0;
    } else if (s > 0) {
      fh = (fh << s) | (fl >> (32 - s));
      fl <<= s;
    }
    E = 1 - s;
  }
  h = (fh << 11) | (fl >> 21);
  l = fl << 11;
}

// Every case the fast path leaves: a zero, subnormal, infinite or NaN
// operand, or a result outside the normal range.
#if defined(__CUDACC__)
static __host__ __device__ __noinline__
#else
static inline
#endif
double mul_rn_slow(double x, double y) {
  const uint64_t a = to_bits(x), b = to_bits(y);
  const uint32_t ahi = (uint32_t)(a >> 32), alo = (uint32_t)a;
  const uint32_t bhi = (uint32_t)(b >> 32), blo = (uint32_t)b;
  const uint32_t sign = (ahi ^ bhi) & 0x80000000u;
  const uint32_t amag = ahi & 0x7fffffffu, bmag = bhi & 0x7fffffffu;
  const bool anan = amag > 0x7ff00000u || (amag == 0x7ff00000u && alo != 0);
  const bool bnan = bmag > 0x7ff00000u || (bmag == 0x7ff00000u && blo != 0);
  const bool ainf = amag == 0x7ff00000u && alo == 0;
  const bool binf = bmag == 0x7ff00000u && blo == 0;
  const bool azero = amag == 0 && alo == 0;
  const bool bzero = bmag == 0 && blo == 0;
  if (anan || bnan || (ainf && bzero) || (binf && azero)) return from_bits(sign | 0x7ff80000u, 0);
  if (ainf || binf) return from_bits(sign | 0x7ff00000u, 0);
  if (azero || bzero) return from_bits(sign, 0);
  uint32_t ah, al, bh, bl;
  int ea, eb;
  unpack(ahi, alo, ah, al, ea);
  unpack(bhi, blo, bh, bl, eb);
  uint32_t h, l;
  bool low_nz;
  mul_hi128(ah, al, bh, bl, h, l, low_nz);
  const int top = (int)(h >> 31);
  if (!top) {
    h = (h << 1) | (l >> 31);
    l <<= 1;
  }
  l |= low_nz ? 1u : 0u;
  int E = ea + eb - 1023 + top;
  if (E >= 2047) return from_bits(sign | 0x7ff00000u, 0);
  if (E < 1) {  // gradual underflow: shift right by 1 - E more bits, keeping a sticky bit
    const int s = 1 - E;
    if (s >= 64) {
      const bool nz = (h | l) != 0;
      h = 0;
      l = nz ? 1u : 0u;
    } else if (s >= 32) {
      const bool nz = l != 0 || (s > 32 && (h << (64 - s)) != 0);
      l = (s == 32) ? h : (h >> (s - 32));
      h = 0;
      l |= nz ? 1u : 0u;
    } else {
      const bool nz = (l << (32 - s)) != 0;
      l = (l >> s) | (h << (32 - s));
      h >>= s;
      l |= nz ? 1u : 0u;
    }
    // with E = 1 the field's added 1 is carried only by a significand that
    // rounds up to 2^52, the smallest normal number
    const uint32_t up = ((l & 0x7ffu) + 0x3ffu + ((l >> 11) & 1u)) >> 11;
    const uint32_t mh = h >> 11;
    const uint32_t ml = (l >> 11) | (h << 21);
    const uint32_t lo = ml + up;
    return from_bits(sign + mh + (lo < up ? 1u : 0u), lo);
  }
  return round_pack(sign, E, h, l);
}

// x * y rounded to nearest even (see the file comment).  The fast path takes
// two normal operands whose product's exponent is in the normal range; all
// else goes to mul_rn_slow.  The exponent stays a field word throughout:
// ew = fa + fb - 1024 * 2^20 (+ 2^20 when P >= 2^127) is the result's biased
// exponent minus one at bit 20, in range exactly when it is below 2046 * 2^20
// as an unsigned number, and the significand's leading bit adds the last 1.
EIG3_HD double mul_rn_int(double x, double y) {
  const uint64_t a = to_bits(x), b = to_bits(y);
  const uint32_t ahi = (uint32_t)(a >> 32), alo = (uint32_t)a;
  const uint32_t bhi = (uint32_t)(b >> 32), blo = (uint32_t)b;
  const uint32_t fa = ahi & 0x7ff00000u, fb = bhi & 0x7ff00000u;
  // significands << 11: (ah, al), (bh, bl) in [2^63, 2^64)
  const uint32_t ah = ((ahi | 0x100000u) << 11) | (alo >> 21), al = alo << 11;
  const uint32_t bh = ((bhi | 0x100000u) << 11) | (blo >> 21), bl = blo << 11;
  const uint64_t t0 = (uint64_t)al * bl;
  const uint64_t t1 = (uint64_t)ah * bl + (t0 >> 32);
  const uint64_t t2 = (uint64_t)al * bh + (uint32_t)t1;
  const uint64_t t3 = (uint64_t)ah * bh + (t1 >> 32) + (t2 >> 32);
  const uint32_t h = (uint32_t)(t3 >> 32), l = (uint32_t)t3;
  const bool top = (int32_t)h < 0;  // P >= 2^127
  const uint32_t hn = top ? h : (h << 1) | (l >> 31);
  const uint32_t ln = top ? l : l << 1;
  const uint32_t ew = fa + fb + (top ? 0xc0100000u : 0xc0000000u);
  const bool fast = (fa - 0x100000u) < 0x7fe00000u && (fb - 0x100000u) < 0x7fe00000u &&
                    ew < 0x7fe00000u;
  if (!fast) return mul_rn_slow(x, y);
  // round at bit 11: up when the rounding bit (10) is set and a lower bit of
  // P (the sticky bit) or the last kept bit (11) is
  const bool sticky = ((ln & 0x3ffu) | (uint32_t)t2 | (uint32_t)t0) != 0;
  const uint32_t up = (ln >> 10) & ((ln >> 11) | (sticky ? 1u : 0u)) & 1u;
  const uint32_t lo = ((ln >> 11) | (hn << 21)) + up;
  const uint32_t hi = ((ahi ^ bhi) & 0x80000000u) + ew + (hn >> 11) + (lo < up ? 1u : 0u);
  return from_bits(hi, lo);
}

}  // namespace softfp
}  // namespace eig3
