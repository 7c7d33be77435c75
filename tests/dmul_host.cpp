// Host build of the integer-pipe binary64 multiplication, for the bit-for-bit
// test against the host's IEEE multiplication (tests/test_dmul.py).
#include <stddef.h>

#include "eig3_dmul.cuh"

extern "C" void dmul_batch(const double *x, const double *y, double *out, size_t n) {
  for (size_t i = 0; i < n; ++i) out[i] = eig3::softfp::mul_rn_int(x[i], y[i]);
}
