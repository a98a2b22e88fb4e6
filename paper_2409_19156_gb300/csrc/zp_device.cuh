// Small device helpers shared by the kernels.
#pragma once

namespace zp {

// x^e for e >= 0 by repeated squaring (the seeds rho^m of the recursion, Sec. 2).
__device__ __forceinline__ double pow_uint(double x, int e) {
  double result = 1.0, base = x;
  while (e) {
    if (e & 1) result *= base;
    base *= base;
    e >>= 1;
  }
  return result;
}

}  // namespace zp
