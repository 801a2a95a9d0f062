// flog64.cuh -- table-driven FP64 natural logarithm for the FP64 pair and self kernels.
//
// Method: P. T. P. Tang, "Table-driven implementation of the logarithm function in IEEE
// floating-point arithmetic", ACM Trans. Math. Software 16 (1990) 378-400 -- reduce x to a
// breakpoint a_k near its mantissa, take log a_k from a table and the rest from a short
// polynomial in u = (m - a_k)/a_k.  This build's own variant:
// x = m 2^e with m in [1, 2); k = the top 7 bits of m's fraction; a_k = 1 + (k + 1/2) / 128, so
// u = (m - a_k) / a_k satisfies |u| <= 1/256; then
//   log x = e ln 2 + log a_k + log1p(u),   log1p(u) = u + u^2 (-1/2 + u/3 - u^2/4 + u^3/5 - u^4/6 + u^5/7),
// the Taylor series of log1p cut after u^7, whose truncation error |u|^8 / 8 < 1e-20.  The
// table holds (a_k, 1/a_k, log a_k), filled once per context by a kernel that calls the CUDA
// log, and ln 2 split into a 32-bit head and a tail so that e * head is exact.  Valid for
// positive, finite, normal x (the pair kernels pass r^2 >= 1e-150).  stokes_check_log64
// evaluates it on caller-given points so that tests can compare it with CUDA's log.
#pragma once
#include <cuda_runtime.h>

namespace stokes {

constexpr int kLogTab = 128;

struct LogTab {
  double a[kLogTab], inv_a[kLogTab], log_a[kLogTab];
  double ln2_hi, ln2_lo;
};

__device__ __forceinline__ double flog64(double x, const LogTab *__restrict__ t) {
  const long long bits = __double_as_longlong(x);
  const int e = int((bits >> 52) & 0x7FF) - 1023;
  const double m = __longlong_as_double((bits & 0x000FFFFFFFFFFFFFLL) | 0x3FF0000000000000LL);
  const int k = int((bits >> 45) & (kLogTab - 1));
  const double u = (m - __ldg(&t->a[k])) * __ldg(&t->inv_a[k]);
  double p = 1.0 / 7.0;
  p = fma(p, u, -1.0 / 6.0);
  p = fma(p, u, 1.0 / 5.0);
  p = fma(p, u, -1.0 / 4.0);
  p = fma(p, u, 1.0 / 3.0);
  p = fma(p, u, -0.5);
  const double l1p = fma(u * u, p, u);
  const double de = double(e);
  return fma(de, __ldg(&t->ln2_hi), __ldg(&t->log_a[k])) + fma(de, __ldg(&t->ln2_lo), l1p);
}

}  // namespace stokes
