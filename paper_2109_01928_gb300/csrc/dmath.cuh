// log, exp and normal deviates as fixed sequences of IEEE double operations.
//
// The dual-annealing kernels draw heavy-tailed moves and accept uphill moves
// with a generalized Metropolis rule, both built on log and exp. CUDA's log/exp
// are accurate to about an ulp but are not a published operation sequence, and
// a last-bit difference can flip an acceptance; these versions are defined by
// their operations, every one correctly rounded (__d*_rn: no contraction into
// FMA), so any implementation of the same sequence returns the same bits:
//   log x:  x = m 2^e, m in [sqrt(1/2), sqrt(2)), f = (m-1)/(m+1),
//           log x = e ln2 + 2 f sum_{j=0}^{12} f^(2j) / (2j+1)   (atanh series);
//   exp x:  k = rint(x / ln2), r = (x - k ln2_hi) - k ln2_lo,
//           exp x = 2^k (1 + r (1 + r/2 (... (1 + r/14))))     (Taylor);
//   normal pair: Marsaglia's polar method, (u, v) sqrt(-2 log s / s).
// Accuracy: a few ulp over the double range.
#pragma once
#include "common.cuh"

namespace debyefit {

constexpr double DM_LN2 = 0.6931471805599453;        // ln 2 rounded to double
constexpr double DM_LN2_HI = 0.6931471803691238;     // ln 2, low 21 mantissa bits cleared
constexpr double DM_LN2_LO = 1.9082149292705877e-10; // ln 2 - DM_LN2_HI (from 50 digits)
constexpr double DM_SQRT_HALF = 0.7071067811865476;
constexpr double DM_EXP_MAX = 709.0;
constexpr double DM_EXP_MIN = -745.0;
constexpr int DM_POLAR_TRIES = 32;

__device__ __forceinline__ double dm_log(double x) {
  int e = 0;
  double m = frexp(x, &e);
  if (m < DM_SQRT_HALF) {
    m = __dmul_rn(m, 2.0);
    e -= 1;
  }
  const double f = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  const double s = __dmul_rn(f, f);
  double p = __ddiv_rn(1.0, 25.0);
#pragma unroll
  for (int j = 11; j >= 0; --j) p = __dadd_rn(__dmul_rn(p, s), __ddiv_rn(1.0, (double)(2 * j + 1)));
  return __dadd_rn(__dmul_rn((double)e, DM_LN2), __dmul_rn(__dmul_rn(2.0, f), p));
}

__device__ __forceinline__ double dm_exp(double x) {
  if (x > DM_EXP_MAX) return INFINITY;
  if (x < DM_EXP_MIN) return 0.0;
  const double k = rint(__ddiv_rn(x, DM_LN2));
  const double r = __dsub_rn(__dsub_rn(x, __dmul_rn(k, DM_LN2_HI)), __dmul_rn(k, DM_LN2_LO));
  double p = 1.0;
#pragma unroll
  for (int j = 14; j >= 1; --j) p = __dadd_rn(1.0, __ddiv_rn(__dmul_rn(p, r), (double)j));
  return ldexp(p, (int)k);
}

}  // namespace debyefit
