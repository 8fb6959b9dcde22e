// FP64 elementary functions of the shower and hard process, evaluated with
// exactly rounded IEEE-754 operations only (+ - * / sqrt, floor, frexp, ldexp;
// the including translation units are built without FMA contraction), so that
// any IEEE-754 machine running the same steps produces the same bits.
//   gm_exp: Cody-Waite reduction x = k ln2 + r (ln2 = 32-bit head + tail),
//           Taylor series of e^r to degree 14 on |r| <= 0.35, times 2^k.
//   gm_log: x = m 2^e, m in [1/sqrt2, sqrt2); ln m = 2 atanh s with
//           s = (m-1)/(m+1), odd series through s^23 (|s| < 0.172).
//   gm_sincos2pi: cos and sin of 2 pi R; R is reduced exactly to
//           v in [-1/8, 1/8] and a quadrant, then Taylor series of degree
//           18 (cos) and 19 (sin) on |2 pi v| <= pi/4.
#pragma once

#include <cmath>

namespace gaps {

constexpr double kGmLn2Hi = 0x1.62e42fee00000p-1;
constexpr double kGmLn2Lo = 0x1.a39ef35793c76p-33;
constexpr double kGmInvLn2 = 0x1.71547652b82fep+0;
constexpr double kGmTwoPi = 0x1.921fb54442d18p+2;
constexpr double kGmSqrtHalf = 0x1.6a09e667f3bcdp-1;

__host__ __device__ inline double gm_exp(double x) {
  if (!(x == x)) return x;
  if (x > 709.8) return HUGE_VAL;
  if (x < -745.2) return 0.0;
  double k = floor(x * kGmInvLn2 + 0.5);
  double r = (x - k * kGmLn2Hi) - k * kGmLn2Lo;
  // 1/j! for j = 14 down to 1
  double p = 1.0 / 87178291200.0;
  p = p * r + 1.0 / 6227020800.0;
  p = p * r + 1.0 / 479001600.0;
  p = p * r + 1.0 / 39916800.0;
  p = p * r + 1.0 / 3628800.0;
  p = p * r + 1.0 / 362880.0;
  p = p * r + 1.0 / 40320.0;
  p = p * r + 1.0 / 5040.0;
  p = p * r + 1.0 / 720.0;
  p = p * r + 1.0 / 120.0;
  p = p * r + 1.0 / 24.0;
  p = p * r + 1.0 / 6.0;
  p = p * r + 1.0 / 2.0;
  p = p * r + 1.0;
  p = p * r + 1.0;
  return ldexp(p, (int)k);
}

__host__ __device__ inline double gm_log(double x) {
  if (!(x == x) || x < 0.0) return NAN;
  if (x == 0.0) return -HUGE_VAL;
  if (x > 1.7976931348623157e308) return x;
  int e;
  double m = frexp(x, &e);
  if (m < kGmSqrtHalf) {
    m = m * 2.0;
    e -= 1;
  }
  double s = (m - 1.0) / (m + 1.0);
  double z = s * s;
  // 1/(2j+1) for j = 11 down to 1, then 1
  double p = 1.0 / 23.0;
  p = p * z + 1.0 / 21.0;
  p = p * z + 1.0 / 19.0;
  p = p * z + 1.0 / 17.0;
  p = p * z + 1.0 / 15.0;
  p = p * z + 1.0 / 13.0;
  p = p * z + 1.0 / 11.0;
  p = p * z + 1.0 / 9.0;
  p = p * z + 1.0 / 7.0;
  p = p * z + 1.0 / 5.0;
  p = p * z + 1.0 / 3.0;
  p = p * z + 1.0;
  double lm = 2.0 * s * p;
  double de = (double)e;
  return de * kGmLn2Hi + (de * kGmLn2Lo + lm);
}

__host__ __device__ inline void gm_sincos2pi(double R, double& c, double& s) {
  double u = R - floor(R + 0.5);
  double n = floor(4.0 * u + 0.5);
  double v = u - 0.25 * n;
  double th = kGmTwoPi * v;
  double z = th * th;
  double ps = -1.0 / 121645100408832000.0;  // -1/19!
  double pc = 1.0 / 6402373705728000.0;     //  1/18!
  ps = ps * z + 1.0 / 355687428096000.0;
  pc = pc * z + -1.0 / 20922789888000.0;
  ps = ps * z + -1.0 / 1307674368000.0;
  pc = pc * z + 1.0 / 87178291200.0;
  ps = ps * z + 1.0 / 6227020800.0;
  pc = pc * z + -1.0 / 479001600.0;
  ps = ps * z + -1.0 / 39916800.0;
  pc = pc * z + 1.0 / 3628800.0;
  ps = ps * z + 1.0 / 362880.0;
  pc = pc * z + -1.0 / 40320.0;
  ps = ps * z + -1.0 / 5040.0;
  pc = pc * z + 1.0 / 720.0;
  ps = ps * z + 1.0 / 120.0;
  pc = pc * z + -1.0 / 24.0;
  ps = ps * z + -1.0 / 6.0;
  pc = pc * z + 1.0 / 2.0;
  double sn = th + th * (z * ps);
  double cn = 1.0 - z * pc;
  int q = (int)n;
  if (q == 0) { c = cn; s = sn; }
  else if (q == 1) { c = -sn; s = cn; }
  else if (q == -1) { c = sn; s = -cn; }
  else { c = -cn; s = -sn; }
}

}  // namespace gaps
