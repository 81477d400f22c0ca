// Double-float arithmetic on the FP32 pipe: a value is an unevaluated pair of
// floats (hi, lo) with |lo| <= ulp(hi)/2, about 48 significant bits.  The
// building blocks are the error-free transformations TwoSum (Knuth, TAOCP
// vol. 2, 4.2.2), Fast2Sum (Dekker 1971) and the FMA form of TwoProduct; the
// pair operations follow Dekker (1971) and the double-double library of
// Hida, Li and Bailey (2001) in their "sloppy" form (error ~2^-48 of the
// operands' magnitude).
//
// On top of them: sin/cos of a double-float angle by table-driven reduction
// (Tang 1990; the table holds sin, cos of k pi/256 as float pairs) with a
// three-part Cody-Waite constant (Cody & Waite 1980) and Taylor terms on the
// reduced argument |r| <= pi/512; atan2 as the FP32 atan2f refined by one
// rotation (the tangent of the residual angle, which is ~1e-7, equals the
// residual to far below double-float rounding).
//
// GB300 issues FP64 at ~1/60 of its FP32 rate: the mixed-precision
// tessellation carries its angles, normals, parameters and vertices in these
// pairs instead of FP64.
//
// Every function is host- and device-callable so that the arithmetic can be
// checked on the CPU.
#pragma once

#include <math.h>
#include <vector_types.h>

#include "ps_sincos_table.h"

#if defined(__CUDACC__)
#define PS_HD __host__ __device__ __forceinline__
#else
#define PS_HD inline
#endif

namespace ps {

struct DF {
  float hi, lo;
};
struct DF2 {
  DF x, y;
};

PS_HD DF df_of(float a) { return DF{a, 0.f}; }
PS_HD float df_f(DF a) { return a.hi + a.lo; }
PS_HD double df_d(DF a) { return (double)a.hi + (double)a.lo; }
PS_HD DF df_from_d(double v) {
  float h = (float)v;
  return DF{h, (float)(v - (double)h)};
}

// |a| >= |b| (or a == 0): s + e == a + b exactly
PS_HD DF fast_two_sum(float a, float b) {
  float s = a + b;
  return DF{s, b - (s - a)};
}
PS_HD DF two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  return DF{s, (a - (s - bb)) + (b - bb)};
}
PS_HD DF two_prod(float a, float b) {
  float p = a * b;
  return DF{p, fmaf(a, b, -p)};
}
PS_HD DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }
PS_HD DF df_add(DF a, DF b) {
  DF s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
PS_HD DF df_sub(DF a, DF b) { return df_add(a, df_neg(b)); }
PS_HD DF df_add_f(DF a, float b) {
  DF s = two_sum(a.hi, b);
  return fast_two_sum(s.hi, s.lo + a.lo);
}
PS_HD DF df_mul(DF a, DF b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return fast_two_sum(p, e);
}
PS_HD DF df_mul_f(DF a, float b) {
  float p = a.hi * b;
  float e = fmaf(a.hi, b, -p);
  e = fmaf(a.lo, b, e);
  return fast_two_sum(p, e);
}
// a / b: the quotient's residual a.hi - q b is exact under an FMA
PS_HD DF df_div_f(DF a, float b) {
  float q = a.hi / b;
  float r = fmaf(-q, b, a.hi);
  return fast_two_sum(q, (r + a.lo) / b);
}
PS_HD DF df_div(DF a, DF b) {
  float q = a.hi / b.hi;
  DF r = df_sub(a, df_mul_f(b, q));
  return fast_two_sum(q, r.hi / b.hi);
}
PS_HD DF df_sqrt(DF a) {
  if (!(a.hi > 0.f)) return DF{0.f, 0.f};
  const float s = sqrtf(a.hi);
  const DF e = df_sub(a, two_prod(s, s));
  return fast_two_sum(s, e.hi / (2.f * s));
}
PS_HD bool df_lt(DF a, DF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
PS_HD bool df_le(DF a, DF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }
PS_HD DF df_abs(DF a) { return (a.hi < 0.f || (a.hi == 0.f && a.lo < 0.f)) ? df_neg(a) : a; }
PS_HD bool df_is0(DF a) { return a.hi == 0.f && a.lo == 0.f; }
// b - a for floats, exactly
PS_HD DF df_diff(float b, float a) { return two_sum(b, -a); }
// a.x b.y - a.y b.x and a.x b.x + a.y b.y
PS_HD DF df_cross(DF2 a, DF2 b) { return df_sub(df_mul(a.x, b.y), df_mul(a.y, b.x)); }
PS_HD DF df_dot(DF2 a, DF2 b) { return df_add(df_mul(a.x, b.x), df_mul(a.y, b.y)); }

// A lazily normalized sum: value s + e, where e gathers the rounding errors of
// the terms added to s (|e| need not be below ulp(s)/2).  Sums of a few exact
// products of pairs reach the same ~2^-48 accuracy as normalized pair
// arithmetic with fewer operations.
struct Acc {
  float s, e;
};
// A += x y (x, y pairs)
PS_HD void acc_prod(Acc& A, DF x, DF y) {
  const float p = x.hi * y.hi;
  const float pe = fmaf(x.hi, y.hi, -p);
  const float s = A.s + p;
  const float bb = s - A.s;
  A.e += ((A.s - (s - bb)) + (p - bb)) + (pe + fmaf(x.hi, y.lo, x.lo * y.hi));
  A.s = s;
}
PS_HD Acc acc_first(DF x, DF y) {
  const float p = x.hi * y.hi;
  return Acc{p, fmaf(x.hi, y.hi, -p) + fmaf(x.hi, y.lo, x.lo * y.hi)};
}
PS_HD DF acc_df(Acc A) { return DF{A.s, A.e}; }  // unnormalized pair
PS_HD float acc_round(Acc A) { return A.s + A.e; }

// a + g + x y rounded once (a a float; g, x, y pairs)
PS_HD float sum_prod_round(DF s1, float gl, DF x, DF y) {
  // s1 = two_sum(a, g.hi), gl = g.lo
  const float p = x.hi * y.hi;
  const float pe = fmaf(x.hi, y.hi, -p);
  const DF s2 = two_sum(s1.hi, p);
  return s2.hi + (s2.lo + ((s1.lo + gl) + (pe + fmaf(x.hi, y.lo, x.lo * y.hi))));
}

PS_HD DF df_pi() { return DF{PS_DF_PI_HI, PS_DF_PI_LO}; }
PS_HD DF df_two_pi() { return DF{PS_DF_TWO_PI_HI, PS_DF_TWO_PI_LO}; }
PS_HD DF df_sqrt2() { return DF{PS_DF_SQRT2_HI, PS_DF_SQRT2_LO}; }

PS_HD float4 sc_tab_load(const float4* tab, int i) {
#if defined(__CUDA_ARCH__)
  return __ldg(tab + i);
#else
  return tab[i];
#endif
}

// sin and cos of x (|x| < 2^10) to ~1e-14 absolute.  tab: the 512 entries of
// ps_sincos_table.h.
//   k = nearest integer to x 256/pi, r = x - k pi/256 (|r| <= pi/512):
//   x.hi - k C1 is exact under an FMA (C1 has 24 bits, the difference is a
//   multiple of 2^-31 below 2^-7); C2 and C3 extend C1 to ~72 bits of pi/256.
//   sin r = r - r^3/6 + r^5/120 and cos r = 1 - (r^2/2 - r^4/24): the omitted
//   terms are below 1e-17 at |r| <= pi/512; the small terms are FP32 (their
//   rounding is ~2^-24 of 4e-8), the leading r and r^2/2 pairs are exact.
//   sin(a + r) = S_a - S_a c + C_a sin r, cos(a + r) = C_a - C_a c - S_a sin r
//   with c = 1 - cos r.
PS_HD void df_sincos(DF x, const float4* tab, DF& s, DF& c) {
  const float kf = rintf(x.hi * PS_256_OVER_PI);
  const int k = (int)kf;
  const float r1 = fmaf(-kf, PS_PI256_1, x.hi);
  DF r = two_sum(r1, x.lo);
  r = df_sub(r, two_prod(kf, PS_PI256_2));
  r = fast_two_sum(r.hi, fmaf(-kf, PS_PI256_3, r.lo));
  const float rh = r.hi, rl = r.lo;
  const float r2 = rh * rh;
  // sin r = rh + (rl - rh^3/6 + rh^5/120 - rl rh^2/2)
  const float st = fmaf(-rh * r2, fmaf(-r2, 1.f / 120.f, 1.f / 6.f), rl * fmaf(-0.5f, r2, 1.f));
  const DF sr = fast_two_sum(rh, st);
  // 1 - cos r = rh^2/2 - rh^4/24 + rh rl
  const DF h2 = two_prod(rh, rh);
  const DF cr = fast_two_sum(0.5f * h2.hi, fmaf(0.5f, h2.lo, fmaf(rh, rl, -r2 * r2 * (1.f / 24.f))));
  const float4 e = sc_tab_load(tab, k & 511);
  const DF Sa{e.x, e.y}, Ca{e.z, e.w};
  // S_a + C_a sin r - S_a c and C_a - S_a sin r - C_a c, the products exact in
  // their high parts, the remaining terms gathered in FP32 (all below 2^-24 of
  // the result's ulp)
  {
    const float p1 = Ca.hi * sr.hi, e1 = fmaf(Ca.hi, sr.hi, -p1);
    const float p2 = Sa.hi * cr.hi, e2 = fmaf(Sa.hi, cr.hi, -p2);
    const DF a = two_sum(Sa.hi, p1);
    const DF b = two_sum(a.hi, -p2);
    const float lo = (a.lo + b.lo) + (Sa.lo + (e1 - e2)) +
                     (fmaf(Ca.hi, sr.lo, Ca.lo * sr.hi) - fmaf(Sa.hi, cr.lo, Sa.lo * cr.hi));
    s = fast_two_sum(b.hi, lo);
  }
  {
    const float p1 = Sa.hi * sr.hi, e1 = fmaf(Sa.hi, sr.hi, -p1);
    const float p2 = Ca.hi * cr.hi, e2 = fmaf(Ca.hi, cr.hi, -p2);
    const DF a = two_sum(Ca.hi, -p1);
    const DF b = two_sum(a.hi, -p2);
    const float lo = (a.lo + b.lo) + (Ca.lo - (e1 + e2)) -
                     (fmaf(Sa.hi, sr.lo, Sa.lo * sr.hi) + fmaf(Ca.hi, cr.lo, Ca.lo * cr.hi));
    c = fast_two_sum(b.hi, lo);
  }
}

// atan2(y, x) in (-pi, pi] to ~1e-14 (y = +0, x < 0 gives +pi).  a0 = atan2f (a few ulp); with
// (S, C) = sincos(a0), the residual angle is atan(u), u = (y C - x S)/(x C + y S),
// and |u| ~ 1e-7 makes atan(u) = u to ~1e-21.  (0, 0) gives atan2f's value.
PS_HD DF df_atan2(DF y, DF x, const float4* tab) {
  const float a0 = atan2f(y.hi, x.hi);
  if (x.hi == 0.f && y.hi == 0.f) return DF{a0, 0.f};
  // directions along an axis give the pair nearest 0, pi/2, pi, -pi/2 exactly,
  // so that exact reversals and right angles are decided as in FP64
  if (y.hi == 0.f && y.lo == 0.f) return x.hi > 0.f ? DF{0.f, 0.f} : df_pi();
  if (x.hi == 0.f && x.lo == 0.f)
    return y.hi > 0.f ? DF{PS_DF_HALF_PI_HI, PS_DF_HALF_PI_LO} : DF{-PS_DF_HALF_PI_HI, -PS_DF_HALF_PI_LO};
  DF S, C;
  df_sincos(DF{a0, 0.f}, tab, S, C);
  const DF num = df_sub(df_mul(y, C), df_mul(x, S));
  const float den = fmaf(x.hi, C.hi, y.hi * S.hi);
  return two_sum(a0, df_f(num) / den);
}

// x modulo 2 pi into [0, 2 pi) for |x| < 4 pi (one or two corrections)
PS_HD DF df_mod2pi(DF x) {
  const DF tp = df_two_pi();
  if (df_lt(x, df_of(0.f))) x = df_add(x, tp);
  if (df_lt(x, df_of(0.f))) x = df_add(x, tp);
  if (df_le(tp, x)) x = df_sub(x, tp);
  if (df_le(tp, x)) x = df_sub(x, tp);
  return x;
}

// a (-) b into (-pi, pi]: the relative angle of Sec. 3.2.2, one correction by
// 2 pi (callers map an exact reversal, -pi, to +pi)
PS_HD DF df_ominus(DF a, DF b) {
  DF d = df_sub(a, b);
  const DF pi = df_pi();
  if (df_lt(pi, d)) return df_sub(d, df_two_pi());
  if (df_lt(d, df_neg(pi))) return df_add(d, df_two_pi());
  return d;
}

}  // namespace ps
