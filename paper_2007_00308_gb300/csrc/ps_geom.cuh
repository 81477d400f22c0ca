// Device geometry of polar stroking: segment forms, the curvature-sign
// polynomial, interval construction, the t(psi) solve and rib evaluation.
#pragma once

#include "ps_internal.cuh"

namespace ps {

struct Seg {
  int type;
  float2 A, B, C, D;
  float w;
};

__device__ __forceinline__ float2 mk(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return mk(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return mk(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 operator*(float2 a, float s) { return mk(a.x * s, a.y * s); }
__device__ __forceinline__ float dot2(float2 a, float2 b) { return a.x * b.x + a.y * b.y; }
__device__ __forceinline__ float cross2(float2 a, float2 b) { return a.x * b.y - a.y * b.x; }
__device__ __forceinline__ bool is0(float2 a) { return a.x == 0.f && a.y == 0.f; }
__device__ __forceinline__ float angf(float2 a) { return atan2f(a.y, a.x); }

struct D2 {
  double x, y;
};
__device__ __forceinline__ D2 dd(float2 a) { return D2{(double)a.x, (double)a.y}; }
__device__ __forceinline__ D2 dsub(D2 a, D2 b) { return D2{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ double dcross(D2 a, D2 b) { return a.x * b.y - a.y * b.x; }
__device__ __forceinline__ double ddot(D2 a, D2 b) { return a.x * b.x + a.y * b.y; }

__device__ __forceinline__ Seg load_seg(const uint8_t* type, const float* pts, const float* wts,
                                        int64_t i) {
  Seg g;
  g.type = type[i];
  const float4* q = reinterpret_cast<const float4*>(pts + 8 * i);
  float4 a = __ldg(q), b = __ldg(q + 1);
  g.A = mk(a.x, a.y);
  g.B = mk(a.z, a.w);
  g.C = mk(b.x, b.y);
  g.D = mk(b.z, b.w);
  g.w = wts ? __ldg(wts + i) : 1.f;
  if (g.type == PS_QUAD || g.type == PS_CONIC) g.C = g.B;
  return g;
}

// All of the form's control points coincide: the segment has no stroke (Sec. 3.3.4).
__device__ __forceinline__ bool zero_length(const Seg& g) {
  switch (g.type) {
    case PS_CUBIC: return is0(g.B - g.A) && is0(g.C - g.A) && is0(g.D - g.A);
    case PS_QUAD: return is0(g.B - g.A) && is0(g.D - g.A);
    case PS_CONIC: return g.w == 0.f ? is0(g.D - g.A) : (is0(g.B - g.A) && is0(g.D - g.A));
    default: return is0(g.D - g.A);
  }
}

// Table 1's normalized end gradients (directions only).  The table's P_C in the
// quadratic and conic rows is their last control point, P_D.
__device__ __forceinline__ float2 end_grad0(const Seg& g) {
  switch (g.type) {
    case PS_CUBIC:
      if (!is0(g.B - g.A)) return g.B - g.A;
      if (!is0(g.C - g.A)) return g.C - g.A;
      return g.D - g.A;
    case PS_QUAD:
      return !is0(g.B - g.A) ? g.B - g.A : g.D - g.A;
    case PS_CONIC:
      if (!is0(g.B - g.A) && g.w != 0.f) return (g.B - g.A) * (g.w > 0.f ? 1.f : -1.f);
      return g.D - g.A;
    default:
      return g.D - g.A;
  }
}
__device__ __forceinline__ float2 end_grad1(const Seg& g) {
  switch (g.type) {
    case PS_CUBIC:
      if (!is0(g.D - g.C)) return g.D - g.C;
      if (!is0(g.D - g.B)) return g.D - g.B;
      return g.D - g.A;
    case PS_QUAD:
      return !is0(g.D - g.B) ? g.D - g.B : g.D - g.A;
    case PS_CONIC:
      if (!is0(g.D - g.B) && g.w != 0.f) return (g.D - g.B) * (g.w > 0.f ? 1.f : -1.f);
      return g.D - g.A;
    default:
      return g.D - g.A;
  }
}

// Hodograph direction H(t) with g'(t) = c(t) H(t), c > 0.
__device__ __forceinline__ float2 hodo(const Seg& g, float t) {
  float u = 1.f - t;
  switch (g.type) {
    case PS_CUBIC:
      return (g.B - g.A) * (u * u) + (g.C - g.B) * (2.f * u * t) + (g.D - g.C) * (t * t);
    case PS_QUAD:
      return (g.B - g.A) * u + (g.D - g.B) * t;
    case PS_CONIC:
      return (g.B - g.A) * (g.w * u * u) + (g.D - g.A) * (u * t) + (g.D - g.B) * (g.w * t * t);
    default:
      return g.D - g.A;
  }
}
__device__ __forceinline__ D2 hodo_d64(const Seg& g, double t) {
  double u = 1.0 - t;
  D2 A = dd(g.A), B = dd(g.B), C = dd(g.C), D = dd(g.D);
  double w = g.w;
  D2 r;
  switch (g.type) {
    case PS_CUBIC:
      r.x = (B.x - A.x) * (u * u) + (C.x - B.x) * (2.0 * u * t) + (D.x - C.x) * (t * t);
      r.y = (B.y - A.y) * (u * u) + (C.y - B.y) * (2.0 * u * t) + (D.y - C.y) * (t * t);
      return r;
    case PS_QUAD:
      r.x = (B.x - A.x) * u + (D.x - B.x) * t;
      r.y = (B.y - A.y) * u + (D.y - B.y) * t;
      return r;
    case PS_CONIC:
      r.x = (B.x - A.x) * (w * u * u) + (D.x - A.x) * (u * t) + (D.x - B.x) * (w * t * t);
      r.y = (B.y - A.y) * (w * u * u) + (D.y - A.y) * (u * t) + (D.y - B.y) * (w * t * t);
      return r;
    default:
      return dsub(D, A);
  }
}

// g(t) - A: the Bernstein weights sum to one, so subtracting A from every control
// point leaves small-magnitude terms; the caller adds A once.
__device__ __forceinline__ float2 g_rel(const Seg& g, float t) {
  float u = 1.f - t;
  switch (g.type) {
    case PS_CUBIC: {
      float b = 3.f * u * u * t, c = 3.f * u * t * t, d = t * t * t;
      return (g.B - g.A) * b + (g.C - g.A) * c + (g.D - g.A) * d;
    }
    case PS_QUAD:
      return (g.B - g.A) * (2.f * u * t) + (g.D - g.A) * (t * t);
    case PS_CONIC: {
      // (1-t)^2 + 2w(1-t)t + t^2 written as (1-2t)^2 + 2(1+w)(1-t)t: for
      // w > -1 both terms are non-negative, so the sum does not cancel when w
      // nears -1 (where the denominator itself nears 0 at t = 1/2)
      float s = 1.f - 2.f * t;
      float den = s * s + 2.f * (1.f + g.w) * u * t;
      float2 num = (g.B - g.A) * (2.f * u * t * g.w) + (g.D - g.A) * (t * t);
      return num * (1.f / den);
    }
    default:
      return (g.D - g.A) * t;
  }
}

// Compensated g(t) - A (PS_PREC_MIXED): the Bernstein sum of (P_i - A) in
// double-float arithmetic -- every product and sum carried as an unevaluated
// pair through error-free transformations (Dekker 1971; Knuth's TwoSum), the
// pair rounded once at the end.  About ten times the flops of g_rel.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF fast_two_sum(float a, float b) {
  float s = a + b;
  return DF{s, b - (s - a)};
}
__device__ __forceinline__ DF two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  return DF{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return fast_two_sum(p, e);
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  DF s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ float2 g_rel_comp(const Seg& g, float t) {
  DF T{t, 0.f};
  DF U = two_sum(1.f, -t);
  DF x{0.f, 0.f}, y{0.f, 0.f};
  DF bx = two_sum(g.B.x, -g.A.x), by = two_sum(g.B.y, -g.A.y);
  DF dx = two_sum(g.D.x, -g.A.x), dy = two_sum(g.D.y, -g.A.y);
  switch (g.type) {
    case PS_CUBIC: {
      DF cx = two_sum(g.C.x, -g.A.x), cy = two_sum(g.C.y, -g.A.y);
      DF ut = df_mul(U, T);
      DF wb = df_mul(df_mul(ut, U), DF{3.f, 0.f});
      DF wc = df_mul(df_mul(ut, T), DF{3.f, 0.f});
      DF wd = df_mul(df_mul(T, T), T);
      x = df_add(df_add(df_mul(bx, wb), df_mul(cx, wc)), df_mul(dx, wd));
      y = df_add(df_add(df_mul(by, wb), df_mul(cy, wc)), df_mul(dy, wd));
      break;
    }
    case PS_QUAD: {
      DF wb = df_mul(df_mul(U, T), DF{2.f, 0.f});
      DF wd = df_mul(T, T);
      x = df_add(df_mul(bx, wb), df_mul(dx, wd));
      y = df_add(df_mul(by, wb), df_mul(dy, wd));
      break;
    }
    case PS_CONIC: {
      DF W{g.w, 0.f};
      DF ut = df_mul(U, T);
      DF wb = df_mul(df_mul(ut, W), DF{2.f, 0.f});
      DF wd = df_mul(T, T);
      DF den = df_add(df_add(df_mul(U, U), wb), wd);
      x = df_add(df_mul(bx, wb), df_mul(dx, wd));
      y = df_add(df_mul(by, wb), df_mul(dy, wd));
      float inv = 1.f / den.hi;
      // one Newton step of the quotient in double-float
      DF qx{x.hi * inv, 0.f}, qy{y.hi * inv, 0.f};
      DF rx = df_add(x, df_mul(DF{-qx.hi, 0.f}, den));
      DF ry = df_add(y, df_mul(DF{-qy.hi, 0.f}, den));
      return mk(qx.hi + rx.hi * inv, qy.hi + ry.hi * inv);
    }
    default:
      x = df_mul(dx, T);
      y = df_mul(dy, T);
  }
  return mk(x.hi + x.lo, y.hi + y.lo);
}

}  // namespace ps
