// Device geometry of polar stroking: segment forms, the curvature-sign
// polynomial, interval construction, the t(psi) solve and rib evaluation.
#pragma once

#include "ps_df.cuh"
#include "ps_internal.cuh"

namespace ps {

// sin, cos of k pi/256 as float pairs (df_sincos); one copy per translation unit
static __device__ const float4 ps_sc_tab[512] = {PS_SINCOS_TABLE_VALUES};

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

// Compensated g(t) - A (PS_PREC_MIXED): the Bernstein sum of (P_i - A) at the
// float t in double-float arithmetic (ps_df.cuh) -- the differences exact as
// pairs, the weights as pairs, the products exact in their high parts and the
// rounding errors gathered lazily; the conic's quotient by one residual step.
__device__ __forceinline__ DF2 g_rel_comp_df(const Seg& g, float t) {
  const DF U = two_sum(1.f, -t);
  const DF bx = two_sum(g.B.x, -g.A.x), by = two_sum(g.B.y, -g.A.y);
  const DF dx = two_sum(g.D.x, -g.A.x), dy = two_sum(g.D.y, -g.A.y);
  switch (g.type) {
    case PS_CUBIC: {
      const DF cx = two_sum(g.C.x, -g.A.x), cy = two_sum(g.C.y, -g.A.y);
      const DF ut3 = df_mul_f(df_mul_f(U, t), 3.f);
      const DF wb = df_mul(ut3, U), wc = df_mul_f(ut3, t), wd = df_mul_f(two_prod(t, t), t);
      Acc x = acc_first(bx, wb), y = acc_first(by, wb);
      acc_prod(x, cx, wc); acc_prod(y, cy, wc);
      acc_prod(x, dx, wd); acc_prod(y, dy, wd);
      return DF2{acc_df(x), acc_df(y)};
    }
    case PS_QUAD: {
      const DF wb = df_mul_f(df_mul_f(U, t), 2.f), wd = two_prod(t, t);
      Acc x = acc_first(bx, wb), y = acc_first(by, wb);
      acc_prod(x, dx, wd); acc_prod(y, dy, wd);
      return DF2{acc_df(x), acc_df(y)};
    }
    case PS_CONIC: {
      const DF ut = df_mul_f(U, t);
      const DF wb = df_mul_f(ut, 2.f * g.w);  // 2w exact
      const DF wd = two_prod(t, t);
      const DF den = df_add(df_add(df_mul(U, U), wb), wd);
      Acc ax = acc_first(bx, wb), ay = acc_first(by, wb);
      acc_prod(ax, dx, wd); acc_prod(ay, dy, wd);
      const DF x = fast_two_sum(ax.s, ax.e), y = fast_two_sum(ay.s, ay.e);
      // the quotient in double-float: q_hi, then the residual's quotient
      const float inv = 1.f / den.hi;
      const float qx = x.hi * inv, qy = y.hi * inv;
      const DF rx = df_sub(x, df_mul_f(den, qx));
      const DF ry = df_sub(y, df_mul_f(den, qy));
      return DF2{fast_two_sum(qx, rx.hi * inv), fast_two_sum(qy, ry.hi * inv)};
    }
    default:
      return DF2{df_mul_f(dx, t), df_mul_f(dy, t)};
  }
}
__device__ __forceinline__ float2 g_rel_comp(const Seg& g, float t) {
  DF2 v = g_rel_comp_df(g, t);
  return mk(df_f(v.x), df_f(v.y));
}

// g'(t) in FP32: c(t) H(t) with c = 3 (cubic), 2 (quadratic), 2/den^2 (conic).
__device__ __forceinline__ float2 deriv_f(const Seg& g, float t) {
  float2 H = hodo(g, t);
  switch (g.type) {
    case PS_CUBIC: return H * 3.f;
    case PS_QUAD: return H * 2.f;
    case PS_CONIC: {
      float u = 1.f - t, s = 1.f - 2.f * t;
      float den = s * s + 2.f * (1.f + g.w) * u * t;
      return H * (2.f / (den * den));
    }
    default: return H;
  }
}

// g(t) - A at a double-float t: the compensated sum at t.hi plus g'(t.hi) t.lo
// (|t.lo| <= 2^-25 t.hi, so the second-order term is below 1e-15 of g'').
__device__ __forceinline__ DF2 g_rel_df(const Seg& g, DF t) {
  DF2 v = g_rel_comp_df(g, t.hi);
  if (t.lo != 0.f) {
    float2 d = deriv_f(g, t.hi);
    v.x = df_add_f(v.x, d.x * t.lo);
    v.y = df_add_f(v.y, d.y * t.lo);
  }
  return v;
}

// The control-point differences of Table 1's end gradients, exactly, as pairs.
__device__ __forceinline__ DF2 df_vec(float2 b, float2 a) {
  return DF2{two_sum(b.x, -a.x), two_sum(b.y, -a.y)};
}
__device__ __forceinline__ DF2 df_scale_sign(DF2 v, float s) {
  return s < 0.f ? DF2{df_neg(v.x), df_neg(v.y)} : v;
}
__device__ __forceinline__ DF2 end_grad0_df(const Seg& g) {
  switch (g.type) {
    case PS_CUBIC:
      if (!is0(g.B - g.A)) return df_vec(g.B, g.A);
      if (!is0(g.C - g.A)) return df_vec(g.C, g.A);
      return df_vec(g.D, g.A);
    case PS_QUAD:
      return !is0(g.B - g.A) ? df_vec(g.B, g.A) : df_vec(g.D, g.A);
    case PS_CONIC:
      if (!is0(g.B - g.A) && g.w != 0.f) return df_scale_sign(df_vec(g.B, g.A), g.w);
      return df_vec(g.D, g.A);
    default:
      return df_vec(g.D, g.A);
  }
}
__device__ __forceinline__ DF2 end_grad1_df(const Seg& g) {
  switch (g.type) {
    case PS_CUBIC:
      if (!is0(g.D - g.C)) return df_vec(g.D, g.C);
      if (!is0(g.D - g.B)) return df_vec(g.D, g.B);
      return df_vec(g.D, g.A);
    case PS_QUAD:
      return !is0(g.D - g.B) ? df_vec(g.D, g.B) : df_vec(g.D, g.A);
    case PS_CONIC:
      if (!is0(g.D - g.B) && g.w != 0.f) return df_scale_sign(df_vec(g.D, g.B), g.w);
      return df_vec(g.D, g.A);
    default:
      return df_vec(g.D, g.A);
  }
}

// Hodograph direction H(t) in double-float at a float t (differences exact).
__device__ __forceinline__ DF2 hodo_df(const Seg& g, float t) {
  DF T{t, 0.f};
  DF U = two_sum(1.f, -t);
  DF2 d0, d1, d2;
  DF b0, b1, b2;
  switch (g.type) {
    case PS_CUBIC:
      d0 = df_vec(g.B, g.A); d1 = df_vec(g.C, g.B); d2 = df_vec(g.D, g.C);
      b0 = df_mul(U, U); b1 = df_mul_f(df_mul(U, T), 2.f); b2 = two_prod(t, t);
      break;
    case PS_QUAD:
      d0 = df_vec(g.B, g.A); d1 = df_vec(g.D, g.B); d2 = DF2{{0.f, 0.f}, {0.f, 0.f}};
      b0 = U; b1 = T; b2 = DF{0.f, 0.f};
      break;
    case PS_CONIC:
      d0 = df_vec(g.B, g.A); d1 = df_vec(g.D, g.A); d2 = df_vec(g.D, g.B);
      b0 = df_mul_f(df_mul(U, U), g.w); b1 = df_mul(U, T); b2 = df_mul_f(two_prod(t, t), g.w);
      break;
    default:
      return df_vec(g.D, g.A);
  }
  DF2 r;
  r.x = df_add(df_add(df_mul(d0.x, b0), df_mul(d1.x, b1)), df_mul(d2.x, b2));
  r.y = df_add(df_add(df_mul(d0.y, b0), df_mul(d1.y, b1)), df_mul(d2.y, b2));
  return r;
}

}  // namespace ps
