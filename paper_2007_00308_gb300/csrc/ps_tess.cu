// Tessellation hot path: per-link intervals and step counts, single-pass rib
// offsets, the rib emitter (t(psi) solve, Eq. 11; ribs, Eq. 14-17) and the
// segmented arc-length scan (Eq. 18).
#include <cuda_runtime.h>

#include "ps_geom.cuh"
#include "ps_internal.cuh"

namespace ps {

// ---------------------------------------------------------------------------
// quadratic roots of a + b t + c t^2 (constant term first), cancellation-free
template <typename R>
__device__ __forceinline__ int quad_roots(R a, R b, R c, R disc, R scale, R tol, R* r) {
  if (c == R(0)) {
    if (b == R(0)) return 0;
    r[0] = -a / b;
    return 1;
  }
  if (disc < R(0)) {
    if (-disc > tol * scale) return 0;
    disc = R(0);
  }
  R sq = sqrt(disc);
  R q = R(-0.5) * (b + (b >= R(0) ? sq : -sq));
  if (q != R(0)) {
    r[0] = q / c;
    r[1] = a / q;
  } else {
    r[0] = R(0);
    r[1] = R(0);
  }
  if (r[0] > r[1]) {
    R s = r[0];
    r[0] = r[1];
    r[1] = s;
  }
  return 2;
}

// f(t) = H(t) . N as a power-form quadratic a + b t + c t^2 (Eq. 11; the conic's
// positive denominator is dropped, Sec. 3.4).
template <typename R, typename V>
__device__ __forceinline__ void solve_coeffs(const Seg& g, V N, R& a, R& b, R& c) {
  R Ax = g.A.x, Ay = g.A.y, Bx = g.B.x, By = g.B.y, Cx = g.C.x, Cy = g.C.y, Dx = g.D.x, Dy = g.D.y;
  switch (g.type) {
    case PS_CUBIC: {
      R al = (Bx - Ax) * N.x + (By - Ay) * N.y;
      R be = (Cx - Bx) * N.x + (Cy - By) * N.y;
      R ga = (Dx - Cx) * N.x + (Dy - Cy) * N.y;
      a = al;
      b = R(2) * (be - al);
      c = al - R(2) * be + ga;
      break;
    }
    case PS_QUAD: {
      R al = (Bx - Ax) * N.x + (By - Ay) * N.y;
      R be = (Dx - Bx) * N.x + (Dy - By) * N.y;
      a = al;
      b = be - al;
      c = R(0);
      break;
    }
    default: {  // conic
      R w = g.w;
      R al = w * ((Bx - Ax) * N.x + (By - Ay) * N.y);
      R be = (Dx - Ax) * N.x + (Dy - Ay) * N.y;
      R ga = w * ((Dx - Bx) * N.x + (Dy - By) * N.y);
      a = al;
      b = be - R(2) * al;
      c = al - be + ga;
    }
  }
}

// The same roots with approximate division and square root (relative error
// ~2^-22): the starting guesses of the mixed path, which Newton steps refine.
__device__ __forceinline__ int quad_roots_fast(float a, float b, float c, float disc, float scale,
                                               float tol, float* r) {
  if (c == 0.f) {
    if (b == 0.f) return 0;
    r[0] = __fdividef(-a, b);
    return 1;
  }
  if (disc < 0.f) {
    if (-disc > tol * scale) return 0;
    disc = 0.f;
  }
  const float sq = disc > 0.f ? disc * rsqrtf(disc) : 0.f;
  const float q = -0.5f * (b + (b >= 0.f ? sq : -sq));
  if (q != 0.f) {
    r[0] = __fdividef(q, c);
    r[1] = __fdividef(a, q);
  } else {
    r[0] = 0.f;
    r[1] = 0.f;
  }
  if (r[0] > r[1]) {
    float s = r[0];
    r[0] = r[1];
    r[1] = s;
  }
  return 2;
}

// t(psi) in [pa, pb] (Sec. 3.4) in FP32: roots of H(t).N(psi) = 0 inside the
// range (with a small slack), the one whose tangent points along psi (largest
// H.T(psi)), else the endpoint with the smaller |H.N|.  Returns whether a root
// was taken, and the power-form coefficients for the caller's refinement.
template <bool FAST = false>
__device__ __forceinline__ bool solve_t32(const Seg& g, float sn, float cs, float pa, float pb,
                                          float& t_out, float& a, float& b, float& c) {
  float2 N = mk(-sn, cs), T = mk(cs, sn);
  solve_coeffs<float>(g, N, a, b, c);
  float disc = b * b - 4.f * a * c, scale = b * b + fabsf(4.f * a * c);
  float r[2];
  int n = FAST ? quad_roots_fast(a, b, c, disc, scale, 1e-5f, r)
               : quad_roots<float>(a, b, c, disc, scale, 1e-5f, r);
  float best = 0.f, bestv = -3.0e38f;
  bool found = false;
  for (int i = 0; i < n; ++i) {
    float t = r[i];
    if (!(t >= pa - 1e-5f && t <= pb + 1e-5f)) continue;
    t = fminf(fmaxf(t, pa), pb);
    float v = dot2(hodo(g, t), T);
    if (!found || v > bestv) {
      bestv = v;
      best = t;
      found = true;
    }
  }
  if (found) {
    t_out = best;
    return true;
  }
  float fa = fabsf(dot2(hodo(g, pa), N)), fb = fabsf(dot2(hodo(g, pb), N));
  t_out = fa < fb ? pa : pb;
  return false;
}

__device__ __forceinline__ float solve_t(const Seg& g, float sn, float cs, float pa, float pb) {
  if (g.type == PS_LINE) return pa;
  float t, a, b, c;
  solve_t32(g, sn, cs, pa, pb, t, a, b, c);
  return t;
}

__device__ __forceinline__ float solve_t(const Seg& g, float psi, float pa, float pb) {
  float sn, cs;
  sincosf(psi, &sn, &cs);
  return solve_t(g, sn, cs, pa, pb);
}

// The roots of H(t).N = 0 in FP64 from a double normal (the near-double-root
// island of PS_PREC_MIXED: there the discriminant cancels).  Returns false when
// no root lies in [pa, pb] (slack 1e-9).
__device__ __noinline__ bool solve_t64(const Seg& g, double sn, double cs, double pa, double pb,
                                       double& t_out) {
  D2 Nd{-sn, cs};
  double a, b, c;
  solve_coeffs<double>(g, Nd, a, b, c);
  double disc = b * b - 4.0 * a * c, scale = b * b + fabs(4.0 * a * c);
  double r[2];
  int n = quad_roots<double>(a, b, c, disc, scale, 1e-12, r);
  double best = 0.0, bestv = -1e300;
  bool found = false;
  for (int i = 0; i < n; ++i) {
    double t = r[i];
    if (!(t >= pa - 1e-9 && t <= pb + 1e-9)) continue;
    t = fmin(fmax(t, pa), pb);
    D2 H = hodo_d64(g, t);
    double v = H.x * cs + H.y * sn;
    if (!found || v > bestv) {
      bestv = v;
      best = t;
      found = true;
    }
  }
  t_out = best;
  return found;
}

// f(t) = H(t).N at a float t in double-float (ps_df.cuh): H = sum_i w_i d_i with
// the differences d_i exact as pairs and the weights as pairs -- cubic
// (B-A) u^2 + 2(C-B) u t + (D-C) t^2, quadratic (B-A) u + (D-B) t, conic
// w(B-A) u^2 + (D-A) u t + w(D-B) t^2 (u = 1 - t exact) -- and N a pair.
// The power-form coefficients of solve_coeffs describe the same function.
__device__ __forceinline__ float hn_resid(const Seg& g, float t, DF nx, DF ny) {
  const DF U = two_sum(1.f, -t);
  DF2 d0, d1, d2;
  DF w0, w1, w2;
  switch (g.type) {
    case PS_CUBIC:
      d0 = df_vec(g.B, g.A); d1 = df_vec(g.C, g.B); d2 = df_vec(g.D, g.C);
      w0 = df_mul(U, U); w1 = df_mul_f(U, 2.f * t); w2 = two_prod(t, t);
      break;
    case PS_QUAD:
      d0 = df_vec(g.B, g.A); d1 = df_vec(g.D, g.B); d2 = d1;
      w0 = U; w1 = DF{t, 0.f}; w2 = DF{0.f, 0.f};
      break;
    default:
      d0 = df_vec(g.B, g.A); d1 = df_vec(g.D, g.A); d2 = df_vec(g.D, g.B);
      w0 = df_mul_f(df_mul(U, U), g.w); w1 = df_mul_f(U, t); w2 = df_mul_f(two_prod(t, t), g.w);
      break;
  }
  Acc hx = acc_first(d0.x, w0), hy = acc_first(d0.y, w0);
  acc_prod(hx, d1.x, w1); acc_prod(hy, d1.y, w1);
  acc_prod(hx, d2.x, w2); acc_prod(hy, d2.y, w2);
  Acc f = acc_first(acc_df(hx), nx);
  acc_prod(f, acc_df(hy), ny);
  return acc_round(f);
}

// H(t).N as a power-form quadratic a + b t + c t^2 with double-float
// coefficients (the differences exact as pairs, N a pair).
__device__ __forceinline__ void hn_coeffs_df(const Seg& g, DF nx, DF ny, DF& a, DF& b, DF& c) {
  DF2 d0, d1, d2;
  switch (g.type) {
    case PS_CUBIC: d0 = df_vec(g.B, g.A); d1 = df_vec(g.C, g.B); d2 = df_vec(g.D, g.C); break;
    case PS_QUAD: d0 = df_vec(g.B, g.A); d1 = df_vec(g.D, g.B); d2 = d1; break;
    default: d0 = df_vec(g.B, g.A); d1 = df_vec(g.D, g.A); d2 = df_vec(g.D, g.B); break;
  }
  auto dotn = [&](DF2 d) {
    Acc A = acc_first(d.x, nx);
    acc_prod(A, d.y, ny);
    return fast_two_sum(A.s, A.e);
  };
  const DF e0 = dotn(d0), e1 = dotn(d1), e2 = dotn(d2);
  switch (g.type) {
    case PS_CUBIC:  // e0 u^2 + 2 e1 u t + e2 t^2
      a = e0;
      b = df_mul_f(df_sub(e1, e0), 2.f);
      c = df_add(df_sub(e0, df_mul_f(e1, 2.f)), e2);
      break;
    case PS_QUAD:  // e0 u + e1 t
      a = e0;
      b = df_sub(e1, e0);
      c = DF{0.f, 0.f};
      break;
    default: {  // w e0 u^2 + e1 u t + w e2 t^2
      const DF we0 = df_mul_f(e0, g.w), we2 = df_mul_f(e2, g.w);
      a = we0;
      b = df_sub(e1, df_mul_f(we0, 2.f));
      c = df_add(df_sub(we0, e1), we2);
    }
  }
}

// t(psi) by the oracle's steps (stable quadratic formula, range test with a
// 1e-12 slack, alias rejection by the largest H.T, endpoint rule) with
// double-float coefficients and roots: the near-double-root case, where the
// FP32 discriminant cancels.  A discriminant within 1e-10 of its scale (a
// double root to double-float precision) is solved in FP64.
__device__ __noinline__ DF solve_t_quad_df(const Seg& g, DF sn, DF cs, DF pa, DF pb) {
  const DF nx = df_neg(sn);
  DF a, b, c;
  hn_coeffs_df(g, nx, cs, a, b, c);
  DF r[2];
  int n = 0;
  if (df_is0(c)) {
    if (!df_is0(b)) r[n++] = df_neg(df_div(a, b));
  } else {
    DF disc = df_sub(df_mul(b, b), df_mul_f(df_mul(a, c), 4.f));
    const float scale = b.hi * b.hi + fabsf(4.f * a.hi * c.hi);
    if (fabsf(disc.hi) < 1e-10f * scale) {
      double td;
      if (solve_t64(g, df_d(sn), df_d(cs), df_d(pa), df_d(pb), td)) return df_from_d(td);
    }
    if (disc.hi < 0.f && -disc.hi <= 1e-12f * scale) disc = DF{0.f, 0.f};
    if (!(disc.hi < 0.f)) {
      const DF sq = df_sqrt(disc);
      const DF q = df_mul_f(df_add(b, b.hi >= 0.f ? sq : df_neg(sq)), -0.5f);
      if (!df_is0(q)) {
        r[n++] = df_div(q, c);
        r[n++] = df_div(a, q);
      }
    }
  }
  const DF lo = df_add_f(pa, -1e-12f), hi = df_add_f(pb, 1e-12f);
  const float2 T = mk(cs.hi, sn.hi);
  DF best = pa;
  float bestv = -3.0e38f;
  bool found = false;
  for (int i = 0; i < n; ++i) {
    DF t = r[i];
    if (df_lt(t, lo) || df_lt(hi, t)) continue;
    if (df_lt(t, pa)) t = pa;
    if (df_lt(pb, t)) t = pb;
    const float v = dot2(hodo(g, t.hi), T);
    if (!found || v > bestv) {
      bestv = v;
      best = t;
      found = true;
    }
  }
  if (found) return best;
  const float2 N = mk(nx.hi, cs.hi);
  const float fa = fabsf(dot2(hodo(g, pa.hi), N)), fb = fabsf(dot2(hodo(g, pb.hi), N));
  return fa < fb ? pa : pb;
}

// t(psi) in PS_PREC_MIXED (Eq. 11), as a double-float pair.  The root is chosen
// in FP32 as above (alias rejection, endpoint rule), then refined by a Newton
// step on H(t).N(psi) = 0 with the residual in double-float from the
// double-float normal (sn, cs), and a second step where the first one's
// quadratic term, c dt^2 / f', could exceed 1e-12.  A near double root (the
// FP32 discriminant below 1e-3 of its scale), or a step that moved t by more
// than 1e-4, takes the double-float quadratic solve instead.
__device__ DF solve_t_mx(const Seg& g, DF sn, DF cs, DF pa, DF pb) {
  if (g.type == PS_LINE) return pa;
  float t0, a, b, c;
  const bool root = solve_t32<true>(g, sn.hi, cs.hi, pa.hi, pb.hi, t0, a, b, c);
  const float disc = b * b - 4.f * a * c, scale = b * b + fabsf(4.f * a * c);
  if (!(c != 0.f && fabsf(disc) < 1e-3f * scale)) {
    if (!root) return t0 == pa.hi ? pa : pb;  // endpoint rule
    const DF nx = df_neg(sn);
    float dt = 0.f;
#pragma unroll 1
    for (int it = 0; it < 2; ++it) {
      if (it == 1) {
        if (!(fabsf(c * dt * dt) > 1e-12f * fabsf(fmaf(2.f * c, t0, b)))) break;
        t0 += dt;
      }
      const float fp = fmaf(2.f * c, t0, b);
      dt = fp != 0.f ? -__fdividef(hn_resid(g, t0, nx, cs), fp) : 0.f;
    }
    if (fabsf(dt) <= 1e-4f) {
      DF t = two_sum(t0, dt);
      if (df_lt(t, pa)) t = pa;
      if (df_lt(pb, t)) t = pb;
      return t;
    }
  }
  return solve_t_quad_df(g, sn, cs, pa, pb);
}

// ---------------------------------------------------------------------------
// a b - c d.  In FP32 with c d's rounding recovered (Kahan's form): exactly 0
// when the two products are equal, within about an ulp otherwise.  A plain
// a * b - c * d is contracted to fma(a, b, -c d), which keeps only c d's
// rounding, so an exactly flat segment could read as slightly curved.  In FP64
// the products of FP32 inputs are exact.
template <typename R>
__device__ __forceinline__ R diff_prod(R a, R b, R c, R d) {
  if constexpr (sizeof(R) == 4) {
    const R w = c * d;
    const R e = fma(-c, d, w);
    return fma(a, b, -w) + e;
  } else {
    return a * b - c * d;
  }
}

// Curvature-sign polynomial C(t) ~ g'(t) x g''(t) in power form c0 + c1 t + c2 t^2.
template <typename R>
struct CrossPoly {
  R c0, c1, c2, disc, scale;
  bool flat;
  __device__ R eval(R t) const { return c0 + t * (c1 + t * c2); }
};

template <typename R>
__device__ CrossPoly<R> cross_poly(const Seg& g) {
  CrossPoly<R> P;
  P.c0 = P.c1 = P.c2 = P.disc = P.scale = R(0);
  P.flat = true;
  R Ax = g.A.x, Ay = g.A.y, Bx = g.B.x, By = g.B.y, Cx = g.C.x, Cy = g.C.y, Dx = g.D.x, Dy = g.D.y;
  switch (g.type) {
    case PS_CUBIC: {
      R d1x = Bx - Ax, d1y = By - Ay, d2x = Cx - Bx, d2y = Cy - By, d3x = Dx - Cx, d3y = Dy - Cy;
      R X12 = diff_prod(d1x, d2y, d1y, d2x), X13 = diff_prod(d1x, d3y, d1y, d3x),
        X23 = diff_prod(d2x, d3y, d2y, d3x);
      P.c0 = X12;
      P.c1 = X13 - R(2) * X12;
      P.c2 = X12 - X13 + X23;
      // discriminant X13^2 - 4 X12 X23 with error-free products: an exact cusp
      // (double root) gives exactly zero
      R h1 = X13 * X13, l1 = fma(X13, X13, -h1);
      R h2 = (R(4) * X12) * X23, l2 = fma(R(4) * X12, X23, -h2);
      P.disc = (h1 - h2) + (l1 - l2);
      P.scale = fabs(h1) + fabs(h2);
      P.flat = (X12 == R(0) && X13 == R(0) && X23 == R(0));
      break;
    }
    case PS_QUAD: {
      R K = diff_prod(Bx - Ax, Dy - By, By - Ay, Dx - Bx);
      P.c0 = K;
      P.flat = (K == R(0));
      break;
    }
    case PS_CONIC: {
      R K = diff_prod(Bx - Ax, Dy - By, By - Ay, Dx - Bx);
      R w = g.w, wK = w * K;
      P.c0 = wK;
      P.c1 = wK * (R(2) * w - R(2));
      P.c2 = wK * (R(2) - R(2) * w);
      P.disc = P.c1 * P.c1 - R(4) * P.c0 * P.c2;
      P.scale = P.c1 * P.c1 + fabs(R(4) * P.c0 * P.c2);
      P.flat = (wK == R(0));
      break;
    }
    default:
      break;
  }
  return P;
}

__device__ __forceinline__ float wrap2pi(float x) {
  if (x < 0.f) x += PS_TWO_PI_F;
  if (x >= PS_TWO_PI_F) x -= PS_TWO_PI_F;
  return x;
}

// Steps for a turning of magnitude ad (Eq. 12).  q is a nominal step: a ratio
// exceeding an integer n by less than STEP_SNAP steps takes n steps, so turnings
// that q divides exactly (caps, 90-degree arcs) do not hinge on q's last bit.
#define STEP_SNAP 1e-4f
__device__ __forceinline__ int ceil_steps(float ad, float q) {
  if (ad == 0.f) return 0;
  int D = (int)ceilf(ad / q - STEP_SNAP);
  return D < 1 ? 1 : D;
}
// MIXED: re-evaluate a step count in double-float when its FP32 argument is within
// rounding of the boundary
__device__ __forceinline__ bool near_integer(float x) {
  x -= STEP_SNAP;
  float f = x - floorf(x);
  return fminf(f, 1.f - f) < 4e-5f * fmaxf(1.f, x);
}

// A link's angle step in FP32 (for the FP32 count decisions), with what the
// mixed kernel needs to recompute it in double-float where a count decision is
// re-taken (step_df).
struct Step {
  float q;
  float q0, tau, r;  // the nominal step and the boost's inputs
  int kind;          // 0: q0 itself, 1: round join or cap, 2: segment
};

__device__ __forceinline__ Step plain_step(float q) { return Step{q, q, 0.f, 0.f, 0}; }

// Reading R21 (Sec. 7 suggests boosting q for links near the scale of pixels).
// With a pixel tolerance tau > 0 a link steps by the largest angle, up to the
// bounds below, at which each boundary edge stays within tau px of the stroke
// boundary it replaces; tau = 0 keeps q.
//   round join / cap (an arc of radius r): max(q, 2 acos(1 - tau/r)), pi once
//     tau >= r -- the arc-to-chord gap of a step phi is r (1 - cos(phi/2));
//   segment: max(q, min(2 atan(tau/L_g), sqrt(pi tau / (2r)), pi/2)), L_g the
//     control polygon's length -- one step's offset piece is no longer than
//     L_g + r phi and lies within (length/2) tan(phi/2) of its chord.
// A conic with w_B <= 0 leaves its control hull and keeps q.
__device__ Step round_step(float q, float tau, float r) {
  if (!(tau > 0.f)) return plain_step(q);
  // 2 acos(1 - x) = 4 asin(sqrt(x/2)), without the cancellation of 1 - x
  float qf = tau >= r ? PS_PI_F : 4.f * asinf(sqrtf(0.5f * tau / r));
  return Step{fmaxf(qf, q), q, tau, r, 1};
}

template <typename R>
__device__ __forceinline__ R leg(float2 a, float2 b) {
  R dx = (R)b.x - (R)a.x, dy = (R)b.y - (R)a.y;
  return sqrt(dx * dx + dy * dy);
}

template <typename R>
__device__ __forceinline__ R polygon_length(const Seg& g) {
  switch (g.type) {
    case PS_LINE: return leg<R>(g.A, g.D);
    case PS_CUBIC: return leg<R>(g.A, g.B) + leg<R>(g.B, g.C) + leg<R>(g.C, g.D);
    default: return leg<R>(g.A, g.B) + leg<R>(g.B, g.D);
  }
}

__device__ Step seg_step(const Seg& g, float q, float tau, float r) {
  if (!(tau > 0.f) || (g.type == PS_CONIC && !(g.w > 0.f))) return plain_step(q);
  float Lg = polygon_length<float>(g);
  float a = Lg > 0.f ? 2.f * atanf(tau / Lg) : PS_PI_F;
  float b = sqrtf(PS_PI_F * tau / (2.f * r));
  return Step{fmaxf(fminf(fminf(a, b), 0.5f * PS_PI_F), q), q, tau, r, 2};
}

// Out-of-line double-float atan2 and sincos for the link set-up, which calls
// them from many places on divergent paths: one copy of each keeps the
// kernel's code small (its warps stalled on instruction fetch); the per-rib
// emitter inlines them.
__device__ __noinline__ DF atan2_ool(DF y, DF x) { return df_atan2(y, x, ps_sc_tab); }
__device__ __noinline__ void sincos_ool(DF x, DF& s, DF& c) { df_sincos(x, ps_sc_tab, s, c); }

__device__ __forceinline__ DF df_max(DF a, DF b) { return df_lt(a, b) ? b : a; }
__device__ __forceinline__ DF df_min(DF a, DF b) { return df_lt(a, b) ? a : b; }

// The link step of the same rule in double-float (g is the segment for kind
// 2), where a count decision is re-taken: 2 acos(1 - x) = 4 asin(sqrt(x/2)) =
// 4 atan2(sqrt(x/2), sqrt(1 - x/2)), atan(tau/L_g) = atan2(tau, L_g).
__device__ __noinline__ DF step_df(const Step& S, const Seg* g) {
  const DF q = df_of(S.q0), tau = df_of(S.tau);
  if (S.kind == 1) {
    if (S.tau >= S.r) return df_max(df_pi(), q);
    const DF h = df_div_f(tau, 2.f * S.r);  // tau / (2 r), 2r exact
    const DF a = atan2_ool(df_sqrt(h), df_sqrt(df_sub(df_of(1.f), h)));
    return df_max(df_mul_f(a, 4.f), q);
  }
  if (S.kind == 2 && g) {
    auto leg = [](float2 a, float2 b) {
      const DF dx = two_sum(b.x, -a.x), dy = two_sum(b.y, -a.y);
      return df_sqrt(df_add(df_mul(dx, dx), df_mul(dy, dy)));
    };
    DF Lg;
    switch (g->type) {
      case PS_LINE: Lg = leg(g->A, g->D); break;
      case PS_CUBIC: Lg = df_add(df_add(leg(g->A, g->B), leg(g->B, g->C)), leg(g->C, g->D)); break;
      default: Lg = df_add(leg(g->A, g->B), leg(g->B, g->D));
    }
    const DF a = df_is0(Lg) ? df_pi() : df_mul_f(atan2_ool(tau, Lg), 2.f);
    const DF b = df_sqrt(df_div_f(df_mul(df_pi(), tau), 2.f * S.r));
    const DF half_pi{PS_DF_HALF_PI_HI, PS_DF_HALF_PI_LO};
    return df_max(df_min(df_min(a, b), half_pi), q);
  }
  return q;
}

// Steps for the turning ad in FP32 (Eq. 12 with the nominal-step snap).
__device__ __forceinline__ int steps32(float ad, const Step& S) { return ceil_steps(ad, S.q); }

// Steps for a double-float turning ad > 0 (PS_PREC_MIXED): decided in FP32,
// re-decided in double-float when the FP32 ratio sits within rounding of a
// boundary, ceil(ad/q - snap) with the pair's exact ceiling.  With the pixel
// boost a re-decided link step comes from its rule in double-float (step_df).
template <bool PX>
__device__ __forceinline__ int steps_mx(DF ad, const Step& S, const Seg* g) {
  if (!near_integer(ad.hi / S.q)) return ceil_steps(ad.hi, S.q);
  DF x;
  if (PX && S.kind != 0) x = df_sub(df_div(ad, step_df(S, g)), DF{PS_DF_SNAP_HI, PS_DF_SNAP_LO});
  else x = df_sub(df_div_f(ad, S.q0), DF{PS_DF_SNAP_HI, PS_DF_SNAP_LO});
  float c = ceilf(x.hi);
  if (c == x.hi && x.lo > 0.f) c += 1.f;
  const int D = (int)c;
  return D < 1 ? 1 : D;
}

// Reversals of a segment with collinear control points: along the common
// direction v, H(t).v is the Bernstein quadratic lam1 u^2 + 2 lam2 u t + lam3 t^2
// (linear lam1 u + lam3 t for the quadratic Bezier).  The direction reverses at
// its simple roots inside (0,1): two when lam2^2 - lam1 lam3 > 0 (sign taken with
// error-free products), none otherwise (a double root is a kink); roots at the
// ends (lam1 = 0, lam3 = 0) are factored out exactly.  R: the arithmetic, T: the
// type of the roots.
template <typename R, typename T>
__device__ int collinear_reversals(const Seg& g, T* rts) {
  float2 vf = end_grad0(g);
  R vx = vf.x, vy = vf.y;
  R Ax = g.A.x, Ay = g.A.y, Bx = g.B.x, By = g.B.y, Cx = g.C.x, Cy = g.C.y, Dx = g.D.x, Dy = g.D.y;
  R l1, l2, l3;
  switch (g.type) {
    case PS_CUBIC:
      l1 = (Bx - Ax) * vx + (By - Ay) * vy;
      l2 = (Cx - Bx) * vx + (Cy - By) * vy;
      l3 = (Dx - Cx) * vx + (Dy - Cy) * vy;
      break;
    case PS_QUAD: {
      R a1 = (Bx - Ax) * vx + (By - Ay) * vy, a3 = (Dx - Bx) * vx + (Dy - By) * vy;
      if ((a1 > R(0) && a3 < R(0)) || (a1 < R(0) && a3 > R(0))) {
        rts[0] = (T)(a1 / (a1 - a3));
        return 1;
      }
      return 0;
    }
    case PS_CONIC: {
      R w = g.w;
      if (w == R(0)) return 0;
      l1 = w * ((Bx - Ax) * vx + (By - Ay) * vy);
      l2 = R(0.5) * ((Dx - Ax) * vx + (Dy - Ay) * vy);
      l3 = w * ((Dx - Bx) * vx + (Dy - By) * vy);
      break;
    }
    default:
      return 0;
  }
  int n = 0;
  if (l1 == R(0) && l3 == R(0)) return 0;
  if (l1 == R(0)) {
    R den = R(2) * l2 - l3;
    if (den != R(0)) {
      R r = R(2) * l2 / den;
      if (r > R(0) && r < R(1)) rts[n++] = (T)r;
    }
    return n;
  }
  if (l3 == R(0)) {
    R den = l1 - R(2) * l2;
    if (den != R(0)) {
      R r = l1 / den;
      if (r > R(0) && r < R(1)) rts[n++] = (T)r;
    }
    return n;
  }
  R h1 = l2 * l2, e1 = fma(l2, l2, -h1);
  R h2 = l1 * l3, e2 = fma(l1, l3, -h2);
  R disc = (h1 - h2) + (e1 - e2);
  if (!(disc > R(0))) return 0;
  R a = l1, b = R(2) * (l2 - l1), c = l1 - R(2) * l2 + l3, r[2];
  int m = quad_roots<R>(a, b, c, R(4) * disc, R(1), R(0), r);
  for (int i = 0; i < m; ++i)
    if (r[i] > R(0) && r[i] < R(1)) rts[n++] = (T)r[i];
  if (n == 2 && rts[0] > rts[1]) {
    T t = rts[0];
    rts[0] = rts[1];
    rts[1] = t;
  }
  return n;
}

// Record fields as pairs (the lo parts stay zero in FP32).
__device__ __forceinline__ void put_psi(LinkRec& L, int k, DF v) { L.psi[k] = v.hi; L.psi_lo[k] = v.lo; }
__device__ __forceinline__ void put_p(LinkRec& L, int k, DF v) { L.p[k] = v.hi; L.p_lo[k] = v.lo; }
__device__ __forceinline__ void put_step(LinkRec& L, int k, DF v) { L.step[k] = v.hi; L.step_lo[k] = v.lo; }

// The curvature-sign polynomial in PS_PREC_MIXED.  A cubic's is formed in
// double-float from the exact control-point differences (X_ij = d_i x d_j as
// pairs) and its roots by the stable quadratic formula in double-float.  FP64
// (the discriminant island) serves a cubic whose cross products are within
// rounding of zero (a flat or nearly flat segment, whose flatness is decided
// exactly) or whose discriminant is within 1e-6 of its scale (near a cusp,
// where the roots need the extra bits), and the quadratic's and conic's
// single-product polynomial.
struct CurvMX {
  bool use64, flat;
  CrossPoly<double> Pd;
  DF c0, c1, c2;
  int nroot;
  DF roots[2];
  __device__ int sign_at(DF t) const {
    if (use64) {
      const double v = Pd.eval(df_d(t));
      return v > 0.0 ? 1 : (v < 0.0 ? -1 : 0);
    }
    const DF v = df_add(c0, df_mul(t, df_add(c1, df_mul(t, c2))));
    return v.hi > 0.f ? 1 : (v.hi < 0.f ? -1 : 0);
  }
};

__device__ __forceinline__ void curv_add_root(CurvMX& C, DF r) {
  if (df_lt(df_of(0.f), r) && df_lt(r, df_of(1.f)) && (C.nroot == 0 || df_lt(C.roots[C.nroot - 1], r)))
    C.roots[C.nroot++] = r;
}

__device__ CurvMX curv_mx(const Seg& g) {
  CurvMX C;
  C.use64 = true;
  C.flat = true;
  C.nroot = 0;
  if (g.type == PS_CUBIC) {
    const DF2 d1 = df_vec(g.B, g.A), d2 = df_vec(g.C, g.B), d3 = df_vec(g.D, g.C);
    const DF X12 = df_cross(d1, d2), X13 = df_cross(d1, d3), X23 = df_cross(d2, d3);
    const float m1 = fabsf(d1.x.hi) + fabsf(d1.y.hi), m2 = fabsf(d2.x.hi) + fabsf(d2.y.hi),
                m3 = fabsf(d3.x.hi) + fabsf(d3.y.hi);
    const float xm = fabsf(X12.hi) + fabsf(X13.hi) + fabsf(X23.hi);
    if (xm > 1e-9f * (m1 * m2 + m1 * m3 + m2 * m3)) {
      // c1^2 - 4 c0 c2 reduces to X13^2 - 4 X12 X23
      const DF disc = df_sub(df_mul(X13, X13), df_mul_f(df_mul(X12, X23), 4.f));
      const float scale = X13.hi * X13.hi + fabsf(4.f * X12.hi * X23.hi);
      if (fabsf(disc.hi) > 1e-6f * scale) {
        C.use64 = false;
        C.flat = false;
        C.c0 = X12;
        C.c1 = df_sub(X13, df_mul_f(X12, 2.f));
        C.c2 = df_add(df_sub(X12, X13), X23);
        if (disc.hi > 0.f) {  // two simple roots (a sign change at each)
          DF r[2];
          int n = 0;
          if (df_is0(C.c2)) {
            if (!df_is0(C.c1)) r[n++] = df_neg(df_div(C.c0, C.c1));
          } else {
            const DF sq = df_sqrt(disc);
            const DF q = df_mul_f(df_add(C.c1, C.c1.hi >= 0.f ? sq : df_neg(sq)), -0.5f);
            if (!df_is0(q)) {
              r[n++] = df_div(q, C.c2);
              r[n++] = df_div(C.c0, q);
            }
          }
          if (n == 2 && df_lt(r[1], r[0])) {
            const DF t = r[0];
            r[0] = r[1];
            r[1] = t;
          }
          for (int i = 0; i < n; ++i) curv_add_root(C, r[i]);
        }
        return C;
      }
    }
  }
  C.Pd = cross_poly<double>(g);
  C.flat = C.Pd.flat;
  if (!C.flat && (C.Pd.c1 != 0.0 || C.Pd.c2 != 0.0)) {
    double r[2];
    int n = quad_roots<double>(C.Pd.c0, C.Pd.c1, C.Pd.c2, C.Pd.disc, C.Pd.scale, 0.0, r);
    if (n == 2 && C.Pd.disc <= 0.0) n = 0;  // a double root: no sign change
    for (int i = 0; i < n; ++i)
      if (r[i] > 0.0 && r[i] < 1.0) curv_add_root(C, df_from_d(r[i]));
  }
  return C;
}

// Interval table of a segment link in FP32 (Sec. 3.3.4-3.3.6, Eq. 4-6, 12-13).
// Returns N (total steps) or -1 if the table does not fit.
template <bool PX>
__device__ int seg_intervals32(const Seg& g, Step S, LinkRec& L) {
  float Psi0 = angf(end_grad0(g)), Psin = angf(end_grad1(g));
  CrossPoly<float> Pf = cross_poly<float>(g);
  int M = 0;
  uint32_t pivots = 0;
  if (Pf.flat) {
    // zero curvature: flat pieces with +pi pivots where H reverses (collinear
    // control points with back-tracking); one quad per flat piece
    float rts[2];
    int nr = collinear_reversals<float, float>(g, rts);
    float psi = Psi0, pp = 0.f;
    for (int i = 0; i <= nr; ++i) {
      float pe = (i < nr) ? rts[i] : 1.f;
      L.p[M] = pp;
      L.psi[M] = psi;
      L.step[M] = 0.f;  // flat: Delta = 1, no interior ribs
      L.dsum[M + 1] = 0;
      M++;
      if (i < nr) {
        L.p[M] = pe;
        L.psi[M] = psi;
        pivots |= 1u << M;
        M++;
        psi = psi + PS_PI_F;
      }
      pp = pe;
    }
    L.p[M] = 1.f;
    L.psi[M] = psi;
    int N = 0;
    L.dsum[0] = 0;
    for (int k = 0; k < M; ++k) {
      int D = 1;
      L.step[k] = 0.f;
      if ((pivots >> k) & 1u) {
        D = steps32(PS_PI_F, S);
        L.step[k] = PS_PI_F / (float)D;
      }
      N += D;
      L.dsum[k + 1] = (uint16_t)N;
    }
    L.meta |= ((uint32_t)M << 4) | (pivots << 8);
    return N;
  }

  // Eq. 4: curvature-sign changes strictly inside (0,1)
  float roots[2];
  int nroot = 0;
  if (Pf.c1 != 0.f || Pf.c2 != 0.f) {
    float r[2];
    int n = quad_roots<float>(Pf.c0, Pf.c1, Pf.c2, Pf.disc, Pf.scale, 0.f, r);
    if (n == 2 && Pf.disc <= 0.f) n = 0;
    for (int i = 0; i < n; ++i)
      if (r[i] > 0.f && r[i] < 1.f && (nroot == 0 || r[i] > roots[nroot - 1])) roots[nroot++] = r[i];
  }
  // Eq. 5
  float p[4], Psi[4];
  int n = 0;
  p[n] = 0.f;
  Psi[n] = Psi0;
  n++;
  for (int i = 0; i < nroot; ++i) {
    p[n] = roots[i];
    Psi[n] = angf(hodo(g, roots[i]));
    n++;
  }
  p[n] = 1.f;
  Psi[n] = Psin;

  // Eq. 6: turning of each interval in the direction of the curvature sign
  for (int k = 0; k < n; ++k) {
    float pa = p[k], pb = p[k + 1];
    float sgn = 0.f;
    float probes[3] = {0.5f * (pa + pb), 0.75f * pa + 0.25f * pb, 0.25f * pa + 0.75f * pb};
    for (int i = 0; i < 3 && sgn == 0.f; ++i) {
      float v = Pf.eval(probes[i]);
      sgn = v > 0.f ? 1.f : (v < 0.f ? -1.f : 0.f);
    }
    float delta = 0.f;
    if (sgn != 0.f) {
      delta = sgn * wrap2pi(sgn * (Psi[k + 1] - Psi[k]));
      if (fabsf(delta) > PS_TWO_PI_F - 1e-5f) delta = 0.f;
    }
    float ad = fabsf(delta);
    if (ad >= PS_PI_F) {
      // Sec. 3.3.5: split at half the turning, p by Eq. 11
      float psi_s = Psi[k] + 0.5f * delta;
      float ps_ = solve_t(g, psi_s, pa, pb);
      int Dh = steps32(0.5f * ad, S);
      if (M + 2 > 6) return -1;
      L.p[M] = pa; L.psi[M] = Psi[k]; L.step[M] = 0.5f * delta / (float)Dh; L.dsum[M + 1] = (uint16_t)Dh; M++;
      L.p[M] = ps_; L.psi[M] = psi_s; L.step[M] = 0.5f * delta / (float)Dh; L.dsum[M + 1] = (uint16_t)Dh;
      L.meta |= META_SPLIT_BIT(M);
      M++;
    } else {
      int D = ad == 0.f ? (pb > pa ? 1 : 0) : steps32(ad, S);
      if (M + 1 > 6) return -1;
      L.p[M] = pa; L.psi[M] = Psi[k]; L.step[M] = D ? delta / (float)D : 0.f; L.dsum[M + 1] = (uint16_t)D; M++;
    }
  }
  L.p[M] = 1.f;
  L.psi[M] = Psin;
  // dsum[k+1] holds Delta_k so far: accumulate into Delta_Sigma
  int N = 0;
  L.dsum[0] = 0;
  for (int k = 0; k < M; ++k) {
    N += L.dsum[k + 1];
    L.dsum[k + 1] = (uint16_t)N;
  }
  L.meta |= ((uint32_t)M << 4);
  return N;
}

// The same table in PS_PREC_MIXED.  Angles, parameters and steps are
// double-float pairs: end angles by the double-float atan2 of the exact
// control-point differences, inflections from the curvature polynomial's
// roots (curv_mx: double-float, FP64 near flatness or a double root), their
// angles from the double-float hodograph, turnings and counts in
// double-float, split points by the double-float t solve.
template <bool PX>
__device__ int seg_intervals_mx(const Seg& g, Step S, LinkRec& L) {
  const DF2 ge0 = end_grad0_df(g), ge1 = end_grad1_df(g);
  const DF Psi0 = atan2_ool(ge0.y, ge0.x), Psin = atan2_ool(ge1.y, ge1.x);
  const CurvMX Cv = curv_mx(g);
  const DF zero = df_of(0.f), one = df_of(1.f);
  int M = 0;
  uint32_t pivots = 0;
  if (Cv.flat) {
    double rts[2];
    int nr = collinear_reversals<double, double>(g, rts);
    DF psi = Psi0, pp = zero;
    for (int i = 0; i <= nr; ++i) {
      DF pe = (i < nr) ? df_from_d(rts[i]) : one;
      put_p(L, M, pp);
      put_psi(L, M, psi);
      put_step(L, M, zero);
      L.dsum[M + 1] = 0;
      M++;
      if (i < nr) {
        put_p(L, M, pe);
        put_psi(L, M, psi);
        pivots |= 1u << M;
        M++;
        psi = df_add(psi, df_pi());
      }
      pp = pe;
    }
    put_p(L, M, one);
    put_psi(L, M, psi);
    int N = 0;
    L.dsum[0] = 0;
    for (int k = 0; k < M; ++k) {
      int D = 1;
      put_step(L, k, zero);
      if ((pivots >> k) & 1u) {
        D = steps_mx<PX>(df_pi(), S, &g);
        put_step(L, k, df_div_f(df_pi(), (float)D));
      }
      N += D;
      L.dsum[k + 1] = (uint16_t)N;
    }
    L.meta |= ((uint32_t)M << 4) | (pivots << 8);
    return N;
  }

  // Eq. 4 (the roots of the curvature polynomial, curv_mx) and Eq. 5: an
  // inflection's angle is insensitive to its parameter to first order (the
  // tangent turns at rate 0 there), so H is taken at the float root
  DF p[4], Psi[4];
  int n = 0;
  p[n] = zero;
  Psi[n] = Psi0;
  n++;
  for (int i = 0; i < Cv.nroot; ++i) {
    p[n] = Cv.roots[i];
    DF2 H = hodo_df(g, p[n].hi);
    Psi[n] = atan2_ool(H.y, H.x);
    n++;
  }
  p[n] = one;
  Psi[n] = Psin;

  // Eq. 6: turning in the direction of the curvature sign, modulo 2 pi
  const DF full = DF{PS_DF_FULL_TURN_SLACK_HI, PS_DF_FULL_TURN_SLACK_LO};
  for (int k = 0; k < n; ++k) {
    const DF pa = p[k], pb = p[k + 1];
    int sgn = 0;
    const DF probes[3] = {df_mul_f(df_add(pa, pb), 0.5f),
                          df_add(df_mul_f(pa, 0.75f), df_mul_f(pb, 0.25f)),
                          df_add(df_mul_f(pa, 0.25f), df_mul_f(pb, 0.75f))};
    for (int i = 0; i < 3 && sgn == 0; ++i) sgn = Cv.sign_at(probes[i]);
    DF delta = zero;
    if (sgn != 0) {
      DF d = df_sub(Psi[k + 1], Psi[k]);
      if (sgn < 0) d = df_neg(d);
      d = df_mod2pi(d);
      if (df_lt(full, d)) d = zero;  // a full turn within rounding: numerically flat
      delta = sgn < 0 ? df_neg(d) : d;
    }
    const DF ad = df_abs(delta);
    if (df_le(df_pi(), ad)) {
      // Sec. 3.3.5: split at half the turning, p by Eq. 11
      const DF half{0.5f * delta.hi, 0.5f * delta.lo};
      const DF psi_s = df_add(Psi[k], half);
      DF sn, cs;
      sincos_ool(psi_s, sn, cs);
      const DF ps_ = solve_t_mx(g, sn, cs, p[k], p[k + 1]);
      const int Dh = steps_mx<PX>(df_abs(half), S, &g);
      const DF st = df_div_f(half, (float)Dh);
      if (M + 2 > 6) return -1;
      put_p(L, M, p[k]); put_psi(L, M, Psi[k]); put_step(L, M, st); L.dsum[M + 1] = (uint16_t)Dh; M++;
      put_p(L, M, ps_); put_psi(L, M, psi_s); put_step(L, M, st); L.dsum[M + 1] = (uint16_t)Dh;
      L.meta |= META_SPLIT_BIT(M);
      M++;
    } else {
      const int D = df_is0(ad) ? (df_lt(pa, pb) ? 1 : 0) : steps_mx<PX>(ad, S, &g);
      if (M + 1 > 6) return -1;
      put_p(L, M, p[k]); put_psi(L, M, Psi[k]);
      put_step(L, M, D ? df_div_f(delta, (float)D) : zero);
      L.dsum[M + 1] = (uint16_t)D;
      M++;
    }
  }
  put_p(L, M, one);
  put_psi(L, M, Psin);
  int N = 0;
  L.dsum[0] = 0;
  for (int k = 0; k < M; ++k) {
    N += L.dsum[k + 1];
    L.dsum[k + 1] = (uint16_t)N;
  }
  L.meta |= ((uint32_t)M << 4);
  return N;
}

__device__ __forceinline__ float ominus_f(float a, float b) {
  float d = a - b;
  if (d > PS_PI_F) return d - PS_TWO_PI_F;
  if (d < -PS_PI_F) return d + PS_TWO_PI_F;
  return d;
}

// J of a join or cap (Sec. 4.3.2-4.3.5; reading R8: bevel 1, triangle 2,
// miters 3, round ceil(|delta|/q); caps: triangle 2, square 4, round
// ceil(pi/q)).  round: the round style's step count.
__device__ __forceinline__ int pivot_count(int kind, int style, bool zero_turn, int round) {
  if (kind == LK_JOIN) {
    if (zero_turn) return 0;
    switch (style) {
      case PS_JOIN_BEVEL: return 1;
      case PS_JOIN_TRIANGLE: return 2;
      case PS_JOIN_MITER:
      case PS_JOIN_MITER_TRUNCATE: return 3;
      case PS_JOIN_ROUND: return round;
      default: return 0;
    }
  }
  switch (style) {
    case PS_CAP_TRIANGLE: return 2;
    case PS_CAP_SQUARE: return 4;
    case PS_CAP_ROUND: return round;
    default: return 0;
  }
}

// Join / cap pivot in FP32 (Sec. 4.3): generator fixed at `at`, psi from Psi0
// through delta in J steps; the outer side is N for delta > 0, P for delta < 0
// and the inner radius is zero.
template <bool PX>
__device__ int pivot_setup32(float2 at, float Psi0, float delta, int kind, int style, float r,
                             float miter, Step S, LinkRec& L) {
  const bool rnd = (kind == LK_JOIN && style == PS_JOIN_ROUND) || (kind == LK_CAP && style == PS_CAP_ROUND);
  const float ad = fabsf(delta);
  int J = pivot_count(kind, style, delta == 0.f, rnd ? steps32(ad, S) : 0);
  if (J == 0) return 0;
  L.P[0] = at;
  L.rN = delta > 0.f ? r : 0.f;
  L.rP = delta > 0.f ? 0.f : r;
  L.psi[0] = Psi0;
  L.psi[1] = Psi0 + delta;
  L.step[0] = delta / (float)J;
  L.dsum[0] = 0;
  L.dsum[1] = (uint16_t)J;
  L.p[0] = 0.f;
  L.p[1] = 1.f;
  L.meta |= (1u << 4) | ((uint32_t)style << 16);
  if (kind == LK_CAP && style == PS_CAP_SQUARE) L.meta |= META_FLAG_SQUARE;
  if (kind == LK_JOIN && (style == PS_JOIN_MITER || style == PS_JOIN_MITER_TRUNCATE)) {
    float sd = delta > 0.f ? -1.f : 1.f;  // outer offset = at + sd * r * n
    float s0, c0, s1, c1, sh, ch;
    sincosf(Psi0, &s0, &c0);
    sincosf(Psi0 + delta, &s1, &c1);
    sincosf(Psi0 + 0.5f * delta, &sh, &ch);
    float2 O0 = at + mk(-s0, c0) * (sd * r);
    float2 O3 = at + mk(-s1, c1) * (sd * r);
    // miter ratio 1/sin(phi/2), phi = pi - |delta|; infinite at a reversal
    float cm = cosf(0.5f * ad);
    float ratio = cm > 0.f ? 1.f / cm : INFINITY;
    float2 v1, v2;
    if (ratio <= miter) {
      float2 tip = at + mk(-sh, ch) * (sd * r * ratio);
      v1 = tip;
      v2 = tip;
    } else if (style == PS_JOIN_MITER) {
      v1 = O0;
      v2 = O3;
    } else {
      float lam = (miter * r - r * cosf(0.5f * ad)) / sinf(0.5f * ad);
      lam = fmaxf(lam, 0.f);
      v1 = O0 + mk(c0, s0) * lam;
      v2 = O3 - mk(c1, s1) * lam;
    }
    L.v1 = v1;
    L.v2 = v2;
    L.meta |= META_FLAG_OVERRIDE;
  }
  return J;
}

// a + b (a float, b a pair) rounded once
__device__ __forceinline__ float add_round(float a, DF b) { return df_f(df_add_f(b, a)); }

// The same pivot in PS_PREC_MIXED: Psi0 and delta are double-float pairs, the
// counts are re-decided in double-float at their boundaries, and the miter
// decision and override vertices are taken in double-float.
template <bool PX>
__device__ int pivot_setup_mx(float2 at, DF Psi0, DF delta, int kind, int style, float r,
                              float miter, Step S, LinkRec& L) {
  const bool rnd = (kind == LK_JOIN && style == PS_JOIN_ROUND) || (kind == LK_CAP && style == PS_CAP_ROUND);
  const DF ad = df_abs(delta);
  int J = pivot_count(kind, style, df_is0(delta), rnd && !df_is0(delta) ? steps_mx<PX>(ad, S, nullptr) : 0);
  if (J == 0) return 0;
  const bool pos = df_lt(df_of(0.f), delta);
  L.P[0] = at;
  L.rN = pos ? r : 0.f;
  L.rP = pos ? 0.f : r;
  put_psi(L, 0, Psi0);
  put_psi(L, 1, df_add(Psi0, delta));
  put_step(L, 0, df_div_f(delta, (float)J));
  L.dsum[0] = 0;
  L.dsum[1] = (uint16_t)J;
  L.p[0] = 0.f;
  L.p[1] = 1.f;
  L.meta |= (1u << 4) | ((uint32_t)style << 16);
  if (kind == LK_CAP && style == PS_CAP_SQUARE) L.meta |= META_FLAG_SQUARE;
  if (kind == LK_JOIN && (style == PS_JOIN_MITER || style == PS_JOIN_MITER_TRUNCATE)) {
    const float sdr = pos ? -r : r;  // outer offset = at + sdr * n, n = (-sin, cos)
    const DF half{0.5f * delta.hi, 0.5f * delta.lo}, ahalf = df_abs(half);
    DF s0, c0, s1, c1, sh, ch, sa, ca;
    sincos_ool(Psi0, s0, c0);
    sincos_ool(df_add(Psi0, delta), s1, c1);
    sincos_ool(df_add(Psi0, half), sh, ch);
    sincos_ool(ahalf, sa, ca);
    // miter ratio 1/cos(|delta|/2) <= limit  <=>  limit cos(|delta|/2) >= 1
    const bool accept = ca.hi > 0.f && df_le(df_of(1.f), df_mul_f(ca, miter));
    DF2 O0{df_mul_f(df_neg(s0), sdr), df_mul_f(c0, sdr)};  // relative to at
    DF2 O3{df_mul_f(df_neg(s1), sdr), df_mul_f(c1, sdr)};
    float2 v1, v2;
    if (accept) {
      const DF len = df_div(df_of(sdr), ca);
      const float tx = add_round(at.x, df_mul(df_neg(sh), len)), ty = add_round(at.y, df_mul(ch, len));
      v1 = mk(tx, ty);
      v2 = v1;
    } else if (style == PS_JOIN_MITER) {
      v1 = mk(add_round(at.x, O0.x), add_round(at.y, O0.y));
      v2 = mk(add_round(at.x, O3.x), add_round(at.y, O3.y));
    } else {
      // truncate: clip at limit * r along the bisector
      DF lam = df_div(df_sub(two_prod(miter, r), df_mul_f(ca, r)), sa);
      if (lam.hi < 0.f) lam = df_of(0.f);
      v1 = mk(add_round(at.x, df_add(O0.x, df_mul(c0, lam))), add_round(at.y, df_add(O0.y, df_mul(s0, lam))));
      v2 = mk(add_round(at.x, df_sub(O3.x, df_mul(c1, lam))), add_round(at.y, df_sub(O3.y, df_mul(s1, lam))));
    }
    L.v1 = v1;
    L.v2 = v2;
    L.meta |= META_FLAG_OVERRIDE;
  }
  return J;
}

// Full setup of link k of path p.  Returns the number of ribs (N+1 or 0).  PX
// compiles the pixel-scale step boost in (tau > 0); without it the link steps by
// q, and the kernel carries none of the boost's code (whose presence alone
// slowed the kernel by 40%).
template <bool MIXED, bool PX>
__device__ int link_setup(const uint8_t* st, const float* sp, const float* sw, int32_t s0, int n,
                          int k, float r, int join, int cap, float miter, bool closed, float q,
                          float tau, LinkRec& L) {
  L.meta = 0;
  L.w = 1.f;
  L.rN = L.rP = r;
  int nrib = 0;
  if (n <= 0) return 0;
  if (k & 1) {
    int i = (k - 1) >> 1;
    Seg g = load_seg(st, sp, sw, s0 + i);
    if (zero_length(g)) return 0;
    // A conic with w_B <= -1 (external parabola / hyperbola) passes through
    // infinity where its denominator vanishes, t = 1/2 +- sqrt(w^2-1)/(2(1-w)):
    // its stroke is unbounded, so it is rejected (an error, no ribs).
    if (g.type == PS_CONIC && !(g.w > -1.f)) return -1;
    L.P[0] = g.A; L.P[1] = g.B; L.P[2] = g.C; L.P[3] = g.D;
    L.w = g.w;
    L.meta = LK_SEG | ((uint32_t)g.type << 2);
    const Step S = PX ? seg_step(g, q, tau, r) : plain_step(q);
    int N = MIXED ? seg_intervals_mx<PX>(g, S, L) : seg_intervals32<PX>(g, S, L);
    if (N < 0) return -1;
    nrib = N > 0 ? N + 1 : 0;
  } else {
    // a cap (k = 0 or 2n of an open path), a join between the nearest
    // non-degenerate segments, or the closing join of a closed path
    int ia = -1, ib = -1;  // incoming / outgoing segment (cap: ia = ib = the end segment)
    int kind;
    if (k == 0 || k == 2 * n) {
      int first = -1, last = -1;
      if (k == 0 || closed) {
        for (int i = 0; i < n; ++i) {
          Seg g = load_seg(st, sp, sw, s0 + i);
          if (!zero_length(g)) { first = i; break; }
        }
      }
      if (k == 2 * n) {
        for (int i = n - 1; i >= 0; --i) {
          Seg g = load_seg(st, sp, sw, s0 + i);
          if (!zero_length(g)) { last = i; break; }
        }
      }
      if (!closed) {
        kind = LK_CAP;
        ia = ib = (k == 0) ? first : last;
        if (ia < 0) return 0;
      } else {
        if (k != 2 * n || first < 0 || last < 0) return 0;
        kind = LK_JOIN;
        ia = last;
        ib = first;
      }
    } else {
      int i = k / 2 - 1;
      Seg b = load_seg(st, sp, sw, s0 + i + 1);
      if (zero_length(b)) return 0;
      for (int m = i; m >= 0; --m) {
        Seg a = load_seg(st, sp, sw, s0 + m);
        if (!zero_length(a)) { ia = m; break; }
      }
      if (ia < 0) return 0;
      ib = i + 1;
      kind = LK_JOIN;
    }
    const Seg a = load_seg(st, sp, sw, s0 + ia), b = load_seg(st, sp, sw, s0 + ib);
    const int style = kind == LK_CAP ? cap : join;
    const bool rnd = (kind == LK_CAP && cap == PS_CAP_ROUND) || (kind == LK_JOIN && join == PS_JOIN_ROUND);
    const Step S = PX && rnd ? round_step(q, tau, r) : plain_step(q);
    const float2 at = kind == LK_CAP ? (k == 0 ? a.A : a.D) : b.A;
    L.meta = kind;
    int J;
    if constexpr (MIXED) {
      DF Psi0, delta;
      if (kind == LK_CAP) {
        // start cap: a pivot from Psi_s + pi through pi; stop cap: from Psi_e (R7)
        const DF2 e = k == 0 ? end_grad0_df(a) : end_grad1_df(a);
        Psi0 = atan2_ool(e.y, e.x);
        if (k == 0) Psi0 = df_add(Psi0, df_pi());
        delta = df_pi();
      } else {
        // Sec. 4.3.1: delta = Psi_1 (-) Psi_0, taken as the angle from the
        // incoming to the outgoing gradient; an exact reversal is +pi (R10)
        const DF2 e1 = end_grad1_df(a), e0 = end_grad0_df(b);
        Psi0 = atan2_ool(e1.y, e1.x);
        delta = atan2_ool(df_cross(e1, e0), df_dot(e1, e0));
      }
      J = pivot_setup_mx<PX>(at, Psi0, delta, kind, style, r, miter, S, L);
    } else {
      float Psi0, delta;
      if (kind == LK_CAP) {
        Psi0 = k == 0 ? angf(end_grad0(a)) + PS_PI_F : angf(end_grad1(a));
        delta = PS_PI_F;
      } else {
        Psi0 = angf(end_grad1(a));
        delta = ominus_f(angf(end_grad0(b)), Psi0);
        if (delta == -PS_PI_F) delta = PS_PI_F;
      }
      J = pivot_setup32<PX>(at, Psi0, delta, kind, style, r, miter, S, L);
    }
    nrib = J > 0 ? J + 1 : 0;
  }
  if (nrib == 0) L.meta = 0;
  return nrib;
}

// Path of link l: the p with lbase(p) <= l < lbase(p+1), lbase(p) = 2 seg_off[p] + p.
__device__ __forceinline__ int find_path(const int32_t* seg_off, int n_path, int64_t l) {
  int lo = 0, hi = n_path;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    int64_t lb = 2 * (int64_t)__ldg(seg_off + mid) + mid;
    if (lb <= l) lo = mid; else hi = mid;
  }
  return lo;
}

// ---- block scans (256 threads) ---------------------------------------------------
template <int NT>
__device__ __forceinline__ long long block_excl_sum(long long v, long long& total, long long* sm) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sm[wid] = x;
  __syncthreads();
  if (wid == 0) {
    long long w = lane < NT / 32 ? sm[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < NT / 32) sm[lane] = w;
  }
  __syncthreads();
  total = sm[NT / 32 - 1];
  long long excl = x - v + (wid > 0 ? sm[wid - 1] : 0);
  __syncthreads();
  return excl;
}

// ---------------------------------------------------------------------------
// K1: link setup + rib counts + single-pass exclusive scan into link offsets.
constexpr int SETUP_NT = 256;
constexpr int SETUP_IPT = 2;  // links per thread by default (tunable: 1, 2, 4)
constexpr int SETUP_TILE = SETUP_NT * SETUP_IPT;

template <bool MIXED, int SETUP_IPT, bool PX = false>
__global__ void __launch_bounds__(SETUP_NT, 2) k_link_setup(
    const uint8_t* __restrict__ st, const float* __restrict__ sp, const float* __restrict__ sw,
    const int32_t* __restrict__ seg_off, const float* __restrict__ width,
    const uint8_t* __restrict__ join, const uint8_t* __restrict__ cap,
    const float* __restrict__ miter, const uint8_t* __restrict__ closed, int n_path,
    int64_t n_link, float q, float tau, LinkRec* __restrict__ recs, int32_t* __restrict__ link_off,
    int32_t* __restrict__ path_off, int64_t* __restrict__ n_rib_out, int64_t capacity,
    uint32_t* tflag, long long* tagg, long long* tincl, int32_t* counters, int32_t* status,
    int64_t n_tiles, int64_t l_begin) {
  __shared__ long long sm[SETUP_NT / 32 + 1];
  __shared__ long long s_prefix;
  __shared__ int s_tile;
  // The tile's links are counting-sorted by class (the segment's type; a
  // join; a cap) so that each warp sets up links of one class: the classes
  // take different branches, and links alternate between segments and joins.
  constexpr int NCLS = 6;
  constexpr int TILE_L = SETUP_NT * SETUP_IPT;
  __shared__ int s_ncls[NCLS];
  __shared__ uint16_t s_perm[TILE_L];
  __shared__ int s_cnt[TILE_L];  // rib count of each local link
  __shared__ int s_pth[TILE_L];  // its path
  __shared__ int s_kk[TILE_L];   // its index within the path
  if (threadIdx.x == 0) s_tile = atomicAdd(&counters[0], 1);
  if (threadIdx.x < NCLS) s_ncls[threadIdx.x] = 0;
  __syncthreads();
  int64_t tile = s_tile;
  if (tile >= n_tiles) return;
  const int64_t l_tile = tile * (int64_t)TILE_L;
  int cls_rank[SETUP_IPT];
  for (int i = 0; i < SETUP_IPT; ++i) {
    const int li = threadIdx.x * SETUP_IPT + i;
    const int64_t l = l_tile + li;
    cls_rank[i] = -1;
    s_cnt[li] = 0;
    if (l < n_link) {
      // local link l is link l_begin + l of the batch (a range call)
      const int64_t lg = l_begin + l;
      const int p = find_path(seg_off, n_path, lg);
      const int32_t s0 = __ldg(seg_off + p), n = __ldg(seg_off + p + 1) - s0;
      const int k = (int)(lg - (2 * (int64_t)s0 + p));
      s_pth[li] = p;
      s_kk[li] = k;
      const int c = (k & 1) ? min((int)__ldg(st + s0 + ((k - 1) >> 1)), 3)
                            : ((k == 0 || k == 2 * n) && !closed[p]) ? 5 : 4;
      cls_rank[i] = c << 16 | atomicAdd(&s_ncls[c], 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int c = 0; c < NCLS; ++c) {
      const int v = s_ncls[c];
      s_ncls[c] = acc;
      acc += v;
    }
  }
  __syncthreads();
  for (int i = 0; i < SETUP_IPT; ++i)
    if (cls_rank[i] >= 0)
      s_perm[s_ncls[cls_rank[i] >> 16] + (cls_rank[i] & 0xffff)] =
          (uint16_t)(threadIdx.x * SETUP_IPT + i);
  __syncthreads();
  const int n_here = (int)min((int64_t)TILE_L, n_link > l_tile ? n_link - l_tile : (int64_t)0);
  for (int i = 0; i < SETUP_IPT; ++i) {
    const int w = i * SETUP_NT + threadIdx.x;  // consecutive lanes, consecutive sorted links
    if (w < n_here) {
      const int li = s_perm[w];
      const int p = s_pth[li], k = s_kk[li];
      const int32_t s0 = __ldg(seg_off + p), s1 = __ldg(seg_off + p + 1);
      LinkRec L = {};
      int nr = link_setup<MIXED, PX>(st, sp, sw, s0, s1 - s0, k, 0.5f * __ldg(width + p), join[p],
                                 cap[p], __ldg(miter + p), closed[p] != 0, q, tau, L);
      if (nr < 0) {
        ps_record_error(status, PS_ERR_INVALID);
        nr = 0;
        L.meta = 0;
      }
      L.pad = 0;
      recs[l_tile + li] = L;
      s_cnt[li] = nr;
    }
  }
  __syncthreads();
  long long local = 0;
  for (int i = 0; i < SETUP_IPT; ++i) local += s_cnt[threadIdx.x * SETUP_IPT + i];
  long long total;
  long long excl = block_excl_sum<SETUP_NT>(local, total, sm);
  if (threadIdx.x < 32) {
    long long pre = lookback_sum_warp(tflag, tagg, tincl, total, tile, status);
    if (threadIdx.x == 0) s_prefix = pre;
  }
  __syncthreads();
  long long off = s_prefix + excl;
  for (int i = 0; i < SETUP_IPT; ++i) {
    const int li = threadIdx.x * SETUP_IPT + i;
    const int64_t l = l_tile + li;
    if (l < n_link) {
      if (off > 0x7fffffffLL) ps_record_error(status, PS_ERR_CAPACITY);
      link_off[l] = (int32_t)off;
      const int p = s_pth[li], kk = s_kk[li];
      if (kk == 0) path_off[p] = (int32_t)off;
      off += s_cnt[li];
      if (l == n_link - 1) {
        link_off[n_link] = (int32_t)off;
        // the end of the last path, when the range ends with that path's last link
        if (kk == 2 * (__ldg(seg_off + p + 1) - __ldg(seg_off + p))) path_off[p + 1] = (int32_t)off;
        *n_rib_out = off;
        if (off > capacity) ps_record_error(status, PS_ERR_CAPACITY);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// K2: ribs.  Each warp takes chunks of EMIT_CHUNK consecutive ribs and works
// through them in slabs of 32, one rib per lane: the lane's link advances
// monotonically from the chunk's first link (found by a 32-way search), the
// rib's psi(j), t(j), g(t(j)) and n(j) are evaluated, and the rib, its tag and
// the chord to the previous rib of the same link (the previous lane, the last
// lane of the previous slab, or for the chunk's first rib a re-evaluation) are
// written.  No block-wide synchronisation.
constexpr int EMIT_NT = 256;
constexpr int EMIT_K = 32;  // slabs of 32 ribs per chunk by default (tunable: 4, 8, 16, 32, 64)

struct RibEval {
  float4 v;      // N.x N.y P.x P.y
  float2 grel;   // g(t) - A (segments) for the chord
  float2 glo;    // its low parts as pairs (0 in FP32)
  float t, tlo;  // t as a pair (tlo = 0 in FP32)
  bool seg;
};

// One rib, FP32 (PS_PREC_FP32).
__device__ __forceinline__ RibEval eval_rib32(const LinkRec* __restrict__ L, int j) {
  // fields are read where needed (L1-cached) instead of copying the record
  RibEval R;
  uint32_t meta = __ldg(&L->meta);
  int kind = META_KIND(meta);
  int M = META_M(meta);
  float4 p01 = __ldg(reinterpret_cast<const float4*>(L->P));
  float rN = __ldg(&L->rN), rP = __ldg(&L->rP);
  R.tlo = 0.f;
  R.glo = mk(0.f, 0.f);
  if (kind == LK_SEG) {
    Seg g;
    float4 p23 = __ldg(reinterpret_cast<const float4*>(L->P) + 1);
    g.type = META_TYPE(meta);
    g.A = mk(p01.x, p01.y); g.B = mk(p01.z, p01.w); g.C = mk(p23.x, p23.y); g.D = mk(p23.z, p23.w);
    g.w = __ldg(&L->w);
    int k = 0;
    while (k < M && j >= (int)__ldg(&L->dsum[k + 1])) ++k;
    // k == M only for j == N; boundary when j == dsum[k]
    float t, psi;
    int dk = (int)__ldg(&L->dsum[k]);
    bool bnd = j == dk;
    psi = bnd ? __ldg(&L->psi[k]) : __ldg(&L->psi[k]) + __ldg(&L->step[k]) * (float)(j - dk);
    float sn, cs;
    sincosf(psi, &sn, &cs);
    float pa = __ldg(&L->p[k]);
    if (bnd || META_PIVOT(meta, k)) t = pa;
    else t = solve_t(g, sn, cs, pa, __ldg(&L->p[k + 1]));
    float2 n = mk(-sn, cs);
    float2 gr = g_rel(g, t);
    float2 Nv = gr - n * rN, Pv = gr + n * rP;
    R.v = make_float4(g.A.x + Nv.x, g.A.y + Nv.y, g.A.x + Pv.x, g.A.y + Pv.y);
    R.grel = gr;
    R.t = t;
    R.seg = true;
  } else {
    int J = (int)__ldg(&L->dsum[1]);
    float psi = (j == J) ? __ldg(&L->psi[1]) : __ldg(&L->psi[0]) + __ldg(&L->step[0]) * (float)j;
    float sn, cs;
    sincosf(psi, &sn, &cs);
    float2 n = mk(-sn, cs);
    float rn = rN, rp = rP;
    if ((meta & META_FLAG_SQUARE) && (j == 1 || j == 3)) {
      rn *= 1.41421356237309515f;
      rp *= 1.41421356237309515f;
    }
    float2 at = mk(p01.x, p01.y);
    float2 Nv = at - n * rn, Pv = at + n * rp;
    if ((meta & META_FLAG_OVERRIDE) && (j == 1 || j == 2)) {
      float4 vv = __ldg(reinterpret_cast<const float4*>(&L->v1));
      float2 v = j == 1 ? mk(vv.x, vv.y) : mk(vv.z, vv.w);
      if (rN > 0.f) Nv = v; else Pv = v;
    }
    R.v = make_float4(Nv.x, Nv.y, Pv.x, Pv.y);
    R.grel = mk(0.f, 0.f);
    R.t = 0.f;
    R.seg = false;
  }
  return R;
}

__device__ __forceinline__ DF ld_pair(const float* hi, const float* lo) { return DF{__ldg(hi), __ldg(lo)}; }

// One rib, PS_PREC_MIXED: psi(j) = Psi_k + step_k (j - Delta_Sigma(k)) as a
// pair, its normal by the double-float sincos (one call for every kind of
// link), t by the double-float solve, g(t) compensated, and each vertex
// coordinate summed in double-float and rounded once (Eq. 14-17).
__device__ __forceinline__ RibEval eval_rib_mx(const LinkRec* __restrict__ L, int j) {
  RibEval R;
  const uint32_t meta = __ldg(&L->meta);
  const int kind = META_KIND(meta);
  const float4 p01 = __ldg(reinterpret_cast<const float4*>(L->P));
  const float rN = __ldg(&L->rN), rP = __ldg(&L->rP);
  const bool seg = kind == LK_SEG;
  // the rib's angle
  int k = 0, dk = 0;
  DF psi;
  if (seg) {
    const int M = META_M(meta);
    while (k < M && j >= (int)__ldg(&L->dsum[k + 1])) ++k;
    dk = (int)__ldg(&L->dsum[k]);
  } else {
    dk = j == (int)__ldg(&L->dsum[1]) ? j : 0;  // the last pivot rib is Psi_1 itself
    k = dk ? 1 : 0;
  }
  psi = ld_pair(&L->psi[k], &L->psi_lo[k]);
  if (j != dk) psi = df_add(psi, df_mul_f(ld_pair(&L->step[k], &L->step_lo[k]), (float)(j - dk)));
  DF sn, cs;
  df_sincos(psi, ps_sc_tab, sn, cs);
  // the generator point, relative parts as a pair
  float ax = p01.x, ay = p01.y;
  DF gx{0.f, 0.f}, gy{0.f, 0.f};
  DF rn = df_of(rN), rp = df_of(rP);
  R.grel = mk(0.f, 0.f);
  R.glo = mk(0.f, 0.f);
  R.t = 0.f;
  R.tlo = 0.f;
  if (seg) {
    Seg g;
    const float4 p23 = __ldg(reinterpret_cast<const float4*>(L->P) + 1);
    g.type = META_TYPE(meta);
    g.A = mk(p01.x, p01.y); g.B = mk(p01.z, p01.w); g.C = mk(p23.x, p23.y); g.D = mk(p23.z, p23.w);
    g.w = __ldg(&L->w);
    const DF pa = ld_pair(&L->p[k], &L->p_lo[k]);
    DF t = pa;
    if (j != dk && !META_PIVOT(meta, k))
      t = solve_t_mx(g, sn, cs, pa, ld_pair(&L->p[k + 1], &L->p_lo[k + 1]));
    const DF2 gr = g_rel_df(g, t);
    gx = gr.x;
    gy = gr.y;
    R.grel = mk(gr.x.hi, gr.y.hi);
    R.glo = mk(gr.x.lo, gr.y.lo);
    R.t = t.hi;
    R.tlo = t.lo;
  } else if ((meta & META_FLAG_SQUARE) && (j == 1 || j == 3)) {
    rn = df_mul_f(df_sqrt2(), rN);
    rp = df_mul_f(df_sqrt2(), rP);
  }
  // N = A + g - rn n, P = A + g + rp n, n = (-sin psi, cos psi)
  const DF sx = two_sum(ax, gx.hi), sy = two_sum(ay, gy.hi);
  float4 v = make_float4(sum_prod_round(sx, gx.lo, sn, rn), sum_prod_round(sy, gy.lo, df_neg(cs), rn),
                         sum_prod_round(sx, gx.lo, df_neg(sn), rp), sum_prod_round(sy, gy.lo, cs, rp));
  if ((meta & META_FLAG_OVERRIDE) && (j == 1 || j == 2)) {
    const float4 vv = __ldg(reinterpret_cast<const float4*>(&L->v1));
    const float2 o = j == 1 ? mk(vv.x, vv.y) : mk(vv.z, vv.w);
    if (rN > 0.f) { v.x = o.x; v.y = o.y; } else { v.z = o.x; v.w = o.y; }
  }
  R.v = v;
  R.seg = seg;
  return R;
}

template <bool MIXED>
__device__ __forceinline__ RibEval eval_rib(const LinkRec* __restrict__ L, int j) {
  if constexpr (MIXED) return eval_rib_mx(L, j);
  else return eval_rib32(L, j);
}

// The same, out of line: the emitter's rare re-evaluation of a chunk's
// preceding rib calls it, so the hot loop holds one copy of the rib code.
template <bool MIXED>
__device__ __noinline__ RibEval eval_rib_ool(const LinkRec* __restrict__ L, int j) {
  return eval_rib<MIXED>(L, j);
}

__device__ __forceinline__ int64_t find_link(const int32_t* off, int64_t lo, int64_t hi, int64_t r) {
  // last l in [lo, hi] with off[l] <= r  (off non-decreasing)
  while (hi > lo) {
    int64_t mid = (lo + hi + 1) >> 1;
    if ((int64_t)__ldg(off + mid) <= r) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Warp-cooperative find_link over [0, n - 1] (off[0] <= r): 32 probes per round.
__device__ __forceinline__ int64_t find_link_warp(const int32_t* off, int64_t n, int64_t r,
                                                  int lane) {
  int64_t lo = 0, hi = n - 1;  // off[lo] <= r, answer in [lo, hi]
  while (hi - lo > 31) {
    int64_t step = (hi - lo + 31) / 32;
    int64_t cand = lo + lane * step;
    bool ok = cand <= hi && (int64_t)__ldg(off + cand) <= r;
    uint32_t b = __ballot_sync(0xffffffffu, ok);
    int m = __popc(b);  // lanes 0 .. m-1 ok (lane 0 always)
    int64_t nlo = lo + (int64_t)(m - 1) * step;
    int64_t nhi = m < 32 ? lo + (int64_t)m * step - 1 : hi;
    lo = nlo;
    hi = nhi < hi ? nhi : hi;
  }
  int64_t cand = lo + lane;
  bool ok = cand <= hi && (int64_t)__ldg(off + cand) <= r;
  uint32_t b = __ballot_sync(0xffffffffu, ok);
  return lo + __popc(b) - 1;
}

template <bool MIXED>
__global__ void __launch_bounds__(EMIT_NT, MIXED ? 2 : 3) k_emit(
    const LinkRec* __restrict__ recs, const int32_t* __restrict__ link_off,
    const int32_t* __restrict__ link_path, int64_t n_link, const int64_t* __restrict__ n_rib,
    int64_t capacity, float4* __restrict__ rib, uint32_t* __restrict__ tag,
    float* __restrict__ chord, float* __restrict__ tout, int emit_k) {
  int64_t R = *n_rib;
  if (R > capacity) R = capacity;
  const int lane = threadIdx.x & 31;
  const int64_t chunk = 32 * (int64_t)emit_k;
  const int64_t n_chunks = (R + chunk - 1) / chunk;
  const int64_t warp0 = ((int64_t)blockIdx.x * EMIT_NT + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * EMIT_NT) >> 5;
  for (int64_t c = warp0; c < n_chunks; c += n_warps) {
    const int64_t r0 = c * chunk;
    int64_t l = find_link_warp(link_off, n_link, r0, lane);
    float2 carry_g = mk(0.f, 0.f), carry_gl = mk(0.f, 0.f);
    float carry_t = 0.f, carry_tl = 0.f;
#pragma unroll 1
    for (int s = 0; s < emit_k; ++s) {
      const int64_t r = r0 + (int64_t)s * 32 + lane;
      const bool active = r < R;
      RibEval E;
      E.grel = mk(0.f, 0.f);
      E.glo = mk(0.f, 0.f);
      E.t = 0.f;
      E.tlo = 0.f;
      E.seg = false;
      int j = 0;
      if (active) {
        while (l + 1 < n_link && (int64_t)__ldg(link_off + l + 1) <= r) ++l;
        j = (int)(r - __ldg(link_off + l));
        E = eval_rib<MIXED>(recs + l, j);
        rib[r] = E.v;
        uint32_t p = (uint32_t)__ldg(link_path + l);
        tag[r] = (p << 2) | (E.seg ? PS_TAG_SEGMENT : 0u) | (j == 0 ? PS_TAG_LINK_START : 0u);
        if (tout) tout[r] = E.t + E.tlo;
      }
      if (chord) {
        // rib r - 1 is in the same link iff j > 0
        float2 pg, pgl = mk(0.f, 0.f);
        pg.x = __shfl_up_sync(0xffffffffu, E.grel.x, 1);
        pg.y = __shfl_up_sync(0xffffffffu, E.grel.y, 1);
        if (MIXED) {
          pgl.x = __shfl_up_sync(0xffffffffu, E.glo.x, 1);
          pgl.y = __shfl_up_sync(0xffffffffu, E.glo.y, 1);
        }
        float pt = __shfl_up_sync(0xffffffffu, E.t, 1);
        float ptl = MIXED ? __shfl_up_sync(0xffffffffu, E.tlo, 1) : 0.f;
        if (lane == 0) {
          pg = carry_g;
          pgl = carry_gl;
          pt = carry_t;
          ptl = carry_tl;
        }
        carry_g.x = __shfl_sync(0xffffffffu, E.grel.x, 31);
        carry_g.y = __shfl_sync(0xffffffffu, E.grel.y, 31);
        if (MIXED) {
          carry_gl.x = __shfl_sync(0xffffffffu, E.glo.x, 31);
          carry_gl.y = __shfl_sync(0xffffffffu, E.glo.y, 31);
        }
        carry_t = __shfl_sync(0xffffffffu, E.t, 31);
        if (MIXED) carry_tl = __shfl_sync(0xffffffffu, E.tlo, 31);
        if (active) {
          float cl = 0.f;
          if (E.seg && j > 0) {
            if (lane == 0 && s == 0) {
              RibEval Ep = eval_rib_ool<MIXED>(recs + l, j - 1);
              pg = Ep.grel;
              pgl = Ep.glo;
              pt = Ep.t;
              ptl = Ep.tlo;
            }
            // Sec. 7: a step whose t decreases adds no length.  The chord is
            // differenced as pairs before rounding (MIXED).
            if (E.t > pt || (E.t == pt && E.tlo >= ptl)) {
              float dx = (E.grel.x - pg.x) + (E.glo.x - pgl.x);
              float dy = (E.grel.y - pg.y) + (E.glo.y - pgl.y);
              cl = sqrtf(dx * dx + dy * dy);
            }
          }
          chord[r] = cl;
        }
      }
    }
  }
}

// Path index of every link (for the rib tags).
__global__ void k_link_path(const int32_t* __restrict__ seg_off, int n_path, int64_t n_link,
                            int32_t* __restrict__ link_path, int64_t l_begin) {
  int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= n_link) return;
  link_path[l] = find_path(seg_off, n_path, l_begin + l);
}

// ---------------------------------------------------------------------------
// K3: segmented inclusive scan of per-rib chords into cumulative arc length
// (Eq. 18), restarting at every path's first rib.  The tessellation runs it in
// place on the chords the emitter wrote into s; it is also the standalone arc
// length of a given rib stream (ps_arclength_scan) and the adjoint's suffix
// sums.
constexpr int SCAN_NT = 256;
constexpr int SCAN_IPT = 16;
constexpr int SCAN_TILE = SCAN_NT * SCAN_IPT;

// Segmented (by path) inclusive scan of per-rib chords into s (Eq. 18), in
// place allowed (chord_in == s_out).  Persistent CTAs claim tiles of 4,096 ribs
// in order (by ticket); thread k of a tile owns ribs 16k..16k+15 and, with VEC (all three
// arrays 16-byte aligned), moves them with 128-bit loads and stores.  Within a
// tile sums are FP32 (relative error ~1e-6 of s); the carry between tiles,
// which runs over a whole path, is a double-float pair from a warp-wide
// look-back.
template <bool VEC>
__global__ void __launch_bounds__(SCAN_NT) k_arclen_scan(
    const float* chord_in, const uint32_t* __restrict__ tag, const int64_t* __restrict__ n_rib,
    int64_t capacity, float* s_out, float* __restrict__ path_len, uint32_t* tflag,
    unsigned long long* tagg, unsigned long long* tincl, int32_t* counters, int32_t* status) {
  __shared__ float sv[SCAN_NT / 32];
  __shared__ int sh[SCAN_NT / 32];
  __shared__ float s_carry[2];
  __shared__ int64_t s_tile;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t R = *n_rib;
  if (R > capacity) R = capacity;
  const int64_t n_tiles = (R + SCAN_TILE - 1) / SCAN_TILE;
  // tiles are claimed by ticket; a tile's successor ticket is claimed as soon as
  // its look-back is done, so that the atomic's latency hides behind the
  // tile's stores (claiming earlier would hold back tiles that later tiles'
  // look-backs wait on)
  __shared__ int64_t s_next;
  if (threadIdx.x == 0) s_tile = atomicAdd(&counters[1], 1);
  __syncthreads();
  for (;;) {
    // every thread reads s_tile before the barriers below, and thread 0
    // rewrites it only after them
    const int64_t tile = s_tile;
    if (tile >= n_tiles) return;
    const int64_t base = tile * SCAN_TILE + (int64_t)threadIdx.x * SCAN_IPT;
    const bool full = base + SCAN_IPT <= R;
    float c[SCAN_IPT];
    uint32_t pth[SCAN_IPT];
    if (VEC && full) {
      const float4* cp = reinterpret_cast<const float4*>(chord_in + base);
      const uint4* tp = reinterpret_cast<const uint4*>(tag + base);
#pragma unroll
      for (int q = 0; q < SCAN_IPT / 4; ++q) {
        float4 a = cp[q];
        uint4 b = __ldg(tp + q);
        c[4 * q] = a.x; c[4 * q + 1] = a.y; c[4 * q + 2] = a.z; c[4 * q + 3] = a.w;
        pth[4 * q] = b.x >> 2; pth[4 * q + 1] = b.y >> 2;
        pth[4 * q + 2] = b.z >> 2; pth[4 * q + 3] = b.w >> 2;
      }
    } else {
#pragma unroll
      for (int i = 0; i < SCAN_IPT; ++i) {
        int64_t r = base + i;
        c[i] = r < R ? chord_in[r] : 0.f;
        pth[i] = r < R ? (__ldg(tag + r) >> 2) : 0xffffffffu;
      }
    }
    // path of the rib before this thread's first: the previous lane's last
    uint32_t prevp = __shfl_up_sync(0xffffffffu, pth[SCAN_IPT - 1], 1);
    if (lane == 0) prevp = (base > 0 && base <= R) ? (__ldg(tag + base - 1) >> 2) : 0xffffffffu;
    uint32_t hm = 0;  // bit i: rib base + i starts a path
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < SCAN_IPT; ++i) {
      uint32_t pp = i ? pth[i - 1] : prevp;
      if (base + i < R && (base + i == 0 || pp != pth[i])) {
        hm |= 1u << i;
        acc = 0.f;
      }
      acc += c[i];
    }
    float v = acc;
    int h = hm != 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      float vy = __shfl_up_sync(0xffffffffu, v, o);
      int hy = __shfl_up_sync(0xffffffffu, h, o);
      if (lane >= o) {
        if (!h) v += vy;
        h |= hy;
      }
    }
    if (lane == 31) {
      sv[wid] = v;
      sh[wid] = h;
    }
    __syncthreads();
    float wcarry = 0.f;
    int whead = 0;
    for (int w = wid - 1; w >= 0; --w) {
      wcarry += sv[w];
      if (sh[w]) { whead = 1; break; }
    }
    if (wid == 0) {
      DF tile_v{0.f, 0.f};
      int tile_h = 0;
      for (int w = SCAN_NT / 32 - 1; w >= 0; --w) {
        tile_v = df_add_f(tile_v, sv[w]);
        if (sh[w]) { tile_h = 1; break; }
      }
      DF carry = lookback_segsum_df(tflag, tagg, tincl, tile_v, tile_h != 0, tile, status);
      if (lane == 0) {
        s_carry[0] = carry.hi;
        s_carry[1] = carry.lo;
        s_next = atomicAdd(&counters[1], 1);
      }
    }
    __syncthreads();
    float vprev = __shfl_up_sync(0xffffffffu, v, 1);
    int hprev = __shfl_up_sync(0xffffffffu, h, 1);
    if (lane == 0) {
      vprev = 0.f;
      hprev = 0;
    }
    // path of the rib after this thread's last: the next lane's first
    uint32_t nextp = __shfl_down_sync(0xffffffffu, pth[0], 1);
    if (lane == 31) nextp = base + SCAN_IPT < R ? (__ldg(tag + base + SCAN_IPT) >> 2) : 0xffffffffu;
    // ribs before this thread's first head continue the running total
    const DF tile_carry = (hprev || whead) ? DF{0.f, 0.f} : DF{s_carry[0], s_carry[1]};
    float run = hprev ? vprev : vprev + wcarry;
    bool after_head = false;
#pragma unroll
    for (int i = 0; i < SCAN_IPT; ++i) {
      if ((hm >> i) & 1u) {
        run = 0.f;
        after_head = true;
      }
      run += c[i];
      c[i] = after_head ? run : df_f(df_add_f(tile_carry, run));
      uint32_t np = i + 1 < SCAN_IPT ? pth[i + 1] : nextp;
      if (path_len && base + i < R && np != pth[i]) path_len[pth[i]] = c[i];
    }
    if (VEC && full) {
      float4* op = reinterpret_cast<float4*>(s_out + base);
#pragma unroll
      for (int q = 0; q < SCAN_IPT / 4; ++q)
        op[q] = make_float4(c[4 * q], c[4 * q + 1], c[4 * q + 2], c[4 * q + 3]);
    } else {
#pragma unroll
      for (int i = 0; i < SCAN_IPT; ++i)
        if (base + i < R) s_out[base + i] = c[i];
    }
    if (threadIdx.x == 0) s_tile = s_next;
    __syncthreads();
  }
}

// Launch of k_arclen_scan with the vector form when every array allows it.
static void launch_arclen_scan(ps_context* ctx, int grid_override, cudaStream_t st,
                               const float* chord, const uint32_t* tag, const int64_t* n_rib,
                               int64_t capacity, float* s_out, float* path_len, uint32_t* flag,
                               double* aggd, double* incld, int32_t* counters, int32_t* status) {
  // the tile states' 8-byte words hold double-float pairs
  unsigned long long* agg = reinterpret_cast<unsigned long long*>(aggd);
  unsigned long long* incl = reinterpret_cast<unsigned long long*>(incld);
  const bool vec = ((reinterpret_cast<uintptr_t>(chord) | reinterpret_cast<uintptr_t>(tag) |
                     reinterpret_cast<uintptr_t>(s_out)) & 15u) == 0;
  const void* fn = vec ? (const void*)k_arclen_scan<true> : (const void*)k_arclen_scan<false>;
  int g = grid_override > 0 ? grid_override : ps_persistent_grid(ctx, fn, SCAN_NT, 0);
  if (vec)
    k_arclen_scan<true><<<g, SCAN_NT, 0, st>>>(chord, tag, n_rib, capacity, s_out, path_len, flag,
                                               agg, incl, counters, status);
  else
    k_arclen_scan<false><<<g, SCAN_NT, 0, st>>>(chord, tag, n_rib, capacity, s_out, path_len,
                                                flag, agg, incl, counters, status);
}

// Chords from rib midpoints (standalone arc length of any rib stream).
__global__ void k_midpoint_chords(const float4* __restrict__ rib, const uint32_t* __restrict__ tag,
                                  const int64_t* __restrict__ n_rib, int64_t capacity,
                                  float* __restrict__ chord) {
  int64_t R = *n_rib;
  if (R > capacity) R = capacity;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R;
       r += (int64_t)gridDim.x * blockDim.x) {
    uint32_t tg = tag[r];
    float c = 0.f;
    if ((tg & PS_TAG_SEGMENT) && !(tg & PS_TAG_LINK_START) && r > 0) {
      float4 a = rib[r - 1], b = rib[r];
      float dx = 0.5f * ((b.x + b.z) - (a.x + a.z)), dy = 0.5f * ((b.y + b.w) - (a.y + a.w));
      c = sqrtf(dx * dx + dy * dy);
    }
    chord[r] = c;
  }
}

}  // namespace ps

using namespace ps;

// ===========================================================================
// host entry points
// Tessellation of the links [l0, l0 + L) of the batch (all of them when called
// for the whole batch): offsets and ribs are local to the range.
static int launch_tessellate(ps_context* ctx, const ps_segments* seg, const ps_paths* paths,
                             float dtheta, int precision, uint32_t flags, ps_tess_out* out,
                             cudaStream_t st, int64_t l0, int64_t L) {
  int P = paths->n_path;
  if (P <= 0) return PS_ERR_INVALID;
  // links per thread: the tuned value, or the default for the boosted kernel
  // (one instantiation only)
  const int ipt = ctx->pixel_tol > 0.f ? SETUP_IPT : ctx->tune[PS_TUNE_SETUP_LINKS];
  int64_t n_tiles = (L + SETUP_NT * ipt - 1) / (SETUP_NT * ipt);
  int rc;
  // the arc-length scan's tiles follow the set-up tiles in the tile states
  if ((rc = ps_ensure_tiles(ctx, n_tiles + (out->capacity + SCAN_TILE - 1) / SCAN_TILE + 2)) != PS_OK)
    return rc;
  if ((rc = ps_ensure_recs(ctx, L)) != PS_OK) return rc;
  // link path indices live after the records
  int32_t* link_path = reinterpret_cast<int32_t*>(ctx->d_recs + ctx->rec_cap);
  cudaMemsetAsync(ctx->d_tile_flag, 0, sizeof(uint32_t) * n_tiles, st);
  cudaMemsetAsync(ctx->d_counters, 0, sizeof(int32_t) * 16, st);
  // a count-only call has no rib buffers to overflow
  int64_t count_cap = (flags & PS_TESS_COUNT_ONLY) ? INT64_MAX : out->capacity;
  { ProfScope ps_(ctx, PK_LINK_PATH, st);
  k_link_path<<<(unsigned)((L + 255) / 256), 256, 0, st>>>(paths->d_seg_off, P, L, link_path, l0); }
  {
  ProfScope ps_(ctx, PK_LINK_SETUP, st);
#define PS_SETUP_ARGS                                                                          \
  seg->d_type, seg->d_pts, seg->d_w, paths->d_seg_off, paths->d_width, paths->d_join,         \
      paths->d_cap, paths->d_miter, paths->d_closed, P, L, dtheta, ctx->pixel_tol, ctx->d_recs, \
      out->d_link_rib_off, out->d_path_rib_off, out->d_n_rib, count_cap, ctx->d_tile_flag,    \
      ctx->d_tile_agg, ctx->d_tile_incl, ctx->d_counters, ctx->d_status, n_tiles, l0
  const unsigned g = (unsigned)n_tiles;
  const bool mx = precision == PS_PREC_MIXED;
  if (ctx->pixel_tol > 0.f) {
    if (mx) k_link_setup<true, SETUP_IPT, true><<<g, SETUP_NT, 0, st>>>(PS_SETUP_ARGS);
    else k_link_setup<false, SETUP_IPT, true><<<g, SETUP_NT, 0, st>>>(PS_SETUP_ARGS);
  } else if (ipt == 1) {
    if (mx) k_link_setup<true, 1><<<g, SETUP_NT, 0, st>>>(PS_SETUP_ARGS);
    else k_link_setup<false, 1><<<g, SETUP_NT, 0, st>>>(PS_SETUP_ARGS);
  } else if (ipt == 4) {
    if (mx) k_link_setup<true, 4><<<g, SETUP_NT, 0, st>>>(PS_SETUP_ARGS);
    else k_link_setup<false, 4><<<g, SETUP_NT, 0, st>>>(PS_SETUP_ARGS);
  } else {
    if (mx) k_link_setup<true, 2><<<g, SETUP_NT, 0, st>>>(PS_SETUP_ARGS);
    else k_link_setup<false, 2><<<g, SETUP_NT, 0, st>>>(PS_SETUP_ARGS);
  }
#undef PS_SETUP_ARGS
  }
  if ((rc = ps_cuda_check(cudaGetLastError())) != PS_OK) return rc;
  if (flags & PS_TESS_COUNT_ONLY) return PS_OK;

  bool arc = (flags & PS_TESS_ARCLENGTH) && out->d_s;
  const void* fn = precision == PS_PREC_MIXED ? (const void*)k_emit<true> : (const void*)k_emit<false>;
  int grid = ps_persistent_grid(ctx, fn, EMIT_NT, 0);
  {
  ProfScope ps_(ctx, PK_EMIT, st);
#define PS_EMIT_ARGS                                                                           \
  ctx->d_recs, out->d_link_rib_off, link_path, L, out->d_n_rib, out->capacity,                 \
      reinterpret_cast<float4*>(out->d_rib), out->d_tag, arc ? out->d_s : nullptr, out->d_t,   \
      ctx->tune[PS_TUNE_EMIT_SLABS]
  if (precision == PS_PREC_MIXED) k_emit<true><<<grid, EMIT_NT, 0, st>>>(PS_EMIT_ARGS);
  else k_emit<false><<<grid, EMIT_NT, 0, st>>>(PS_EMIT_ARGS);
#undef PS_EMIT_ARGS
  }
  if ((rc = ps_cuda_check(cudaGetLastError())) != PS_OK) return rc;
  if (arc) {
    // the emitter wrote each rib's chord into s; the segmented scan turns them
    // into cumulative arc length in place
    int64_t scan_tiles = (out->capacity + SCAN_TILE - 1) / SCAN_TILE;
    cudaMemsetAsync(ctx->d_tile_flag + n_tiles + 1, 0, sizeof(uint32_t) * (scan_tiles + 1), st);
    if (out->d_path_len) cudaMemsetAsync(out->d_path_len, 0, sizeof(float) * P, st);
    ProfScope ps_(ctx, PK_ARCLEN, st);
    launch_arclen_scan(ctx, 0, st, out->d_s, out->d_tag, out->d_n_rib, out->capacity, out->d_s,
                       out->d_path_len, ctx->d_tile_flag + n_tiles + 1,
                       ctx->d_tile_aggd + n_tiles + 1, ctx->d_tile_incld + n_tiles + 1,
                       ctx->d_counters, ctx->d_status);
    if ((rc = ps_cuda_check(cudaGetLastError())) != PS_OK) return rc;
  }
  return PS_OK;
}

// An empty batch (no paths, no segments): R = 0 and the single zero entry of
// each offset array; no kernel runs.
static int empty_batch(ps_tess_out* out, cudaStream_t st) {
  if (!out->d_link_rib_off || !out->d_path_rib_off || !out->d_n_rib) return PS_ERR_INVALID;
  int rc = ps_cuda_check(cudaMemsetAsync(out->d_n_rib, 0, sizeof(int64_t), st));
  if (rc == PS_OK) rc = ps_cuda_check(cudaMemsetAsync(out->d_link_rib_off, 0, sizeof(int32_t), st));
  if (rc == PS_OK) rc = ps_cuda_check(cudaMemsetAsync(out->d_path_rib_off, 0, sizeof(int32_t), st));
  return rc;
}

extern "C" int ps_tessellate_strokes(ps_context* ctx, const ps_segments* seg,
                                     const ps_paths* paths, float dtheta, int precision,
                                     uint32_t flags, ps_tess_out* out, void* stream) {
  if (!ctx || !seg || !paths || !out) return PS_ERR_INVALID;
  if (!(dtheta >= 1e-4f && dtheta <= 3.14159265f)) return PS_ERR_INVALID;
  if (precision != PS_PREC_FP32 && precision != PS_PREC_MIXED) return PS_ERR_INVALID;
  if (seg->n_seg < 0 || paths->n_path < 0 || seg->n_seg > (int64_t)1 << 29) return PS_ERR_INVALID;
  if (paths->n_path == 0) {
    if (seg->n_seg != 0) return PS_ERR_INVALID;
    ctx->last_stream = stream;
    return empty_batch(out, (cudaStream_t)stream);
  }
  if (seg->n_seg > 0 && (!seg->d_type || !seg->d_pts)) return PS_ERR_INVALID;
  if (!paths->d_seg_off || !paths->d_width || !paths->d_join || !paths->d_cap ||
      !paths->d_miter || !paths->d_closed)
    return PS_ERR_INVALID;
  if (!out->d_link_rib_off || !out->d_path_rib_off || !out->d_n_rib) return PS_ERR_INVALID;
  if (!(flags & PS_TESS_COUNT_ONLY) && (!out->d_rib || !out->d_tag || out->capacity < 0))
    return PS_ERR_INVALID;
  if ((flags & PS_TESS_ARCLENGTH) && !(flags & PS_TESS_COUNT_ONLY) && !out->d_s)
    return PS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = stream;
  return launch_tessellate(ctx, seg, paths, dtheta, precision, flags, out, st, 0,
                           2 * seg->n_seg + paths->n_path);
}

extern "C" int ps_count_ribs_sync(ps_context* ctx, const ps_segments* seg, const ps_paths* paths,
                                  float dtheta, int precision, ps_tess_out* out, void* stream,
                                  int64_t* h_n_rib) {
  if (!h_n_rib) return PS_ERR_INVALID;
  int rc = ps_tessellate_strokes(ctx, seg, paths, dtheta, precision, PS_TESS_COUNT_ONLY, out,
                                 stream);
  if (rc != PS_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  rc = ps_cuda_check(cudaMemcpyAsync(h_n_rib, out->d_n_rib, sizeof(int64_t),
                                     cudaMemcpyDeviceToHost, st));
  if (rc != PS_OK) return rc;
  return ps_cuda_check(cudaStreamSynchronize(st));
}

extern "C" int ps_tessellate_links(ps_context* ctx, const ps_segments* seg,
                                   const ps_paths* paths, float dtheta, int precision,
                                   uint32_t flags, int64_t link_begin, int64_t link_end,
                                   ps_tess_out* out, void* stream) {
  if (!ctx || !seg || !paths || !out) return PS_ERR_INVALID;
  if (!(dtheta >= 1e-4f && dtheta <= 3.14159265f)) return PS_ERR_INVALID;
  if (precision != PS_PREC_FP32 && precision != PS_PREC_MIXED) return PS_ERR_INVALID;
  if (seg->n_seg < 0 || paths->n_path <= 0 || seg->n_seg > (int64_t)1 << 29) return PS_ERR_INVALID;
  const int64_t L_all = 2 * seg->n_seg + paths->n_path;
  if (link_begin < 0 || link_end <= link_begin || link_end > L_all) return PS_ERR_INVALID;
  if (seg->n_seg > 0 && (!seg->d_type || !seg->d_pts)) return PS_ERR_INVALID;
  if (!paths->d_seg_off || !paths->d_width || !paths->d_join || !paths->d_cap ||
      !paths->d_miter || !paths->d_closed)
    return PS_ERR_INVALID;
  if (!out->d_link_rib_off || !out->d_path_rib_off || !out->d_n_rib) return PS_ERR_INVALID;
  if (!(flags & PS_TESS_COUNT_ONLY) && (!out->d_rib || !out->d_tag || out->capacity < 0))
    return PS_ERR_INVALID;
  if ((flags & PS_TESS_ARCLENGTH) && !(flags & PS_TESS_COUNT_ONLY) && !out->d_s)
    return PS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = stream;
  // paths whose first link lies outside the range keep -1: no rib of the range
  // starts them
  int rc = ps_cuda_check(cudaMemsetAsync(out->d_path_rib_off, 0xff,
                                         sizeof(int32_t) * (paths->n_path + 1), st));
  if (rc != PS_OK) return rc;
  return launch_tessellate(ctx, seg, paths, dtheta, precision, flags, out, st, link_begin,
                           link_end - link_begin);
}

// s += carry on the leading ribs of the stream that belong to `path` (the path
// that runs into a link range from the ranks before it), and on its length.
__global__ void k_add_s_carry(float* __restrict__ s, const uint32_t* __restrict__ tag,
                              const int64_t* __restrict__ n_rib, int64_t capacity, uint32_t path,
                              float carry_hi, float carry_lo, float* __restrict__ path_len,
                              int with_len) {
  int64_t R = *n_rib;
  if (R > capacity) R = capacity;
  const DF carry{carry_hi, carry_lo};
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R;
       r += (int64_t)gridDim.x * blockDim.x) {
    if ((__ldg(tag + r) >> 2) != path) break;  // ribs of one path are consecutive
    s[r] = df_f(df_add_f(carry, s[r]));
  }
  if (with_len && path_len && blockIdx.x == 0 && threadIdx.x == 0)
    path_len[path] = df_f(df_add_f(carry, path_len[path]));
}

extern "C" int ps_add_s_carry(ps_context* ctx, float* d_s, const uint32_t* d_tag,
                              const int64_t* d_n_rib, int64_t capacity, int32_t path,
                              double carry, float* d_path_len, int with_len, void* stream) {
  if (!ctx || !d_s || !d_tag || !d_n_rib || capacity < 0 || path < 0) return PS_ERR_INVALID;
  if (with_len && !d_path_len) return PS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = stream;
  const float hi = (float)carry, lo = (float)(carry - (double)hi);
  const int grid = ps_persistent_grid(ctx, (const void*)k_add_s_carry, 256, 0);
  k_add_s_carry<<<grid, 256, 0, st>>>(d_s, d_tag, d_n_rib, capacity, (uint32_t)path, hi, lo,
                                      d_path_len, with_len);
  return ps_cuda_check(cudaGetLastError());
}

extern "C" int ps_arclength_scan(ps_context* ctx, const float* d_rib, const uint32_t* d_tag,
                                 const int64_t* d_n_rib, int64_t capacity, float* d_s,
                                 float* d_path_len, int32_t n_path, void* stream) {
  if (!ctx || !d_rib || !d_tag || !d_n_rib || !d_s || capacity < 0 || n_path < 0)
    return PS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = stream;
  int64_t scan_tiles = (capacity + SCAN_TILE - 1) / SCAN_TILE;
  int rc = ps_ensure_tiles(ctx, scan_tiles + 2);
  if (rc != PS_OK) return rc;
  cudaMemsetAsync(ctx->d_tile_flag, 0, sizeof(uint32_t) * (scan_tiles + 1), st);
  cudaMemsetAsync(ctx->d_counters, 0, sizeof(int32_t) * 16, st);
  if (d_path_len && n_path > 0) cudaMemsetAsync(d_path_len, 0, sizeof(float) * n_path, st);
  int g = ps_persistent_grid(ctx, (const void*)k_midpoint_chords, 256, 0);
  { ProfScope ps_(ctx, PK_MIDCHORD, st);
  k_midpoint_chords<<<g, 256, 0, st>>>(reinterpret_cast<const float4*>(d_rib), d_tag, d_n_rib,
                                       capacity, d_s); }
  ProfScope ps_(ctx, PK_ARCLEN, st);
  launch_arclen_scan(ctx, 0, st, d_s, d_tag, d_n_rib, capacity, d_s, d_path_len, ctx->d_tile_flag,
                     ctx->d_tile_aggd, ctx->d_tile_incld, ctx->d_counters, ctx->d_status);
  return ps_cuda_check(cudaGetLastError());
}

// ===========================================================================
// Allocation-free tessellation.
//
// ps_tessellate_strokes keeps its workspace (per-link records, scan tile states)
// in a context that grows it with cudaMalloc.  Some callers cannot allocate
// device memory at the point where they stroke: code that runs where another
// allocator owns the device's memory budget, or code that must not risk a
// failed or blocking allocation in the middle of its work.  For them this
// variant takes its workspace from a fixed array that is part of the loaded
// library image, so it makes no allocation of any kind.
namespace {
constexpr int64_t NOALLOC_MAX_LINKS = 16384;
constexpr int64_t NOALLOC_MAX_RIBS = 4194304;
constexpr int64_t NOALLOC_SETUP_TILES = NOALLOC_MAX_LINKS / SETUP_TILE + 1;
constexpr int64_t NOALLOC_SCAN_TILES = NOALLOC_MAX_RIBS / SCAN_TILE + 1;
constexpr int64_t NOALLOC_TILES = NOALLOC_SETUP_TILES + 1 + NOALLOC_SCAN_TILES + 1;
// byte offsets of the workspace parts (each 256-byte aligned)
constexpr size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t NA_RECS = 0;
constexpr size_t NA_PATH = al256(NA_RECS + sizeof(LinkRec) * NOALLOC_MAX_LINKS);
constexpr size_t NA_FLAG = al256(NA_PATH + sizeof(int32_t) * NOALLOC_MAX_LINKS);
constexpr size_t NA_AGG = al256(NA_FLAG + sizeof(uint32_t) * NOALLOC_TILES);
constexpr size_t NA_INCL = al256(NA_AGG + sizeof(long long) * NOALLOC_TILES);
constexpr size_t NA_AGGD = al256(NA_INCL + sizeof(long long) * NOALLOC_TILES);
constexpr size_t NA_INCLD = al256(NA_AGGD + sizeof(double) * NOALLOC_TILES);
constexpr size_t NA_CNT = al256(NA_INCLD + sizeof(double) * NOALLOC_TILES);
constexpr size_t NA_BYTES = al256(NA_CNT + sizeof(int32_t) * 16);
}  // namespace

// The workspace: about 4.0 MB held by every device that loads the library until
// the process exits.  Host code must not take this name as a device address; it
// asks the runtime for the address on each device (below).
static __device__ __align__(256) unsigned char ps_noalloc_scratch[NA_BYTES];

namespace {
constexpr int NOALLOC_MAX_DEVICES = 64;
unsigned char* g_noalloc_ptr[NOALLOC_MAX_DEVICES];
int g_noalloc_sms[NOALLOC_MAX_DEVICES];
}  // namespace

extern "C" int ps_tessellate_strokes_noalloc(const ps_segments* seg, const ps_paths* paths,
                                             float dtheta, int precision, uint32_t flags,
                                             ps_tess_out* out, int32_t* d_status, void* stream) {
  if (!seg || !paths || !out || !d_status) return PS_ERR_INVALID;
  if (!(dtheta >= 1e-4f && dtheta <= 3.14159265f)) return PS_ERR_INVALID;
  if (precision != PS_PREC_FP32 && precision != PS_PREC_MIXED) return PS_ERR_INVALID;
  if (seg->n_seg < 0 || paths->n_path < 0) return PS_ERR_INVALID;
  if (paths->n_path == 0)
    return seg->n_seg != 0 ? PS_ERR_INVALID : empty_batch(out, (cudaStream_t)stream);
  if (seg->n_seg > 0 && (!seg->d_type || !seg->d_pts)) return PS_ERR_INVALID;
  if (!paths->d_seg_off || !paths->d_width || !paths->d_join || !paths->d_cap ||
      !paths->d_miter || !paths->d_closed)
    return PS_ERR_INVALID;
  if (!out->d_link_rib_off || !out->d_path_rib_off || !out->d_n_rib) return PS_ERR_INVALID;
  bool count_only = (flags & PS_TESS_COUNT_ONLY) != 0;
  if (!count_only && (!out->d_rib || !out->d_tag || out->capacity < 0)) return PS_ERR_INVALID;
  bool arc = !count_only && (flags & PS_TESS_ARCLENGTH);
  if (arc && !out->d_s) return PS_ERR_INVALID;
  int64_t L = 2 * seg->n_seg + paths->n_path;
  // the fixed workspace bounds the problem size
  if (L > NOALLOC_MAX_LINKS) return PS_ERR_CAPACITY;
  if (arc && out->capacity > NOALLOC_MAX_RIBS) return PS_ERR_CAPACITY;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return PS_ERR_CUDA;
  if (!g_noalloc_ptr[dev]) {
    // one-time set-up on this device (with it current): the device address of
    // the workspace, and the SM count for the persistent grids
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, ps_noalloc_scratch) != cudaSuccess || !p) return PS_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      return PS_ERR_CUDA;
    g_noalloc_sms[dev] = sms;
    g_noalloc_ptr[dev] = (unsigned char*)p;
  }
  unsigned char* base = g_noalloc_ptr[dev];
  LinkRec* recs = reinterpret_cast<LinkRec*>(base + NA_RECS);
  int32_t* link_path = reinterpret_cast<int32_t*>(base + NA_PATH);
  uint32_t* tflag = reinterpret_cast<uint32_t*>(base + NA_FLAG);
  long long* tagg = reinterpret_cast<long long*>(base + NA_AGG);
  long long* tincl = reinterpret_cast<long long*>(base + NA_INCL);
  double* taggd = reinterpret_cast<double*>(base + NA_AGGD);
  double* tincld = reinterpret_cast<double*>(base + NA_INCLD);
  int32_t* counters = reinterpret_cast<int32_t*>(base + NA_CNT);

  cudaStream_t st = (cudaStream_t)stream;
  int P = paths->n_path;
  int64_t n_tiles = (L + SETUP_TILE - 1) / SETUP_TILE;
  // the array keeps the previous call's contents: reset what must start at zero
  if (cudaMemsetAsync(tflag, 0, sizeof(uint32_t) * NOALLOC_TILES, st) != cudaSuccess ||
      cudaMemsetAsync(counters, 0, sizeof(int32_t) * 16, st) != cudaSuccess)
    return PS_ERR_CUDA;
  int64_t count_cap = count_only ? INT64_MAX : out->capacity;
  k_link_path<<<(unsigned)((L + 255) / 256), 256, 0, st>>>(paths->d_seg_off, P, L, link_path, (int64_t)0);
  if (precision == PS_PREC_MIXED)
    k_link_setup<true, SETUP_IPT><<<(unsigned)n_tiles, SETUP_NT, 0, st>>>(
        seg->d_type, seg->d_pts, seg->d_w, paths->d_seg_off, paths->d_width, paths->d_join,
        paths->d_cap, paths->d_miter, paths->d_closed, P, L, dtheta, 0.f, recs, out->d_link_rib_off,
        out->d_path_rib_off, out->d_n_rib, count_cap, tflag, tagg, tincl, counters, d_status,
        n_tiles, (int64_t)0);
  else
    k_link_setup<false, SETUP_IPT><<<(unsigned)n_tiles, SETUP_NT, 0, st>>>(
        seg->d_type, seg->d_pts, seg->d_w, paths->d_seg_off, paths->d_width, paths->d_join,
        paths->d_cap, paths->d_miter, paths->d_closed, P, L, dtheta, 0.f, recs, out->d_link_rib_off,
        out->d_path_rib_off, out->d_n_rib, count_cap, tflag, tagg, tincl, counters, d_status,
        n_tiles, (int64_t)0);
  if (cudaGetLastError() != cudaSuccess) return PS_ERR_CUDA;
  if (count_only) return PS_OK;
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, precision == PS_PREC_MIXED ? (const void*)k_emit<true> : (const void*)k_emit<false>,
      EMIT_NT, 0);
  int grid = g_noalloc_sms[dev] * (per_sm > 0 ? per_sm : 1);
  if (precision == PS_PREC_MIXED)
    k_emit<true><<<grid, EMIT_NT, 0, st>>>(recs, out->d_link_rib_off, link_path, L, out->d_n_rib,
                                           out->capacity, reinterpret_cast<float4*>(out->d_rib),
                                           out->d_tag, arc ? out->d_s : nullptr, out->d_t, EMIT_K);
  else
    k_emit<false><<<grid, EMIT_NT, 0, st>>>(recs, out->d_link_rib_off, link_path, L, out->d_n_rib,
                                            out->capacity, reinterpret_cast<float4*>(out->d_rib),
                                            out->d_tag, arc ? out->d_s : nullptr, out->d_t, EMIT_K);
  if (cudaGetLastError() != cudaSuccess) return PS_ERR_CUDA;
  if (arc) {
    if (out->d_path_len && cudaMemsetAsync(out->d_path_len, 0, sizeof(float) * P, st) != cudaSuccess)
      return PS_ERR_CUDA;
    int per_sm2 = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, (const void*)k_arclen_scan<true>,
                                                  SCAN_NT, 0);
    int g2 = g_noalloc_sms[dev] * (per_sm2 > 0 ? per_sm2 : 1);
    int64_t o = NOALLOC_SETUP_TILES + 1;
    launch_arclen_scan(nullptr, g2, st, out->d_s, out->d_tag, out->d_n_rib, out->capacity,
                       out->d_s, out->d_path_len, tflag + o, taggd + o, tincld + o, counters,
                       d_status);
    if (cudaGetLastError() != cudaSuccess) return PS_ERR_CUDA;
  }
  return PS_OK;
}

// ---------------------------------------------------------------------------
int ps_run_link_setup(ps_context* ctx, const ps_segments* seg, const ps_paths* paths, float dtheta,
                      int precision, int32_t* d_link_off, int32_t* d_path_off, int64_t* d_n_rib,
                      cudaStream_t st) {
  int64_t S = seg->n_seg;
  int P = paths->n_path;
  int64_t L = 2 * S + P;
  int64_t n_tiles = (L + SETUP_TILE - 1) / SETUP_TILE;
  int rc;
  if ((rc = ps_ensure_tiles(ctx, n_tiles + 2)) != PS_OK) return rc;
  if ((rc = ps_ensure_recs(ctx, L)) != PS_OK) return rc;
  int32_t* link_path = reinterpret_cast<int32_t*>(ctx->d_recs + ctx->rec_cap);
  cudaMemsetAsync(ctx->d_tile_flag, 0, sizeof(uint32_t) * n_tiles, st);
  cudaMemsetAsync(ctx->d_counters, 0, sizeof(int32_t) * 16, st);
  k_link_path<<<(unsigned)((L + 255) / 256), 256, 0, st>>>(paths->d_seg_off, P, L, link_path, (int64_t)0);
  const bool px = ctx->pixel_tol > 0.f;
  if (precision == PS_PREC_MIXED && px)
    k_link_setup<true, SETUP_IPT, true><<<(unsigned)n_tiles, SETUP_NT, 0, st>>>(
        seg->d_type, seg->d_pts, seg->d_w, paths->d_seg_off, paths->d_width, paths->d_join,
        paths->d_cap, paths->d_miter, paths->d_closed, P, L, dtheta, ctx->pixel_tol, ctx->d_recs,
        d_link_off, d_path_off, d_n_rib, INT64_MAX, ctx->d_tile_flag, ctx->d_tile_agg,
        ctx->d_tile_incl, ctx->d_counters, ctx->d_status, n_tiles, (int64_t)0);
  else if (px)
    k_link_setup<false, SETUP_IPT, true><<<(unsigned)n_tiles, SETUP_NT, 0, st>>>(
        seg->d_type, seg->d_pts, seg->d_w, paths->d_seg_off, paths->d_width, paths->d_join,
        paths->d_cap, paths->d_miter, paths->d_closed, P, L, dtheta, ctx->pixel_tol, ctx->d_recs,
        d_link_off, d_path_off, d_n_rib, INT64_MAX, ctx->d_tile_flag, ctx->d_tile_agg,
        ctx->d_tile_incl, ctx->d_counters, ctx->d_status, n_tiles, (int64_t)0);
  else if (precision == PS_PREC_MIXED)
    k_link_setup<true, SETUP_IPT><<<(unsigned)n_tiles, SETUP_NT, 0, st>>>(
        seg->d_type, seg->d_pts, seg->d_w, paths->d_seg_off, paths->d_width, paths->d_join,
        paths->d_cap, paths->d_miter, paths->d_closed, P, L, dtheta, ctx->pixel_tol, ctx->d_recs,
        d_link_off,
        d_path_off, d_n_rib, INT64_MAX, ctx->d_tile_flag, ctx->d_tile_agg, ctx->d_tile_incl,
        ctx->d_counters, ctx->d_status, n_tiles, (int64_t)0);
  else
    k_link_setup<false, SETUP_IPT><<<(unsigned)n_tiles, SETUP_NT, 0, st>>>(
        seg->d_type, seg->d_pts, seg->d_w, paths->d_seg_off, paths->d_width, paths->d_join,
        paths->d_cap, paths->d_miter, paths->d_closed, P, L, dtheta, ctx->pixel_tol, ctx->d_recs,
        d_link_off,
        d_path_off, d_n_rib, INT64_MAX, ctx->d_tile_flag, ctx->d_tile_agg, ctx->d_tile_incl,
        ctx->d_counters, ctx->d_status, n_tiles, (int64_t)0);
  return ps_cuda_check(cudaGetLastError());
}

int ps_run_segmented_prefix(ps_context* ctx, float* d_vals, const uint32_t* d_tag,
                            const int64_t* d_n_rib, int64_t capacity, float* d_path_tot,
                            int32_t n_path, cudaStream_t st) {
  int64_t scan_tiles = (capacity + SCAN_TILE - 1) / SCAN_TILE;
  int rc = ps_ensure_tiles(ctx, scan_tiles + 2);
  if (rc != PS_OK) return rc;
  cudaMemsetAsync(ctx->d_tile_flag, 0, sizeof(uint32_t) * (scan_tiles + 1), st);
  cudaMemsetAsync(ctx->d_counters, 0, sizeof(int32_t) * 16, st);
  if (d_path_tot && n_path > 0) cudaMemsetAsync(d_path_tot, 0, sizeof(float) * n_path, st);
  launch_arclen_scan(ctx, 0, st, d_vals, d_tag, d_n_rib, capacity, d_vals, d_path_tot,
                     ctx->d_tile_flag, ctx->d_tile_aggd, ctx->d_tile_incld, ctx->d_counters,
                     ctx->d_status);
  return ps_cuda_check(cudaGetLastError());
}
