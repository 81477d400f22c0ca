/*
 * Polar stroking oracle — a plain, slow FP64 CPU restatement of the method of
 * M. J. Kilgard, "Polar Stroking: New Theory and Methods for Stroking Paths",
 * ACM TOG 39(4), 2020.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library loads this file;
 * only the test-suite, the package smoke check and the benchmark's CPU-baseline
 * leg do.  It shares no code, header, table or constant with the CUDA path:
 * the enum values below are the public interface's numbers, written out here
 * independently.
 *
 * Parts
 *   O1  orc_tessellate            tessellation + cumulative arc length
 *                                 (Sec. 3.1-3.4, Sec. 4.2-4.4, Sec. 5, Eq. 18)
 *   O1b orc_dash                  dashing by cumulative arc length (Sec. 5.2)
 *   O2  orc_raster                16-sample fixed-point coverage of a rib stream
 *   O3  orc_centreline_distance   brute-force distance to the generator curves
 *
 * Every step follows the paper's order and notation.  Where the paper is
 * silent or self-contradictory the reading taken is stated at the step,
 * numbered R1..R21.
 *
 * Compile with -ffp-contract=off so that no multiply-add is fused behind the
 * source's back: the results are then the same on x86-64 and aarch64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- public interface numbers ------------------------------------------ */
enum { ORC_LINE = 0, ORC_QUAD = 1, ORC_CUBIC = 2, ORC_CONIC = 3 };
enum { ORC_JOIN_NONE = 0, ORC_JOIN_BEVEL = 1, ORC_JOIN_MITER = 2,
       ORC_JOIN_MITER_TRUNCATE = 3, ORC_JOIN_ROUND = 4, ORC_JOIN_TRIANGLE = 5 };
enum { ORC_CAP_BUTT = 0, ORC_CAP_SQUARE = 1, ORC_CAP_ROUND = 2, ORC_CAP_TRIANGLE = 3 };
/* per-rib tag: bit0 first rib of its link, bit1 rib of a segment link,
 * bits 2.. path index */
#define TAG_LINK_START 1u
#define TAG_SEGMENT 2u
/* per-link info bits */
#define INFO_FRAGILE64 1u
#define INFO_FRAGILE32 2u
#define INFO_KIND_SHIFT 2 /* 0 empty, 1 segment, 2 join, 3 cap */

#define ORC_OK 0
#define ORC_ERR_INVALID (-1)
#define ORC_ERR_CAPACITY (-2)

#define PI 3.14159265358979323846
#define TWO_PI (2.0 * PI)
#define MAXI 12 /* intervals per link: <= 3 curve intervals, each split once,
                   plus collinear pivots (<= 2) and their flat pieces */
/* Reading R13: q is a nominal step.  A turning whose ratio to q exceeds an
 * integer n by less than STEP_SNAP steps takes n steps, not n + 1, so that
 * exactly-divisible turnings (a 180-degree cap at q = 2 degrees, say) do not
 * depend on the last bit of q's rounding.  Every step then turns at most
 * q (1 + STEP_SNAP). */
#define STEP_SNAP 1e-4

/* steps for a turning of magnitude ad > 0 (Eq. 12 with R13) */
static int step_count(double ad, double q) {
  int D = (int)ceil(ad / q - STEP_SNAP);
  return D < 1 ? 1 : D;
}
/* distance of a count's argument to its rounding boundary, in steps */
static double step_margin(double ad, double q) {
  double x = ad / q - STEP_SNAP;
  double f = x - floor(x);
  return f < 1.0 - f ? f : 1.0 - f;
}

typedef struct { double x, y; } V2;
static V2 mk(double x, double y) { V2 r; r.x = x; r.y = y; return r; }
static V2 add(V2 a, V2 b) { return mk(a.x + b.x, a.y + b.y); }
static V2 sub(V2 a, V2 b) { return mk(a.x - b.x, a.y - b.y); }
static V2 mul(V2 a, double s) { return mk(a.x * s, a.y * s); }
static double dot(V2 a, V2 b) { return a.x * b.x + a.y * b.y; }
static double cross(V2 a, V2 b) { return a.x * b.y - a.y * b.x; }
static double len(V2 a) { return sqrt(a.x * a.x + a.y * a.y); }
static int is_zero(V2 a) { return a.x == 0.0 && a.y == 0.0; }
static double ang(V2 a) { return atan2(a.y, a.x); }
/* unit normal of tangent angle psi: <-sin psi, cos psi> (Sec. 3.3.1, Eq. 15) */
static V2 normal_of(double psi) { return mk(-sin(psi), cos(psi)); }
static V2 tangent_of(double psi) { return mk(cos(psi), sin(psi)); }
/* x mod 2pi in [0, 2pi) */
static double mod2pi(double x) {
  double r = fmod(x, TWO_PI);
  if (r < 0) r += TWO_PI;
  if (r >= TWO_PI) r -= TWO_PI;
  return r;
}
/* relative angle difference theta1 (-) theta2, Sec. 3.2.2 */
static double ominus(double a, double b) {
  double d = a - b;
  if (d > PI) return d - TWO_PI;
  if (d < -PI) return d + TWO_PI;
  return d;
}

/* ---- segment forms (Table 1) -------------------------------------------- */
typedef struct {
  int type;
  V2 A, B, C, D; /* quadratic and conic use A, B, D (their last point is P_D) */
  double w;      /* conic weight w_B */
} Seg;

/* generator curve g_f(t), Table 1 */
static V2 seg_eval(const Seg* g, double t) {
  double u = 1.0 - t;
  switch (g->type) {
    case ORC_CUBIC:
      return add(add(mul(g->A, u * u * u), mul(g->B, 3.0 * u * u * t)),
                 add(mul(g->C, 3.0 * u * t * t), mul(g->D, t * t * t)));
    case ORC_QUAD:
      return add(add(mul(g->A, u * u), mul(g->B, 2.0 * u * t)), mul(g->D, t * t));
    case ORC_CONIC: {
      double den = u * u + 2.0 * u * t * g->w + t * t;
      V2 num = add(add(mul(g->A, u * u), mul(g->B, 2.0 * u * t * g->w)), mul(g->D, t * t));
      return mul(num, 1.0 / den);
    }
    default:
      return add(mul(g->A, u), mul(g->D, t));
  }
}

/* Hodograph direction H(t): g'(t) = c(t) H(t) with c(t) > 0.
 *   cubic:     g' = 3 [u^2 (B-A) + 2ut (C-B) + t^2 (D-C)]        (Bernstein derivative)
 *   quadratic: g' = 2 [u (B-A) + t (D-B)]
 *   conic:     g' = 2 [w u^2 (B-A) + u t (D-A) + w t^2 (D-B)] / den(t)^2
 *              (quotient rule on Table 1's rational form; the cubic terms
 *               of the numerator cancel)
 *   line:      g' = D - A                                                    */
static V2 hodo(const Seg* g, double t) {
  double u = 1.0 - t;
  switch (g->type) {
    case ORC_CUBIC:
      return add(add(mul(sub(g->B, g->A), u * u), mul(sub(g->C, g->B), 2.0 * u * t)),
                 mul(sub(g->D, g->C), t * t));
    case ORC_QUAD:
      return add(mul(sub(g->B, g->A), u), mul(sub(g->D, g->B), t));
    case ORC_CONIC:
      return add(add(mul(sub(g->B, g->A), g->w * u * u), mul(sub(g->D, g->A), u * t)),
                 mul(sub(g->D, g->B), g->w * t * t));
    default:
      return sub(g->D, g->A);
  }
}
/* dH/dt */
static V2 hodo_d(const Seg* g, double t) {
  double u = 1.0 - t;
  switch (g->type) {
    case ORC_CUBIC: {
      V2 d1 = sub(g->B, g->A), d2 = sub(g->C, g->B), d3 = sub(g->D, g->C);
      return mul(add(mul(sub(d2, d1), u), mul(sub(d3, d2), t)), 2.0);
    }
    case ORC_QUAD:
      return sub(sub(g->D, g->B), sub(g->B, g->A));
    case ORC_CONIC: {
      V2 h0 = mul(sub(g->B, g->A), g->w), h1 = sub(g->D, g->A), h2 = mul(sub(g->D, g->B), g->w);
      return add(add(mul(h0, -2.0 * u), mul(h1, u - t)), mul(h2, 2.0 * t));
    }
    default:
      return mk(0, 0);
  }
}
/* positive factor c(t) with g' = c H */
static double hodo_scale(const Seg* g, double t) {
  double u = 1.0 - t, den;
  switch (g->type) {
    case ORC_CUBIC: return 3.0;
    case ORC_QUAD: return 2.0;
    case ORC_CONIC: den = u * u + 2.0 * u * t * g->w + t * t; return 2.0 / (den * den);
    default: return 1.0;
  }
}

/* Zero-length test: all of the form's control points coincide (Sec. 3.3.4). */
static int seg_zero_length(const Seg* g) {
  V2 a = g->A;
  switch (g->type) {
    case ORC_CUBIC:
      return is_zero(sub(g->B, a)) && is_zero(sub(g->C, a)) && is_zero(sub(g->D, a));
    case ORC_QUAD:
      return is_zero(sub(g->B, a)) && is_zero(sub(g->D, a));
    case ORC_CONIC:
      if (g->w == 0.0) return is_zero(sub(g->D, a));
      return is_zero(sub(g->B, a)) && is_zero(sub(g->D, a));
    default:
      return is_zero(sub(g->D, a));
  }
}

/* Normalized end gradients (Table 1).  Reading R1: the table's "P_C" for the
 * quadratic and conic rows is their last point P_D, and the line row's
 * "P_B - P_A" is P_D - P_A, matching the generator functions in the same rows.
 * Only the direction matters (angles are taken with atan2). */
static V2 end_grad0(const Seg* g) {
  switch (g->type) {
    case ORC_CUBIC:
      if (!is_zero(sub(g->B, g->A))) return sub(g->B, g->A);
      if (!is_zero(sub(g->C, g->A))) return sub(g->C, g->A);
      return sub(g->D, g->A);
    case ORC_QUAD:
      if (!is_zero(sub(g->B, g->A))) return sub(g->B, g->A);
      return sub(g->D, g->A);
    case ORC_CONIC:
      if (!is_zero(sub(g->B, g->A)) && g->w != 0.0)
        return mul(sub(g->B, g->A), g->w > 0 ? 1.0 : -1.0);
      return sub(g->D, g->A);
    default:
      return sub(g->D, g->A);
  }
}
static V2 end_grad1(const Seg* g) {
  switch (g->type) {
    case ORC_CUBIC:
      if (!is_zero(sub(g->D, g->C))) return sub(g->D, g->C);
      if (!is_zero(sub(g->D, g->B))) return sub(g->D, g->B);
      return sub(g->D, g->A);
    case ORC_QUAD:
      if (!is_zero(sub(g->D, g->B))) return sub(g->D, g->B);
      return sub(g->D, g->A);
    case ORC_CONIC:
      if (!is_zero(sub(g->D, g->B)) && g->w != 0.0)
        return mul(sub(g->D, g->B), g->w > 0 ? 1.0 : -1.0);
      return sub(g->D, g->A);
    default:
      return sub(g->D, g->A);
  }
}

/* ---- the curvature-sign polynomial C(t) = H(t) x H'(t) ------------------- */
/* sgn C(t) = sgn kappa(t) (Sec. 3.1; kappa's numerator is g' x g'' . z, reading
 * R2 for the printed ". g").  C is at most quadratic for every form:
 *   cubic:     C = 2 [u^2 X12 + u t X13 + t^2 X23],  Xij = d_i x d_j
 *              (d1 = B-A, d2 = C-B, d3 = D-C; the Loop-Blinn inflection
 *               quadratic of Sec. 3.3.2 written in Bernstein form)
 *   quadratic: C = (B-A) x (D-B)              (constant: no inflection)
 *   conic:     C = w K den(t), K = (B-A) x (D-B)
 *   line:      C = 0
 * Returned in power form C = c0 + c1 t + c2 t^2 (common positive factors
 * dropped), with the discriminant c1^2 - 4 c0 c2 computed with error-free
 * products so that an exact double root (an exact cusp) gives exactly 0. */
typedef struct { double c0, c1, c2, disc, disc_scale; int flat; } CrossPoly;

static double two_prod_err(double a, double b, double p) { return fma(a, b, -p); }

static CrossPoly cross_poly(const Seg* g) {
  CrossPoly P;
  memset(&P, 0, sizeof P);
  switch (g->type) {
    case ORC_CUBIC: {
      V2 d1 = sub(g->B, g->A), d2 = sub(g->C, g->B), d3 = sub(g->D, g->C);
      double X12 = cross(d1, d2), X13 = cross(d1, d3), X23 = cross(d2, d3);
      P.c0 = X12;
      P.c1 = X13 - 2.0 * X12;
      P.c2 = X12 - X13 + X23;
      /* c1^2 - 4 c0 c2 simplifies to X13^2 - 4 X12 X23 */
      double h1 = X13 * X13, l1 = two_prod_err(X13, X13, h1);
      double h2 = (4.0 * X12) * X23, l2 = two_prod_err(4.0 * X12, X23, h2);
      P.disc = (h1 - h2) + (l1 - l2);
      P.disc_scale = fabs(h1) + fabs(h2);
      P.flat = (X12 == 0.0 && X13 == 0.0 && X23 == 0.0);
      break;
    }
    case ORC_QUAD: {
      double K = cross(sub(g->B, g->A), sub(g->D, g->B));
      P.c0 = K;
      P.flat = (K == 0.0);
      break;
    }
    case ORC_CONIC: {
      double K = cross(sub(g->B, g->A), sub(g->D, g->B));
      double wK = g->w * K;
      /* den(t) = 1 + (2w - 2) t + (2 - 2w) t^2 */
      P.c0 = wK;
      P.c1 = wK * (2.0 * g->w - 2.0);
      P.c2 = wK * (2.0 - 2.0 * g->w);
      P.disc = P.c1 * P.c1 - 4.0 * P.c0 * P.c2;
      P.disc_scale = P.c1 * P.c1 + fabs(4.0 * P.c0 * P.c2);
      P.flat = (wK == 0.0);
      break;
    }
    default:
      P.flat = 1;
  }
  return P;
}
static double cross_eval(const CrossPoly* P, double t) { return P->c0 + t * (P->c1 + t * P->c2); }

/* Real roots of a + b t + c t^2 = 0 (note: constant term first) with the
 * cancellation-free formula q = -(b + sgn(b) sqrt(disc))/2, roots q/c, a/q.
 * Returns the count; roots sorted ascending.  disc < 0 is treated as a double
 * root when it is within rounding of zero (|disc| <= tol * scale). */
static int quad_roots(double a, double b, double c, double disc, double scale, double tol,
                      double* r) {
  if (c == 0.0) {
    if (b == 0.0) return 0;
    r[0] = -a / b;
    return 1;
  }
  if (disc < 0.0) {
    if (-disc > tol * scale) return 0;
    disc = 0.0;
  }
  double sq = sqrt(disc);
  double q = -0.5 * (b + (b >= 0 ? sq : -sq));
  int n = 0;
  if (q != 0.0) {
    r[n++] = q / c;
    r[n++] = a / q;
  } else {
    r[n++] = 0.0; /* b == 0 and disc == 0: double root at 0 */
    r[n++] = 0.0;
  }
  if (r[0] > r[1]) { double s = r[0]; r[0] = r[1]; r[1] = s; }
  return n;
}

/* ---- t(psi): Eq. 11 and the endpoint fallback of Sec. 3.4 --------------- */
/* Solve H(t) . N(psi) = 0 for t in [pa, pb].  H . N is quadratic in t for
 * cubics and conics (the conic's positive denominator is dropped, Sec. 3.4),
 * linear for quadratics.  Among roots inside the range (slack 1e-12) the one
 * whose tangent points along psi is chosen: largest H(t) . T(psi); this
 * rejects the psi + pi alias and prefers an exact cusp (H = 0) to the alias
 * (reading R3).  No root in range: the paper's endpoint rule. */
static double solve_t(const Seg* g, double psi, double pa, double pb) {
  V2 N = normal_of(psi), T = tangent_of(psi);
  double a, b, c; /* f(t) = a + b t + c t^2 */
  switch (g->type) {
    case ORC_CUBIC: {
      double al = dot(sub(g->B, g->A), N), be = dot(sub(g->C, g->B), N), ga = dot(sub(g->D, g->C), N);
      /* al u^2 + 2 be u t + ga t^2 */
      a = al; b = 2.0 * (be - al); c = al - 2.0 * be + ga;
      break;
    }
    case ORC_QUAD: {
      double al = dot(sub(g->B, g->A), N), be = dot(sub(g->D, g->B), N);
      a = al; b = be - al; c = 0.0;
      break;
    }
    case ORC_CONIC: {
      double al = g->w * dot(sub(g->B, g->A), N), be = dot(sub(g->D, g->A), N),
             ga = g->w * dot(sub(g->D, g->B), N);
      /* al u^2 + be u t + ga t^2 */
      a = al; b = be - 2.0 * al; c = al - be + ga;
      break;
    }
    default:
      return pa;
  }
  double disc = b * b - 4.0 * a * c, scale = b * b + fabs(4.0 * a * c);
  double r[2];
  int n = quad_roots(a, b, c, disc, scale, 1e-12, r);
  double best_t = 0.0, best_v = -INFINITY;
  int found = 0;
  for (int i = 0; i < n; ++i) {
    double t = r[i];
    if (!(t >= pa - 1e-12 && t <= pb + 1e-12)) continue;
    if (t < pa) t = pa;
    if (t > pb) t = pb;
    double v = dot(hodo(g, t), T);
    if (!found || v > best_v) { best_v = v; best_t = t; found = 1; }
  }
  if (found) return best_t;
  double fa = fabs(dot(hodo(g, pa), N)), fb = fabs(dot(hodo(g, pb), N));
  return fa < fb ? pa : pb;
}

/* ---- intervals of a link (Sec. 3.3.4-3.3.6, Eq. 4-6, 12-13) ------------- */
typedef struct {
  int M;                  /* number of intervals */
  double p[MAXI + 1];     /* parameter at interval boundaries (Eq. 4) */
  double Psi[MAXI + 1];   /* tangent angle at boundaries (Eq. 5) */
  double delta[MAXI];     /* signed turning of each interval (Eq. 6, reading R4) */
  int Delta[MAXI];        /* steps per interval (Eq. 12) */
  int pivot[MAXI];        /* interval pivots at a fixed t (collinear reversal) */
  int split[MAXI + 1];    /* boundary k is a split point (Sec. 3.3.5), t from Eq. 11 */
  int N;                  /* total steps Delta_Sigma(M) (Eq. 13) */
  int fragile64, fragile32;
} Intervals;

/* Fragility: a count that another correct evaluation order could legitimately
 * change.  ceil(|delta|/q) within eps of an integer, a discriminant within
 * rounding of zero, a root within eps of an interval end, a turning within
 * eps of zero. */
static void mark_count_fragility(Intervals* I, double q) {
  for (int k = 0; k < I->M; ++k) {
    if (I->pivot[k]) continue;
    double x = fabs(I->delta[k]) / q;
    double dist = step_margin(fabs(I->delta[k]), q);
    if (x > 0 && dist < 1e-9 * (1.0 + x)) I->fragile64 = 1;
    if (x > 0 && dist < 2e-5 * (1.0 + x)) I->fragile32 = 1;
    if (I->delta[k] != 0.0 && fabs(I->delta[k]) < 1e-4) I->fragile32 = 1;
    if (fabs(fabs(I->delta[k]) - PI) < 1e-5) I->fragile32 = 1; /* split decision */
    if (fabs(fabs(I->delta[k]) - PI) < 1e-12) I->fragile64 = 1;
  }
}

static void finish_counts(Intervals* I, double q) {
  I->N = 0;
  for (int k = 0; k < I->M; ++k) {
    double ad = fabs(I->delta[k]);
    int D;
    if (ad == 0.0)
      D = (I->p[k + 1] > I->p[k]) ? 1 : 0; /* flat interval: one quad (R5) */
    else
      D = step_count(ad, q);
    I->Delta[k] = D;
    I->N += D;
  }
  mark_count_fragility(I, q);
}

/* Reversals of a segment whose control points are collinear (reading R5): along
 * the common direction v, H(t) . v is a Bernstein quadratic
 *   lam1 u^2 + 2 lam2 u t + lam3 t^2
 * (a linear one, lam1 u + lam3 t, for the quadratic Bezier).  The direction
 * reverses at its simple roots strictly inside (0,1): two when
 * lam2^2 - lam1 lam3 > 0, none when it is <= 0 (a double root is a kink, where
 * g' touches zero and resumes its direction).  Roots at t = 0 or 1 (lam1 = 0 or
 * lam3 = 0) are factored out exactly.  lam_i are dot products of FP32
 * differences, exact in FP64; the discriminant uses error-free products. */
static int collinear_reversals(const Seg* g, double* rts) {
  V2 v = end_grad0(g);
  double l1, l2, l3;
  switch (g->type) {
    case ORC_CUBIC:
      l1 = dot(sub(g->B, g->A), v); l2 = dot(sub(g->C, g->B), v); l3 = dot(sub(g->D, g->C), v);
      break;
    case ORC_QUAD: {
      double a1 = dot(sub(g->B, g->A), v), a3 = dot(sub(g->D, g->B), v);
      if ((a1 > 0 && a3 < 0) || (a1 < 0 && a3 > 0)) { rts[0] = a1 / (a1 - a3); return 1; }
      return 0;
    }
    case ORC_CONIC:
      if (g->w == 0.0) return 0;
      /* w(B-A) u^2 + (D-A) u t + w(D-B) t^2 : middle Bernstein coefficient (D-A)/2 */
      l1 = g->w * dot(sub(g->B, g->A), v); l2 = 0.5 * dot(sub(g->D, g->A), v);
      l3 = g->w * dot(sub(g->D, g->B), v);
      break;
    default:
      return 0;
  }
  int n = 0;
  if (l1 == 0.0 && l3 == 0.0) return 0;
  if (l1 == 0.0) { /* t (2 l2 u + l3 t): other root where 2 l2 u + l3 t = 0 */
    double den = 2.0 * l2 - l3;
    if (den != 0.0) { double r = 2.0 * l2 / den; if (r > 0.0 && r < 1.0) rts[n++] = r; }
    return n;
  }
  if (l3 == 0.0) { /* u (l1 u + 2 l2 t) */
    double den = l1 - 2.0 * l2;
    if (den != 0.0) { double r = l1 / den; if (r > 0.0 && r < 1.0) rts[n++] = r; }
    return n;
  }
  double h1 = l2 * l2, e1 = two_prod_err(l2, l2, h1);
  double h2 = l1 * l3, e2 = two_prod_err(l1, l3, h2);
  double disc = (h1 - h2) + (e1 - e2);
  if (!(disc > 0.0)) return 0;
  /* power form: a + b t + c t^2 with a = l1, b = 2(l2 - l1), c = l1 - 2 l2 + l3 */
  double a = l1, b = 2.0 * (l2 - l1), c = l1 - 2.0 * l2 + l3, r[2];
  int m = quad_roots(a, b, c, 4.0 * disc, 1.0, 0.0, r);
  for (int i = 0; i < m; ++i)
    if (r[i] > 0.0 && r[i] < 1.0) rts[n++] = r[i];
  if (n == 2 && rts[0] > rts[1]) { double t = rts[0]; rts[0] = rts[1]; rts[1] = t; }
  return n;
}

/* Segment link intervals. */
static void seg_intervals(const Seg* g, double q, Intervals* I) {
  memset(I, 0, sizeof *I);
  double Psi0 = ang(end_grad0(g)), Psin = ang(end_grad1(g));
  CrossPoly P = cross_poly(g);

  if (P.flat) {
    /* Zero curvature everywhere (Sec. 3.3.6 "flat interval").  Reading R5:
     * the direction can still reverse where H passes through 0 (collinear
     * control points with back-tracking); each such reversal is a pivot of
     * +pi at a fixed t, and the flat pieces between pivots are one quad each. */
    double rts[2];
    int nr = collinear_reversals(g, rts);
    double psi = Psi0, pp = 0.0;
    int M = 0;
    for (int i = 0; i <= nr; ++i) {
      double pe = (i < nr) ? rts[i] : 1.0;
      I->p[M] = pp; I->Psi[M] = psi; I->delta[M] = 0.0; I->pivot[M] = 0; M++;
      if (i < nr) {
        I->p[M] = pe; I->Psi[M] = psi; I->delta[M] = PI; I->pivot[M] = 1; M++;
        psi = psi + PI;
      }
      pp = pe;
    }
    I->p[M] = 1.0;
    I->Psi[M] = psi;
    I->M = M;
    finish_counts(I, q);
    return;
  }

  /* Eq. 4: parameter values of curvature-sign changes strictly inside (0,1) */
  double roots[2];
  int nroot = 0;
  if (P.c1 != 0.0 || P.c2 != 0.0) {
    double r[2];
    int n = quad_roots(P.c0, P.c1, P.c2, P.disc, P.disc_scale, 0.0, r);
    if (n == 2 && P.disc <= 0.0) n = 0; /* double root: curvature keeps its sign */
    for (int i = 0; i < n; ++i)
      if (r[i] > 0.0 && r[i] < 1.0 && (nroot == 0 || r[i] > roots[nroot - 1]))
        roots[nroot++] = r[i];
    if (P.c2 != 0.0 && fabs(P.disc) <= 1e-12 * P.disc_scale && P.disc != 0.0) I->fragile64 = 1;
    if (P.c2 != 0.0 && fabs(P.disc) <= 1e-5 * P.disc_scale) I->fragile32 = 1;
    for (int i = 0; i < n; ++i) {
      if (fabs(r[i]) < 1e-9 || fabs(r[i] - 1.0) < 1e-9) I->fragile64 = 1;
      if (fabs(r[i]) < 1e-4 || fabs(r[i] - 1.0) < 1e-4) I->fragile32 = 1;
    }
  }
  /* Eq. 5 */
  double p[4], Psi[4];
  int n = 0;
  p[n] = 0.0; Psi[n] = Psi0; n++;
  for (int i = 0; i < nroot; ++i) { p[n] = roots[i]; Psi[n] = ang(hodo(g, roots[i])); n++; }
  p[n] = 1.0; Psi[n] = Psin;

  /* Eq. 6 with reading R4: the turning of interval k is (Psi_k - Psi_{k-1})
   * taken modulo 2pi in the direction given by the curvature sign on the
   * interval.  A result within 1e-9 of a full turn is a numerically flat
   * interval whose end angles straddle by rounding. */
  int M = 0;
  for (int k = 0; k < n; ++k) {
    double pa = p[k], pb = p[k + 1];
    double sgn = 0.0;
    double probes[3] = {0.5 * (pa + pb), 0.75 * pa + 0.25 * pb, 0.25 * pa + 0.75 * pb};
    for (int i = 0; i < 3 && sgn == 0.0; ++i) {
      double v = cross_eval(&P, probes[i]);
      sgn = (v > 0) ? 1.0 : (v < 0 ? -1.0 : 0.0);
    }
    double delta = 0.0;
    if (sgn != 0.0) {
      delta = sgn * mod2pi(sgn * (Psi[k + 1] - Psi[k]));
      if (fabs(delta) > TWO_PI - 1e-9) { delta = 0.0; I->fragile64 = 1; I->fragile32 = 1; }
      if (fabs(delta) > TWO_PI - 1e-4) I->fragile32 = 1;
    }
    /* the split decision below (|delta| >= pi) is fragile when the turning is
     * within rounding of pi: splitting or not changes the count unless q
     * divides pi/2 */
    if (fabs(fabs(delta) - PI) < 1e-5) I->fragile32 = 1;
    if (fabs(fabs(delta) - PI) < 1e-12) I->fragile64 = 1;
    if (fabs(delta) >= PI) {
      /* Sec. 3.3.5: split at half the turning (reading R6), p by Eq. 11 */
      double psi_s = Psi[k] + 0.5 * delta;
      double ps = solve_t(g, psi_s, pa, pb);
      I->p[M] = pa; I->Psi[M] = Psi[k]; I->delta[M] = 0.5 * delta; M++;
      I->split[M] = 1;
      I->p[M] = ps; I->Psi[M] = psi_s; I->delta[M] = 0.5 * delta; M++;
    } else {
      I->p[M] = pa; I->Psi[M] = Psi[k]; I->delta[M] = delta; M++;
    }
  }
  I->p[M] = 1.0;
  I->Psi[M] = Psin;
  I->M = M;
  finish_counts(I, q);
}

/* ---- links of a path (Sec. 4.3-4.4) -------------------------------------- */
typedef struct {
  int kind;        /* 0 empty, 1 segment, 2 join, 3 cap */
  int seg;         /* segment index for kind 1 */
  V2 at;           /* join / cap point */
  double Psi0, delta; /* join / cap pivot (Sec. 4.3.1) */
  int style;       /* join or cap style */
  double miter_limit;
} Link;

static Seg load_seg(int64_t i, const uint8_t* type, const double* pts, const double* wts) {
  Seg g;
  g.type = type[i];
  const double* q = pts + 8 * i;
  g.A = mk(q[0], q[1]);
  g.B = mk(q[2], q[3]);
  g.C = mk(q[4], q[5]);
  g.D = mk(q[6], q[7]);
  g.w = wts ? wts[i] : 1.0;
  return g;
}

/* Reading R21 (Sec. 7 leaves a pixel-scale boost of q to heuristics).  With a
 * pixel tolerance tau > 0 each link steps by its own q_link >= q, the largest
 * step (up to the bounds below) at which every boundary edge of its quads
 * stays within tau px of the stroke boundary it replaces; tau = 0 keeps q.
 *
 * Round join or cap: the outer boundary is an arc of radius r = w/2, and one
 * step of phi leaves a gap of r (1 - cos(phi/2)) between arc and chord, so
 *   q_link = max(q, 2 acos(1 - tau / r))    (pi when tau >= r).
 *
 * Segment: the boundary piece of one step is the offset of a curve piece
 * that turns by phi <= pi/2 in one direction; its length is at most
 * l + r phi, l the curve piece's length, and l <= L_g, the length of the
 * control polygon (a polynomial Bezier's or a positive-weight conic's arc is
 * no longer than its control polygon).  A convex arc turning by phi lies in
 * the triangle of its chord c and end tangents, at most (c/2) tan(phi/2) from
 * the chord.  Splitting tau between the two terms of c, and using
 * tan(x) <= 4x/pi on [0, pi/4]:
 *   q_link = max(q, min(2 atan(tau / L_g), sqrt(pi tau / (2 r)), pi/2)).
 * The bound holds on the outer side and on an inner side whose radius of
 * curvature stays >= r (elsewhere the inner side folds inside the stroke).  A
 * conic with w_B <= 0 leaves its control hull and keeps q. */
static double polygon_length(const Seg* g) {
  switch (g->type) {
    case ORC_LINE: return len(sub(g->D, g->A));
    case ORC_QUAD: return len(sub(g->B, g->A)) + len(sub(g->D, g->B));
    case ORC_CUBIC: return len(sub(g->B, g->A)) + len(sub(g->C, g->B)) + len(sub(g->D, g->C));
    case ORC_CONIC: return g->w > 0.0 ? len(sub(g->B, g->A)) + len(sub(g->D, g->B)) : -1.0;
  }
  return -1.0;
}

static double seg_step(const Seg* g, double q, double tau, double r) {
  if (!(tau > 0.0)) return q;
  double Lg = polygon_length(g);
  if (Lg < 0.0) return q;
  double a = Lg > 0.0 ? 2.0 * atan(tau / Lg) : PI;
  double b = sqrt(PI * tau / (2.0 * r));
  double qp = a < b ? a : b;
  if (qp > 0.5 * PI) qp = 0.5 * PI;
  return qp > q ? qp : q;
}

static double round_step(double q, double tau, double r) {
  if (!(tau > 0.0)) return q;
  double qp = tau >= r ? PI : 2.0 * acos(1.0 - tau / r);
  return qp > q ? qp : q;
}

/* Round-style counts J = ceil(|delta|/q) (Sec. 4.3.2, 4.3.4) */
static int round_count(double delta, double q) {
  double ad = fabs(delta);
  if (ad == 0.0) return 0;
  return step_count(ad, q);
}

static int join_count(int style, double delta, double q) {
  if (delta == 0.0) return 0; /* tangent-continuous: no join region */
  switch (style) {
    case ORC_JOIN_NONE: return 0;
    case ORC_JOIN_BEVEL: return 1;
    case ORC_JOIN_TRIANGLE: return 2;
    case ORC_JOIN_MITER:
    case ORC_JOIN_MITER_TRUNCATE: return 3;
    case ORC_JOIN_ROUND: return round_count(delta, q);
    default: return 0;
  }
}
static int cap_count(int style, double q) {
  switch (style) {
    case ORC_CAP_BUTT: return 0;
    case ORC_CAP_TRIANGLE: return 2;
    case ORC_CAP_SQUARE: return 4;
    case ORC_CAP_ROUND: return round_count(PI, q);
    default: return 0;
  }
}

/* Emit the ribs of a join or cap link j = 0..J (Sec. 4.3.1-4.3.5).
 * The generator is the fixed point `at`; psi(j) = Psi0 + delta j / J.
 * Reading R7: the outer side is N (= g - r n) when delta > 0 and P when
 * delta < 0; the inner radius is forced to zero.  Miter variants override the
 * outer vertices of ribs 1 and 2 (R8); square caps push ribs 1 and 3 out to
 * sqrt(2) w/2 (R9). */
static void emit_pivot(const Link* L, int J, double r, V2* Nv, V2* Pv, double* psiv) {
  double rN = L->delta > 0 ? r : 0.0, rP = L->delta > 0 ? 0.0 : r;
  for (int j = 0; j <= J; ++j) {
    double psi = (j == J) ? L->Psi0 + L->delta : L->Psi0 + L->delta * (double)j / (double)J;
    double rn = rN, rp = rP;
    if (L->kind == 3 && L->style == ORC_CAP_SQUARE && (j == 1 || j == 3)) {
      rn *= sqrt(2.0);
      rp *= sqrt(2.0);
    }
    V2 n = normal_of(psi);
    Nv[j] = sub(L->at, mul(n, rn));
    Pv[j] = add(L->at, mul(n, rp));
    psiv[j] = psi;
  }
  if (L->kind == 2 && (L->style == ORC_JOIN_MITER || L->style == ORC_JOIN_MITER_TRUNCATE) && J == 3) {
    double sd = L->delta > 0 ? -1.0 : 1.0; /* outer offset = at + sd * r * n */
    double ad = fabs(L->delta);
    V2 O0 = add(L->at, mul(normal_of(L->Psi0), sd * r));
    V2 O3 = add(L->at, mul(normal_of(L->Psi0 + L->delta), sd * r));
    /* miter ratio = miter length / stroke width = 1 / sin(phi/2), phi = pi - |delta| */
    double cm = cos(0.5 * ad);
    double ratio = cm > 0.0 ? 1.0 / cm : INFINITY;
    V2 v1, v2;
    if (ratio <= L->miter_limit) {
      V2 tip = add(L->at, mul(normal_of(L->Psi0 + 0.5 * L->delta), sd * r * ratio));
      v1 = tip; v2 = tip;
    } else if (L->style == ORC_JOIN_MITER) {
      v1 = O0; v2 = O3; /* revert to bevel */
    } else {
      /* truncate: clip the miter at distance limit * w/2 along the bisector */
      double dc = L->miter_limit * r;
      double lam = (dc - r * cos(0.5 * ad)) / sin(0.5 * ad);
      if (lam < 0) lam = 0;
      v1 = add(O0, mul(tangent_of(L->Psi0), lam));
      v2 = sub(O3, mul(tangent_of(L->Psi0 + L->delta), lam));
    }
    if (L->delta > 0) { Nv[1] = v1; Nv[2] = v2; } else { Pv[1] = v1; Pv[2] = v2; }
  }
}

/* ---- O1: tessellation + arc length -------------------------------------- */
/* Inputs use the library's layout (FP32 values, converted exactly):
 *   seg_type[S], seg_pts[S][4][2] (A,B,C,D), seg_w[S]
 *   path_seg_off[P+1], path_width[P], path_join[P], path_cap[P],
 *   path_miter[P], path_closed[P]
 * Links of path p: 2 n_p + 1 slots in the order start-cap, seg 0, join 0/1,
 * seg 1, ..., seg n-1, end-cap (open) or closing join (closed).
 * Outputs (any may be NULL to only count):
 *   link_nrib[L]   ribs of each link (N+1 when N > 0, else 0)
 *   link_info[L]   fragility and kind bits
 *   rib[4R]        N.x N.y P.x P.y per rib (Eq. 16-17)
 *   s[R]           cumulative arc length per path (Eq. 18, Sec. 5.1)
 *   t[R], psi[R]   t(j) and psi(j) of each rib (Eq. 14)
 *   rho[R]         radius of curvature at solved ribs, 0 at boundaries and
 *                  pivots (used to state a conditioning-aware tolerance)
 *   tag[R]         link start / segment bits and path index
 *   path_len[P]    total arc length per path
 */
int orc_tessellate_f64(int64_t n_seg, const uint8_t* seg_type, const double* seg_pts,
                       const double* seg_w, int32_t n_path, const int32_t* path_seg_off,
                       const double* path_width, const uint8_t* path_join,
                       const uint8_t* path_cap, const double* path_miter,
                       const uint8_t* path_closed, double q0, double tau, int64_t* link_nrib,
                       uint8_t* link_info, int64_t rib_cap, double* rib, double* s_out,
                       double* t_out, double* psi_out, double* rho_out, uint32_t* tag_out,
                       double* path_len, int64_t* n_rib_total) {
  if (!(q0 > 0.0) || !(tau >= 0.0) || n_seg < 0 || n_path < 0) return ORC_ERR_INVALID;
  int64_t R = 0;
  int overflow = 0;
  enum { MAXR = 8192 };
  static V2 Nv[MAXR], Pv[MAXR];
  static double tv[MAXR], psiv[MAXR], rhov[MAXR];

  for (int32_t p = 0; p < n_path; ++p) {
    int32_t s0 = path_seg_off[p], s1 = path_seg_off[p + 1];
    int n = s1 - s0;
    if (n < 0 || s0 < 0 || s1 > n_seg) return ORC_ERR_INVALID;
    double r = 0.5 * path_width[p];
    int closed = path_closed ? path_closed[p] : 0;
    int64_t lbase = 2 * (int64_t)s0 + p;
    double s_run = 0.0;
    /* first / last non-degenerate segment of the path */
    int first_nd = -1, last_nd = -1;
    for (int i = 0; i < n; ++i) {
      Seg g = load_seg(s0 + i, seg_type, seg_pts, seg_w);
      if (!seg_zero_length(&g)) { if (first_nd < 0) first_nd = i; last_nd = i; }
    }
    for (int k = 0; k <= 2 * n; ++k) {
      int64_t l = lbase + k;
      Link L;
      memset(&L, 0, sizeof L);
      Intervals I;
      memset(&I, 0, sizeof I);
      Seg g;
      memset(&g, 0, sizeof g);
      int J = 0;
      if (first_nd >= 0) {
        if (k % 2 == 1) {
          int i = (k - 1) / 2;
          g = load_seg(s0 + i, seg_type, seg_pts, seg_w);
          if (!seg_zero_length(&g)) {
            L.kind = 1;
            L.seg = i;
          }
        } else if (k == 0 || k == 2 * n) {
          if (!closed) {
            int i = (k == 0) ? first_nd : last_nd;
            Seg c = load_seg(s0 + i, seg_type, seg_pts, seg_w);
            L.kind = 3;
            L.style = path_cap[p];
            L.delta = PI;
            if (k == 0) { /* start cap: pivot from Psi_s + pi through pi (R7) */
              L.at = c.A;
              L.Psi0 = ang(end_grad0(&c)) + PI;
            } else {      /* stop cap: pivot from Psi_e through pi */
              L.at = c.D;
              L.Psi0 = ang(end_grad1(&c));
            }
          } else if (k == 2 * n) { /* closing join: last -> first */
            Seg a = load_seg(s0 + last_nd, seg_type, seg_pts, seg_w);
            Seg b = load_seg(s0 + first_nd, seg_type, seg_pts, seg_w);
            L.kind = 2;
            L.style = path_join[p];
            L.at = b.A;
            L.Psi0 = ang(end_grad1(&a));
            L.delta = ominus(ang(end_grad0(&b)), L.Psi0);
          }
        } else {
          /* join after segment i = k/2 - 1, into segment i + 1 */
          int i = k / 2 - 1;
          Seg b = load_seg(s0 + i + 1, seg_type, seg_pts, seg_w);
          int inc = -1;
          for (int m = i; m >= 0; --m) {
            Seg a = load_seg(s0 + m, seg_type, seg_pts, seg_w);
            if (!seg_zero_length(&a)) { inc = m; break; }
          }
          if (!seg_zero_length(&b) && inc >= 0) {
            Seg a = load_seg(s0 + inc, seg_type, seg_pts, seg_w);
            L.kind = 2;
            L.style = path_join[p];
            L.at = b.A;
            L.Psi0 = ang(end_grad1(&a));
            /* Sec. 4.3.1: delta_1 = Psi_1 (-) Psi_0; an exact reversal is +pi (R10) */
            L.delta = ominus(ang(end_grad0(&b)), L.Psi0);
          }
        }
      }
      if (L.kind == 2 && L.delta == -PI) L.delta = PI;
      L.miter_limit = path_miter ? path_miter[p] : 4.0;
      /* the link's step (R21; q0 itself when tau = 0) */
      double q = q0;
      if (L.kind == 1) q = seg_step(&g, q0, tau, r);
      else if (L.kind == 2 && L.style == ORC_JOIN_ROUND) q = round_step(q0, tau, r);
      else if (L.kind == 3 && L.style == ORC_CAP_ROUND) q = round_step(q0, tau, r);

      int nrib = 0;
      uint8_t info = 0;
      if (L.kind == 1) {
        /* A conic with w_B <= -1 is an external parabola (w = -1) or hyperbola
         * (w < -1): its denominator (1-t)^2 + 2w(1-t)t + t^2 vanishes at
         * t = 1/2 +- sqrt(w^2-1)/(2(1-w)) in [0,1] (Sec. 3.3.3 with the
         * corrected root formula), where the curve passes through infinity and
         * its stroke is unbounded.  Such a segment is rejected. */
        if (g.type == ORC_CONIC && !(g.w > -1.0)) return ORC_ERR_INVALID;
        seg_intervals(&g, q, &I);
        if (I.N > 0) nrib = I.N + 1;
        info |= (I.fragile64 ? INFO_FRAGILE64 : 0) | (I.fragile32 ? INFO_FRAGILE32 : 0);
      } else if (L.kind == 2) {
        J = join_count(L.style, L.delta, q);
        if (J > 0) nrib = J + 1;
        if (L.style == ORC_JOIN_ROUND && L.delta != 0.0) {
          double x = fabs(L.delta) / q, dd = step_margin(fabs(L.delta), q);
          if (dd < 1e-9 * (1 + x)) info |= INFO_FRAGILE64;
          if (dd < 2e-5 * (1 + x)) info |= INFO_FRAGILE32;
        }
        if (fabs(L.delta) < 1e-4) info |= INFO_FRAGILE32;
        if (L.style == ORC_JOIN_MITER || L.style == ORC_JOIN_MITER_TRUNCATE) {
          double ratio = 1.0 / cos(0.5 * fabs(L.delta));
          if (fabs(ratio - L.miter_limit) < 1e-5 * L.miter_limit) info |= INFO_FRAGILE32;
          if (fabs(ratio - L.miter_limit) < 1e-12 * L.miter_limit) info |= INFO_FRAGILE64;
        }
      } else if (L.kind == 3) {
        J = cap_count(L.style, q);
        if (J > 0) nrib = J + 1;
        if (L.style == ORC_CAP_ROUND) {
          double x = PI / q, dd = step_margin(PI, q);
          if (dd < 1e-9 * (1 + x)) info |= INFO_FRAGILE64;
          if (dd < 2e-5 * (1 + x)) info |= INFO_FRAGILE32;
        }
      }
      if (nrib == 0) L.kind = L.kind ? L.kind : 0;
      info |= (uint8_t)((nrib > 0 ? L.kind : 0) << INFO_KIND_SHIFT);
      if (link_nrib) link_nrib[l] = nrib;
      if (link_info) link_info[l] = info;
      if (nrib == 0) continue;
      if (nrib > MAXR) return ORC_ERR_INVALID;

      /* ribs of this link */
      if (L.kind == 1) {
        /* Eq. 14-15: rib j is a boundary rib when j = Delta_Sigma(k) for some
         * k (t = p_k, normal from Psi_k), else interior to interval k with
         * psi(j) = Psi_k + (delta_k / Delta_k)(j - Delta_Sigma(k)) (reading
         * R4 fixes the interval index of the step). */
        int kb = 0, base = 0;
        for (int j = 0; j <= I.N; ++j) {
          while (kb < I.M && j >= base + I.Delta[kb]) { base += I.Delta[kb]; kb++; }
          double t, psi, rho = 0.0;
          if (j == base) {
            t = I.p[kb];
            psi = I.Psi[kb];
            if (I.split[kb]) {
              /* a split point is solved from Eq. 11 like an interior rib: its
               * radius of curvature is reported for the tolerance */
              V2 H = hodo(&g, t), Hd = hodo_d(&g, t);
              double cr = fabs(cross(H, Hd)), hl = len(H);
              rho = cr > 0 ? hodo_scale(&g, t) * hl * hl * hl / cr : 1e300;
            }
          } else {
            psi = I.Psi[kb] + I.delta[kb] / (double)I.Delta[kb] * (double)(j - base);
            if (I.pivot[kb]) {
              t = I.p[kb];
            } else {
              t = solve_t(&g, psi, I.p[kb], I.p[kb + 1]);
              V2 H = hodo(&g, t), Hd = hodo_d(&g, t);
              double cr = fabs(cross(H, Hd)), hl = len(H);
              rho = cr > 0 ? hodo_scale(&g, t) * hl * hl * hl / cr : 1e300;
            }
          }
          V2 c = seg_eval(&g, t), nn = normal_of(psi);
          Nv[j] = sub(c, mul(nn, r));
          Pv[j] = add(c, mul(nn, r));
          tv[j] = t;
          psiv[j] = psi;
          rhov[j] = rho;
        }
      } else {
        emit_pivot(&L, J, r, Nv, Pv, psiv);
        for (int j = 0; j <= J; ++j) { tv[j] = 0.0; rhov[j] = 0.0; }
      }

      /* Eq. 18 with Sec. 7's rule: a step whose t decreases adds 0; joins
       * and caps add 0; the first rib of a link continues the running total. */
      for (int j = 0; j < nrib; ++j) {
        if (L.kind == 1 && j > 0 && tv[j] >= tv[j - 1]) {
          V2 c1 = seg_eval(&g, tv[j]), c0 = seg_eval(&g, tv[j - 1]);
          s_run += len(sub(c1, c0));
        }
        if (R < rib_cap) {
          if (rib) {
            rib[4 * R + 0] = Nv[j].x; rib[4 * R + 1] = Nv[j].y;
            rib[4 * R + 2] = Pv[j].x; rib[4 * R + 3] = Pv[j].y;
          }
          if (s_out) s_out[R] = s_run;
          if (t_out) t_out[R] = tv[j];
          if (psi_out) psi_out[R] = psiv[j];
          if (rho_out) rho_out[R] = rhov[j];
          if (tag_out)
            tag_out[R] = ((uint32_t)p << 2) | (j == 0 ? TAG_LINK_START : 0u) |
                         (L.kind == 1 ? TAG_SEGMENT : 0u);
        } else {
          overflow = 1;
        }
        R++;
      }
    }
    if (path_len) path_len[p] = s_run;
  }
  if (n_rib_total) *n_rib_total = R;
  return overflow ? ORC_ERR_CAPACITY : ORC_OK;
}

/* The library's FP32 input layout: converted exactly to FP64 and tessellated. */
int orc_tessellate(int64_t n_seg, const uint8_t* seg_type, const float* seg_pts,
                   const float* seg_w, int32_t n_path, const int32_t* path_seg_off,
                   const float* path_width, const uint8_t* path_join, const uint8_t* path_cap,
                   const float* path_miter, const uint8_t* path_closed, double q, double tau,
                   int64_t* link_nrib, uint8_t* link_info, int64_t rib_cap, double* rib,
                   double* s_out, double* t_out, double* psi_out, double* rho_out,
                   uint32_t* tag_out, double* path_len, int64_t* n_rib_total) {
  double* pts = (double*)malloc(sizeof(double) * (size_t)(8 * n_seg + 1));
  double* w = (double*)malloc(sizeof(double) * (size_t)(n_seg + 1));
  double* wid = (double*)malloc(sizeof(double) * (size_t)(n_path + 1));
  double* mit = (double*)malloc(sizeof(double) * (size_t)(n_path + 1));
  if (!pts || !w || !wid || !mit) { free(pts); free(w); free(wid); free(mit); return ORC_ERR_INVALID; }
  for (int64_t i = 0; i < 8 * n_seg; ++i) pts[i] = seg_pts[i];
  for (int64_t i = 0; i < n_seg; ++i) w[i] = seg_w ? seg_w[i] : 1.0;
  for (int32_t p = 0; p < n_path; ++p) {
    wid[p] = path_width[p];
    mit[p] = path_miter ? path_miter[p] : 4.0;
  }
  int rc = orc_tessellate_f64(n_seg, seg_type, pts, w, n_path, path_seg_off, wid, path_join,
                              path_cap, mit, path_closed, q, tau, link_nrib, link_info, rib_cap, rib,
                              s_out, t_out, psi_out, rho_out, tag_out, path_len, n_rib_total);
  free(pts); free(w); free(wid); free(mit);
  return rc;
}

/* Interval table of one segment (for tests). Returns M; fills p, Psi, delta,
 * Delta (arrays of MAXI+1). */
int orc_segment_intervals(int type, const float* pts8, float w, double q, double* p,
                          double* Psi, double* delta, int32_t* Delta, int32_t* pivot,
                          int32_t* flags) {
  Seg g;
  g.type = type;
  g.A = mk(pts8[0], pts8[1]); g.B = mk(pts8[2], pts8[3]);
  g.C = mk(pts8[4], pts8[5]); g.D = mk(pts8[6], pts8[7]);
  g.w = w;
  Intervals I;
  seg_intervals(&g, q, &I);
  for (int k = 0; k <= I.M; ++k) { p[k] = I.p[k]; Psi[k] = I.Psi[k]; }
  for (int k = 0; k < I.M; ++k) { delta[k] = I.delta[k]; Delta[k] = I.Delta[k]; pivot[k] = I.pivot[k]; }
  *flags = (I.fragile64 ? 1 : 0) | (I.fragile32 ? 2 : 0);
  return I.M;
}

/* Geometry probes (for tests that pin the formulas above against finite
 * differences and closed forms). what: 0 g(t), 1 H(t), 2 H'(t), 3 c(t),
 * 4 C(t) (x holds C, y holds 0) */
void orc_segment_probe(int type, const float* pts8, float w, int what, int n, const double* t,
                       double* out) {
  Seg g;
  g.type = type;
  g.A = mk(pts8[0], pts8[1]); g.B = mk(pts8[2], pts8[3]);
  g.C = mk(pts8[4], pts8[5]); g.D = mk(pts8[6], pts8[7]);
  g.w = w;
  CrossPoly P = cross_poly(&g);
  for (int i = 0; i < n; ++i) {
    V2 v = mk(0, 0);
    switch (what) {
      case 0: v = seg_eval(&g, t[i]); break;
      case 1: v = hodo(&g, t[i]); break;
      case 2: v = hodo_d(&g, t[i]); break;
      case 3: v = mk(hodo_scale(&g, t[i]), 0); break;
      case 4: v = mk(cross_eval(&P, t[i]), 0); break;
    }
    out[2 * i] = v.x;
    out[2 * i + 1] = v.y;
  }
}

/* ---- O1b: dashing (Sec. 5.2) -------------------------------------------- */
/* Reading R11: the pattern (on, off, on, off, ...; an odd count is repeated
 * twice) restarts at s = 0 of every path, shifted by `offset`; "on" stretches
 * are half-open [a, b).  Each quad [s_{j-1}, s_j] of a rib strip is clipped
 * to the on-stretches by interpolating both rib vertices at
 * f = (s - s_{j-1}) / (s_j - s_{j-1}); every clipped piece is an independent
 * 2-rib strip (its first rib carries the link-start bit).  A quad of zero
 * length (join, cap, cusp pivot) is kept whole iff its s lies in an on
 * stretch.  Dash ends are butt.
 * Inputs: rib[4R], s[R], tag[R]; pattern[m]; offset.
 * Outputs (NULL to count): out_rib[4 cap], out_s[cap], out_tag[cap],
 * out_src[cap] (index of the source quad's end rib j), *n_out. */
static void dash_put(int64_t n, int64_t cap, const double* rib, int64_t j, double f0, double f1,
                     double s0, double s1, uint32_t tg, double* out_rib, double* out_s,
                     uint32_t* out_tag, int64_t* out_src) {
  if (!out_rib || n + 2 > cap) return;
  for (int c = 0; c < 4; ++c) {
    double v0 = rib[4 * (j - 1) + c], v1 = rib[4 * j + c];
    out_rib[4 * n + c] = v0 + f0 * (v1 - v0);
    out_rib[4 * n + 4 + c] = v0 + f1 * (v1 - v0);
  }
  out_s[n] = s0;
  out_s[n + 1] = s1;
  out_tag[n] = tg | TAG_LINK_START;
  out_tag[n + 1] = tg;
  out_src[n] = j;
  out_src[n + 1] = j;
}

int orc_dash(int64_t R, const double* rib, const double* s, const uint32_t* tag,
             const double* pattern, int m, double offset, int64_t cap, double* out_rib,
             double* out_s, uint32_t* out_tag, int64_t* out_src, int64_t* n_out) {
  if (m <= 0 || m > 32) return ORC_ERR_INVALID;
  int m2 = (m % 2) ? 2 * m : m;
  double cum[65];
  cum[0] = 0.0;
  for (int i = 0; i < m2; ++i) {
    double d = pattern[i % m];
    if (!(d >= 0.0)) return ORC_ERR_INVALID;
    cum[i + 1] = cum[i] + d;
  }
  double period = cum[m2];
  if (!(period > 0.0)) return ORC_ERR_INVALID;
  int64_t n = 0;
  for (int64_t j = 1; j < R; ++j) {
    if (tag[j] & TAG_LINK_START) continue;
    double sa = s[j - 1], sb = s[j];
    uint32_t tg = tag[j] & ~TAG_LINK_START;
    /* on-stretch i of period k: [k*period + cum[2i] - offset, k*period + cum[2i+1] - offset) */
    double k0 = floor((sa + offset) / period) - 1.0;
    for (double k = k0;; k += 1.0) {
      double base = k * period;
      if (base - offset > sb) break;
      for (int i = 0; i < m2; i += 2) {
        double a = (base + cum[i]) - offset, b = (base + cum[i + 1]) - offset;
        if (!(b > a)) continue;
        if (sb > sa) {
          double lo = a > sa ? a : sa, hi = b < sb ? b : sb;
          if (hi > lo) {
            dash_put(n, cap, rib, j, (lo - sa) / (sb - sa), (hi - sa) / (sb - sa), lo, hi, tg,
                     out_rib, out_s, out_tag, out_src);
            n += 2;
          }
        } else if (sa >= a && sa < b) { /* zero-length quad kept whole */
          dash_put(n, cap, rib, j, 0.0, 1.0, sa, sb, tg, out_rib, out_s, out_tag, out_src);
          n += 2;
        }
      }
    }
  }
  *n_out = n;
  return n > cap ? ORC_ERR_CAPACITY : ORC_OK;
}

/* ---- O2: fixed-point sample coverage of a rib stream --------------------- */
/* Reading R12 (the paper leaves rasterization to the GPU's API):
 *  - quad j of a strip (ribs j-1, j of one link) is the two triangles
 *    (N_{j-1}, P_{j-1}, P_j) and (N_{j-1}, P_j, N_j) (Sec. 4.1: GPUs split
 *    quads into two triangles);
 *  - vertices snap to integers round-half-even(v * 256) (8-bit subpixel);
 *  - pixel (x, y) has 16 samples k = 0..15 at
 *      (256 x + 16 k + 8, 256 y + 16 ((5 k) mod 16) + 8)  in 1/256 px;
 *  - a sample is covered by a triangle iff, with the triangle oriented
 *    counter-clockwise, all three edge functions are >= 0 (zero-area
 *    triangles cover nothing);
 *  - the coverage of a path is the union over its triangles (Sec. 3.3.6:
 *    the support of a path is the maximum over its parts); the canvas is the
 *    union over paths; covered[p] counts path p's samples.
 * Samples outside [0,W) x [0,H) are ignored. */
static int64_t snap256(double v) { return (int64_t)nearbyint(v * 256.0); }
static int64_t floor_div(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
static int64_t ceil_div(int64_t a, int64_t b) { return -floor_div(-a, b); }

static void raster_tri(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t cx, int64_t cy,
                       uint16_t* mask, int64_t x0c, int64_t y0c, int64_t x1c, int64_t y1c) {
  int64_t wc = x1c - x0c + 1;
  int64_t area = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
  if (area == 0) return;
  if (area < 0) { int64_t tx = bx, ty = by; bx = cx; by = cy; cx = tx; cy = ty; }
  int64_t minx = ax < bx ? (ax < cx ? ax : cx) : (bx < cx ? bx : cx);
  int64_t maxx = ax > bx ? (ax > cx ? ax : cx) : (bx > cx ? bx : cx);
  int64_t miny = ay < by ? (ay < cy ? ay : cy) : (by < cy ? by : cy);
  int64_t maxy = ay > by ? (ay > cy ? ay : cy) : (by > cy ? by : cy);
  /* pixels whose sample window [256x+8, 256x+248] can meet the bbox */
  int64_t px0 = ceil_div(minx - 248, 256), px1 = floor_div(maxx - 8, 256);
  int64_t py0 = ceil_div(miny - 248, 256), py1 = floor_div(maxy - 8, 256);
  if (px0 < x0c) px0 = x0c;
  if (py0 < y0c) py0 = y0c;
  if (px1 > x1c) px1 = x1c;
  if (py1 > y1c) py1 = y1c;
  for (int64_t y = py0; y <= py1; ++y) {
    for (int64_t x = px0; x <= px1; ++x) {
      uint16_t m = 0;
      for (int k = 0; k < 16; ++k) {
        int64_t sx = 256 * x + 16 * k + 8, sy = 256 * y + 16 * ((5 * k) % 16) + 8;
        int64_t e0 = (bx - ax) * (sy - ay) - (by - ay) * (sx - ax);
        int64_t e1 = (cx - bx) * (sy - by) - (cy - by) * (sx - bx);
        int64_t e2 = (ax - cx) * (sy - cy) - (ay - cy) * (sx - cx);
        if (e0 >= 0 && e1 >= 0 && e2 >= 0) m |= (uint16_t)(1u << k);
      }
      if (m) mask[(y - y0c) * wc + (x - x0c)] |= m;
    }
  }
}

/* rib[4R] in px (any precision; snapped here), tag[R].  canvas[W*H] is ORed
 * into (the caller zeroes it); covered[n_path] is added to. */
/* Reading R19 (Sec. 4.1, Sec. 7: quads rasterized as quads, bow-ties as such):
 * the exact coverage of quad (N0, P0, P1, N1) is its polygon N0 -> P0 -> P1 ->
 * N1 -> N0 filled by the crossing rule: a sample is covered iff the ray from it
 * towards +x crosses an odd number of the four edges, where edge a -> b is
 * crossed iff a.y <= y < b.y with the sample strictly left of a -> b, or
 * b.y <= y < a.y with the sample strictly right of it (integer edge function).
 * A closed polyline of four edges winds at most once around a point, so odd
 * crossings = nonzero winding: convex, concave and bow-tie quads alike. */
static void raster_quad_exact(const int64_t* vx, const int64_t* vy, uint16_t* mask, int64_t x0c,
                              int64_t y0c, int64_t x1c, int64_t y1c) {
  int64_t wc = x1c - x0c + 1;
  int64_t minx = vx[0], maxx = vx[0], miny = vy[0], maxy = vy[0];
  for (int i = 1; i < 4; ++i) {
    if (vx[i] < minx) minx = vx[i];
    if (vx[i] > maxx) maxx = vx[i];
    if (vy[i] < miny) miny = vy[i];
    if (vy[i] > maxy) maxy = vy[i];
  }
  int64_t px0 = ceil_div(minx - 248, 256), px1 = floor_div(maxx - 8, 256);
  int64_t py0 = ceil_div(miny - 248, 256), py1 = floor_div(maxy - 8, 256);
  if (px0 < x0c) px0 = x0c;
  if (py0 < y0c) py0 = y0c;
  if (px1 > x1c) px1 = x1c;
  if (py1 > y1c) py1 = y1c;
  for (int64_t y = py0; y <= py1; ++y) {
    for (int64_t x = px0; x <= px1; ++x) {
      uint16_t m = 0;
      for (int k = 0; k < 16; ++k) {
        int64_t sx = 256 * x + 16 * k + 8, sy = 256 * y + 16 * ((5 * k) % 16) + 8;
        int cross = 0;
        for (int i = 0; i < 4; ++i) {
          int64_t ax = vx[i], ay = vy[i], bx = vx[(i + 1) & 3], by = vy[(i + 1) & 3];
          int64_t e = (bx - ax) * (sy - ay) - (by - ay) * (sx - ax);
          if (ay <= sy && sy < by && e > 0) cross ^= 1;
          if (by <= sy && sy < ay && e < 0) cross ^= 1;
        }
        if (cross) m |= (uint16_t)(1u << k);
      }
      mask[(y - y0c) * wc + (x - x0c)] |= m;
    }
  }
}

static int raster_impl(int64_t R, const double* rib, const uint32_t* tag, int W, int H,
                       int32_t n_path, int exact, uint16_t* canvas, uint64_t* covered);

int orc_raster(int64_t R, const double* rib, const uint32_t* tag, int W, int H,
               int32_t n_path, uint16_t* canvas, uint64_t* covered) {
  return raster_impl(R, rib, tag, W, H, n_path, 0, canvas, covered);
}

/* O2 with the exact quad coverage of reading R19. */
int orc_raster_exact(int64_t R, const double* rib, const uint32_t* tag, int W, int H,
                     int32_t n_path, uint16_t* canvas, uint64_t* covered) {
  return raster_impl(R, rib, tag, W, H, n_path, 1, canvas, covered);
}

static int raster_impl(int64_t R, const double* rib, const uint32_t* tag, int W, int H,
                       int32_t n_path, int exact, uint16_t* canvas, uint64_t* covered) {
  if (W <= 0 || H <= 0) return ORC_ERR_INVALID;
  uint16_t* mask = (uint16_t*)calloc((size_t)W * H, sizeof(uint16_t));
  if (!mask) return ORC_ERR_INVALID;
  int64_t j = 0;
  while (j < R) {
    uint32_t path = tag[j] >> 2;
    int64_t j1 = j;
    while (j1 < R && (tag[j1] >> 2) == path) j1++;
    /* path's ribs are [j, j1) */
    int64_t bx0 = INT64_MAX, by0 = INT64_MAX, bx1 = INT64_MIN, by1 = INT64_MIN;
    for (int64_t i = j; i < j1; ++i)
      for (int c = 0; c < 2; ++c) {
        int64_t X = snap256(rib[4 * i + 2 * c]), Y = snap256(rib[4 * i + 2 * c + 1]);
        if (X < bx0) bx0 = X;
        if (X > bx1) bx1 = X;
        if (Y < by0) by0 = Y;
        if (Y > by1) by1 = Y;
      }
    int64_t x0 = floor_div(bx0, 256) - 1, x1 = floor_div(bx1, 256) + 1;
    int64_t y0 = floor_div(by0, 256) - 1, y1 = floor_div(by1, 256) + 1;
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (x1 > W - 1) x1 = W - 1;
    if (y1 > H - 1) y1 = H - 1;
    if (x0 <= x1 && y0 <= y1) {
      int wc = (int)(x1 - x0 + 1), hc = (int)(y1 - y0 + 1);
      memset(mask, 0, (size_t)wc * hc * sizeof(uint16_t));
      for (int64_t i = j + 1; i < j1; ++i) {
        if (tag[i] & TAG_LINK_START) continue;
        const double* a = rib + 4 * (i - 1);
        const double* b = rib + 4 * i;
        int64_t Nax = snap256(a[0]), Nay = snap256(a[1]), Pax = snap256(a[2]), Pay = snap256(a[3]);
        int64_t Nbx = snap256(b[0]), Nby = snap256(b[1]), Pbx = snap256(b[2]), Pby = snap256(b[3]);
        if (exact) {
          int64_t qx[4] = {Nax, Pax, Pbx, Nbx}, qy[4] = {Nay, Pay, Pby, Nby};
          raster_quad_exact(qx, qy, mask, x0, y0, x1, y1);
        } else {
          raster_tri(Nax, Nay, Pax, Pay, Pbx, Pby, mask, x0, y0, x1, y1);
          raster_tri(Nax, Nay, Pbx, Pby, Nbx, Nby, mask, x0, y0, x1, y1);
        }
      }
      uint64_t cnt = 0;
      for (int yy = 0; yy < hc; ++yy)
        for (int xx = 0; xx < wc; ++xx) {
          uint16_t m = mask[yy * wc + xx];
          if (!m) continue;
          canvas[(y0 + yy) * (int64_t)W + (x0 + xx)] |= m;
          for (int b = 0; b < 16; ++b) cnt += (m >> b) & 1u;
        }
      if (path < (uint32_t)n_path) covered[path] += cnt;
    }
    j = j1;
  }
  free(mask);
  return ORC_OK;
}

/* ---- O3: brute-force distance from samples to the generator curves ------- */
/* For each of the W*H*16 samples (pattern of O2), the distance to the union of
 * the path's generator curves g(t), t in [0,1]: dense sampling (n_dense
 * points per segment) followed by golden-section refinement around every
 * local minimum of the sampled distance.  With round joins and caps the
 * stroked region is exactly {x : dist(x, curves) <= w/2} (Sec. 3.2: normal
 * segments of length w/2 cover every point whose nearest curve point is
 * interior; caps, joins and cusp pivots are discs at the remaining nearest
 * points).  out_dist[(y*W + x)*16 + k]. */
static double seg_dist2(const Seg* g, V2 S, double t) {
  V2 d = sub(seg_eval(g, t), S);
  return dot(d, d);
}

int orc_centreline_distance(int64_t n_seg, const uint8_t* seg_type, const float* seg_pts,
                            const float* seg_w, int W, int H, int n_dense, double* out_dist) {
  if (n_dense < 16 || W <= 0 || H <= 0) return ORC_ERR_INVALID;
  V2* dense = (V2*)malloc(sizeof(V2) * (size_t)n_seg * (n_dense + 1));
  if (!dense) return ORC_ERR_INVALID;
  Seg* segs = (Seg*)malloc(sizeof(Seg) * (size_t)(n_seg ? n_seg : 1));
  for (int64_t i = 0; i < n_seg; ++i) {
    double q8[8];
    for (int c = 0; c < 8; ++c) q8[c] = seg_pts[8 * i + c];
    double wi = seg_w ? (double)seg_w[i] : 1.0;
    segs[i] = load_seg(0, seg_type + i, q8, &wi);
    for (int m = 0; m <= n_dense; ++m)
      dense[i * (n_dense + 1) + m] = seg_eval(&segs[i], (double)m / n_dense);
  }
  const double gr = 0.5 * (sqrt(5.0) - 1.0);
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x)
      for (int k = 0; k < 16; ++k) {
        V2 S = mk(x + (16.0 * k + 8.0) / 256.0, y + (16.0 * ((5 * k) % 16) + 8.0) / 256.0);
        double best = INFINITY;
        for (int64_t i = 0; i < n_seg; ++i) {
          const V2* D = dense + i * (n_dense + 1);
          for (int m = 0; m <= n_dense; ++m) {
            V2 dd = sub(D[m], S);
            double d2 = dot(dd, dd);
            double dl = m > 0 ? dot(sub(D[m - 1], S), sub(D[m - 1], S)) : INFINITY;
            double dr = m < n_dense ? dot(sub(D[m + 1], S), sub(D[m + 1], S)) : INFINITY;
            if (d2 < best) best = d2;
            if (d2 <= dl && d2 <= dr) {
              /* refine on [t_{m-1}, t_{m+1}] by golden section */
              double lo = (m > 0 ? m - 1 : 0) / (double)n_dense;
              double hi = (m < n_dense ? m + 1 : n_dense) / (double)n_dense;
              double c1 = hi - gr * (hi - lo), c2 = lo + gr * (hi - lo);
              double f1 = seg_dist2(&segs[i], S, c1), f2 = seg_dist2(&segs[i], S, c2);
              for (int it = 0; it < 60; ++it) {
                if (f1 < f2) { hi = c2; c2 = c1; f2 = f1; c1 = hi - gr * (hi - lo); f1 = seg_dist2(&segs[i], S, c1); }
                else { lo = c1; c1 = c2; f1 = f2; c2 = lo + gr * (hi - lo); f2 = seg_dist2(&segs[i], S, c2); }
              }
              double fm = f1 < f2 ? f1 : f2;
              if (fm < best) best = fm;
            }
          }
        }
        out_dist[((int64_t)y * W + x) * 16 + k] = sqrt(best);
      }
  free(dense);
  free(segs);
  return ORC_OK;
}

/* ---- uniform parametric tessellation and facet angles (Sec. 8.1) --------- */
/* The comparison of Sec. 8.1 strokes a segment with Eq. 1 sampled at uniform
 * parameters: rib j of N+1 at t_j = j/N is g(t_j) -+ r n(t_j), with n(t) the
 * unit left normal of g'(t) (the same N/P convention as the polar ribs).  Where
 * g'(t) = 0 (an exact cusp) the direction of g''(t) stands in for the tangent;
 * a segment whose hodograph vanishes everywhere uses its chord.  N is set by
 * the caller (the polar quad count of the same segment). */
int orc_uniform_ribs(int type, const double* pts8, double w, int N, double r, double* rib) {
  if (N < 1 || !pts8 || !rib) return ORC_ERR_INVALID;
  Seg g;
  g.type = type;
  g.A = mk(pts8[0], pts8[1]); g.B = mk(pts8[2], pts8[3]);
  g.C = mk(pts8[4], pts8[5]); g.D = mk(pts8[6], pts8[7]);
  g.w = w;
  for (int j = 0; j <= N; ++j) {
    double t = (double)j / (double)N;
    V2 p = seg_eval(&g, t);
    V2 T = hodo(&g, t);
    double L = sqrt(T.x * T.x + T.y * T.y);
    if (L == 0.0) {
      T = hodo_d(&g, t);
      L = sqrt(T.x * T.x + T.y * T.y);
    }
    if (L == 0.0) {
      T = sub(g.D, g.A);
      L = sqrt(T.x * T.x + T.y * T.y);
    }
    V2 n = L > 0.0 ? mk(-T.y / L, T.x / L) : mk(0.0, 0.0);
    rib[4 * j + 0] = p.x - r * n.x;
    rib[4 * j + 1] = p.y - r * n.y;
    rib[4 * j + 2] = p.x + r * n.x;
    rib[4 * j + 3] = p.y + r * n.y;
  }
  return ORC_OK;
}

/* Facet angles of one run of ribs (one segment's quads): for each interior rib
 * j and each side X in {N, P}, the angle in [0, pi] between the boundary edges
 * X_j - X_{j-1} and X_{j+1} - X_j, where one quad meets the next (Sec. 4.2's
 * facet angle).  Sec. 4.2 bounds it by 2q except next to offset cusps: an
 * offset arc without a cusp has its chord direction between the tangent
 * directions at its ends, and those are the generator's (the offset's tangent
 * is the generator's, reversed only through a cusp).  So a facet is ordinary
 * when each of its two edges points within the angle between the tangents of
 * its end ribs (the rib P - N is the left normal, turned clockwise it is the
 * tangent), within a slack (unit-vector cross products; 1e-12 for FP64 ribs).
 * A rib of zero length carries no tangent; there an
 * edge counts when it advances with the centreline edge ((N+P)/2) of the same
 * index.  angle[2j+s] is -1 where an edge has zero length (ribs 0 and n-1 have
 * no facet). */
static int edge_regular(const double* rib, int64_t i0, int64_t i1, int s, V2 e, double eps) {
  V2 v0 = mk(rib[4 * i0 + 2] - rib[4 * i0], rib[4 * i0 + 3] - rib[4 * i0 + 1]);
  V2 v1 = mk(rib[4 * i1 + 2] - rib[4 * i1], rib[4 * i1 + 3] - rib[4 * i1 + 1]);
  double l0 = sqrt(v0.x * v0.x + v0.y * v0.y), l1 = sqrt(v1.x * v1.x + v1.y * v1.y);
  double le = sqrt(e.x * e.x + e.y * e.y);
  if (l0 == 0.0 || l1 == 0.0) {
    V2 m0 = mk(0.5 * (rib[4 * i0] + rib[4 * i0 + 2]), 0.5 * (rib[4 * i0 + 1] + rib[4 * i0 + 3]));
    V2 m1 = mk(0.5 * (rib[4 * i1] + rib[4 * i1 + 2]), 0.5 * (rib[4 * i1 + 1] + rib[4 * i1 + 3]));
    V2 m = sub(m1, m0);
    (void)s;
    return e.x * m.x + e.y * m.y > 0.0;
  }
  V2 T0 = mk(v0.y / l0, -v0.x / l0), T1 = mk(v1.y / l1, -v1.x / l1);
  V2 u = mk(e.x / le, e.y / le);
  double c01 = T0.x * T1.y - T0.y * T1.x;
  double c0u = T0.x * u.y - T0.y * u.x, cu1 = u.x * T1.y - u.y * T1.x;
  if (u.x * (T0.x + T1.x) + u.y * (T0.y + T1.y) <= 0.0) return 0;  /* backwards */
  if (c01 >= 0.0) return c0u >= -eps && cu1 >= -eps;  /* counter-clockwise step */
  return c0u <= eps && cu1 <= eps;                     /* clockwise step */
}

int orc_facet_angles(int64_t n, const double* rib, double slack, double* angle,
                     uint8_t* ordinary) {
  if (n < 0 || (n > 0 && (!rib || !angle || !ordinary))) return ORC_ERR_INVALID;
  for (int64_t j = 0; j < n; ++j) {
    for (int s = 0; s < 2; ++s) {
      angle[2 * j + s] = -1.0;
      ordinary[2 * j + s] = 0;
      if (j == 0 || j == n - 1) continue;
      V2 a = mk(rib[4 * (j - 1) + 2 * s], rib[4 * (j - 1) + 2 * s + 1]);
      V2 b = mk(rib[4 * j + 2 * s], rib[4 * j + 2 * s + 1]);
      V2 c = mk(rib[4 * (j + 1) + 2 * s], rib[4 * (j + 1) + 2 * s + 1]);
      V2 e0 = sub(b, a), e1 = sub(c, b);
      if ((e0.x == 0.0 && e0.y == 0.0) || (e1.x == 0.0 && e1.y == 0.0)) continue;
      angle[2 * j + s] = fabs(atan2(e0.x * e1.y - e0.y * e1.x, e0.x * e1.x + e0.y * e1.y));
      ordinary[2 * j + s] =
          (edge_regular(rib, j - 1, j, s, e0, slack) && edge_regular(rib, j, j + 1, s, e1, slack))
              ? 1 : 0;
    }
  }
  return ORC_OK;
}

/* ---- dashing with capped dash ends (Sec. 5.2, reading R18) ---------------- */
/* As orc_dash, and every on-stretch [a, b) gets the path's cap style at its
 * ends inside the path: a start cap where 0 < a lies in a segment quad
 * [s_{j-1}, s_j), an end cap where b lies in (s_{j-1}, s_j].  A cap is the
 * path cap of Sec. 4.3.5 (reading R7) about the boundary rib: centre the rib's
 * midpoint, radius half its length, tangent the rib turned clockwise; a start
 * cap pivots from psi + pi, an end cap from psi, both through +pi.  Its J+1
 * ribs (J from the cap style, none for butt) form a strip of their own at the
 * boundary's s, written right before the stretch's first piece (start cap) or
 * right after its last piece (end cap).  path_cap[p] is path p's cap style. */
static int64_t dash_cap(int64_t n, int64_t cap, const double* rib, int64_t j, double f, double sv,
                        uint32_t path, int style, double q, int start, double* out_rib,
                        double* out_s, uint32_t* out_tag, int64_t* out_src) {
  int J = cap_count(style, q);
  if (J <= 0) return 0;
  double v[4];
  for (int c = 0; c < 4; ++c) {
    double v0 = rib[4 * (j - 1) + c], v1 = rib[4 * j + c];
    v[c] = v0 + f * (v1 - v0);
  }
  double vx = v[2] - v[0], vy = v[3] - v[1];
  double r = 0.5 * sqrt(vx * vx + vy * vy);
  double psi = atan2(-vx, vy); /* the rib is 2r n(psi), n = (-sin psi, cos psi) */
  Link L;
  memset(&L, 0, sizeof L);
  L.kind = 3;
  L.style = style;
  L.at = mk(0.5 * (v[0] + v[2]), 0.5 * (v[1] + v[3]));
  L.Psi0 = start ? psi + PI : psi;
  L.delta = PI;
  if (out_rib && n + J + 1 <= cap) {
    V2* Nv = (V2*)malloc(sizeof(V2) * (size_t)(J + 1));
    V2* Pv = (V2*)malloc(sizeof(V2) * (size_t)(J + 1));
    double* ps_ = (double*)malloc(sizeof(double) * (size_t)(J + 1));
    if (!Nv || !Pv || !ps_) {
      free(Nv); free(Pv); free(ps_);
      return 0;
    }
    emit_pivot(&L, J, r, Nv, Pv, ps_);
    for (int k = 0; k <= J; ++k) {
      out_rib[4 * (n + k) + 0] = Nv[k].x;
      out_rib[4 * (n + k) + 1] = Nv[k].y;
      out_rib[4 * (n + k) + 2] = Pv[k].x;
      out_rib[4 * (n + k) + 3] = Pv[k].y;
      out_s[n + k] = sv;
      out_tag[n + k] = (path << 2) | (k == 0 ? TAG_LINK_START : 0u);
      out_src[n + k] = j;
    }
    free(Nv); free(Pv); free(ps_);
  }
  return J + 1;
}

int orc_dash_capped(int64_t R, const double* rib, const double* s, const uint32_t* tag,
                    const double* pattern, int m, double offset, const uint8_t* path_cap,
                    int64_t n_path, double q, int64_t cap, double* out_rib, double* out_s,
                    uint32_t* out_tag, int64_t* out_src, int64_t* n_out) {
  if (m <= 0 || m > 32 || !(q > 0.0) || (n_path > 0 && !path_cap)) return ORC_ERR_INVALID;
  int m2 = (m % 2) ? 2 * m : m;
  double cum[65];
  cum[0] = 0.0;
  for (int i = 0; i < m2; ++i) {
    double d = pattern[i % m];
    if (!(d >= 0.0)) return ORC_ERR_INVALID;
    cum[i + 1] = cum[i] + d;
  }
  double period = cum[m2];
  if (!(period > 0.0)) return ORC_ERR_INVALID;
  int64_t n = 0;
  for (int64_t j = 1; j < R; ++j) {
    if (tag[j] & TAG_LINK_START) continue;
    double sa = s[j - 1], sb = s[j];
    uint32_t tg = tag[j] & ~TAG_LINK_START;
    uint32_t path = tag[j] >> 2;
    if ((int64_t)path >= n_path) return ORC_ERR_INVALID;
    int style = path_cap[path];
    double k0 = floor((sa + offset) / period) - 1.0;
    for (double k = k0;; k += 1.0) {
      double base = k * period;
      if (base - offset > sb) break;
      for (int i = 0; i < m2; i += 2) {
        double a = (base + cum[i]) - offset, b = (base + cum[i + 1]) - offset;
        if (!(b > a)) continue;
        if (sb > sa) {
          double lo = a > sa ? a : sa, hi = b < sb ? b : sb;
          if (hi > lo) {
            double f0 = (lo - sa) / (sb - sa), f1 = (hi - sa) / (sb - sa);
            if (a >= sa && a < sb && a > 0.0)
              n += dash_cap(n, cap, rib, j, f0, lo, path, style, q, 1, out_rib, out_s, out_tag,
                            out_src);
            dash_put(n, cap, rib, j, f0, f1, lo, hi, tg, out_rib, out_s, out_tag, out_src);
            n += 2;
            if (b > sa && b <= sb)
              n += dash_cap(n, cap, rib, j, f1, hi, path, style, q, 0, out_rib, out_s, out_tag,
                            out_src);
          }
        } else if (sa >= a && sa < b) { /* zero-length quad kept whole */
          dash_put(n, cap, rib, j, 0.0, 1.0, sa, sb, tg, out_rib, out_s, out_tag, out_src);
          n += 2;
        }
      }
    }
  }
  *n_out = n;
  return n > cap ? ORC_ERR_CAPACITY : ORC_OK;
}
