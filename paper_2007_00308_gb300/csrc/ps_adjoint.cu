// Adjoint of the tessellation: gradients of the rib vertices (N_j, P_j) and of
// the cumulative arc length s_j with respect to the control points and the
// stroke widths, at the forward pass's fixed step counts.
//
// Each rib depends on the control points through its centreline point g(t_j)
// and its normal angle psi_j (Eq. 14-17).  For a rib solved by Eq. 11,
// F(t, psi, P) = H(t; P) . N(psi) = 0 is differentiated implicitly:
//   dt = -(dF/dP dP + dF/dpsi dpsi) / (dF/dt),  dF/dpsi = -H . T(psi).
// psi_j interpolates the interval's boundary angles (psi(j) of Sec. 4.2.1), so
// its adjoint is split between the two boundaries; boundary angles come from
// Table 1's end gradients, from H at an inflection (where H x H' = 0, so the
// inflection's own motion drops out), or from a split (their mean).  An
// inflection point's parameter moves with the root of the curvature polynomial.
// Arc length is the sum of chords (Eq. 18): a reverse (suffix) sum of dL/ds
// weights each chord's direction.
#include <cuda_runtime.h>

#include "ps_geom.cuh"
#include "ps_internal.cuh"

namespace {
using namespace ps;

// link sources: kind, main segment (segment / capped segment), incoming and
// outgoing segments of a join, cap end (0 start, 1 stop)
struct LinkSrc {
  int kind, seg, seg_in, seg_out, cap_end, path;
};

__device__ __forceinline__ int find_path_a(const int32_t* seg_off, int n_path, int64_t l) {
  int lo = 0, hi = n_path;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    int64_t lb = 2 * (int64_t)__ldg(seg_off + mid) + mid;
    if (lb <= l) lo = mid; else hi = mid;
  }
  return lo;
}

// The segments a link reads (same rules as the forward's link setup).
__device__ LinkSrc link_src(const uint8_t* st, const float* sp, const float* sw,
                            const int32_t* seg_off, const uint8_t* closed, int n_path, int64_t l) {
  LinkSrc R{0, -1, -1, -1, 0, 0};
  int p = find_path_a(seg_off, n_path, l);
  R.path = p;
  int s0 = __ldg(seg_off + p), n = __ldg(seg_off + p + 1) - s0;
  int k = (int)(l - (2 * (int64_t)s0 + p));
  bool cl = closed[p] != 0;
  if (n <= 0) return R;
  if (k & 1) {
    R.kind = LK_SEG;
    R.seg = s0 + (k - 1) / 2;
    return R;
  }
  auto nd = [&](int i) { return !zero_length(load_seg(st, sp, sw, s0 + i)); };
  if (k == 0 || k == 2 * n) {
    int first = -1, last = -1;
    for (int i = 0; i < n; ++i)
      if (nd(i)) { first = i; break; }
    for (int i = n - 1; i >= 0; --i)
      if (nd(i)) { last = i; break; }
    if (first < 0) return R;
    if (!cl) {
      R.kind = LK_CAP;
      R.seg = s0 + (k == 0 ? first : last);
      R.cap_end = k == 0 ? 0 : 1;
    } else if (k == 2 * n) {
      R.kind = LK_JOIN;
      R.seg_in = s0 + last;
      R.seg_out = s0 + first;
    }
    return R;
  }
  int i = k / 2 - 1;
  if (!nd(i + 1)) return R;
  for (int m = i; m >= 0; --m)
    if (nd(m)) {
      R.kind = LK_JOIN;
      R.seg_in = s0 + m;
      R.seg_out = s0 + i + 1;
      break;
    }
  return R;
}

// ---- per-form weights ------------------------------------------------------
// g(t) = sum_i b[i] P_i and H(t) = sum_i beta[i] P_i over the slots A, B, C, D
// (the quadratic and conic have no C: their middle point is B).
__device__ __forceinline__ void weights(const Seg& g, float t, float* b, float* beta, float& c,
                                        float2& H, float2& Hd) {
  float u = 1.f - t;
  switch (g.type) {
    case PS_CUBIC:
      b[0] = u * u * u; b[1] = 3.f * u * u * t; b[2] = 3.f * u * t * t; b[3] = t * t * t;
      beta[0] = -u * u; beta[1] = u * u - 2.f * u * t; beta[2] = 2.f * u * t - t * t; beta[3] = t * t;
      c = 3.f;
      Hd = (g.B - g.A) * (-2.f * u) + (g.C - g.B) * (2.f * (u - t)) + (g.D - g.C) * (2.f * t);
      break;
    case PS_QUAD:
      b[0] = u * u; b[1] = 2.f * u * t; b[2] = 0.f; b[3] = t * t;
      beta[0] = -u; beta[1] = u - t; beta[2] = 0.f; beta[3] = t;
      c = 2.f;
      Hd = (g.D - g.B) - (g.B - g.A);
      break;
    case PS_CONIC: {
      // the denominator in its cancellation-free form (as in g_rel)
      float w = g.w, s12 = 1.f - 2.f * t, den = s12 * s12 + 2.f * (1.f + w) * u * t;
      b[0] = u * u / den; b[1] = 2.f * u * t * w / den; b[2] = 0.f; b[3] = t * t / den;
      beta[0] = -w * u * u - u * t; beta[1] = w * u * u - w * t * t; beta[2] = 0.f;
      beta[3] = u * t + w * t * t;
      c = 2.f / (den * den);
      Hd = (g.B - g.A) * (-2.f * u * w) + (g.D - g.A) * (u - t) + (g.D - g.B) * (2.f * t * w);
      break;
    }
    default:
      b[0] = u; b[1] = 0.f; b[2] = 0.f; b[3] = t;
      beta[0] = -1.f; beta[1] = 0.f; beta[2] = 0.f; beta[3] = 1.f;
      c = 1.f;
      Hd = mk(0.f, 0.f);
  }
  H = hodo(g, t);
}

// Control points (slot order A, B, C, D) that Table 1's end gradient reads, with
// signs: e = sum_i coef[i] P_i.
__device__ __forceinline__ float2 end_grad_coef(const Seg& g, int end, float* coef) {
  coef[0] = coef[1] = coef[2] = coef[3] = 0.f;
  float sg = g.w > 0.f ? 1.f : -1.f;
  if (end == 0) {
    switch (g.type) {
      case PS_CUBIC:
        if (!is0(g.B - g.A)) { coef[1] = 1.f; coef[0] = -1.f; }
        else if (!is0(g.C - g.A)) { coef[2] = 1.f; coef[0] = -1.f; }
        else { coef[3] = 1.f; coef[0] = -1.f; }
        break;
      case PS_QUAD:
        if (!is0(g.B - g.A)) { coef[1] = 1.f; coef[0] = -1.f; }
        else { coef[3] = 1.f; coef[0] = -1.f; }
        break;
      case PS_CONIC:
        if (!is0(g.B - g.A) && g.w != 0.f) { coef[1] = sg; coef[0] = -sg; }
        else { coef[3] = 1.f; coef[0] = -1.f; }
        break;
      default:
        coef[3] = 1.f; coef[0] = -1.f;
    }
    return end_grad0(g);
  }
  switch (g.type) {
    case PS_CUBIC:
      if (!is0(g.D - g.C)) { coef[3] = 1.f; coef[2] = -1.f; }
      else if (!is0(g.D - g.B)) { coef[3] = 1.f; coef[1] = -1.f; }
      else { coef[3] = 1.f; coef[0] = -1.f; }
      break;
    case PS_QUAD:
      if (!is0(g.D - g.B)) { coef[3] = 1.f; coef[1] = -1.f; }
      else { coef[3] = 1.f; coef[0] = -1.f; }
      break;
    case PS_CONIC:
      if (!is0(g.D - g.B) && g.w != 0.f) { coef[3] = sg; coef[1] = -sg; }
      else { coef[3] = 1.f; coef[0] = -1.f; }
      break;
    default:
      coef[3] = 1.f; coef[0] = -1.f;
  }
  return end_grad1(g);
}

// gradient slot of control point i of segment s (quadratic / conic C -> B)
__device__ __forceinline__ void add_pt(float* gp, int64_t s, int type, int i, float2 v) {
  if (v.x == 0.f && v.y == 0.f) return;
  int slot = (i == 2 && (type == PS_QUAD || type == PS_CONIC)) ? 1 : i;
  atomicAdd(gp + 8 * s + 2 * slot, v.x);
  atomicAdd(gp + 8 * s + 2 * slot + 1, v.y);
}

// d atan2(v) / dv
__device__ __forceinline__ float2 dang(float2 v) {
  float l2 = dot2(v, v);
  return l2 > 0.f ? mk(-v.y / l2, v.x / l2) : mk(0.f, 0.f);
}

__device__ __forceinline__ int find_link_a(const int32_t* off, int64_t lo, int64_t hi, int64_t r) {
  while (hi > lo) {
    int64_t mid = (lo + hi + 1) >> 1;
    if ((int64_t)__ldg(off + mid) <= r) lo = mid; else hi = mid - 1;
  }
  return (int)lo;
}

__global__ void k_adj_links(const uint8_t* st, const float* sp, const float* sw,
                            const int32_t* seg_off, const uint8_t* closed, int n_path,
                            int64_t n_link, int4* src) {
  int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= n_link) return;
  LinkSrc R = link_src(st, sp, sw, seg_off, closed, n_path, l);
  int a = R.kind == LK_JOIN ? R.seg_in : R.seg;
  int b = R.kind == LK_JOIN ? R.seg_out : R.cap_end;
  src[l] = make_int4(R.kind, a, b, R.path);
}

// Sum of v over the lanes from this one to the end of its run of equal keys
// (runs of a key are contiguous); exact at the run's first lane.
__device__ __forceinline__ float run_sum(float v, long long key) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    float y = __shfl_down_sync(0xffffffffu, v, o);
    long long ky = __shfl_down_sync(0xffffffffu, key, o);
    if (lane + o < 32 && ky == key) v += y;
  }
  return v;
}

__device__ __forceinline__ bool run_head(long long key) {
  long long kp = __shfl_up_sync(0xffffffffu, key, 1);
  return (threadIdx.x & 31) == 0 || kp != key;
}

// Per rib: gradients of g(t_j), psi_j, r, for the control points, the link's
// boundary-angle adjoints and the path width.  A warp takes 32 consecutive
// ribs (mostly of one link), sums their contributions per target with
// segmented shuffles, and the first lane of each run adds them atomically:
// every rib of a segment adds to the same few words, so adding per rib would
// serialize on them.
__global__ void __launch_bounds__(256) k_adj_ribs(
    const LinkRec* __restrict__ recs, const int4* __restrict__ src,
    const int32_t* __restrict__ link_off, int64_t n_link, const int64_t* __restrict__ n_rib,
    int64_t capacity, const float4* __restrict__ rib, const float* __restrict__ tf,
    const float4* __restrict__ grib, const float* __restrict__ suffix,
    const uint8_t* __restrict__ stype, float* __restrict__ gpts, float* __restrict__ adj_psi,
    float* __restrict__ gwidth) {
  int64_t R = *n_rib;
  if (R > capacity) R = capacity;
  const int lane = threadIdx.x & 31;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < R;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = base + lane;
    const bool act = r < R;
    // link of rib r: one search for the warp's first rib, then a short walk
    int l = 0;
    if (lane == 0) l = find_link_a(link_off, 0, n_link - 1, base);
    l = __shfl_sync(0xffffffffu, l, 0);
    if (act)
      while (l + 1 < n_link && (int64_t)__ldg(link_off + l + 1) <= r) ++l;
    // this rib's contributions: point gradients of segment seg_t (slots 0..3),
    // the path width, and the boundary angles kslot, kslot + 1 of link l
    float P8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int seg_t = -1, path_t = -1, kslot = 0;
    float gw = 0.f, psA = 0.f, psB = 0.f;
    const LinkRec* L = recs + l;
    const uint32_t meta = act ? __ldg(&L->meta) : 0u;
    const int kind = META_KIND(meta);
    const int j = act ? (int)(r - __ldg(link_off + l)) : 0;
    const int nr = act ? __ldg(link_off + l + 1) - __ldg(link_off + l) : 0;
    // The chords of Eq. 18 beside this rib: their directions from the
    // centreline points g(t) - A in double-float, differenced before rounding
    // (a short chord between points far from A keeps its direction); the
    // neighbours' points come from the neighbouring lanes of the same link.
    Seg g;
    float t = 0.f;
    DF2 gc{{0.f, 0.f}, {0.f, 0.f}};
    if (kind == LK_SEG) {
      const float4 p01 = __ldg(reinterpret_cast<const float4*>(L->P));
      const float4 p23 = __ldg(reinterpret_cast<const float4*>(L->P) + 1);
      g.type = META_TYPE(meta);
      g.A = mk(p01.x, p01.y); g.B = mk(p01.z, p01.w); g.C = mk(p23.x, p23.y); g.D = mk(p23.z, p23.w);
      g.w = __ldg(&L->w);
      t = __ldg(tf + r);
      gc = g_rel_comp_df(g, t);
    }
    DF2 gprev, gnext;
    gprev.x.hi = __shfl_up_sync(0xffffffffu, gc.x.hi, 1);
    gprev.x.lo = __shfl_up_sync(0xffffffffu, gc.x.lo, 1);
    gprev.y.hi = __shfl_up_sync(0xffffffffu, gc.y.hi, 1);
    gprev.y.lo = __shfl_up_sync(0xffffffffu, gc.y.lo, 1);
    gnext.x.hi = __shfl_down_sync(0xffffffffu, gc.x.hi, 1);
    gnext.x.lo = __shfl_down_sync(0xffffffffu, gc.x.lo, 1);
    gnext.y.hi = __shfl_down_sync(0xffffffffu, gc.y.hi, 1);
    gnext.y.lo = __shfl_down_sync(0xffffffffu, gc.y.lo, 1);
    if (kind == LK_SEG) {
      if (lane == 0 && j > 0) gprev = g_rel_comp_df(g, __ldg(tf + r - 1));
      if (lane == 31 && j + 1 < nr) gnext = g_rel_comp_df(g, __ldg(tf + r + 1));
    }
    if (act) {
    int4 sc = __ldg(src + l);
    float4 G = __ldg(grib + r);
    float2 GN = mk(G.x, G.y), GP = mk(G.z, G.w);
    float rN = __ldg(&L->rN), rP = __ldg(&L->rP);
    if (kind == LK_SEG) {
      int M = META_M(meta);
      int k = 0;
      while (k < M && j >= (int)__ldg(&L->dsum[k + 1])) ++k;
      int dk = (int)__ldg(&L->dsum[k]);
      bool boundary = (j == dk);
      float psi, lam = 0.f;
      if (boundary) psi = __ldg(&L->psi[k]);
      else {
        int Dk = (int)__ldg(&L->dsum[k + 1]) - dk;
        psi = __ldg(&L->psi[k]) + __ldg(&L->step[k]) * (float)(j - dk);
        lam = (float)(j - dk) / (float)Dk;
      }
      float sn, cs;
      sincosf(psi, &sn, &cs);
      float2 n = mk(-sn, cs), T = mk(cs, sn);
      // upstream on the centreline point: both vertices, and the chords to the
      // neighbouring ribs of this link (Eq. 18; a step with decreasing t adds 0)
      float2 Gg = GN + GP;
      if (j > 0 && t >= __ldg(tf + r - 1)) {
        float2 d = mk(df_f(df_sub(gc.x, gprev.x)), df_f(df_sub(gc.y, gprev.y)));
        float len = sqrtf(dot2(d, d));
        if (len > 0.f) Gg = Gg + d * (__ldg(suffix + r) / len);
      }
      if (j + 1 < nr && __ldg(tf + r + 1) >= t) {
        float2 d = mk(df_f(df_sub(gnext.x, gc.x)), df_f(df_sub(gnext.y, gc.y)));
        float len = sqrtf(dot2(d, d));
        if (len > 0.f) Gg = Gg - d * (__ldg(suffix + r + 1) / len);
      }
      // N = g - rN n, P = g + rP n: dN/dpsi = rN T, dP/dpsi = -rP T
      float Gpsi = rN * dot2(T, GN) - rP * dot2(T, GP);
      float Gr = -dot2(n, GN) + dot2(n, GP);  // rN = rP = w/2 on segment links
      gw = 0.5f * Gr;
      path_t = sc.w;
      float b[4], beta[4], c;
      float2 H, Hd;
      weights(g, t, b, beta, c, H, Hd);
      float2 Nn = n;  // N(psi) = <-sin, cos>
      bool pivot = META_PIVOT(meta, k) && !boundary;
      bool solved = !boundary && !pivot && g.type != PS_LINE;
      bool at_split = boundary && k > 0 && k < M && META_SPLIT(meta, k);
      bool at_infl = boundary && k > 0 && k < M && !META_SPLIT(meta, k) && !META_PIVOT(meta, k) &&
                     !(k > 0 && META_PIVOT(meta, k - 1)) && g.type == PS_CUBIC;
      float dLdt = c * dot2(Gg, H);
      float pt[4][2];
      for (int i = 0; i < 4; ++i) {
        pt[i][0] = b[i] * Gg.x;
        pt[i][1] = b[i] * Gg.y;
      }
      if (solved || at_split) {
        float Ft = dot2(Hd, Nn);
        if (fabsf(Ft) > 1e-20f) {
          float kap = -dLdt / Ft;
          for (int i = 0; i < 4; ++i) {
            pt[i][0] += kap * beta[i] * Nn.x;
            pt[i][1] += kap * beta[i] * Nn.y;
          }
          Gpsi += kap * (-dot2(H, T));
        }
      } else if (at_infl) {
        // t = p, a root of the curvature polynomial C(t) = X12 u^2 + X13 u t + X23 t^2
        float2 d1 = g.B - g.A, d2 = g.C - g.B, d3 = g.D - g.C;
        float u = 1.f - t;
        float X12 = cross2(d1, d2), X13 = cross2(d1, d3), X23 = cross2(d2, d3);
        float Cp = -2.f * u * X12 + (u - t) * X13 + 2.f * t * X23;
        if (fabsf(Cp) > 1e-20f) {
          auto J = [](float2 v) { return mk(v.y, -v.x); };
          float2 c1 = J(d2) * (u * u) + J(d3) * (u * t);
          float2 c2 = J(d1) * (-u * u) + J(d3) * (t * t);
          float2 c3 = J(d1) * (-u * t) + J(d2) * (-t * t);
          float2 dC[4] = {c1 * -1.f, c1 - c2, c2 - c3, c3};
          float f = -dLdt / Cp;
          for (int i = 0; i < 4; ++i) {
            pt[i][0] += f * dC[i].x;
            pt[i][1] += f * dC[i].y;
          }
        }
      }
      seg_t = sc.y;
      for (int i = 0; i < 4; ++i) {
        // quadratic / conic: C's gradient goes to B's slot
        int slot = (i == 2 && (g.type == PS_QUAD || g.type == PS_CONIC)) ? 1 : i;
        P8[2 * slot] += pt[i][0];
        P8[2 * slot + 1] += pt[i][1];
      }
      // psi's adjoint to the interval's boundary angles
      kslot = k;
      psA = boundary ? Gpsi : (1.f - lam) * Gpsi;
      psB = boundary ? 0.f : lam * Gpsi;
    } else if (kind == LK_JOIN || kind == LK_CAP) {
      int J = (int)__ldg(&L->dsum[1]);
      float psi = (j == J) ? __ldg(&L->psi[1]) : __ldg(&L->psi[0]) + __ldg(&L->step[0]) * (float)j;
      float sn, cs;
      sincosf(psi, &sn, &cs);
      float2 n = mk(-sn, cs), T = mk(cs, sn);
      float sq = ((meta & META_FLAG_SQUARE) && (j == 1 || j == 3)) ? 1.41421356237309515f : 1.f;
      bool ovr = (meta & META_FLAG_OVERRIDE) && (j == 1 || j == 2);
      // the pivot point: the outgoing segment's A (join), the capped end (cap)
      float2 Gat = GN + GP;
      seg_t = kind == LK_JOIN ? sc.z : sc.y;
      int pslot = (kind == LK_CAP && sc.z == 1) ? 3 : 0;
      P8[2 * pslot] = Gat.x;
      P8[2 * pslot + 1] = Gat.y;
      path_t = sc.w;
      if (!ovr) {  // miter tips: the tip's motion with the angles and width is not followed
        float Gpsi, Gr;
        if (rN > 0.f) {  // N = at - sq r n
          Gpsi = sq * rN * dot2(T, GN);
          Gr = -sq * dot2(n, GN);
        } else {         // P = at + sq r n
          Gpsi = -sq * rP * dot2(T, GP);
          Gr = sq * dot2(n, GP);
        }
        gw = 0.5f * Gr;
        float fr = (float)j / (float)J;
        kslot = 0;
        if (kind == LK_JOIN) {
          psA = (1.f - fr) * Gpsi;
          psB = fr * Gpsi;
        } else {
          psA = Gpsi;  // delta = pi is constant
        }
      }
    }
    }  // act
    // sums per link (points, width) and per (link, interval) (angles)
    const long long key1 = act ? (long long)l : -1 - (long long)lane;
    const long long key2 = act ? 8 * (long long)l + kslot : -1 - (long long)lane;
    const bool h1 = run_head(key1), h2 = run_head(key2);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float v = run_sum(P8[i], key1);
      if (h1 && seg_t >= 0 && v != 0.f) atomicAdd(gpts + 8 * (int64_t)seg_t + i, v);
    }
    {
      float v = run_sum(gw, key1);
      if (h1 && path_t >= 0 && v != 0.f) atomicAdd(gwidth + path_t, v);
    }
    {
      float a = run_sum(psA, key2), b = run_sum(psB, key2);
      if (h2 && act) {
        if (a != 0.f) atomicAdd(adj_psi + 8 * (int64_t)l + kslot, a);
        if (b != 0.f) atomicAdd(adj_psi + 8 * (int64_t)l + kslot + 1, b);
      }
    }
  }
}

// Per link: boundary-angle adjoints -> control points.
__global__ void k_adj_finalize(const LinkRec* __restrict__ recs, const int4* __restrict__ src,
                               int64_t n_link, const uint8_t* st, const float* sp, const float* sw,
                               const float* __restrict__ adj_psi, float* __restrict__ gpts) {
  int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= n_link) return;
  int4 sc = src[l];
  const LinkRec* L = recs + l;
  uint32_t meta = L->meta;
  int kind = META_KIND(meta);
  if (kind == LK_EMPTY) return;
  float a[8];
  for (int k = 0; k < 8; ++k) a[k] = adj_psi[8 * l + k];
  float coef[4];
  if (kind == LK_SEG) {
    int M = META_M(meta);
    Seg g = load_seg(st, sp, sw, sc.y);
    bool flat = false;
    for (int k = 0; k < M; ++k) flat = flat || META_PIVOT(meta, k);
    if (flat) return;  // collinear pieces: angles fixed by the line direction
    // a split angle is the mean of its neighbours (Sec. 3.3.5)
    for (int k = 1; k < M; ++k)
      if (META_SPLIT(meta, k)) {
        a[k - 1] += 0.5f * a[k];
        a[k + 1] += 0.5f * a[k];
        a[k] = 0.f;
      }
    for (int k = 0; k <= M; ++k) {
      if (a[k] == 0.f) continue;
      if (k == 0 || k == M) {
        float2 e = end_grad_coef(g, k == 0 ? 0 : 1, coef);
        float2 dv = dang(e) * a[k];
        for (int i = 0; i < 4; ++i) add_pt(gpts, sc.y, g.type, i, dv * coef[i]);
      } else {
        // inflection: Psi = atan2 H(p); H x H' = 0 there, so only dH/dP counts
        float b[4], beta[4], c;
        float2 H, Hd;
        weights(g, L->p[k], b, beta, c, H, Hd);
        float2 dv = dang(H) * a[k];
        for (int i = 0; i < 4; ++i) add_pt(gpts, sc.y, g.type, i, dv * beta[i]);
      }
    }
  } else if (kind == LK_JOIN) {
    Seg ga = load_seg(st, sp, sw, sc.y), gb = load_seg(st, sp, sw, sc.z);
    float2 e1 = end_grad_coef(ga, 1, coef);
    float2 dv = dang(e1) * a[0];
    for (int i = 0; i < 4; ++i) add_pt(gpts, sc.y, ga.type, i, dv * coef[i]);
    float2 e0 = end_grad_coef(gb, 0, coef);
    dv = dang(e0) * a[1];
    for (int i = 0; i < 4; ++i) add_pt(gpts, sc.z, gb.type, i, dv * coef[i]);
  } else {
    Seg gc = load_seg(st, sp, sw, sc.y);
    float2 e = end_grad_coef(gc, sc.z == 0 ? 0 : 1, coef);
    float2 dv = dang(e) * a[0];
    for (int i = 0; i < 4; ++i) add_pt(gpts, sc.y, gc.type, i, dv * coef[i]);
  }
}

// suffix[r] = sum of dL/ds over ribs >= r of r's path = total - prefix + own
__global__ void k_adj_suffix(float* suf, const float* g, const float* tot, const uint32_t* tag,
                             const int64_t* n_rib, int64_t cap) {
  int64_t R = *n_rib;
  if (R > cap) R = cap;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R;
       r += (int64_t)gridDim.x * blockDim.x)
    suf[r] = tot[tag[r] >> 2] - suf[r] + g[r];
}

}  // namespace

extern "C" int ps_tessellate_backward(ps_context* ctx, const ps_segments* seg,
                                      const ps_paths* paths, float dtheta, int precision,
                                      const ps_tess_out* fwd, const float* d_grad_rib,
                                      const float* d_grad_s, float* d_grad_pts,
                                      float* d_grad_width, void* stream) {
  if (!ctx || !seg || !paths || !fwd) return PS_ERR_INVALID;
  // an empty batch has no gradients to write
  if (paths->n_path == 0 && seg->n_seg == 0) return PS_OK;
  if (!d_grad_rib || !d_grad_pts || !d_grad_width) return PS_ERR_INVALID;
  if (!fwd->d_rib || !fwd->d_tag || !fwd->d_t || !fwd->d_n_rib || fwd->capacity < 0)
    return PS_ERR_INVALID;
  if (precision != PS_PREC_FP32 && precision != PS_PREC_MIXED) return PS_ERR_INVALID;
  if (paths->n_path <= 0 || seg->n_seg < 0) return PS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = stream;
  int64_t S = seg->n_seg;
  int P = paths->n_path;
  int64_t L = 2 * S + P;
  int64_t cap = fwd->capacity;
  // workspace: offsets, link sources, boundary adjoints, suffix sums, path totals, n_rib
  size_t o_loff = 0;
  size_t o_poff = o_loff + sizeof(int32_t) * (L + 1);
  size_t o_src = (o_poff + sizeof(int32_t) * (P + 1) + 15) & ~(size_t)15;
  size_t o_adj = o_src + sizeof(int4) * L;
  size_t o_suf = o_adj + sizeof(float) * 8 * L;
  size_t o_tot = o_suf + sizeof(float) * (cap + 1);
  size_t o_nr = (o_tot + sizeof(float) * (P + 1) + 15) & ~(size_t)15;
  size_t bytes = o_nr + 16;
  if (bytes > ctx->adj_bytes) {
    if (ctx->d_adj) cudaFree(ctx->d_adj);
    ctx->d_adj = nullptr;
    if (cudaMalloc(&ctx->d_adj, bytes) != cudaSuccess) return PS_ERR_CUDA;
    ctx->adj_bytes = bytes;
  }
  char* w = (char*)ctx->d_adj;
  int32_t* loff = (int32_t*)(w + o_loff);
  int32_t* poff = (int32_t*)(w + o_poff);
  int4* src = (int4*)(w + o_src);
  float* adj = (float*)(w + o_adj);
  float* suf = (float*)(w + o_suf);
  float* tot = (float*)(w + o_tot);
  int64_t* nr = (int64_t*)(w + o_nr);
  int rc = ps_run_link_setup(ctx, seg, paths, dtheta, precision, loff, poff, nr, st);
  if (rc != PS_OK) return rc;
  k_adj_links<<<(unsigned)((L + 255) / 256), 256, 0, st>>>(seg->d_type, seg->d_pts, seg->d_w,
                                                          paths->d_seg_off, paths->d_closed, P, L,
                                                          src);
  // suffix sums of dL/ds within each path: total - inclusive prefix + own value
  cudaMemsetAsync(suf, 0, sizeof(float) * (cap + 1), st);
  if (d_grad_s) {
    cudaMemcpyAsync(suf, d_grad_s, sizeof(float) * cap, cudaMemcpyDeviceToDevice, st);
    if ((rc = ps_run_segmented_prefix(ctx, suf, fwd->d_tag, fwd->d_n_rib, cap, tot, P, st)) != PS_OK)
      return rc;
  }
  cudaMemsetAsync(adj, 0, sizeof(float) * 8 * L, st);
  cudaMemsetAsync(d_grad_pts, 0, sizeof(float) * 8 * S, st);
  cudaMemsetAsync(d_grad_width, 0, sizeof(float) * P, st);
  // convert prefix -> suffix in place
  if (d_grad_s)
    k_adj_suffix<<<ctx->num_sms * 8, 256, 0, st>>>(suf, d_grad_s, tot, fwd->d_tag, fwd->d_n_rib,
                                                  cap);
  int grid = ctx->num_sms * 8;
  k_adj_ribs<<<grid, 256, 0, st>>>(ctx->d_recs, src, fwd->d_link_rib_off, L, fwd->d_n_rib, cap,
                                   reinterpret_cast<const float4*>(fwd->d_rib), fwd->d_t,
                                   reinterpret_cast<const float4*>(d_grad_rib), suf, seg->d_type,
                                   d_grad_pts, adj, d_grad_width);
  k_adj_finalize<<<(unsigned)((L + 255) / 256), 256, 0, st>>>(ctx->d_recs, src, L, seg->d_type,
                                                              seg->d_pts, seg->d_w, adj,
                                                              d_grad_pts);
  return ps_cuda_check(cudaGetLastError());
}
