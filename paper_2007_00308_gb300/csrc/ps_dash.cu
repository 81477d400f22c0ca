// Dashing by cumulative arc length (Sec. 5.2).
//
// On-stretch i of period k covers s in [k*period + cum[2i] - offset,
// k*period + cum[2i+1] - offset).  Each quad [s_{r-1}, s_r] of a rib strip is
// clipped to those stretches by interpolating both rib vertices; every piece is
// an independent 2-rib strip.  A quad of zero length (join, cap, cusp pivot) is
// kept whole iff its s is "on".  Stretch boundaries are evaluated in FP64 with
// explicitly rounded operations (no contraction).
//
// With cap styles (ps_dash_capped), every stretch also gets its path's cap at
// its ends inside the path: a start cap where 0 < a lies in [s_{r-1}, s_r), an
// end cap where b lies in (s_{r-1}, s_r], each the path cap of Sec. 4.3.5
// (pivot through +pi, outer side N, inner radius 0) about the boundary rib --
// centre its midpoint, radius half its length, tangent the rib turned
// clockwise -- as a strip of its own at the boundary's s, written before the
// stretch's first piece or after its last.
#include <cuda_runtime.h>

#include "ps_internal.cuh"

namespace {

struct DashPattern {
  double cum[65];
  double period;
  double offset;
  float cum_f[65];             // the same in FP32, for the prefilter
  float period_f, period_lo;   // period = period_f + period_lo (+ ~2^-48 period)
  float offset_f;
  int m2;
  int j_round;                 // ribs - 1 of a round cap at this dtheta
  const uint8_t* path_cap;     // cap style per path, or null: butt dash ends
  int n_path;
};

__device__ __forceinline__ int cap_steps(const DashPattern& P, uint32_t path) {
  if (!P.path_cap || (int)path >= P.n_path) return 0;
  switch (P.path_cap[path]) {
    case PS_CAP_TRIANGLE: return 2;
    case PS_CAP_SQUARE: return 4;
    case PS_CAP_ROUND: return P.j_round;
    default: return 0;
  }
}

// Ribs k = 0..J of a dash cap about boundary rib v (start: pivot from psi + pi,
// end: from psi; both through +pi).
__device__ __forceinline__ void emit_cap(float4 v, int J, bool square, bool start, uint32_t tg,
                                         float sv, int32_t src, int64_t o, float4* out_rib,
                                         float* out_s, uint32_t* out_tag, int32_t* out_src) {
  const float PI_F = 3.14159265358979323846f;
  float cx = 0.5f * (v.x + v.z), cy = 0.5f * (v.y + v.w);
  float vx = v.z - v.x, vy = v.w - v.y;
  float r = 0.5f * sqrtf(vx * vx + vy * vy);
  float psi = atan2f(-vx, vy);  // the rib is 2r n(psi), n = (-sin psi, cos psi)
  float psi0 = start ? psi + PI_F : psi;
  for (int k = 0; k <= J; ++k) {
    float ang = k == J ? psi0 + PI_F : psi0 + PI_F * (float)k / (float)J;
    float sn, cs;
    sincosf(ang, &sn, &cs);
    float rn = (square && (k == 1 || k == 3)) ? r * 1.41421356237309515f : r;
    out_rib[o + k] = make_float4(cx + rn * sn, cy - rn * cs, cx, cy);
    out_s[o + k] = sv;
    out_tag[o + k] = (tg & ~(PS_TAG_SEGMENT | PS_TAG_LINK_START)) | (k == 0 ? PS_TAG_LINK_START : 0u);
    if (out_src) out_src[o + k] = src;
  }
}

constexpr int DASH_NT = 256;
constexpr int DASH_QPT = 4;  // quads per thread
constexpr int DASH_TILE = DASH_NT * DASH_QPT;

// End vertex of a whole quad as dash_quad computes it (f1 = 1): a0 + (a1 - a0)
// in FP64, which is a1 itself whenever a1 - a0 is exact in FP64 (exponents at
// most 28 apart, or a zero); otherwise the FP64 sum is taken as is.
__device__ __forceinline__ float whole_end(float a0, float a1) {
  const int e0 = (int)((__float_as_uint(a0) >> 23) & 0xffu);
  const int e1 = (int)((__float_as_uint(a1) >> 23) & 0xffu);
  if (a0 == 0.f || a1 == 0.f || abs(e0 - e1) <= 28) return a1;
  return (float)__dadd_rn((double)a0, __dsub_rn((double)a1, (double)a0));
}

// FP32 prefilter: whether the quad [sa, sb] lies inside one interval of the
// pattern (an on-stretch or a gap) with a margin eps above the FP32 error of
// its phase.  The phase of sa is computed with error-free steps: sa + offset as
// an exact float pair (TwoSum), k period_f exactly with its FMA residual, and
// the period's low part; what remains is a few roundings of values below two
// periods plus k * 2^-48 period, under 1e-6 of the period for k < 2^24, while
// the pattern's own FP32 rounding adds at most 2^-24 of it.  eps is 1e-4 of the
// period.  1: inside an on-stretch (the quad is emitted whole), 0: inside a gap
// (nothing), -1: within eps of a boundary (decided in FP64 by dash_quad).
__device__ __forceinline__ int dash_quick(const DashPattern& P, float sa, float sb) {
  const float per = P.period_f;
  const float eps = 1e-4f * per;
  const float u = sa + P.offset_f;  // TwoSum: u + ul == sa + offset exactly
  const float bv = u - sa;
  const float ul = (sa - (u - bv)) + (P.offset_f - bv);
  const float k = floorf(u / per);
  if (!(fabsf(k) < 16777216.f)) return -1;
  const float kp = k * per;
  const float ke = fmaf(k, per, -kp);  // k per == kp + ke exactly
  const float ph = (((u - kp) + ul) - ke) - k * P.period_lo;  // phase of sa
  if (!(ph >= 0.f && ph < per)) return -1;
  const float pe = ph + (sb - sa);  // phase of sb, beyond the period if it wraps
  int j = 0;  // interval [cum_f[j], cum_f[j+1]) holding ph
  while (j + 1 < P.m2 && P.cum_f[j + 1] <= ph) ++j;
  if (ph - P.cum_f[j] > eps && P.cum_f[j + 1] - pe > eps) return (j & 1) ? 0 : 1;
  return -1;
}

template <bool EMIT>
__device__ __forceinline__ int dash_quad(const DashPattern& P, double sa, double sb, int64_t r,
                                         const float4* rib, float sa_f, float sb_f,
                                         uint32_t tg, int64_t out0, float4* out_rib,
                                         float* out_s, uint32_t* out_tag, int32_t* out_src,
                                         int64_t out_cap, int32_t* status) {
  int n = 0;  // output ribs
  const int J = cap_steps(P, tg >> 2);
  const bool square = J == 4 && P.path_cap && P.path_cap[tg >> 2] == PS_CAP_SQUARE;
  double k0 = floor(__ddiv_rn(__dadd_rn(sa, P.offset), P.period)) - 1.0;
  float4 v0, v1;
  if (EMIT) {
    v0 = rib[r - 1];
    v1 = rib[r];
  }
  for (int guard = 0; guard < (1 << 20); ++guard) {
    double k = k0 + (double)guard;
    double base = __dmul_rn(k, P.period);
    if (__dsub_rn(base, P.offset) > sb) break;
    for (int i = 0; i < P.m2; i += 2) {
      double a = __dsub_rn(__dadd_rn(base, P.cum[i]), P.offset);
      double b = __dsub_rn(__dadd_rn(base, P.cum[i + 1]), P.offset);
      if (!(b > a)) continue;
      double lo, hi;
      bool keep;
      if (sb > sa) {
        lo = a > sa ? a : sa;
        hi = b < sb ? b : sb;
        keep = hi > lo;
      } else {
        lo = sa;
        hi = sb;
        keep = (sa >= a && sa < b);
      }
      if (!keep) continue;
      const bool cap0 = J > 0 && sb > sa && a >= sa && a < sb && a > 0.0;
      const bool cap1 = J > 0 && sb > sa && b > sa && b <= sb;
      const int nr = 2 + (cap0 ? J + 1 : 0) + (cap1 ? J + 1 : 0);
      if (EMIT) {
        int64_t o = out0 + n + (cap0 ? J + 1 : 0);
        if (out0 + n + nr <= out_cap) {
          double f0 = 0.0, f1 = 1.0;
          if (sb > sa) {
            double d = __dsub_rn(sb, sa);
            f0 = __ddiv_rn(__dsub_rn(lo, sa), d);
            f1 = __ddiv_rn(__dsub_rn(hi, sa), d);
          }
          float a0[4] = {v0.x, v0.y, v0.z, v0.w}, a1[4] = {v1.x, v1.y, v1.z, v1.w};
          float p0[4], p1[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            double dv = __dsub_rn((double)a1[c], (double)a0[c]);
            p0[c] = (float)__dadd_rn((double)a0[c], __dmul_rn(f0, dv));
            p1[c] = (float)__dadd_rn((double)a0[c], __dmul_rn(f1, dv));
          }
          out_rib[o] = make_float4(p0[0], p0[1], p0[2], p0[3]);
          out_rib[o + 1] = make_float4(p1[0], p1[1], p1[2], p1[3]);
          out_s[o] = (float)lo;
          out_s[o + 1] = (float)hi;
          out_tag[o] = tg | PS_TAG_LINK_START;
          out_tag[o + 1] = tg;
          if (out_src) {
            out_src[o] = (int32_t)r;
            out_src[o + 1] = (int32_t)r;
          }
          if (cap0)
            emit_cap(out_rib[o], J, square, true, tg, (float)lo, (int32_t)r, out0 + n, out_rib,
                     out_s, out_tag, out_src);
          if (cap1)
            emit_cap(out_rib[o + 1], J, square, false, tg, (float)hi, (int32_t)r, o + 2, out_rib,
                     out_s, out_tag, out_src);
        } else {
          ps_record_error(status, PS_ERR_CAPACITY);
        }
      }
      n += nr;
    }
  }
  return n;
}

// One pass over tiles of 1,024 quads (4 per thread): the FP32 prefilter
// settles most quads; the rest (near a stretch boundary) are queued in shared
// memory and run through the FP64 dash_quad densely -- the FP64 pipe is slow,
// and quads left in place would keep almost every warp on it.  Then a block
// scan of the piece counts, a warp-wide decoupled look-back for the tile's
// output offset, and emission (queued quads again densely).
__global__ void __launch_bounds__(DASH_NT) k_dash(
    const float4* __restrict__ rib, const float* __restrict__ s, const uint32_t* __restrict__ tag,
    const int64_t* __restrict__ n_rib, int64_t capacity, DashPattern P,
    float4* __restrict__ out_rib, float* __restrict__ out_s, uint32_t* __restrict__ out_tag,
    int32_t* __restrict__ out_src, int64_t* __restrict__ n_out, int64_t out_cap, uint32_t* tflag,
    long long* tagg, long long* tincl, int32_t* counters, int32_t* status) {
  __shared__ long long sm[DASH_NT / 32];
  __shared__ int smq[DASH_NT / 32];
  __shared__ long long s_prefix;
  __shared__ int64_t s_tile;
  __shared__ uint16_t s_queue[DASH_TILE];    // tile-local quads for the FP64 path
  __shared__ int s_cnt[DASH_TILE];           // their piece counts
  __shared__ long long s_out[DASH_TILE];     // their output offsets
  int64_t R = *n_rib;
  if (R > capacity) R = capacity;
  int64_t n_tiles = (R + DASH_TILE - 1) / DASH_TILE;
  if (n_tiles == 0) n_tiles = 1;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(&counters[3], 1);
    __syncthreads();
    const int64_t tile = s_tile;
    __syncthreads();
    if (tile >= n_tiles) return;
    const int64_t t0 = tile * DASH_TILE;
    const int q0 = (int)threadIdx.x * DASH_QPT;  // tile-local index of this thread's first quad
    int mode[DASH_QPT];
    float sa[DASH_QPT], sb[DASH_QPT];
    uint32_t tg[DASH_QPT];
    int nq = 0;
#pragma unroll
    for (int q = 0; q < DASH_QPT; ++q) {
      const int64_t r = t0 + q0 + q;
      mode[q] = 0;
      tg[q] = 0u;
      sa[q] = sb[q] = 0.f;
      if (r >= 1 && r < R) {
        tg[q] = __ldg(tag + r);
        if (!(tg[q] & PS_TAG_LINK_START)) {
          sa[q] = __ldg(s + r - 1);
          sb[q] = __ldg(s + r);
          mode[q] = dash_quick(P, sa[q], sb[q]);
          nq += mode[q] < 0;
        }
      }
    }
    // queue positions of this thread's FP64 quads (block exclusive scan)
    int xq = nq;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, xq, o);
      if (lane >= o) xq += y;
    }
    if (lane == 31) smq[wid] = xq;
    __syncthreads();
    int qpre = 0, qtot = 0;
    for (int w = 0; w < DASH_NT / 32; ++w) {
      if (w < wid) qpre += smq[w];
      qtot += smq[w];
    }
    int qp = qpre + xq - nq;
#pragma unroll
    for (int q = 0; q < DASH_QPT; ++q)
      if (mode[q] < 0) s_queue[qp++] = (uint16_t)(q0 + q);
    __syncthreads();
    for (int i = threadIdx.x; i < qtot; i += DASH_NT) {
      const int lq = s_queue[i];
      const int64_t r = t0 + lq;
      s_cnt[lq] = dash_quad<false>(P, (double)__ldg(s + r - 1), (double)__ldg(s + r), r, rib, 0.f,
                                   0.f, __ldg(tag + r), 0, nullptr, nullptr, nullptr, nullptr, 0,
                                   status);
    }
    __syncthreads();
    int cnt[DASH_QPT];
    int mine = 0;
#pragma unroll
    for (int q = 0; q < DASH_QPT; ++q) {
      cnt[q] = mode[q] == 1 ? 2 : mode[q] < 0 ? s_cnt[q0 + q] : 0;
      mine += cnt[q];
    }
    long long x = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) sm[wid] = x;
    __syncthreads();
    long long total = 0, wpre = 0;
    for (int w = 0; w < DASH_NT / 32; ++w) {
      if (w < wid) wpre += sm[w];
      total += sm[w];
    }
    if (wid == 0) {
      long long pre = lookback_sum_warp(tflag, tagg, tincl, total, tile, status);
      if (lane == 0) s_prefix = pre;
    }
    __syncthreads();
    int64_t o = s_prefix + wpre + x - mine;
#pragma unroll
    for (int q = 0; q < DASH_QPT; ++q) {
      const int64_t r = t0 + q0 + q;
      if (mode[q] < 0) {
        s_out[q0 + q] = o;  // emitted from the queue below
      } else if (mode[q] == 1) {
        // inside an on-stretch: the quad itself (f0 = 0, f1 = 1 in dash_quad)
        const uint32_t tq = tg[q] & ~PS_TAG_LINK_START;
        if (o + 2 <= out_cap) {
          const float4 v0 = __ldg(rib + r - 1), v1 = __ldg(rib + r);
          out_rib[o] = v0;
          out_rib[o + 1] = make_float4(whole_end(v0.x, v1.x), whole_end(v0.y, v1.y),
                                       whole_end(v0.z, v1.z), whole_end(v0.w, v1.w));
          out_s[o] = sa[q];
          out_s[o + 1] = sb[q];
          out_tag[o] = tq | PS_TAG_LINK_START;
          out_tag[o + 1] = tq;
          if (out_src) {
            out_src[o] = (int32_t)r;
            out_src[o + 1] = (int32_t)r;
          }
        } else {
          ps_record_error(status, PS_ERR_CAPACITY);
        }
      }
      o += cnt[q];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < qtot; i += DASH_NT) {
      const int lq = s_queue[i];
      if (s_cnt[lq] == 0) continue;
      const int64_t r = t0 + lq;
      dash_quad<true>(P, (double)__ldg(s + r - 1), (double)__ldg(s + r), r, rib, 0.f, 0.f,
                      __ldg(tag + r) & ~PS_TAG_LINK_START, s_out[lq], out_rib, out_s, out_tag,
                      out_src, out_cap, status);
    }
    if (tile == n_tiles - 1 && threadIdx.x == DASH_NT - 1) {
      long long tot = s_prefix + total;
      *n_out = tot;
      if (tot > out_cap) ps_record_error(status, PS_ERR_CAPACITY);
    }
    __syncthreads();
  }
}

}  // namespace

extern "C" int ps_dash_capped(ps_context* ctx, const float* d_rib, const float* d_s,
                              const uint32_t* d_tag, const int64_t* d_n_rib, int64_t capacity,
                              const float* h_pattern, int n_pattern, float offset,
                              const uint8_t* d_path_cap, int32_t n_path, float dtheta,
                              float* d_out_rib, float* d_out_s, uint32_t* d_out_tag,
                              int32_t* d_out_src, int64_t* d_n_out, int64_t out_capacity,
                              void* stream) {
  if (!ctx || !d_rib || !d_s || !d_tag || !d_n_rib || !h_pattern || !d_out_rib || !d_out_s ||
      !d_out_tag || !d_n_out || capacity < 0 || out_capacity < 0)
    return PS_ERR_INVALID;
  if (d_path_cap && (n_path < 0 || !(dtheta >= 1e-4f && dtheta <= 3.14159265f)))
    return PS_ERR_INVALID;
  if (n_pattern < 1 || n_pattern > 32 || !(offset == offset)) return PS_ERR_INVALID;
  DashPattern P;
  P.m2 = (n_pattern % 2) ? 2 * n_pattern : n_pattern;
  P.cum[0] = 0.0;
  for (int i = 0; i < P.m2; ++i) {
    double d = (double)h_pattern[i % n_pattern];
    if (!(d >= 0.0)) return PS_ERR_INVALID;
    P.cum[i + 1] = P.cum[i] + d;
  }
  P.period = P.cum[P.m2];
  P.offset = (double)offset;
  for (int i = 0; i <= P.m2; ++i) P.cum_f[i] = (float)P.cum[i];
  P.period_f = (float)P.period;
  P.period_lo = (float)(P.period - (double)P.period_f);
  P.offset_f = offset;
  P.path_cap = d_path_cap;
  P.n_path = d_path_cap ? n_path : 0;
  P.j_round = 0;
  if (d_path_cap) {
    // a round cap turns pi in steps of at most q (a ratio within 1e-4 step above
    // an integer takes that integer, as for every turning count)
    double x = 3.14159265358979323846 / (double)dtheta;
    int J = (int)ceil(x - 1e-4);
    P.j_round = J < 1 ? 1 : J;
  }
  if (!(P.period > 0.0)) return PS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = stream;
  int64_t n_tiles = (capacity + DASH_TILE - 1) / DASH_TILE + 1;
  int rc = ps_ensure_tiles(ctx, n_tiles + 1);
  if (rc != PS_OK) return rc;
  cudaMemsetAsync(ctx->d_tile_flag, 0, sizeof(uint32_t) * (n_tiles + 1), st);
  cudaMemsetAsync(ctx->d_counters, 0, sizeof(int32_t) * 16, st);
  int grid = ps_persistent_grid(ctx, (const void*)k_dash, DASH_NT, 0);
  ProfScope ps_(ctx, PK_DASH, st);
  k_dash<<<grid, DASH_NT, 0, st>>>(reinterpret_cast<const float4*>(d_rib), d_s, d_tag, d_n_rib,
                                    capacity, P, reinterpret_cast<float4*>(d_out_rib), d_out_s,
                                    d_out_tag, d_out_src, d_n_out, out_capacity, ctx->d_tile_flag,
                                    ctx->d_tile_agg, ctx->d_tile_incl, ctx->d_counters,
                                    ctx->d_status);
  return ps_cuda_check(cudaGetLastError());
}

extern "C" int ps_dash(ps_context* ctx, const float* d_rib, const float* d_s,
                       const uint32_t* d_tag, const int64_t* d_n_rib, int64_t capacity,
                       const float* h_pattern, int n_pattern, float offset, float* d_out_rib,
                       float* d_out_s, uint32_t* d_out_tag, int32_t* d_out_src, int64_t* d_n_out,
                       int64_t out_capacity, void* stream) {
  return ps_dash_capped(ctx, d_rib, d_s, d_tag, d_n_rib, capacity, h_pattern, n_pattern, offset,
                        nullptr, 0, 1.f, d_out_rib, d_out_s, d_out_tag, d_out_src, d_n_out,
                        out_capacity, stream);
}
