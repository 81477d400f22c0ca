// Uniform parametric tessellation and facet-angle statistics (Sec. 8.1).
//
// The paper compares polar stroking with the stroke of Eq. 1 sampled at
// uniform parameters, at equal quad counts, by the facet angles where one
// quad's boundary edge meets the next (Sec. 4.2 bounds the ordinary ones by
// 2q).  k_uniform_ribs writes, for every segment link of a polar tessellation,
// the same number of ribs at t_j = j/N; k_facet_stats reduces the ordinary
// facet angles of a rib stream per link.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ps_geom.cuh"
#include "ps_internal.cuh"

namespace {

using namespace ps;

constexpr int FC_NT = 256;

__device__ __forceinline__ int64_t last_le(const int32_t* off, int64_t lo, int64_t hi, int64_t r) {
  // last l in [lo, hi] with off[l] <= r (off non-decreasing)
  while (hi > lo) {
    int64_t mid = (lo + hi + 1) >> 1;
    if ((int64_t)__ldg(off + mid) <= r) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// dH/dt of the hodograph direction (H of ps_geom.cuh), for the tangent at an
// exact cusp.
__device__ __forceinline__ float2 hodo_dt(const Seg& g, float t) {
  float u = 1.f - t;
  switch (g.type) {
    case PS_CUBIC: {
      float2 d1 = g.B - g.A, d2 = g.C - g.B, d3 = g.D - g.C;
      return ((d2 - d1) * u + (d3 - d2) * t) * 2.f;
    }
    case PS_QUAD:
      return (g.D - g.B) - (g.B - g.A);
    case PS_CONIC: {
      float2 h0 = (g.B - g.A) * g.w, h1 = g.D - g.A, h2 = (g.D - g.B) * g.w;
      return h0 * (-2.f * u) + h1 * (u - t) + h2 * (2.f * t);
    }
    default:
      return mk(0.f, 0.f);
  }
}

// One thread per rib: segment links get g(t) -+ r n(t) at t = j / (n - 1), with
// n(t) the unit left normal of g'(t) (g'' at an exact cusp, the chord if the
// hodograph vanishes everywhere); joins and caps keep the polar ribs.
__global__ void __launch_bounds__(FC_NT) k_uniform_ribs(
    const uint8_t* __restrict__ st, const float* __restrict__ sp, const float* __restrict__ sw,
    const int32_t* __restrict__ seg_off, const float* __restrict__ width, int n_path,
    const int32_t* __restrict__ link_off, int64_t n_link, const int64_t* __restrict__ n_rib,
    int64_t capacity, const float4* __restrict__ polar, float4* __restrict__ out) {
  int64_t R = *n_rib;
  if (R > capacity) R = capacity;
  for (int64_t r = (int64_t)blockIdx.x * FC_NT + threadIdx.x; r < R;
       r += (int64_t)gridDim.x * FC_NT) {
    int64_t l = last_le(link_off, 0, n_link - 1, r);
    int64_t j = r - __ldg(link_off + l), n = (int64_t)__ldg(link_off + l + 1) - __ldg(link_off + l);
    // path of link l: its links start at 2 seg_off[p] + p
    int lo = 0, hi = n_path - 1;
    while (hi > lo) {
      int mid = (lo + hi + 1) >> 1;
      if (2 * (int64_t)__ldg(seg_off + mid) + mid <= l) lo = mid; else hi = mid - 1;
    }
    const int p = lo;
    const int64_t k = l - (2 * (int64_t)__ldg(seg_off + p) + p);
    if (!(k & 1) || n < 2) {
      out[r] = __ldg(polar + r);
      continue;
    }
    Seg g = load_seg(st, sp, sw, __ldg(seg_off + p) + (int)((k - 1) >> 1));
    float t = (float)j / (float)(n - 1);
    float2 c = g_rel_comp(g, t) + g.A;
    float2 H = hodo(g, t);
    if (is0(H)) H = hodo_dt(g, t);
    if (is0(H)) H = g.D - g.A;
    float L = sqrtf(H.x * H.x + H.y * H.y);
    float2 nv = L > 0.f ? mk(-H.y / L, H.x / L) : mk(0.f, 0.f);
    float rr = 0.5f * __ldg(width + p);
    out[r] = make_float4(c.x - rr * nv.x, c.y - rr * nv.y, c.x + rr * nv.x, c.y + rr * nv.y);
  }
}

// Does boundary edge e (from rib a to rib b) point between the tangents of
// ribs a and b?  The rib P - N is the left normal; turned clockwise it is the
// tangent.  Ribs of zero length: the edge must advance with the centreline.
__device__ __forceinline__ bool edge_regular(float4 a, float4 b, float2 e, float slack) {
  float2 v0 = mk(a.z - a.x, a.w - a.y), v1 = mk(b.z - b.x, b.w - b.y);
  float l0 = sqrtf(dot2(v0, v0)), l1 = sqrtf(dot2(v1, v1)), le = sqrtf(dot2(e, e));
  if (l0 == 0.f || l1 == 0.f) {
    float2 m = mk(0.5f * (b.x + b.z) - 0.5f * (a.x + a.z), 0.5f * (b.y + b.w) - 0.5f * (a.y + a.w));
    return dot2(e, m) > 0.f;
  }
  float2 T0 = mk(v0.y / l0, -v0.x / l0), T1 = mk(v1.y / l1, -v1.x / l1), u = e * (1.f / le);
  if (dot2(u, T0 + T1) <= 0.f) return false;
  float c01 = cross2(T0, T1), c0u = cross2(T0, u), cu1 = cross2(u, T1);
  if (c01 >= 0.f) return c0u >= -slack && cu1 >= -slack;
  return c0u <= slack && cu1 <= slack;
}

// One thread per rib: the two facets (N and P sides) at an interior rib of a
// segment link, reduced per link into (max, sum, sum of squares, count) of the
// ordinary ones; lanes of a warp on the same link reduce first.  Link ids stay
// below 2^31.
__global__ void __launch_bounds__(FC_NT) k_facet_stats(
    const float4* __restrict__ rib, const uint32_t* __restrict__ tag,
    const int32_t* __restrict__ link_off, int64_t n_link, const int64_t* __restrict__ n_rib,
    int64_t capacity, float slack, float* __restrict__ stats) {
  int64_t R = *n_rib;
  if (R > capacity) R = capacity;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * FC_NT;
  for (int64_t base = (int64_t)blockIdx.x * FC_NT; base < R; base += stride) {
    const int64_t r = base + threadIdx.x;
    float mx = 0.f, sum = 0.f, sq = 0.f, cnt = 0.f;
    int64_t link = -1;
    if (r >= 1 && r + 1 < R) {
      uint32_t tg = __ldg(tag + r), tn = __ldg(tag + r + 1);
      if ((tg & PS_TAG_SEGMENT) && !(tg & PS_TAG_LINK_START) && !(tn & PS_TAG_LINK_START)) {
        link = last_le(link_off, 0, n_link - 1, r);
        float4 a = __ldg(rib + r - 1), b = __ldg(rib + r), c = __ldg(rib + r + 1);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          float2 A = s ? mk(a.z, a.w) : mk(a.x, a.y), B = s ? mk(b.z, b.w) : mk(b.x, b.y),
                 C = s ? mk(c.z, c.w) : mk(c.x, c.y);
          float2 e0 = B - A, e1 = C - B;
          if (is0(e0) || is0(e1)) continue;
          if (!edge_regular(a, b, e0, slack) || !edge_regular(b, c, e1, slack)) continue;
          float ang = fabsf(atan2f(cross2(e0, e1), dot2(e0, e1)));
          mx = fmaxf(mx, ang);
          sum += ang;
          sq += ang * ang;
          cnt += 1.f;
        }
      }
    }
    // A link's interior ribs sit on consecutive lanes, so a down-shuffle that
    // only adds a lane of the same link leaves lane i with the totals over
    // lanes [i, i + 2^k) of its run after step k; the run's first lane writes.
    const int key = (int)link;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int okey = __shfl_down_sync(0xffffffffu, key, o);
      float omx = __shfl_down_sync(0xffffffffu, mx, o), osum = __shfl_down_sync(0xffffffffu, sum, o),
            osq = __shfl_down_sync(0xffffffffu, sq, o), ocnt = __shfl_down_sync(0xffffffffu, cnt, o);
      if (lane + o < 32 && okey == key) {
        mx = fmaxf(mx, omx);
        sum += osum;
        sq += osq;
        cnt += ocnt;
      }
    }
    const int pkey = __shfl_up_sync(0xffffffffu, key, 1);
    const bool head = lane == 0 || pkey != key;
    if (link >= 0 && head && cnt > 0.f) {
      float* o = stats + 4 * link;
      atomicMax(reinterpret_cast<int*>(o), __float_as_int(mx));  // non-negative floats
      atomicAdd(o + 1, sum);
      atomicAdd(o + 2, sq);
      atomicAdd(o + 3, cnt);
    }
  }
}

}  // namespace

extern "C" int ps_uniform_tessellate(ps_context* ctx, const ps_segments* seg, const ps_paths* paths,
                                     const ps_tess_out* fwd, float* d_rib_out, void* stream) {
  if (!ctx || !seg || !paths || !fwd) return PS_ERR_INVALID;
  if (paths->n_path == 0 && seg->n_seg == 0) return PS_OK;  // empty batch: no ribs
  if (!d_rib_out || !fwd->d_rib || !fwd->d_link_rib_off || !fwd->d_n_rib) return PS_ERR_INVALID;
  if (paths->n_path <= 0 || seg->n_seg < 0 || fwd->capacity < 0) return PS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = stream;
  int64_t L = 2 * seg->n_seg + paths->n_path;
  int grid = ps_persistent_grid(ctx, (const void*)k_uniform_ribs, FC_NT, 0);
  k_uniform_ribs<<<grid, FC_NT, 0, st>>>(seg->d_type, seg->d_pts, seg->d_w, paths->d_seg_off,
                                        paths->d_width, paths->n_path, fwd->d_link_rib_off, L,
                                        fwd->d_n_rib, fwd->capacity,
                                        reinterpret_cast<const float4*>(fwd->d_rib),
                                        reinterpret_cast<float4*>(d_rib_out));
  return ps_cuda_check(cudaGetLastError());
}

extern "C" int ps_facet_stats(ps_context* ctx, const float* d_rib, const uint32_t* d_tag,
                              const int32_t* d_link_rib_off, int64_t n_link, const int64_t* d_n_rib,
                              int64_t capacity, float slack, float* d_stats, void* stream) {
  if (!ctx || !d_rib || !d_tag || !d_link_rib_off || !d_n_rib || !d_stats) return PS_ERR_INVALID;
  if (n_link <= 0 || capacity < 0 || !(slack >= 0.f)) return PS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = stream;
  cudaMemsetAsync(d_stats, 0, sizeof(float) * 4 * (size_t)n_link, st);
  int grid = ps_persistent_grid(ctx, (const void*)k_facet_stats, FC_NT, 0);
  k_facet_stats<<<grid, FC_NT, 0, st>>>(reinterpret_cast<const float4*>(d_rib), d_tag,
                                       d_link_rib_off, n_link, d_n_rib, capacity, slack, d_stats);
  return ps_cuda_check(cudaGetLastError());
}
