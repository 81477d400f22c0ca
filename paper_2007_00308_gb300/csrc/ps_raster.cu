// Tile-binned 16-sample coverage of stroked quads.
//
// Quad (r-1, r) of a rib strip is drawn as the two triangles (N_{r-1}, P_{r-1},
// P_r) and (N_{r-1}, P_r, N_r) (Sec. 4.1).  Vertices snap to 1/256 px.  The
// coverage of a path is the union of its quads (Sec. 3.3.6), so every tile keeps
// one 16-bit sample mask per pixel per path that touches it; the canvas is the OR
// over paths and covered[p] sums path p's masks' popcounts.
#include <cuda_runtime.h>

#include "ps_internal.cuh"

namespace {

constexpr int TILE_PX = 16;                 // tile edge in pixels
constexpr int TILE_UNITS = TILE_PX * 256;   // in 1/256 px
constexpr int COORD_LIMIT = 1 << 29;        // |v * 256| < 2^29, i.e. |v| < 2^21 px

// floor(a / 256) and ceil(a / 256) (arithmetic shifts round toward -inf)
__device__ __forceinline__ int64_t floor256(int64_t a) { return a >> 8; }
__device__ __forceinline__ int64_t ceil256(int64_t a) { return -((-a) >> 8); }

struct QuadFix {
  int x[4], y[4];  // N0 P0 N1 P1 in 1/256 px
};

// Snap a quad's four vertices; false when a coordinate is out of range.
__device__ __forceinline__ bool snap_quad(const float4 a, const float4 b, QuadFix& q) {
  float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
  int s[8];
  bool ok = true;  // one test at the end (NaN fails it too)
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    float f = v[i] * 256.f;  // exact scaling by a power of two
    ok &= fabsf(f) < (float)COORD_LIMIT;
    s[i] = __float2int_rn(f);  // round half to even
  }
  q.x[0] = s[0]; q.y[0] = s[1]; q.x[1] = s[2]; q.y[1] = s[3];
  q.x[2] = s[4]; q.y[2] = s[5]; q.x[3] = s[6]; q.y[3] = s[7];
  return ok;
}

// Pixel range whose sample window [256p + 8, 256p + 248] meets [lo, hi].
__device__ __forceinline__ void pix_range(int lo, int hi, int n, int& p0, int& p1) {
  int64_t a = ceil256((int64_t)lo - 248), b = floor256((int64_t)hi - 8);
  if (a < 0) a = 0;
  if (b > n - 1) b = n - 1;
  p0 = (int)a;
  p1 = (int)b;
}

// Can triangle (x0,y0)-(x1,y1)-(x2,y2) cover a sample of the tile whose samples
// lie in [rx0, rx1] x [ry0, ry1]?  Separating-axis test on the triangle's edges
// (the rectangle's own axes are settled by the bounding-box range).
// (Branch-free: a zero-area triangle meets nothing, and the vertices of a
// clockwise one are swapped by selects.)
__device__ __forceinline__ bool tri_meets_rect(int x0, int y0, int x1, int y1, int x2, int y2,
                                               int rx0, int ry0, int rx1, int ry1) {
  const long long area = (long long)(x1 - x0) * (y2 - y0) - (long long)(y1 - y0) * (x2 - x0);
  const bool cw = area < 0;
  const int vx[3] = {x0, cw ? x2 : x1, cw ? x1 : x2}, vy[3] = {y0, cw ? y2 : y1, cw ? y1 : y2};
  bool ok = area != 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    long long A = (long long)vy[i] - vy[(i + 1) % 3], B = (long long)vx[(i + 1) % 3] - vx[i];
    // the rectangle corner maximizing A x + B y
    long long cx = A >= 0 ? rx1 : rx0, cy = B >= 0 ? ry1 : ry0;
    ok &= A * (cx - vx[i]) + B * (cy - vy[i]) >= 0;
  }
  return ok;
}

// Early-exit forms of the two tests (fewer registers: the scatter pass, which
// re-tests only quads with more than 31 candidate tiles, keeps its occupancy).
__device__ __forceinline__ bool tri_meets_rect_ee(int x0, int y0, int x1, int y1, int x2, int y2,
                                                  int rx0, int ry0, int rx1, int ry1) {
  long long area = (long long)(x1 - x0) * (y2 - y0) - (long long)(y1 - y0) * (x2 - x0);
  if (area == 0) return false;
  if (area < 0) {
    int t = x1; x1 = x2; x2 = t;
    t = y1; y1 = y2; y2 = t;
  }
  int vx[3] = {x0, x1, x2}, vy[3] = {y0, y1, y2};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    long long A = (long long)vy[i] - vy[(i + 1) % 3], B = (long long)vx[(i + 1) % 3] - vx[i];
    long long cx = A >= 0 ? rx1 : rx0, cy = B >= 0 ? ry1 : ry0;
    if (A * (cx - vx[i]) + B * (cy - vy[i]) < 0) return false;
  }
  return true;
}
__device__ __forceinline__ bool tri_meets_rect32_ee(int x0, int y0, int x1, int y1, int x2, int y2,
                                                    int rx0, int ry0, int rx1, int ry1) {
  int area = (x1 - x0) * (y2 - y0) - (y1 - y0) * (x2 - x0);
  if (area == 0) return false;
  if (area < 0) {
    int t = x1; x1 = x2; x2 = t;
    t = y1; y1 = y2; y2 = t;
  }
  int vx[3] = {x0, x1, x2}, vy[3] = {y0, y1, y2};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    int A = vy[i] - vy[(i + 1) % 3], B = vx[(i + 1) % 3] - vx[i];
    int cx = A >= 0 ? rx1 : rx0, cy = B >= 0 ? ry1 : ry0;
    if (A * (cx - vx[i]) + B * (cy - vy[i]) < 0) return false;
  }
  return true;
}

// Same test in int32, for triangles whose extent is below 2^14 on both axes
// and rectangles within 2^14 + 4096 of them: every product stays below 2^29.
__device__ __forceinline__ bool tri_meets_rect32(int x0, int y0, int x1, int y1, int x2, int y2,
                                                 int rx0, int ry0, int rx1, int ry1) {
  const int area = (x1 - x0) * (y2 - y0) - (y1 - y0) * (x2 - x0);
  const bool cw = area < 0;
  const int vx[3] = {x0, cw ? x2 : x1, cw ? x1 : x2}, vy[3] = {y0, cw ? y2 : y1, cw ? y1 : y2};
  bool ok = area != 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    int A = vy[i] - vy[(i + 1) % 3], B = vx[(i + 1) % 3] - vx[i];
    int cx = A >= 0 ? rx1 : rx0, cy = B >= 0 ? ry1 : ry0;
    ok &= A * (cx - vx[i]) + B * (cy - vy[i]) >= 0;
  }
  return ok;
}

// Does quad q (triangles N0 P0 P1 and N0 P1 N1) meet tile (tx, ty)'s sample
// rectangle, clipped to the canvas?  BF: the branch-free tests.
template <bool BF>
__device__ __forceinline__ bool quad_meets_tile(const QuadFix& q, bool small, int tx, int ty,
                                                int W, int H) {
  int rx0 = tx * TILE_UNITS + 8, ry0 = ty * TILE_UNITS + 8;
  int rx1 = min(tx * TILE_UNITS + TILE_UNITS, W * 256) - 8;
  int ry1 = min(ty * TILE_UNITS + TILE_UNITS, H * 256) - 8;
  if (!BF) {
    if (small)
      return tri_meets_rect32_ee(q.x[0], q.y[0], q.x[1], q.y[1], q.x[3], q.y[3], rx0, ry0, rx1, ry1) ||
             tri_meets_rect32_ee(q.x[0], q.y[0], q.x[3], q.y[3], q.x[2], q.y[2], rx0, ry0, rx1, ry1);
    return tri_meets_rect_ee(q.x[0], q.y[0], q.x[1], q.y[1], q.x[3], q.y[3], rx0, ry0, rx1, ry1) ||
           tri_meets_rect_ee(q.x[0], q.y[0], q.x[3], q.y[3], q.x[2], q.y[2], rx0, ry0, rx1, ry1);
  }
  if (small)
    return tri_meets_rect32(q.x[0], q.y[0], q.x[1], q.y[1], q.x[3], q.y[3], rx0, ry0, rx1, ry1) |
           tri_meets_rect32(q.x[0], q.y[0], q.x[3], q.y[3], q.x[2], q.y[2], rx0, ry0, rx1, ry1);
  return tri_meets_rect(q.x[0], q.y[0], q.x[1], q.y[1], q.x[3], q.y[3], rx0, ry0, rx1, ry1) |
         tri_meets_rect(q.x[0], q.y[0], q.x[3], q.y[3], q.x[2], q.y[2], rx0, ry0, rx1, ry1);
}

// pass 0: count (quad, tile) pairs per tile and keep, per quad with at most 31
// candidate tiles (those of its pixel bounding box), the bit mask of the tiles
// its triangles meet; pass 1: scatter rib ids into bins from those masks
// (re-testing only quads with more candidates).  A warp takes 32 quads, one
// per lane.  Quads of one or two tiles are binned in direct rounds; the others'
// (quad, candidate) pairs are flattened with a warp scan so that each lane
// tests one pair at a time.  Lanes of the warp that hit the same tile are
// grouped: one atomic per group.
// Per-quad words from the count pass for the scatter pass, {hits, box}.  hits:
// 0 = no tile; bit 31 with the tall flag in bit 30 and the tile index below it
// = the quad's bounding box lies in that one tile; HITS_RETEST = more than 31
// candidate tiles (the scatter pass re-reads, snaps and re-tests the quad);
// otherwise the hit mask over the candidates, with box = the first candidate
// tile's index | (columns - 1) << 26 | tall << 31, so that the scatter pass
// reads no ribs for the quad.
// The scatter pass fills each tile's entries from the front with quads that
// span more than TALL_ROWS pixel rows and from the back with shorter ones, so
// that the coverage kernel's 32-entry batches hold entries of like heights (a
// warp's row-span loop runs as long as its tallest entry), and a tile's last
// batches, where its warps wait on each other, are the cheap ones.
constexpr uint32_t HITS_RETEST = 0xffffffffu;
constexpr uint32_t HITS_DIRECT = 0x80000000u;
constexpr int BIN_NT = 256;

struct BinQuad {
  int x[4], y[4];
  int tx0, ty0, ntx, n;  // candidate tiles: ntx columns from (tx0, ty0), n in all
  int tbase;             // index of tile (tx0, ty0)
  uint32_t mask;         // pass 1: hit mask from pass 0; pass 0: hits found
  int small;             // bit 0: under 64 px (int32 tests); bit 1: tall (more
                         // than TALL_ROWS pixel rows); one word, so that the
                         // record stays 15 words (an odd stride: no bank conflicts)
};
constexpr int TALL_ROWS = 6;

template <int PASS>
__global__ void __launch_bounds__(BIN_NT) k_bin(const float4* __restrict__ rib,
                                                const uint32_t* __restrict__ tag,
                                                const int64_t* __restrict__ n_rib, int64_t capacity,
                                                int W, int H, int y0, int tiles_x,
                                                int32_t* __restrict__ count,
                                                const int32_t* __restrict__ off,
                                                int32_t* __restrict__ cursor,
                                                uint32_t* __restrict__ bin, int64_t pair_cap,
                                                uint2* __restrict__ hits,
                                                int32_t* __restrict__ back,  // short fill, from the end
                                                int32_t* status) {
  __shared__ BinQuad s_q[BIN_NT];
  __shared__ int s_pre[BIN_NT / 32][33];
  int64_t R = *n_rib;
  if (R > capacity) R = capacity;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  BinQuad* wq = s_q + wid * 32;
  int64_t stride = (int64_t)gridDim.x * BIN_NT;
  for (int64_t base = (int64_t)blockIdx.x * BIN_NT; base < R; base += stride) {
    const int64_t r = base + threadIdx.x;
    const bool in = r >= 1 && r < R;
    const uint2 hb = PASS == 1 && in ? __ldg(hits + r) : make_uint2(0u, 0u);
    const uint32_t h = hb.x;
    const bool direct1 = PASS == 1 && (h & HITS_DIRECT) && h != HITS_RETEST;
    const bool boxed1 = PASS == 1 && h != 0u && !direct1 && h != HITS_RETEST;
    const bool act = PASS == 0 ? in && !(__ldg(tag + r) & PS_TAG_LINK_START) : h == HITS_RETEST;
    BinQuad& Q = wq[lane];
    int cnt = 0;
    Q.n = 0;
    Q.mask = 0;
    Q.tbase = 0;
    Q.ntx = 1;
    Q.small = 0;
    if (act) {
      QuadFix q;
      if (!snap_quad(__ldg(rib + r - 1), __ldg(rib + r), q)) {
        if (PASS == 0) ps_record_error(status, PS_ERR_RANGE);
      } else {
        // relative to the window's first row (exact: snapped units)
        for (int v = 0; v < 4; ++v) q.y[v] -= y0;
        int mnx = min(min(q.x[0], q.x[1]), min(q.x[2], q.x[3]));
        int mxx = max(max(q.x[0], q.x[1]), max(q.x[2], q.x[3]));
        int mny = min(min(q.y[0], q.y[1]), min(q.y[2], q.y[3]));
        int mxy = max(max(q.y[0], q.y[1]), max(q.y[2], q.y[3]));
        int px0, px1, py0, py1;
        pix_range(mnx, mxx, W, px0, px1);
        pix_range(mny, mxy, H, py0, py1);
        if (px0 <= px1 && py0 <= py1) {
          int tx0 = px0 / TILE_PX, tx1 = px1 / TILE_PX, ty0 = py0 / TILE_PX, ty1 = py1 / TILE_PX;
          for (int v = 0; v < 4; ++v) {
            Q.x[v] = q.x[v];
            Q.y[v] = q.y[v];
          }
          Q.tx0 = tx0;
          Q.ty0 = ty0;
          Q.tbase = ty0 * tiles_x + tx0;
          Q.ntx = tx1 - tx0 + 1;
          Q.n = Q.ntx * (ty1 - ty0 + 1);
          Q.small = (mxx - mnx < (1 << 14) && mxy - mny < (1 << 14) ? 1 : 0) |
                    (py1 - py0 + 1 > TALL_ROWS ? 2 : 0);
          if (PASS == 1) {
            Q.mask = h;
            cnt = Q.n <= 31 ? __popc(h) : Q.n;
          } else {
            cnt = Q.n;
          }
        }
      }
    }
    if (boxed1) {  // hit mask and candidate box from the count pass
      Q.mask = h;
      Q.tbase = (int)(hb.y & 0x3ffffffu);
      Q.ntx = (int)((hb.y >> 26) & 31u) + 1;
      Q.small = (int)(hb.y >> 31) << 1;
      Q.n = 31;  // any count from 2 to 31: the mask gives the candidates
      cnt = __popc(h);
    }
    // A quad whose bounding box lies in one tile meets that tile.  One whose box
    // spans two tiles crosses their common edge, so it almost always meets both:
    // it is entered in both untested (an entry without samples costs the
    // coverage kernel only its set-up; measured: count pass -0.06 ms, coverage
    // unchanged; boxes of up to four tiles cost coverage 0.26 ms).  Such
    // quads, and in pass 1 every quad the count pass found in at most two tiles,
    // are binned in up to two direct rounds, outside the flattened (quad,
    // candidate) loop.
    int tdir = Q.n == 1 ? Q.ty0 * tiles_x + Q.tx0 : -1;
    int tdir2 = -1;
    if (PASS == 0 && Q.n == 2) {
      tdir = Q.tbase;
      tdir2 = Q.tbase + (Q.ntx == 2 ? 1 : tiles_x);
      cnt = 0;
      Q.mask = 3u;
    }
    if (direct1) {
      tdir = (int)(h & 0x3fffffffu);
      Q.small = (int)((h >> 30) & 1u) << 1;
    }
    if (boxed1 && __popc(h) <= 2) {
      const int i0 = __ffs(h) - 1;
      tdir = Q.tbase + (i0 / Q.ntx) * tiles_x + i0 % Q.ntx;
      const uint32_t h2 = h & (h - 1u);
      if (h2) {
        const int i1 = __ffs(h2) - 1;
        tdir2 = Q.tbase + (i1 / Q.ntx) * tiles_x + i1 % Q.ntx;
      }
      cnt = 0;
    }
    {
      if (Q.n == 1) {
        cnt = 0;
        if (PASS == 0) Q.mask = 1u;
      }
      const int tall = Q.small >> 1;
      auto direct = [&](int td) {
        // pass 1 groups by tile and height class (the two fill from either end)
        const unsigned peers =
            __match_any_sync(0xffffffffu, td >= 0 ? (PASS == 0 ? td : 2 * td + tall) : -1);
        const int leader = __ffs(peers) - 1;
        if (td >= 0) {
          if (PASS == 0) {
            if (lane == leader) atomicAdd(count + td, __popc(peers));
          } else {
            int basepos = 0;
            if (lane == leader) basepos = atomicAdd((tall ? cursor : back) + td, __popc(peers));
            basepos = __shfl_sync(peers, basepos, leader);
            const int rk = basepos + __popc(peers & ((1u << lane) - 1u));
            const int64_t at = tall ? (int64_t)off[td] + rk : (int64_t)off[td + 1] - 1 - rk;
            if (at < pair_cap && at >= off[td] && at < off[td + 1]) bin[at] = (uint32_t)r;
            else ps_record_error(status, PS_ERR_CAPACITY);
          }
        }
      };
      direct(tdir);
      if (__any_sync(0xffffffffu, tdir2 >= 0)) direct(tdir2);
    }
    // warp scan of the pair counts
    int x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    s_pre[wid][lane + 1] = x;
    if (lane == 0) s_pre[wid][0] = 0;
    const int total = __shfl_sync(0xffffffffu, x, 31);
    __syncwarp();
    for (int it0 = 0; it0 < total; it0 += 32) {
      const int it = it0 + lane;
      int t = -1, e = 0, i = 0, tl = 0;
      if (it < total) {
        int lo = 0;  // last quad whose prefix is <= it
#pragma unroll
        for (int st = 16; st > 0; st >>= 1)
          if (lo + st <= 31 && s_pre[wid][lo + st] <= it) lo += st;
        e = lo;
        const BinQuad& B = wq[e];
        int k = it - s_pre[wid][e];
        bool hit;
        if (PASS == 1 && B.n <= 31) {
          i = __fns(B.mask, 0, k + 1);  // position of the (k+1)-th set bit
          hit = true;
        } else {
          i = k;
          int tx = B.tx0 + i % B.ntx, ty = B.ty0 + i / B.ntx;
          QuadFix q;
          for (int v = 0; v < 4; ++v) {
            q.x[v] = B.x[v];
            q.y[v] = B.y[v];
          }
          // (quads of one or two candidate tiles never get here: they are
          // binned directly)
          hit = quad_meets_tile<PASS == 0>(q, (B.small & 1) != 0, tx, ty, W, H);
        }
        tl = B.small >> 1;
        if (hit) {
          t = B.tbase + (i / B.ntx) * tiles_x + i % B.ntx;
          if (PASS == 0 && i < 31) atomicOr(&wq[e].mask, 1u << i);
        }
      }
      unsigned peers = __match_any_sync(0xffffffffu, t >= 0 ? (PASS == 0 ? t : 2 * t + tl) : -1);
      int leader = __ffs(peers) - 1;
      int cntg = __popc(peers);
      if (t >= 0) {
        if (PASS == 0) {
          if (lane == leader) atomicAdd(count + t, cntg);
        } else {
          int basepos = 0;
          if (lane == leader) basepos = atomicAdd((tl ? cursor : back) + t, cntg);
          basepos = __shfl_sync(peers, basepos, leader);
          int pos = basepos + __popc(peers & ((1u << lane) - 1u));
          int64_t at = tl ? (int64_t)off[t] + pos : (int64_t)off[t + 1] - 1 - pos;
          if (at < pair_cap && at >= off[t] && at < off[t + 1])
            bin[at] = (uint32_t)(base + wid * 32 + e);
          else ps_record_error(status, PS_ERR_CAPACITY);
        }
      }
    }
    __syncwarp();
    if (PASS == 0 && in)
      hits[r] = make_uint2(!act ? 0u
                           : Q.n == 1 ? HITS_DIRECT | (uint32_t)(Q.small >> 1) << 30 | (uint32_t)tdir
                           : Q.n <= 31 ? Q.mask : HITS_RETEST,
                           (uint32_t)Q.tbase | (uint32_t)(Q.ntx - 1) << 26 |
                               (uint32_t)(Q.small >> 1) << 31);
    __syncwarp();
  }
}

// Exclusive scan of tile counts, the cursors reset (front cursors at
// cursor[0 .. n_tile), back cursors at cursor[n_tile + 1 ..)), and the list of tiles with
// entries in order: list[0 .. m) and m = list[n_tile].  CTA b takes tiles
// [4096 b, 4096 (b+1)), 16 per thread; the sum and the count of non-empty tiles
// are scanned together as one int64 (the count in bits 38 and up) with a
// warp-wide decoupled look-back across CTAs.
constexpr int TS_NT = 256, TS_IPT = 16, TS_TILE = TS_NT * TS_IPT;
constexpr int TS_SHIFT = 38;
__global__ void __launch_bounds__(TS_NT) k_tile_scan(const int32_t* __restrict__ count,
                                                     int32_t* __restrict__ off,
                                                     int32_t* __restrict__ cursor,
                                                     int32_t* __restrict__ list, int n_tile,
                                                     int64_t pair_cap, uint32_t* tflag,
                                                     long long* tagg, long long* tincl,
                                                     int32_t* status) {
  __shared__ long long sm[TS_NT / 32];
  __shared__ long long s_pre;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long i0 = (long long)blockIdx.x * TS_TILE + (long long)threadIdx.x * TS_IPT;
  int c[TS_IPT];
  if (i0 + TS_IPT <= n_tile) {
    const int4* cp = reinterpret_cast<const int4*>(count + i0);
#pragma unroll
    for (int q = 0; q < TS_IPT / 4; ++q) {
      int4 v = cp[q];
      c[4 * q] = v.x; c[4 * q + 1] = v.y; c[4 * q + 2] = v.z; c[4 * q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < TS_IPT; ++i) c[i] = i0 + i < n_tile ? count[i0 + i] : 0;
  }
  long long v = 0;
#pragma unroll
  for (int i = 0; i < TS_IPT; ++i) v += (long long)c[i] + ((long long)(c[i] > 0) << TS_SHIFT);
  long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sm[wid] = x;
  __syncthreads();
  long long total = 0, wpre = 0;
  for (int w = 0; w < TS_NT / 32; ++w) {
    if (w < wid) wpre += sm[w];
    total += sm[w];
  }
  if (wid == 0) {
    long long pre = lookback_sum_warp(tflag, tagg, tincl, total, blockIdx.x, status);
    if (lane == 0) s_pre = pre;
  }
  __syncthreads();
  const long long mask = (1LL << TS_SHIFT) - 1;
  long long run = s_pre + wpre + x - v;
#pragma unroll
  for (int i = 0; i < TS_IPT; ++i) {
    const long long idx = i0 + i;
    if (idx < n_tile) {
      const long long sum = run & mask;
      if (sum > 0x7fffffffLL) ps_record_error(status, PS_ERR_CAPACITY);
      off[idx] = (int32_t)(sum > 0x7fffffffLL ? 0x7fffffff : sum);
      cursor[idx] = 0;
      cursor[n_tile + 1 + idx] = 0;  // the short entries' cursor (filled from the end)
      if (c[i] > 0) list[run >> TS_SHIFT] = (int32_t)idx;
      run += (long long)c[i] + ((long long)(c[i] > 0) << TS_SHIFT);
      if (idx == n_tile - 1) {
        const long long tot = run & mask;
        off[n_tile] = (int32_t)(tot > 0x7fffffffLL ? 0x7fffffff : tot);
        list[n_tile] = (int32_t)(run >> TS_SHIFT);
        if (tot > pair_cap) ps_record_error(status, PS_ERR_CAPACITY);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Coverage.  Two 256-thread CTAs per SM (one's warps issue while the other's
// wait at a tile barrier), persistent over tiles.  Per tile each
// warp runs its own queue: it takes the next 32 bin entries, each lane sets one
// up (the path's mask slot from a shared hash, the edge functions relative to
// the tile, the pixel span of every pixel row the quad can reach), a warp scan
// flattens the entries' pixels so that every lane gets two pixels at a time, and
// each pixel's 16-sample mask is ORed into the path's mask in shared memory.
// Block-wide barriers only open and close a tile: per-path popcounts and the
// canvas OR are taken there.  Paths beyond SLOTS per tile take further passes.
constexpr int CV_NT = 256;
constexpr int CV_WARPS = CV_NT / 32;
constexpr int SLOTS = 96;            // per-path masks resident in shared memory
constexpr int HKEYS = 1024;          // hash of path ids (max distinct paths per tile)
constexpr int MASK_WORDS = TILE_PX * TILE_PX / 2;

struct Edge {
  int A, B;       // E(x, y) = A (x - ex) + B (y - ey), tile-relative 1/256 px
  int ex, ey;     // the edge's start vertex
};

// General form: convex quad in e[0..3], else triangle 0 in e[0..2] and
// triangle 1 in e[3..5], each edge as {A, B, ex, ey}.  Fast forms: one convex
// polygon of at most four edges in e[0..3] (bit5), or the union of two
// triangles e[0..2], e[3..5] (bit6), each edge stored as {A, B, C15, i1}:
// A (x - 8) + B (y - 8) + C' is the edge function (C' clamped, see
// to_fast_edge), C15 = C' + 240 A + 176 B its value at sample 15 (see
// fast_mask), and i1 = 16 A + 80 B the step between consecutive samples whose
// sample row advances by 5.
struct __align__(16) EntrySetup {
  Edge e[6];               // 16 bytes each, read as int4
  uint16_t rowpre[17];     // prefix of span widths (16-byte aligned; 0xffff past the last row)
  uint8_t x0[16];          // first pixel of each row's span (rows row0 ..)
  uint16_t slot;           // mask slot of this pass
  uint8_t valid;           // bit0 tri 0, bit1 tri 1, bit2 int64 path, bit3 convex quad,
                           // bit4 int32 path, bit5 fast convex form, bit6 fast two-triangle
                           // form
  uint8_t row0, nrow;
};

static_assert(sizeof(Edge) == 16 && sizeof(EntrySetup) % 16 == 0 && offsetof(EntrySetup, e) == 0,
              "edges are loaded as int4 from shared memory");
static_assert(offsetof(EntrySetup, rowpre) % 16 == 0, "rowpre is filled with two 16-byte stores");

__device__ __forceinline__ void make_edges(int x0, int y0, int x1, int y1, int x2, int y2, Edge* e,
                                           bool& valid, bool& big) {
  long long area = (long long)(x1 - x0) * (y2 - y0) - (long long)(y1 - y0) * (x2 - x0);
  valid = area != 0;
  if (area < 0) {
    int t = x1; x1 = x2; x2 = t;
    t = y1; y1 = y2; y2 = t;
  }
  int vx[3] = {x0, x1, x2}, vy[3] = {y0, y1, y2};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    int ax = vx[i], ay = vy[i], bx = vx[(i + 1) % 3], by = vy[(i + 1) % 3];
    long long A = (long long)ay - by, B = (long long)bx - ax;  // E = (bx-ax)(y-ay) - (by-ay)(x-ax)
    e[i].A = (int)A;
    e[i].B = (int)B;
    e[i].ex = ax;
    e[i].ey = ay;
    if (llabs(A) + llabs(B) >= (1ll << 22)) big = true;
  }
}

// 16-sample mask of one edge given its value Ec at the pixel corner: sample k
// passes iff Ec + A (16k+8) + B (16((5k) mod 16)+8) >= 0.
__device__ __forceinline__ uint32_t edge_mask(const Edge& e, long long Ec, bool big) {
  if (!big) {
    long long D = 248ll * (llabs((long long)e.A) + llabs((long long)e.B));
    if (Ec - D >= 0) return 0xffffu;
    if (Ec + D < 0) return 0u;
    int E0 = (int)Ec, A = e.A, B = e.B;  // |E0| < D < 2^30: sums fit in int32
    uint32_t em = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      int v = E0 + A * (16 * k + 8) + B * (16 * ((5 * k) & 15) + 8);
      em |= (v >= 0 ? 1u : 0u) << k;
    }
    return em;
  }
  uint32_t em = 0;
  for (int k = 0; k < 16; ++k) {
    long long v = Ec + (long long)e.A * (16 * k + 8) + (long long)e.B * (16 * ((5 * k) & 15) + 8);
    em |= (v >= 0 ? 1u : 0u) << k;
  }
  return em;
}

// Same with every quantity known to fit in int32 (edges shorter than 64 px whose
// start vertices lie within 128 px of the tile).
__device__ __forceinline__ uint32_t edge_mask32(const Edge& e, int Ec) {
  int D = 248 * (abs(e.A) + abs(e.B));
  if (Ec - D >= 0) return 0xffffu;
  if (Ec + D < 0) return 0u;
  uint32_t em = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    int v = Ec + e.A * (16 * k + 8) + e.B * (16 * ((5 * k) & 15) + 8);
    em |= (v >= 0 ? 1u : 0u) << k;
  }
  return em;
}

// {A, B, ex, ey} -> fast form {A, B, C15, i1} (requires |A| + |B| < 2^18).
__device__ __forceinline__ void to_fast_edge(Edge& ed) {
  long long A = ed.A, B = ed.B, S = llabs(A) + llabs(B);
  // value at sample 0 of the tile's first pixel: A (8 - ex) + B (8 - ey)
  long long c = A * (8ll - ed.ex) + B * (8ll - ed.ey);
  // Over the tile the value moves by at most 3840 S between pixel corners and
  // 240 S between samples: beyond +-(4080 S + 1) the sign of every sample is
  // fixed, so clamping there changes no sample.
  long long lim = 4080ll * S + 1;
  c = c > lim ? lim : (c < -lim ? -lim : c);
  // stored as the value at sample 15 (15 columns, 11 sample rows further),
  // where the masks start
  ed.ex = (int)(c + 240 * A + 176 * B);
  ed.ey = (int)(16 * A + 80 * B);
}

// Pixel rows whose sample band [256 ly + 8, 256 ly + 248] meets [ymin, ymax].
// (ymin, ymax are tile-relative: snapped coordinates and tile origins are both
// below 2^29 in magnitude, so int32 holds every step.)
__device__ __forceinline__ int entry_rows(int ymin, int ymax, int th, EntrySetup& E) {
  const int c0 = -((248 - ymin) >> 8), c1 = (ymax - 8) >> 8;  // ceil, floor of / 256
  int ly0 = c0 < 0 ? 0 : c0;
  int ly1 = c1 > th - 1 ? th - 1 : c1;
  if (ly1 < ly0) return 0;
  E.row0 = (uint8_t)ly0;
  E.nrow = (uint8_t)(ly1 - ly0 + 1);
  return ly1 - ly0 + 1;
}

// Edge lists of the fast forms as pairs of polygon vertex indices (polygon
// order N0 P0 P1 N1 = 0 1 2 3), 4 bits per edge (start | end << 2), six edges;
// 0x0 (start = end) is the always-true edge A = B = 0.
constexpr uint32_t EL_CONVEX_POS = 0x4u | 0x9u << 4 | 0xEu << 8 | 0x3u << 12;  // 0->1 1->2 2->3 3->0
constexpr uint32_t EL_CONVEX_NEG = 0xCu | 0xBu << 4 | 0x6u << 8 | 0x1u << 12;  // 0->3 3->2 2->1 1->0
constexpr uint32_t EL_TRI0_POS = 0x4u | 0x9u << 4 | 0x2u << 8;   // 0->1 1->2 2->0
constexpr uint32_t EL_TRI0_NEG = 0x8u | 0x6u << 4 | 0x1u << 8;   // 0->2 2->1 1->0
constexpr uint32_t EL_TRI1_POS = 0x8u | 0xEu << 4 | 0x3u << 8;   // 0->2 2->3 3->0
constexpr uint32_t EL_TRI1_NEG = 0xCu | 0xBu << 4 | 0x2u << 8;   // 0->3 3->2 2->0

// Setup of a quad whose extent is below 2^16 (256 px) on both axes: the cross
// products of vertex differences are formed in int64, every edge has
// |A| + |B| < 2^17 (inside the fast form's 2^18), and the fast-form constant
// A (8 - x) + B (8 - y) is formed in int64 (|8 - x| < 2^16 + 4104, as the quad
// meets the tile) and clamped into int32.  One code path serves all classes.
__device__ __forceinline__ int setup_small(const QuadFix& q, int ymin, int ymax, int tw, int th,
                                           EntrySetup& E, int* __restrict__ sc) {
  const int X0 = q.x[0], Y0 = q.y[0], X1 = q.x[1], Y1 = q.y[1];  // N0 P0
  const int X2 = q.x[3], Y2 = q.y[3], X3 = q.x[2], Y3 = q.y[2];  // P1 N1
  auto cross = [](int ax, int ay, int bx, int by) {
    return (long long)ax * by - (long long)ay * bx;
  };
  const long long a0 = cross(X1 - X0, Y1 - Y0, X2 - X0, Y2 - Y0);  // N0 P0 P1
  const long long a1 = cross(X2 - X0, Y2 - Y0, X3 - X0, Y3 - Y0);  // N0 P1 N1
  if (a0 == 0 && a1 == 0) return 0;
  // turns at the four corners of N0 P0 P1 N1
  const long long c0 = cross(X1 - X0, Y1 - Y0, X2 - X1, Y2 - Y1);
  const long long c1 = cross(X2 - X1, Y2 - Y1, X3 - X2, Y3 - Y2);
  const long long c2 = cross(X3 - X2, Y3 - Y2, X0 - X3, Y0 - Y3);
  const long long c3 = cross(X0 - X3, Y0 - Y3, X1 - X0, Y1 - Y0);
  bool pos = c0 >= 0 && c1 >= 0 && c2 >= 0 && c3 >= 0;
  bool neg = c0 <= 0 && c1 <= 0 && c2 <= 0 && c3 <= 0;
  uint32_t el0 = a0 > 0 ? EL_TRI0_POS : EL_TRI0_NEG;
  uint32_t el1 = a1 > 0 ? EL_TRI1_POS : EL_TRI1_NEG;
  // class and edge list by selects: a convex quad, two triangles (diagonal
  // first, as triangle 0 orients it, then the other two edges of each
  // triangle; slot 5 unused), or the one real triangle
  const bool both = a0 != 0 && a1 != 0, convex = both && (pos || neg);
  const uint32_t d0 = a0 > 0 ? 0x2u : 0x8u;            // 2->0 or 0->2
  const uint32_t t0 = a0 > 0 ? (0x4u | 0x9u << 4)      // 0->1 1->2
                             : (0x6u | 0x1u << 4);     // 2->1 1->0
  const uint32_t t1 = a1 > 0 ? (0xEu | 0x3u << 4)      // 2->3 3->0
                             : (0xCu | 0xBu << 4);     // 0->3 3->2
  const uint32_t el = convex ? (pos ? EL_CONVEX_POS : EL_CONVEX_NEG)
                      : both ? (d0 | t0 << 4 | t1 << 12)
                             : (a0 != 0 ? el0 : el1);
  const uint8_t cls = convex ? (8 | 32) : both ? 64 : 32;
  const bool two = cls == 64;
  // Per edge, the line A X + B Y + C' = 0 (X = x - 8, Y = y - 8) as X = k Y + u.
  // An edge with A > 0 bounds X from below: over a row's sample band
  // Y in [Y0, Y0 + 240] by k Y0 + u + min(0, 240 k) - eps, kept as wl(Y0) =
  // fma(k, Y0, ul).  A < 0 bounds X from above; its bound is kept negated,
  // wh(Y0) = fma(-k, Y0, uh), so both kinds reduce with max.  Edges with A = 0
  // (horizontal, or the always-true edge) bound nothing here.  eps covers the
  // float rounding of k, u and the fma (a few 2^-24 relative to |u| + 4096 |k|).
  // Each edge keeps ul and uh, the side it does not bound set to -inf, so that
  // a row reduces both sides with one fma and one max each.
  float kq[6], ul[6], uh[6];
  float k0 = 0.f, u0 = 0.f, eps0 = 0.f;
  bool apos0 = false, anz0 = false;
  // The polygon's vertices, parked in the lane's column of a warp scratch
  // (sc: one int per lane per row, so that the lanes' accesses fall in
  // distinct banks) so that each edge reads its end points by index instead
  // of through chains of selects.
  sc[0] = X0; sc[32] = X1; sc[64] = X2; sc[96] = X3;     // x of vertex v at sc[32 v],
  sc[128] = Y0; sc[160] = Y1; sc[192] = Y2; sc[224] = Y3;  // y at sc[32 (4 + v)]
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    int ia = (el >> (4 * i)) & 3, ib = (el >> (4 * i + 2)) & 3;
    int xa = sc[32 * ia], ya = sc[32 * (4 + ia)], xb = sc[32 * ib], yb = sc[32 * (4 + ib)];
    int A = ya - yb, B = xb - xa, S = abs(A) + abs(B);
    long long c64 = (long long)A * (8 - xa) + (long long)B * (8 - ya);
    int lim = 4080 * S + 1;
    int c = (int)(c64 > lim ? lim : (c64 < -lim ? -lim : c64));
    *reinterpret_cast<int4*>(&E.e[i]) = make_int4(A, B, c + 240 * A + 176 * B, 16 * A + 80 * B);
    float fa = (float)A;
    float k = __fdividef((float)-B, fa), u = __fdividef((float)-c, fa);
    float eps = 4.f + 1e-6f * (fabsf(u) + 4096.f * fabsf(k));
    float k240 = 240.f * k;
    if (i == 0) {
      k0 = k;
      u0 = u;
      eps0 = eps;
      apos0 = A > 0;
      anz0 = A != 0;
    }
    // branch-free: k and u are not finite when A = 0, and are not used then
    const float lo_b = u + fminf(0.f, k240) - eps, hi_b = -(u + fmaxf(0.f, k240) + eps);
    kq[i] = A > 0 ? k : (A < 0 ? -k : 0.f);
    ul[i] = A > 0 ? lo_b : -INFINITY;
    uh[i] = A < 0 ? hi_b : -INFINITY;
  }
  E.valid = cls | (a0 != 0 ? 1 : 0) | (a1 != 0 ? 2 : 0);
  if (two) {
    // With F(p) = cross(P1 - N0, p - N0), triangle 0's diagonal edge is
    // -sgn(a0) F and triangle 1's is sgn(a1) F.  When a0 and a1 have the same
    // sign the triangles lie on opposite sides and triangle 1 needs e[0] <= 0,
    // taken as e[0] < 0 (the sign bit of ~e[0]): a sample on the diagonal inside
    // triangle 1 lies on the segment N0 P1, which triangle 0 also covers.
    // Otherwise triangle 1 needs e[0] >= 0 like triangle 0.  e[5].A holds the
    // word XORed into e[0] for triangle 1's test.
    E.e[5].A = (a0 > 0) == (a1 > 0) ? -1 : 0;
  }
  if (entry_rows(ymin, ymax, th, E) == 0) return 0;
  {
    // slot 5 for spans: triangle 1's diagonal bound (e[0] reversed when the
    // triangles lie on opposite sides, else e[0] itself); a horizontal diagonal
    // bounds no x and leaves slot 5 as the always-true edge (branch-free)
    const bool use5 = two && anz0;
    const bool lo5 = ((a0 > 0) == (a1 > 0)) ? !apos0 : apos0;
    const float k240 = 240.f * k0;
    kq[5] = use5 ? (lo5 ? k0 : -k0) : kq[5];
    ul[5] = use5 ? (lo5 ? u0 + fminf(0.f, k240) - eps0 : -INFINITY) : ul[5];
    uh[5] = use5 ? (lo5 ? -INFINITY : -(u0 + fmaxf(0.f, k240) + eps0)) : uh[5];
  }
  // row spans: group 0 = edges 0..3 (triangle 0 and, for a convex quad, the
  // fourth edge), group 1 = edges 3..5 of the two-triangle form; union of groups
  const bool e3g1 = two;
  // The loop runs the entry's own rows only (a warp runs the most any of its
  // lanes has); prefixes past the last row stay 0xffff, above every item index.
  int tot = 0;
  reinterpret_cast<uint4*>(E.rowpre)[0] = make_uint4(~0u, ~0u, ~0u, ~0u);
  reinterpret_cast<uint4*>(E.rowpre)[1] = make_uint4(~0u, ~0u, ~0u, ~0u);
  E.rowpre[0] = 0;
  const int nrow = E.nrow;
  for (int j = 0; j < nrow; ++j) {
    int wj = 0, aj = 0;
    {
      const float Yb = 256.f * (float)(E.row0 + j);
      float L0 = -INFINITY, M0 = -INFINITY, L1 = -INFINITY, M1 = -INFINITY;
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        // both bounds in one packed fma (each lane of it rounds as fmaf does)
        const float2 w2 = __ffma2_rn(make_float2(kq[i], kq[i]), make_float2(Yb, Yb),
                                     make_float2(ul[i], uh[i]));
        const float wl = w2.x, wh = w2.y;
        if (i >= 4) {
          L1 = fmaxf(L1, wl);
          M1 = fmaxf(M1, wh);
        } else if (i == 3) {
          L1 = e3g1 ? fmaxf(L1, wl) : L1;
          M1 = e3g1 ? fmaxf(M1, wh) : M1;
          L0 = e3g1 ? L0 : fmaxf(L0, wl);
          M0 = e3g1 ? M0 : fmaxf(M0, wh);
        } else {
          L0 = fmaxf(L0, wl);
          M0 = fmaxf(M0, wh);
        }
      }
      const float hi0 = -M0, hi1 = -M1;
      const bool ok0 = L0 <= hi0, ok1 = two && L1 <= hi1;
      // union of the groups' extents (an empty group adds nothing); the
      // float-to-int conversions saturate, so an unbounded side (+-inf) gives
      // pixel 0 or tw - 1 and an empty row gives pb < pa
      const float lo = fminf(ok0 ? L0 : INFINITY, ok1 ? L1 : INFINITY);
      const float hi = fmaxf(ok0 ? hi0 : -INFINITY, ok1 ? hi1 : -INFINITY);
      const int pa = max(0, __float2int_ru((lo - 240.f) * (1.f / 256.f)));
      const int pb = min(tw - 1, __float2int_rd(hi * (1.f / 256.f)));
      if (pb >= pa) {
        aj = pa;
        wj = pb - pa + 1;
      }
      E.x0[j] = (uint8_t)aj;
    }
    tot += wj;
    E.rowpre[j + 1] = (uint16_t)tot;
  }
  return tot;
}

__device__ __forceinline__ void row_span(const EntrySetup& E, int ly, int tw, int& a, int& w);
__device__ __forceinline__ void row_span_fast(const EntrySetup& E, int ly, int tw, int& a, int& w);

// Row spans of an entry set up by the general path (per row, as above).
__device__ __forceinline__ int finish_spans(EntrySetup& E, int tw) {
  int tot = 0;
  E.rowpre[0] = 0;
  for (int j = 0; j < 16; ++j) {
    if (j < E.nrow) {
      int a0, w0;
      if (E.valid & 32) row_span_fast(E, E.row0 + j, tw, a0, w0);
      else row_span(E, E.row0 + j, tw, a0, w0);
      E.x0[j] = (uint8_t)a0;
      tot += w0;
    }
    E.rowpre[j + 1] = (uint16_t)tot;
  }
  return tot;
}

// Exact quad coverage (the crossing rule: a sample is covered iff the ray from
// it towards +x crosses an odd number of the edges of N0 -> P0 -> P1 -> N1 ->
// N0; edge a -> b is crossed iff a.y <= y < b.y with the sample strictly left
// of it, or b.y <= y < a.y with the sample strictly right of it).  Per edge the
// function is stored sign-normalised, F = -E for edges going up (b.y > a.y)
// and E otherwise, so that a crossing is F < 0 inside the edge's y-range
// [ylo, yhi) (empty for horizontal edges).  The y-ranges go to e[4] and e[5];
// the edges to e[0..3], in the fast form (|A| + |B| < 2^18) or else as
// {A, B, ex, ey} for the int64 path.  Runs after the spans were taken from the
// class edges (spans of the two diagonal-split triangles contain the polygon).
__device__ __forceinline__ void store_exact(const QuadFix& q, EntrySetup& E) {
  const int px[4] = {q.x[0], q.x[1], q.x[3], q.x[2]}, py[4] = {q.y[0], q.y[1], q.y[3], q.y[2]};
  long long smax = 0;
  long long A[4], B[4];
  int yr[8];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int ax = px[i], ay = py[i], bx = px[(i + 1) & 3], by = py[(i + 1) & 3];
    long long a = (long long)ay - by, b = (long long)bx - ax;
    if (by > ay) {  // going up: F = -E
      a = -a;
      b = -b;
    }
    A[i] = a;
    B[i] = b;
    smax = max(smax, llabs(a) + llabs(b));
    yr[2 * i] = min(ay, by);
    yr[2 * i + 1] = max(ay, by);
  }
  if (smax < (1ll << 18)) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      long long S = llabs(A[i]) + llabs(B[i]);
      long long c = A[i] * (8ll - px[i]) + B[i] * (8ll - py[i]);
      long long lim = 4080ll * S + 1;
      c = c > lim ? lim : (c < -lim ? -lim : c);
      E.e[i].A = (int)A[i];
      E.e[i].B = (int)B[i];
      E.e[i].ex = (int)(c + 240 * A[i] + 176 * B[i]);  // at sample 15, as in to_fast_edge
      E.e[i].ey = (int)(16 * A[i] + 80 * B[i]);
    }
    E.valid = (E.valid & ~(64 | 8)) | 32;
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      E.e[i].A = (int)A[i];
      E.e[i].B = (int)B[i];
      E.e[i].ex = px[i];
      E.e[i].ey = py[i];
    }
    E.valid = E.valid & ~(32 | 64 | 8);
  }
  *reinterpret_cast<int4*>(&E.e[4]) = make_int4(yr[0], yr[1], yr[2], yr[3]);
  *reinterpret_cast<int4*>(&E.e[5]) = make_int4(yr[4], yr[5], yr[6], yr[7]);
}

// Bits k of the samples whose sample row (5k mod 16) lies in [a, b): the
// y-range masks of the exact mode, rowmask[17 a + b].
__device__ __forceinline__ uint32_t row_range_mask(int a, int b) {
  uint32_t m = 0;
  for (int k = 0; k < 16; ++k) {
    int sk = (5 * k) & 15;
    if (sk >= a && sk < b) m |= 1u << k;
  }
  return m;
}

__device__ __forceinline__ uint32_t exact_yrange(int lo, int hi, int base,
                                                 const uint16_t* __restrict__ rowmask) {
  // samples of the row at y = base + 16 s: in range iff ceil((lo-base)/16) <= s < ceil((hi-base)/16)
  int a = (lo - base + 15) >> 4, b = (hi - base + 15) >> 4;
  a = min(max(a, 0), 16);
  b = min(max(b, 0), 16);
  return rowmask[17 * a + b];
}

// Fast exact mask: the four sign-normalised edge values stepped from sample to
// sample as in fast_mask (the same clamped C', C15 and int32 bounds), one sign
// mask per edge, each limited to its edge's y-range; the parity of the
// crossings.
__device__ __forceinline__ uint32_t exact_mask(const EntrySetup& E, int cx, int cy,
                                               const uint16_t* __restrict__ rowmask) {
  int v[4], i1[4], i2[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int4 ed = *reinterpret_cast<const int4*>(&E.e[i]);
    v[i] = ed.z + ed.x * cx + ed.y * cy;  // at sample 15
    i1[i] = ed.w;
    i2[i] = ed.w - ed.y * 256;
  }
  // samples from 15 down to 0, as in fast_mask
  uint32_t sg[4] = {0u, 0u, 0u, 0u};
#pragma unroll
  for (int k = 15; k >= 0; --k) {
#pragma unroll
    for (int i = 0; i < 4; ++i) sg[i] = __funnelshift_l((uint32_t)v[i], sg[i], 1);
    if (k > 0) {
      const bool up = ((5 * (k - 1)) & 15) <= 10;
#pragma unroll
      for (int i = 0; i < 4; ++i) v[i] -= up ? i1[i] : i2[i];
    }
  }
  const int4 ya = *reinterpret_cast<const int4*>(&E.e[4]);
  const int4 yb = *reinterpret_cast<const int4*>(&E.e[5]);
  const int base = cy + 8;
  uint32_t c = (sg[0] & exact_yrange(ya.x, ya.y, base, rowmask)) ^
               (sg[1] & exact_yrange(ya.z, ya.w, base, rowmask)) ^
               (sg[2] & exact_yrange(yb.x, yb.y, base, rowmask)) ^
               (sg[3] & exact_yrange(yb.z, yb.w, base, rowmask));
  return c & 0xffffu;
}

// The same rule in int64 for quads with an edge of |A| + |B| >= 2^18.
__device__ __forceinline__ uint32_t exact_mask_general(const EntrySetup& E, int lx, int ly) {
  const int4 ya = *reinterpret_cast<const int4*>(&E.e[4]);
  const int4 yb = *reinterpret_cast<const int4*>(&E.e[5]);
  const int lo[4] = {ya.x, ya.z, yb.x, yb.z}, hi[4] = {ya.y, ya.w, yb.y, yb.w};
  uint32_t m = 0;
  for (int k = 0; k < 16; ++k) {
    long long sx = 256ll * lx + 16 * k + 8, sy = 256ll * ly + 16 * ((5 * k) & 15) + 8;
    uint32_t c = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      long long F = (long long)E.e[i].A * (sx - E.e[i].ex) + (long long)E.e[i].B * (sy - E.e[i].ey);
      c ^= (sy >= lo[i] && sy < hi[i] && F < 0) ? 1u : 0u;
    }
    m |= c << k;
  }
  return m;
}

// Edges and row spans of the quad between ribs ra, rb in tile (ox, oy);
// returns the number of pixels in its spans (0: nothing to draw).
template <bool EXACT>
__device__ __forceinline__ int setup_edges(const float4 ra, const float4 rb, int slot, int ox,
                                           int oy, int tw, int th, EntrySetup& E,
                                           int* __restrict__ sc) {
  E.slot = (uint16_t)slot;
  E.valid = 0;
  E.row0 = 0;
  E.nrow = 0;
  QuadFix q;
  if (!snap_quad(ra, rb, q)) return 0;
  for (int v = 0; v < 4; ++v) {
    q.x[v] -= ox;
    q.y[v] -= oy;
  }
  {
    int mnx = min(min(q.x[0], q.x[1]), min(q.x[2], q.x[3]));
    int mxx = max(max(q.x[0], q.x[1]), max(q.x[2], q.x[3]));
    int mny = min(min(q.y[0], q.y[1]), min(q.y[2], q.y[3]));
    int mxy = max(max(q.y[0], q.y[1]), max(q.y[2], q.y[3]));
    if (mxx - mnx < (1 << 16) && mxy - mny < (1 << 16)) {
      int tot = setup_small(q, mny, mxy, tw, th, E, sc);
      if (EXACT && tot > 0) store_exact(q, E);
      return tot;
    }
  }
  bool v0, v1, big = false;
  make_edges(q.x[0], q.y[0], q.x[1], q.y[1], q.x[3], q.y[3], E.e, v0, big);      // N0 P0 P1
  make_edges(q.x[0], q.y[0], q.x[3], q.y[3], q.x[2], q.y[2], E.e + 3, v1, big);  // N0 P1 N1
  if (!v0 && !v1) return 0;
  uint8_t flags = (v0 ? 1 : 0) | (v1 ? 2 : 0);
  if (v0 && v1) {
    // both triangles real and the polygon N0 P0 P1 N1 convex (no turn of the
    // opposite sense): their union is the polygon, four edges instead of six
    int px_[4] = {q.x[0], q.x[1], q.x[3], q.x[2]}, py_[4] = {q.y[0], q.y[1], q.y[3], q.y[2]};
    bool pos = true, neg = true;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int j = (i + 1) & 3, k2 = (i + 2) & 3;
      long long c = (long long)(px_[j] - px_[i]) * (py_[k2] - py_[j]) -
                    (long long)(py_[j] - py_[i]) * (px_[k2] - px_[j]);
      pos = pos && c >= 0;
      neg = neg && c <= 0;
    }
    if (pos || neg) {
      bool bigq = false;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        int a0 = neg ? (4 - i) & 3 : i, a1 = neg ? (3 - i) & 3 : (i + 1) & 3;
        long long A = (long long)py_[a0] - py_[a1], B = (long long)px_[a1] - px_[a0];
        E.e[i].A = (int)A;
        E.e[i].B = (int)B;
        E.e[i].ex = px_[a0];
        E.e[i].ey = py_[a0];
        if (llabs(A) + llabs(B) >= (1ll << 22)) bigq = true;
      }
      big = bigq;
      flags |= 8;
    }
  }
  // int32 evaluation is exact when |A|,|B| < 2^14 and every start vertex is
  // within 2^15 (128 px) of the tile: |A (x - ex)| + |B (y - ey)| < 2^31
  bool small = !big;
  int ne = (flags & 8) ? 4 : 6;
  for (int i = 0; i < ne; ++i) {
    const Edge& ed = E.e[i];
    if ((i < 3 && !(flags & 1) && !(flags & 8)) || (i >= 3 && !(flags & 2))) continue;
    small = small && abs(ed.A) < (1 << 14) && abs(ed.B) < (1 << 14) && ed.ex > -(1 << 15) &&
            ed.ex < (1 << 15) + TILE_UNITS && ed.ey > -(1 << 15) && ed.ey < (1 << 15) + TILE_UNITS;
  }
  E.valid = flags | (big ? 4 : 0) | (small ? 16 : 0);
  // fast form: a convex quad or a single triangle whose edges all have
  // |A| + |B| < 2^18 (shorter than 1024 px); every value of fast_mask then
  // fits in int32 (see fast_mask)
  int nf = (flags & 8) ? 4 : ((flags & 3) == 1 || (flags & 3) == 2) ? 3 : 0;
  if (nf && !big) {
    const Edge* src = (flags & 8) || (flags & 1) ? E.e : E.e + 3;
    long long smax = 0;
    for (int i = 0; i < nf; ++i) smax = max(smax, llabs((long long)src[i].A) + llabs((long long)src[i].B));
    if (smax < (1ll << 18)) {
      Edge f[4];
      for (int i = 0; i < nf; ++i) {
        f[i] = src[i];
        to_fast_edge(f[i]);
      }
      if (nf == 3) {  // always-true fourth edge
        f[3].A = 0;
        f[3].B = 0;
        f[3].ex = 1;
        f[3].ey = 0;
      }
      for (int i = 0; i < 4; ++i) E.e[i] = f[i];
      E.valid |= 32;
    }
  }
  int ymin = min(min(q.y[0], q.y[1]), min(q.y[2], q.y[3]));
  int ymax = max(max(q.y[0], q.y[1]), max(q.y[2], q.y[3]));
  if (entry_rows(ymin, ymax, th, E) == 0) return 0;
  int tot = finish_spans(E, tw);
  if (EXACT && tot > 0) store_exact(q, E);
  return tot;
}

// x-extent of the region where the given edges are all >= 0, over the sample
// band of pixel row ly (conservative: float, widened by eps).  Each edge with
// A != 0 bounds x on one side: x >= xe(y) for A > 0, x <= xe(y) for A < 0, with
// xe(y) = ex - (B / A)(y - ey); over the band the weakest bound is taken.
__device__ __forceinline__ bool band_extent(const Edge* e, int ne, int ly, float& lo, float& hi) {
  float ylo = 256.f * ly + 8.f, yhi = 256.f * ly + 248.f;
  lo = -3.4e38f;
  hi = 3.4e38f;
  for (int i = 0; i < ne; ++i) {
    float A = (float)e[i].A, B = (float)e[i].B, ex = (float)e[i].ex, ey = (float)e[i].ey;
    if (e[i].A == 0) {
      // E = B (y - ey): some sample row of the band must have E >= 0
      float m = fmaxf(B * (ylo - ey), B * (yhi - ey));
      if (m < -4.f * fabsf(B) - 1.f) return false;
      continue;
    }
    float k = B / A;
    float xa = ex - k * (ylo - ey), xb = ex - k * (yhi - ey);
    float eps = 4.f + 1e-6f * (fabsf(ex) + fabsf(xa) + fabsf(xb) + fabsf(ey) + 4096.f);
    if (e[i].A > 0) lo = fmaxf(lo, fminf(xa, xb) - eps);
    else hi = fminf(hi, fmaxf(xa, xb) + eps);
  }
  return hi >= lo;
}

__device__ __forceinline__ void row_span(const EntrySetup& E, int ly, int tw, int& a, int& w) {
  float lo, hi;
  bool ok;
  if (E.valid & 8) {
    ok = band_extent(E.e, 4, ly, lo, hi);
  } else {
    float l0 = 3.4e38f, h0 = -3.4e38f, l1, h1;
    ok = false;
    if ((E.valid & 1) && band_extent(E.e, 3, ly, l1, h1)) {
      l0 = fminf(l0, l1);
      h0 = fmaxf(h0, h1);
      ok = true;
    }
    if ((E.valid & 2) && band_extent(E.e + 3, 3, ly, l1, h1)) {
      l0 = fminf(l0, l1);
      h0 = fmaxf(h0, h1);
      ok = true;
    }
    lo = l0;
    hi = h0;
  }
  a = 0;
  w = 0;
  if (!ok) return;
  // pixels whose samples x in [256 lx + 8, 256 lx + 248] can lie in [lo, hi]
  lo = fmaxf(lo, -1e9f);
  hi = fminf(hi, 1e9f);
  int pa = max(0, (int)ceilf((lo - 248.f) / 256.f));
  int pb = min(tw - 1, (int)floorf((hi - 8.f) / 256.f));
  if (pb >= pa) {
    a = pa;
    w = pb - pa + 1;
  }
}

// 16-sample mask of a fast-form entry at pixel corner (cx, cy) (tile-relative,
// 1/256 px).  Per edge, v = C15 + A cx + B cy is the value at sample 15, with
// C15 = C' + 240 A + 176 B, and stepping visits the values at the other
// samples.  Each is C' + A (x - 8) + B (y - 8) at a sample (x, y) of the tile,
// 0 <= x - 8, y - 8 <= 4080; with S = |A| + |B| < 2^18 and |C'| <= 4080 S + 1
// it stays within 8160 S + 1 < 2^31, and the clamp of C' (see to_fast_edge)
// changed no sign.  A sample is covered iff no edge is negative there: the
// sign bit of the OR of the four values.  The samples are visited from 15 down
// to 0, so that each sign bit enters the mask with one funnel shift.
__device__ __forceinline__ uint32_t fast_mask(const EntrySetup& E, int cx, int cy) {
  int v[4], i1[4], i2[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int4 ed = *reinterpret_cast<const int4*>(&E.e[i]);
    v[i] = ed.z + ed.x * cx + ed.y * cy;  // at sample 15
    i1[i] = ed.w;                 // sample row + 5
    i2[i] = ed.w - ed.y * 256;    // sample row - 11
  }
  uint32_t neg = 0;
#pragma unroll
  for (int k = 15; k >= 0; --k) {
    uint32_t o = (uint32_t)(v[0] | v[1] | v[2] | v[3]);
    neg = __funnelshift_l(o, neg, 1);  // neg << 1 | o >> 31
    if (k > 0) {
      const bool up = ((5 * (k - 1)) & 15) <= 10;  // sample k's row is 5 above sample k-1's
#pragma unroll
      for (int i = 0; i < 4; ++i) v[i] -= up ? i1[i] : i2[i];
    }
  }
  return ~neg & 0xffffu;
}

// Two-triangle fast form: e[0] is the shared diagonal (as triangle 0 orients
// it), e[1], e[2] triangle 0's other edges, e[3], e[4] triangle 1's, and
// e[5].A the word XORed into e[0] for triangle 1 (see setup_small).  A sample
// is covered iff one triangle has no failing edge there (same bounds as
// fast_mask).
__device__ __forceinline__ uint32_t fast_mask2(const EntrySetup& E, int cx, int cy) {
  const uint32_t x1 = (uint32_t)E.e[5].A;
  int v[5], i1[5], i2[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int4 ed = *reinterpret_cast<const int4*>(&E.e[i]);
    v[i] = ed.z + ed.x * cx + ed.y * cy;  // at sample 15
    i1[i] = ed.w;
    i2[i] = ed.w - ed.y * 256;
  }
  uint32_t neg = 0;
#pragma unroll
  for (int k = 15; k >= 0; --k) {
    uint32_t f0 = (uint32_t)(v[0] | v[1] | v[2]);
    uint32_t f1 = ((uint32_t)v[0] ^ x1) | (uint32_t)(v[3] | v[4]);
    neg = __funnelshift_l(f0 & f1, neg, 1);
    if (k > 0) {
      const bool up = ((5 * (k - 1)) & 15) <= 10;
#pragma unroll
      for (int i = 0; i < 5; ++i) v[i] -= up ? i1[i] : i2[i];
    }
  }
  return ~neg & 0xffffu;
}

// Conservative pixel span of a fast-form entry on pixel row ly: each edge with
// A != 0 bounds x on one side over the row's sample band, x >= or <= 8 - (B
// (y - 8) + C') / A; an edge with A == 0 rules the row out when it is negative
// on the whole band.  Float, widened by eps.
template <int N>
__device__ __forceinline__ bool band_extent_fast(const Edge* e, float y0, float& lo, float& hi) {
  float y1 = y0 + 240.f;  // sample rows y - 8 of the band: [y0, y0 + 240]
  lo = -3.4e38f;
  hi = 3.4e38f;
  bool dead = false;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const int4 ed = *reinterpret_cast<const int4*>(&e[i]);
    // the stored constant is the value at sample 15; C' is the one at sample 0
    float A = (float)ed.x, B = (float)ed.y, C = (float)(ed.z - 240 * ed.x - 176 * ed.y);
    float n0 = fmaf(B, y0, C), n1 = fmaf(B, y1, C);
    float mag = fabsf(C) + 4096.f * fabsf(B);
    if (ed.x == 0) {
      dead = dead || fmaxf(n0, n1) < -(4.f + 1e-6f * mag);
      continue;
    }
    float r = __frcp_rn(A);
    float xa = 8.f - n0 * r, xb = 8.f - n1 * r;
    float eps = 4.f + 1e-6f * (mag * fabsf(r) + fabsf(xa) + fabsf(xb));
    if (ed.x > 0) lo = fmaxf(lo, fminf(xa, xb) - eps);
    else hi = fminf(hi, fmaxf(xa, xb) + eps);
  }
  return !dead && hi >= lo;
}

__device__ __forceinline__ void row_span_fast(const EntrySetup& E, int ly, int tw, int& a, int& w) {
  float y0 = 256.f * ly;
  float lo, hi;
  bool ok;
  ok = band_extent_fast<4>(E.e, y0, lo, hi);  // convex fast form (general path)
  a = 0;
  w = 0;
  if (!ok) return;
  lo = fmaxf(lo, -1e9f);
  hi = fminf(hi, 1e9f);
  int pa = max(0, (int)ceilf((lo - 248.f) * (1.f / 256.f)));
  int pb = min(tw - 1, (int)floorf((hi - 8.f) * (1.f / 256.f)));
  if (pb >= pa) {
    a = pa;
    w = pb - pa + 1;
  }
}

// The general form's mask (quads of 256 px or more: int64 or int32 edge
// values, up to six edges), out of line: it is rare, and inlined into the item
// loop it slowed the fast forms (12.25 ms against 12.02 out of line on the
// bench workload; moving the general form's set-up out of line as well cost
// more than it saved).
__device__ __noinline__ uint32_t tri_or_quad_mask(const EntrySetup& E, int lx, int ly) {
  int cx = lx * 256, cy = ly * 256;
  bool big = (E.valid & 4) != 0;
  if (E.valid & 16) {  // int32 path
    if (E.valid & 8) {
      uint32_t m = 0xffffu;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        int Ec = E.e[i].A * (cx - E.e[i].ex) + E.e[i].B * (cy - E.e[i].ey);
        m &= edge_mask32(E.e[i], Ec);
        if (!m) return 0u;
      }
      return m;
    }
    uint32_t m0 = 0, m1 = 0;
    if (E.valid & 1) {
      m0 = 0xffffu;
      for (int i = 0; i < 3 && m0; ++i)
        m0 &= edge_mask32(E.e[i], E.e[i].A * (cx - E.e[i].ex) + E.e[i].B * (cy - E.e[i].ey));
    }
    if ((E.valid & 2) && m0 != 0xffffu) {
      m1 = 0xffffu;
      for (int i = 3; i < 6 && m1; ++i)
        m1 &= edge_mask32(E.e[i], E.e[i].A * (cx - E.e[i].ex) + E.e[i].B * (cy - E.e[i].ey));
    }
    return m0 | m1;
  }
  auto ev = [&](const Edge& ed) {
    return (long long)ed.A * (cx - ed.ex) + (long long)ed.B * (cy - ed.ey);
  };
  if (E.valid & 8) {
    uint32_t m = 0xffffu;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      m &= edge_mask(E.e[i], ev(E.e[i]), big);
      if (!m) return 0u;
    }
    return m;
  }
  uint32_t m0 = 0, m1 = 0;
  if (E.valid & 1) {
    m0 = 0xffffu;
    for (int i = 0; i < 3 && m0; ++i) m0 &= edge_mask(E.e[i], ev(E.e[i]), big);
  }
  if ((E.valid & 2) && m0 != 0xffffu) {
    m1 = 0xffffu;
    for (int i = 3; i < 6 && m1; ++i) m1 &= edge_mask(E.e[i], ev(E.e[i]), big);
  }
  return m0 | m1;
}

// Asynchronous global -> shared copies (cp.async, completion tracked per thread).
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <bool EXACT>
__global__ void __launch_bounds__(CV_NT, 2) k_coverage(
    const float4* __restrict__ rib, const uint32_t* __restrict__ tag,
    const int32_t* __restrict__ off, const uint32_t* __restrict__ bin, int64_t pair_cap, int W,
    int H, int y0, int tiles_x, int n_tile, const int32_t* __restrict__ tile_list,
    uint16_t* __restrict__ canvas,
    unsigned long long* __restrict__ covered, int n_path, int32_t* counters, int32_t* status,
    unsigned long long* __restrict__ stats) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* s_mask = reinterpret_cast<uint32_t*>(smem);                          // SLOTS*MASK_WORDS
  EntrySetup* s_ent = reinterpret_cast<EntrySetup*>(s_mask + SLOTS * MASK_WORDS);  // CV_NT
  static_assert((sizeof(uint32_t) * SLOTS * MASK_WORDS) % 16 == 0, "entry array alignment");
  uint32_t* s_keys = reinterpret_cast<uint32_t*>(s_ent + CV_NT);                 // HKEYS
  uint16_t* s_slot_of = reinterpret_cast<uint16_t*>(s_keys + HKEYS);             // HKEYS
  uint32_t* s_slot_path = reinterpret_cast<uint32_t*>(s_slot_of + HKEYS);        // HKEYS
  __shared__ int s_tile, s_nslot, s_next;
  __shared__ uint8_t s_own[CV_WARPS][32];
  __shared__ uint8_t s_own2[CV_WARPS][32];
  __shared__ uint32_t s_canvas[MASK_WORDS];
  __shared__ uint16_t s_rowmask[EXACT ? 17 * 17 : 1];
  // each lane's next bin entry (its two ribs and tag), copied in while the
  // current batch's pixels are processed; between reading a batch's copies and
  // issuing the next ones, a warp's 256 floats are its set-up scratch
  __shared__ __align__(16) float4 s_pre_rib[CV_WARPS][2][32];
  __shared__ uint32_t s_pre_tag[CV_WARPS][32];

  for (int i = threadIdx.x; i < SLOTS * MASK_WORDS; i += CV_NT) s_mask[i] = 0u;
  for (int i = threadIdx.x; i < MASK_WORDS; i += CV_NT) s_canvas[i] = 0u;
  if (EXACT)
    for (int i = threadIdx.x; i < 17 * 17; i += CV_NT)
      s_rowmask[i] = (uint16_t)row_range_mask(i / 17, i % 17);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  EntrySetup* my = s_ent + wid * 32;
  // work counters (items: per warp, the same in every lane; rows: per lane),
  // added to the global ones at tile ends: one atomic per warp and tile
  unsigned long long st_items = 0, st_rows = 0;
  int st_batches = 0;
  auto flush_stats = [&]() {
    for (int o = 16; o > 0; o >>= 1) st_rows += __shfl_xor_sync(0xffffffffu, st_rows, o);
    if (lane == 0 && stats && (st_items | st_rows)) {
      unsigned long long f0 = st_items & 0x1fffffu, f1 = (st_items >> 21) & 0x1fffffu,
                         f2 = st_items >> 42;
      atomicAdd(stats, f0 + f1 + f2);
      atomicAdd(stats + 1, f0);
      atomicAdd(stats + 2, f1);
      atomicAdd(stats + 3, f2);
      atomicAdd(stats + 6, st_rows);
    }
    st_items = 0;
    st_rows = 0;
    st_batches = 0;
  };
  // tiles are claimed by ticket; the next ticket's atomic is issued when a
  // tile's last pass reaches its flush, and read when the tile ends, so its
  // latency hides behind the flush (claiming earlier would hold a tile back
  // from an idle CTA)
  const int n_list = tile_list[n_tile];  // tiles with entries (the canvas is cleared)
  if (threadIdx.x == 0) s_tile = atomicAdd(&counters[2], 1);
  bool dirty = true;  // the path hash holds the previous tile's keys
  for (;;) {
    if (dirty)
      for (int i = threadIdx.x; i < HKEYS; i += CV_NT) {
        s_keys[i] = 0u;
        s_slot_of[i] = 0xffffu;
      }
    if (threadIdx.x == 0) s_nslot = 0;
    __syncthreads();
    const int ticket = s_tile;
    int t_next = 0;
    flush_stats();
    if (ticket >= n_list) return;
    const int t = tile_list[ticket];
    int tx = t % tiles_x, ty = t / tiles_x;
    int ox = tx * TILE_UNITS, oy = ty * TILE_UNITS;
    int64_t b0 = off[t], b1 = off[t + 1];
    if (b1 > pair_cap) b1 = pair_cap;
    int n = (int)(b1 > b0 ? b1 - b0 : 0);
    int tw = min(TILE_PX, W - tx * TILE_PX), th = min(TILE_PX, H - ty * TILE_PX);
    dirty = n > 0;
    if (n == 0) {  // listed but its entries are beyond the bin capacity
      if (threadIdx.x == 0) t_next = atomicAdd(&counters[2], 1);
      __syncthreads();  // every thread has read s_tile before it is rewritten
    }
    for (int pass = 0; n > 0; ++pass) {
      int slot_lo = pass * SLOTS;
      if (threadIdx.x == 0) s_next = 0;
      __syncthreads();
      // batches of 32 bin entries per warp; the next batch's entries are
      // fetched while this one is processed, and each entry's tag and two ribs
      // are gathered together
      int base_next = 0;
      if (lane == 0) base_next = atomicAdd(&s_next, 32);
      base_next = __shfl_sync(0xffffffffu, base_next, 0);
      uint32_t r_next = base_next + lane < n ? bin[b0 + base_next + lane] : 0u;
      if (base_next + lane < n) {
        cp_async4(&s_pre_tag[wid][lane], tag + r_next);
        cp_async16(&s_pre_rib[wid][0][lane], rib + r_next - 1);
        cp_async16(&s_pre_rib[wid][1][lane], rib + r_next);
      }
      cp_async_commit();
      for (;;) {
        const int base = base_next;
        if (base >= n) break;
        const int e = base + lane;
        const bool valid = e < n;
        uint32_t tg = 0u;
        float4 ra = make_float4(0.f, 0.f, 0.f, 0.f), rb = ra;
        cp_async_wait_all();
        if (valid) {
          tg = s_pre_tag[wid][lane];
          ra = s_pre_rib[wid][0][lane];
          rb = s_pre_rib[wid][1][lane];
        }
        if (lane == 0) base_next = atomicAdd(&s_next, 32);
        base_next = __shfl_sync(0xffffffffu, base_next, 0);
        if (base_next + lane < n) r_next = bin[b0 + base_next + lane];
        // slot of the entry's path: one hash probe per distinct path in the warp
        const uint32_t key = valid ? (tg >> 2) + 1u : 0u;
        const uint32_t peers = __match_any_sync(0xffffffffu, key);
        const int leader = __ffs(peers) - 1;
        int slot = -1;
        if (valid && lane == leader) {
          uint32_t h = (key * 2654435761u) & (HKEYS - 1);
          for (int it = 0; it < HKEYS; ++it) {
            uint32_t prev = pass == 0 ? atomicCAS(&s_keys[h], 0u, key) : s_keys[h];
            if (prev == 0u && pass == 0) {
              int sl = atomicAdd(&s_nslot, 1);
              if (sl < HKEYS) s_slot_path[sl] = key - 1u;
              s_slot_of[h] = (uint16_t)min(sl, HKEYS - 1);
              slot = sl;
              break;
            }
            if (prev == key) {
              uint16_t so;
              int spin = 0;
              do {  // the inserting warp may not have published the slot yet
                so = ((volatile uint16_t*)s_slot_of)[h];
              } while (so == 0xffffu && ++spin < (1 << 20));
              slot = so;
              break;
            }
            if (prev == 0u) break;
            h = (h + 1) & (HKEYS - 1);
          }
          // a full table (more than HKEYS paths on the tile) leaves the path
          // without a slot; a slot never published ends the bounded wait above
          if (slot < 0) ps_record_error(status, PS_ERR_CAPACITY);
          else if (slot >= HKEYS) ps_record_error(status, PS_ERR_TIMEOUT);
        }
        slot = __shfl_sync(0xffffffffu, slot, leader);
        __syncwarp();  // the batch's copies are read: their buffer is the set-up's scratch
        unsigned long long packed = 0;
        if (valid && slot >= slot_lo && slot < slot_lo + SLOTS && slot < HKEYS) {
          EntrySetup& E = my[lane];
          int tot = setup_edges<EXACT>(ra, rb, slot - slot_lo, ox, oy + y0, tw, th, E,
                                        reinterpret_cast<int*>(&s_pre_rib[wid][0][0]) + lane);
          if (tot > 0) {
            st_rows += E.nrow;
            // pixel items per class in 21-bit fields (at most 32 x 256 each):
            // convex fast form, two-triangle fast form, general form
            int cls = (E.valid & 32) ? 0 : (E.valid & 64) ? 1 : 2;
            packed = (unsigned long long)tot << (21 * cls);
          }
        }
        __syncwarp();
        unsigned long long xp = packed;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          unsigned long long y = __shfl_up_sync(0xffffffffu, xp, o);
          if (lane >= o) xp += y;
        }
        const unsigned long long tot3 = __shfl_sync(0xffffffffu, xp, 31);
        const unsigned long long excl3 = xp - packed;
        // the next batch's ribs and tag (each lane reads only its own copies,
        // which it has already read for this batch)
        if (base_next + lane < n) {
          cp_async4(&s_pre_tag[wid][lane], tag + r_next);
          cp_async16(&s_pre_rib[wid][0][lane], rib + r_next - 1);
          cp_async16(&s_pre_rib[wid][1][lane], rib + r_next);
        }
        cp_async_commit();
        st_items += tot3;  // three 21-bit fields of at most 8192 per batch
        if (++st_batches == 200) flush_stats();
#pragma unroll 1
        for (int cls = 0; cls < 3; ++cls) {
          const int sh = 21 * cls;
          const int total = (int)((tot3 >> sh) & 0x1fffffu);
          // this lane's entry: first item and item count in the class
          const int pe = (int)((excl3 >> sh) & 0x1fffffu);
          const int ce = (int)((packed >> sh) & 0x1fffffu);
          for (int it0 = 0; it0 < total; it0 += 64) {
            // Items it0 .. it0 + 63 go two per lane (it0 + lane and it0 + 32 +
            // lane), so that each lane has two independent decode and mask
            // chains in flight.  Per 32-item window, entries whose first item
            // falls inside it (after its first position) mark their start bit;
            // an item's entry is the last start at or before it, else the
            // entry holding the window's first item.
            __syncwarp();
            const int spa = pe - it0, spb = spa - 32;
            const bool sta = ce > 0 && spa > 0 && spa < 32;
            const bool stb = ce > 0 && spb > 0 && spb < 32;
            const uint32_t startsA = __reduce_or_sync(0xffffffffu, sta ? 1u << spa : 0u);
            const uint32_t startsB = __reduce_or_sync(0xffffffffu, stb ? 1u << spb : 0u);
            if (sta) s_own[wid][spa] = (uint8_t)lane;
            if (stb) s_own2[wid][spb] = (uint8_t)lane;
            const uint32_t heldA = __ballot_sync(0xffffffffu, ce > 0 && pe <= it0);
            const uint32_t heldB = __ballot_sync(0xffffffffu, ce > 0 && pe <= it0 + 32);
            const int ebaseA = 31 - __clz(heldA);
            const int ebaseB = heldB ? 31 - __clz(heldB) : 0;
            const int pebaseA = __shfl_sync(0xffffffffu, pe, ebaseA);
            const int pebaseB = __shfl_sync(0xffffffffu, pe, ebaseB);
            __syncwarp();
            const int itA = it0 + lane, itB = it0 + 32 + lane;
            // decode (every index stays in range for items past the end, whose
            // masks are dropped)
            auto decode = [&](int it, int w0, uint32_t starts, const uint8_t* own, int ebase,
                              int pebase, int& e, int& lx, int& ly) {
              const uint32_t sm = starts & ((2u << lane) - 1u);
              const int p = sm ? 31 - __clz(sm) : 0;
              const int eo = own[p];
              e = sm ? eo : ebase;
              const int first = sm ? w0 + p : pebase;
              const EntrySetup& E = my[e];
              const int li = it - first;
              // the item's row: the last k with rowpre[k] <= li, as a binary
              // search in two rounds of three independent loads
              const int r4 = E.rowpre[4], r8 = E.rowpre[8], r12 = E.rowpre[12];
              int k = r8 <= li ? 8 : 0;
              const int rk0 = k ? r8 : 0;
              const int rk4 = k ? r12 : r4;
              const bool s4 = rk4 <= li;
              k += s4 ? 4 : 0;
              const int rb = s4 ? rk4 : rk0;  // rowpre[k]
              const int q1 = E.rowpre[k + 1], q2 = E.rowpre[k + 2], q3 = E.rowpre[k + 3];
              const bool s2 = q2 <= li;
              const int rodd = s2 ? q3 : q1;  // rowpre[k + 2 s2 + 1]
              const bool s1 = rodd <= li;
              const int pre = s1 ? rodd : (s2 ? q2 : rb);
              k += (s2 ? 2 : 0) + (s1 ? 1 : 0);
              ly = E.row0 + k;
              lx = E.x0[k] + (li - pre);
            };
            auto mask_of = [&](int e, int lx, int ly, bool ok) -> uint32_t {
              const EntrySetup& E = my[e];
              if (EXACT)
                return cls == 0 ? exact_mask(E, lx * 256, ly * 256, s_rowmask)
                                : (ok ? exact_mask_general(E, lx, ly) : 0u);
              return cls == 0 ? fast_mask(E, lx * 256, ly * 256)
                     : cls == 1 ? fast_mask2(E, lx * 256, ly * 256)
                                : (ok ? tri_or_quad_mask(E, lx, ly) : 0u);
            };
            auto put = [&](int e, int lx, int ly, uint32_t m) {
              const int lp = ly * TILE_PX + lx;
              atomicOr(&s_mask[my[e].slot * MASK_WORDS + (lp >> 1)], m << (16 * (lp & 1)));
            };
            if (it0 + 32 < total) {  // warp-uniform: both halves hold items
              int eA, lxA, lyA, eB, lxB, lyB;
              decode(itA, it0, startsA, s_own[wid], ebaseA, pebaseA, eA, lxA, lyA);
              decode(itB, it0 + 32, startsB, s_own2[wid], ebaseB, pebaseB, eB, lxB, lyB);
              const uint32_t mA = mask_of(eA, lxA, lyA, true);
              const uint32_t mB = mask_of(eB, lxB, lyB, itB < total);
              if (mA) put(eA, lxA, lyA, mA);
              if (itB < total && mB) put(eB, lxB, lyB, mB);
            } else {
              int eA, lxA, lyA;
              decode(itA, it0, startsA, s_own[wid], ebaseA, pebaseA, eA, lxA, lyA);
              const uint32_t mA = mask_of(eA, lxA, lyA, itA < total);
              if (itA < total && mA) put(eA, lxA, lyA, mA);
            }
          }
        }
        __syncwarp();
      }
      __syncthreads();
      // per-path popcounts, OR into the tile's canvas words, and clear: one
      // warp per slot
      int nslot = min(s_nslot, HKEYS);
      int nhere = min(SLOTS, nslot - slot_lo);
      if (threadIdx.x == 0 && slot_lo + SLOTS >= nslot) t_next = atomicAdd(&counters[2], 1);
      for (int s2 = wid; s2 < nhere; s2 += CV_WARPS) {
        uint32_t* ms = s_mask + s2 * MASK_WORDS;
        unsigned c = 0;
#pragma unroll
        for (int w = lane; w < MASK_WORDS; w += 32) {
          const uint32_t v = ms[w];
          ms[w] = 0u;
          c += __popc(v);
          if (v) atomicOr(&s_canvas[w], v);
        }
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0 && c) {
          uint32_t p = s_slot_path[slot_lo + s2];
          if ((int)p < n_path) atomicAdd(covered + p, (unsigned long long)c);
        }
      }
      if (threadIdx.x == 0) {
        if (s_nslot > HKEYS) ps_record_error(status, PS_ERR_CAPACITY);
        if (stats) {
          atomicAdd(stats + 5, 1ull);
          if (pass == 0) atomicAdd(stats + 4, (unsigned long long)nslot);
        }
      }
      __syncthreads();
      for (int w = threadIdx.x; w < MASK_WORDS; w += CV_NT) {
        uint32_t v = s_canvas[w];
        s_canvas[w] = 0u;
        int lp = 2 * w;
        int py = ty * TILE_PX + lp / TILE_PX, px = tx * TILE_PX + lp % TILE_PX;
        if (py < H) {
          if (pass > 0) {  // later passes OR into what earlier passes wrote
            if (px < W) v |= canvas[(int64_t)py * W + px];
            if (px + 1 < W) v |= (uint32_t)canvas[(int64_t)py * W + px + 1] << 16;
          }
          if (px < W) canvas[(int64_t)py * W + px] = (uint16_t)(v & 0xffffu);
          if (px + 1 < W) canvas[(int64_t)py * W + px + 1] = (uint16_t)(v >> 16);
        }
      }
      if (slot_lo + SLOTS >= nslot) break;
    }
    // a non-empty tile's barriers already follow every read of s_tile and
    // s_nslot
    if (threadIdx.x == 0) s_tile = t_next;
  }
}

size_t coverage_smem_bytes() {
  return sizeof(uint32_t) * SLOTS * MASK_WORDS + sizeof(EntrySetup) * CV_NT +
         sizeof(uint32_t) * HKEYS + sizeof(uint16_t) * HKEYS + sizeof(uint32_t) * HKEYS;
}

}  // namespace

// The canvas holds pixel rows [row0, row0 + height) of the picture (row0 a
// multiple of the tile size); quads are snapped in picture coordinates and
// moved to the window's origin after snapping, so every tile of the window is
// covered exactly as in a canvas that starts at row 0.
static int rasterize(ps_context* ctx, const float* d_rib, const uint32_t* d_tag,
                     const int64_t* d_n_rib, int64_t capacity, int32_t n_path, int width,
                     int row0, int height, int spp, uint16_t* d_canvas, uint64_t* d_covered,
                     void* stream, bool exact) {
  if (!ctx || !d_rib || !d_tag || !d_n_rib || !d_canvas || !d_covered) return PS_ERR_INVALID;
  if (spp != 16 || width <= 0 || height <= 0 || capacity < 0 || n_path < 0) return PS_ERR_INVALID;
  if (row0 < 0 || row0 % TILE_PX != 0) return PS_ERR_INVALID;
  if ((int64_t)width * 256 >= COORD_LIMIT || ((int64_t)row0 + height) * 256 >= COORD_LIMIT)
    return PS_ERR_INVALID;
  const int y0 = row0 * 256;
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = stream;
  int tiles_x = (width + TILE_PX - 1) / TILE_PX, tiles_y = (height + TILE_PX - 1) / TILE_PX;
  int64_t n_tile = (int64_t)tiles_x * tiles_y;
  if (n_tile > (1 << 26)) return PS_ERR_INVALID;
  // default bin capacity: 4 entries per rib unless reserved larger
  int64_t want_pairs = ctx->pair_cap > 0 ? ctx->pair_cap : 4 * capacity + 1024;
  int rc = ps_ensure_raster(ctx, n_tile, want_pairs);
  if (rc != PS_OK) return rc;
  if ((rc = ps_ensure_quad_hits(ctx, capacity)) != PS_OK) return rc;
  if ((rc = ps_ensure_tiles(ctx, (n_tile + TS_TILE - 1) / TS_TILE + 1)) != PS_OK) return rc;
  size_t cov_smem = coverage_smem_bytes();
  const void* kcov = exact ? (const void*)k_coverage<true> : (const void*)k_coverage<false>;
  // the dynamic shared-memory limit is a per-device attribute of the kernel:
  // set once per context (a context lives on one device)
  if (!ctx->cov_attr_done[exact]) {
    if ((rc = ps_cuda_check(cudaFuncSetAttribute(kcov, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)cov_smem))) != PS_OK)
      return rc;
    ctx->cov_attr_done[exact] = 1;
  }
  int grid_cov = ps_persistent_grid(ctx, kcov, CV_NT, cov_smem);
  ctx->last_n_tile = n_tile;
  cudaMemsetAsync(ctx->d_tile_count, 0, sizeof(int32_t) * (n_tile + 1), st);
  cudaMemsetAsync(ctx->d_tile_flag, 0, sizeof(uint32_t) * ((n_tile + TS_TILE - 1) / TS_TILE + 1), st);
  cudaMemsetAsync(ctx->d_counters, 0, sizeof(int32_t) * 16, st);
  cudaMemsetAsync(d_covered, 0, sizeof(uint64_t) * (size_t)n_path, st);
  // tiles without entries are never visited by the coverage kernel
  cudaMemsetAsync(d_canvas, 0, sizeof(uint16_t) * (size_t)width * (size_t)height, st);
  cudaMemsetAsync(ctx->d_scratch64, 0, 7 * sizeof(int64_t), st);
  // persistent grids, each pass at its own occupancy (the count pass holds more
  // registers)
  int grid_bin = ctx->tune[PS_TUNE_BIN_BLOCKS] > 0
                     ? ctx->num_sms * ctx->tune[PS_TUNE_BIN_BLOCKS]
                     : ps_persistent_grid(ctx, (const void*)k_bin<0>, BIN_NT, 0);
  int grid_bin1 = ctx->tune[PS_TUNE_BIN_BLOCKS] > 0
                      ? grid_bin
                      : ps_persistent_grid(ctx, (const void*)k_bin<1>, BIN_NT, 0);
  const float4* rib = reinterpret_cast<const float4*>(d_rib);
  { ProfScope ps_(ctx, PK_BIN_COUNT, st);
  k_bin<0><<<grid_bin, BIN_NT, 0, st>>>(rib, d_tag, d_n_rib, capacity, width, height, y0, tiles_x,
                                      ctx->d_tile_count, ctx->d_tile_off, ctx->d_tile_cursor,
                                      ctx->d_bin, ctx->pair_cap, reinterpret_cast<uint2*>(ctx->d_quad_hits), ctx->d_tile_cursor + n_tile + 1,
                                      ctx->d_status); }
  { ProfScope ps_(ctx, PK_TILE_SCAN, st);
  const int ts_grid = (int)((n_tile + TS_TILE - 1) / TS_TILE);
  k_tile_scan<<<ts_grid, TS_NT, 0, st>>>(ctx->d_tile_count, ctx->d_tile_off, ctx->d_tile_cursor,
                                         ctx->d_tile_list, (int)n_tile, ctx->pair_cap,
                                         ctx->d_tile_flag, ctx->d_tile_agg, ctx->d_tile_incl,
                                         ctx->d_status); }
  { ProfScope ps_(ctx, PK_BIN_SCATTER, st);
  k_bin<1><<<grid_bin1, BIN_NT, 0, st>>>(rib, d_tag, d_n_rib, capacity, width, height, y0, tiles_x,
                                      ctx->d_tile_count, ctx->d_tile_off, ctx->d_tile_cursor,
                                      ctx->d_bin, ctx->pair_cap, reinterpret_cast<uint2*>(ctx->d_quad_hits), ctx->d_tile_cursor + n_tile + 1,
                                      ctx->d_status); }
  { ProfScope ps_(ctx, PK_COVERAGE, st);
#define PS_COV_ARGS                                                                              \
  rib, d_tag, ctx->d_tile_off, ctx->d_bin, ctx->pair_cap, width, height, y0, tiles_x, (int)n_tile, \
      ctx->d_tile_list, d_canvas, reinterpret_cast<unsigned long long*>(d_covered), n_path, ctx->d_counters,      \
      ctx->d_status, reinterpret_cast<unsigned long long*>(ctx->d_scratch64)
  if (exact) k_coverage<true><<<grid_cov, CV_NT, cov_smem, st>>>(PS_COV_ARGS);
  else k_coverage<false><<<grid_cov, CV_NT, cov_smem, st>>>(PS_COV_ARGS);
#undef PS_COV_ARGS
  }
  return ps_cuda_check(cudaGetLastError());
}

extern "C" int ps_rasterize_coverage(ps_context* ctx, const float* d_rib, const uint32_t* d_tag,
                                     const int64_t* d_n_rib, int64_t capacity, int32_t n_path,
                                     int width, int height, int spp, uint16_t* d_canvas,
                                     uint64_t* d_covered, void* stream) {
  return rasterize(ctx, d_rib, d_tag, d_n_rib, capacity, n_path, width, 0, height, spp, d_canvas,
                   d_covered, stream, false);
}

extern "C" int ps_rasterize_coverage_exact(ps_context* ctx, const float* d_rib,
                                           const uint32_t* d_tag, const int64_t* d_n_rib,
                                           int64_t capacity, int32_t n_path, int width, int height,
                                           int spp, uint16_t* d_canvas, uint64_t* d_covered,
                                           void* stream) {
  return rasterize(ctx, d_rib, d_tag, d_n_rib, capacity, n_path, width, 0, height, spp, d_canvas,
                   d_covered, stream, true);
}

extern "C" int ps_rasterize_coverage_rows(ps_context* ctx, const float* d_rib,
                                          const uint32_t* d_tag, const int64_t* d_n_rib,
                                          int64_t capacity, int32_t n_path, int width,
                                          int row_begin, int height, int spp,
                                          uint16_t* d_canvas, uint64_t* d_covered, int exact,
                                          void* stream) {
  return rasterize(ctx, d_rib, d_tag, d_n_rib, capacity, n_path, width, row_begin, height, spp,
                   d_canvas, d_covered, stream, exact != 0);
}

// ---------------------------------------------------------------------------
// Routing quads to the ranks that own their pixel rows, for a raster split of
// the canvas by tile rows over several GPUs: rank d owns rows [row_begin[d],
// row_begin[d + 1]).  A quad goes to every owner of a pixel row its snapped
// bounding box reaches (the rows the binning would test it against), as its
// two ribs and tags; the receiving rank covers its rows from the quads of all
// ranks, so each of its tiles sees every quad of every path that reaches it.
namespace {

constexpr int ROUTE_NT = 256;

// the last d in [0, n_dest) with row_begin[d] <= py (0 when there is none)
__device__ __forceinline__ int owner_of_row(const int32_t* __restrict__ row_begin, int n_dest,
                                            int py) {
  int lo = 0, hi = n_dest - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(row_begin + mid) <= py) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// pass 0 counts the quads of every destination; pass 1 writes them at the
// destination's offset (count[] restarts from 0 between the passes).
template <int PASS>
__global__ void __launch_bounds__(ROUTE_NT) k_route(const float4* __restrict__ rib,
                                                    const uint32_t* __restrict__ tag,
                                                    const int64_t* __restrict__ n_rib,
                                                    int64_t capacity, int W, int H, int n_dest,
                                                    const int32_t* __restrict__ row_begin,
                                                    unsigned long long* __restrict__ count,
                                                    const long long* __restrict__ off,
                                                    float4* __restrict__ out_rib,
                                                    uint32_t* __restrict__ out_tag,
                                                    int64_t out_cap, int32_t* status) {
  int64_t R = *n_rib;
  if (R > capacity) R = capacity;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * ROUTE_NT;
  for (int64_t base = (int64_t)blockIdx.x * ROUTE_NT; base < R; base += stride) {
    const int64_t r = base + threadIdx.x;
    int q0 = 0, nq = 0;  // destinations q0 .. q0 + nq - 1
    uint32_t tg = 0u;
    float4 ra = make_float4(0.f, 0.f, 0.f, 0.f), rb = ra;
    if (r >= 1 && r < R) {
      tg = __ldg(tag + r);
      if (!(tg & PS_TAG_LINK_START)) {
        ra = __ldg(rib + r - 1);
        rb = __ldg(rib + r);
        QuadFix q;
        if (!snap_quad(ra, rb, q)) {
          if (PASS == 0) ps_record_error(status, PS_ERR_RANGE);
        } else {
          const int mnx = min(min(q.x[0], q.x[1]), min(q.x[2], q.x[3]));
          const int mxx = max(max(q.x[0], q.x[1]), max(q.x[2], q.x[3]));
          const int mny = min(min(q.y[0], q.y[1]), min(q.y[2], q.y[3]));
          const int mxy = max(max(q.y[0], q.y[1]), max(q.y[2], q.y[3]));
          int px0, px1, py0, py1;
          pix_range(mnx, mxx, W, px0, px1);
          pix_range(mny, mxy, H, py0, py1);
          if (px0 <= px1 && py0 <= py1) {
            q0 = owner_of_row(row_begin, n_dest, py0);
            nq = owner_of_row(row_begin, n_dest, py1) - q0 + 1;
          }
        }
      }
    }
    // round k takes every lane's k-th destination; lanes bound for one rank
    // are grouped, one atomic per group
    const int kmax = __reduce_max_sync(0xffffffffu, (unsigned)max(nq, 0));
    for (int k = 0; k < kmax; ++k) {
      int d = k < nq ? q0 + k : -1;
      if (d >= 0 && __ldg(row_begin + d) >= __ldg(row_begin + d + 1)) d = -1;  // empty window
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      const int leader = __ffs(peers) - 1;
      if (d >= 0) {
        if (PASS == 0) {
          if (lane == leader) atomicAdd(count + d, (unsigned long long)__popc(peers));
        } else {
          unsigned long long b = 0;
          if (lane == leader) b = atomicAdd(count + d, (unsigned long long)__popc(peers));
          b = __shfl_sync(peers, b, leader);
          const long long pos = off[d] + (long long)b + __popc(peers & ((1u << lane) - 1u));
          if (pos < out_cap && pos < off[d + 1]) {
            out_rib[2 * pos] = ra;
            out_rib[2 * pos + 1] = rb;
            out_tag[2 * pos] = tg | PS_TAG_LINK_START;  // a pair starts a link: one quad
            out_tag[2 * pos + 1] = tg;
          } else {
            ps_record_error(status, PS_ERR_CAPACITY);
          }
        }
      }
    }
  }
}

// offsets of the destinations' blocks; the counts restart for pass 1 (kept
// when the call only counts)
__global__ void k_route_scan(unsigned long long* count, long long* off, int n_dest,
                             int64_t out_cap, bool count_only, int32_t* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  long long acc = 0;
  for (int d = 0; d < n_dest; ++d) {
    off[d] = acc;
    acc += (long long)count[d];
    if (!count_only) count[d] = 0ull;
  }
  off[n_dest] = acc;
  if (!count_only && acc > out_cap) ps_record_error(status, PS_ERR_CAPACITY);
}

}  // namespace

extern "C" int ps_route_quads(ps_context* ctx, const float* d_rib, const uint32_t* d_tag,
                              const int64_t* d_n_rib, int64_t capacity, int32_t width,
                              int32_t height, int32_t n_dest, const int32_t* d_row_begin,
                              float* d_out_rib, uint32_t* d_out_tag, int64_t out_capacity,
                              int64_t* d_dest_count, int64_t* d_dest_off, void* stream) {
  if (!ctx || !d_rib || !d_tag || !d_n_rib || !d_row_begin || !d_dest_count || !d_dest_off)
    return PS_ERR_INVALID;
  if (capacity < 0 || out_capacity < 0 || width <= 0 || height <= 0 || n_dest < 1 ||
      n_dest > 4096)
    return PS_ERR_INVALID;
  const bool count_only = !d_out_rib && !d_out_tag && out_capacity == 0;
  if (!count_only && (!d_out_rib || !d_out_tag)) return PS_ERR_INVALID;
  if ((int64_t)width * 256 >= COORD_LIMIT || (int64_t)height * 256 >= COORD_LIMIT)
    return PS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = stream;
  int rc = ps_cuda_check(cudaMemsetAsync(d_dest_count, 0, sizeof(int64_t) * n_dest, st));
  if (rc != PS_OK) return rc;
  const float4* rib = reinterpret_cast<const float4*>(d_rib);
  float4* orib = reinterpret_cast<float4*>(d_out_rib);
  auto* cnt = reinterpret_cast<unsigned long long*>(d_dest_count);
  auto* off = reinterpret_cast<long long*>(d_dest_off);
  const int grid = ps_persistent_grid(ctx, (const void*)k_route<0>, ROUTE_NT, 0);
  k_route<0><<<grid, ROUTE_NT, 0, st>>>(rib, d_tag, d_n_rib, capacity, width, height, n_dest,
                                        d_row_begin, cnt, off, orib, d_out_tag, out_capacity,
                                        ctx->d_status);
  k_route_scan<<<1, 32, 0, st>>>(cnt, off, n_dest, out_capacity, count_only, ctx->d_status);
  if (!count_only)
    k_route<1><<<grid, ROUTE_NT, 0, st>>>(rib, d_tag, d_n_rib, capacity, width, height, n_dest,
                                          d_row_begin, cnt, off, orib, d_out_tag, out_capacity,
                                          ctx->d_status);
  return ps_cuda_check(cudaGetLastError());
}

extern "C" int ps_raster_stats(ps_context* ctx, int64_t* h_counts, int n_counts) {
  if (!ctx || !h_counts || n_counts < 0) return PS_ERR_INVALID;
  int64_t v[PS_RSTAT_COUNT] = {0, 0, 0, 0, 0, 0, 0, 0};
  int rc = PS_OK;
  if (ctx->d_tile_off && ctx->last_n_tile > 0) {
    int32_t pairs = 0;
    cudaStream_t st = (cudaStream_t)ctx->last_stream;
    rc = ps_cuda_check(cudaMemcpyAsync(&pairs, ctx->d_tile_off + ctx->last_n_tile, sizeof(int32_t),
                                       cudaMemcpyDeviceToHost, st));
    if (rc == PS_OK)
      rc = ps_cuda_check(cudaMemcpyAsync(v + 1, ctx->d_scratch64, 7 * sizeof(int64_t),
                                         cudaMemcpyDeviceToHost, st));
    if (rc == PS_OK) rc = ps_cuda_check(cudaStreamSynchronize(st));
    v[0] = pairs;
  }
  for (int i = 0; i < n_counts; ++i) h_counts[i] = i < PS_RSTAT_COUNT ? v[i] : 0;
  return rc;
}
