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

__device__ __forceinline__ int64_t floor_div(int64_t a, int64_t b) {
  return a >= 0 ? a / b : -((-a + b - 1) / b);
}
__device__ __forceinline__ int64_t ceil_div(int64_t a, int64_t b) { return -floor_div(-a, b); }

struct QuadFix {
  int x[4], y[4];  // N0 P0 N1 P1 in 1/256 px
};

// Snap a quad's four vertices; false when a coordinate is out of range.
__device__ __forceinline__ bool snap_quad(const float4 a, const float4 b, QuadFix& q) {
  float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
  int s[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    float f = v[i] * 256.f;  // exact scaling by a power of two
    if (!(fabsf(f) < (float)COORD_LIMIT)) return false;
    s[i] = __float2int_rn(f);  // round half to even
  }
  q.x[0] = s[0]; q.y[0] = s[1]; q.x[1] = s[2]; q.y[1] = s[3];
  q.x[2] = s[4]; q.y[2] = s[5]; q.x[3] = s[6]; q.y[3] = s[7];
  return true;
}

// Pixel range whose sample window [256p + 8, 256p + 248] meets [lo, hi].
__device__ __forceinline__ void pix_range(int lo, int hi, int n, int& p0, int& p1) {
  int64_t a = ceil_div((int64_t)lo - 248, 256), b = floor_div((int64_t)hi - 8, 256);
  if (a < 0) a = 0;
  if (b > n - 1) b = n - 1;
  p0 = (int)a;
  p1 = (int)b;
}

__device__ __forceinline__ void quad_pixels(const QuadFix& q, int W, int H, int& px0, int& px1,
                                            int& py0, int& py1) {
  int mnx = min(min(q.x[0], q.x[1]), min(q.x[2], q.x[3]));
  int mxx = max(max(q.x[0], q.x[1]), max(q.x[2], q.x[3]));
  int mny = min(min(q.y[0], q.y[1]), min(q.y[2], q.y[3]));
  int mxy = max(max(q.y[0], q.y[1]), max(q.y[2], q.y[3]));
  pix_range(mnx, mxx, W, px0, px1);
  pix_range(mny, mxy, H, py0, py1);
}

// Can triangle (x0,y0)-(x1,y1)-(x2,y2) cover a sample of the tile whose samples
// lie in [rx0, rx1] x [ry0, ry1]?  Separating-axis test on the triangle's edges
// (the rectangle's own axes are settled by the bounding-box range).
__device__ __forceinline__ bool tri_meets_rect(int x0, int y0, int x1, int y1, int x2, int y2,
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
    // the rectangle corner maximizing A x + B y
    long long cx = A >= 0 ? rx1 : rx0, cy = B >= 0 ? ry1 : ry0;
    if (A * (cx - vx[i]) + B * (cy - vy[i]) < 0) return false;
  }
  return true;
}

// pass 0: count (quad, tile) pairs per tile; pass 1: scatter rib ids into bins.
// Lanes of a warp that hit the same tile are grouped: one atomic per group.
template <int PASS>
__global__ void __launch_bounds__(256) k_bin(const float4* __restrict__ rib,
                                             const uint32_t* __restrict__ tag,
                                             const int64_t* __restrict__ n_rib, int64_t capacity,
                                             int W, int H, int tiles_x, int32_t* __restrict__ count,
                                             const int32_t* __restrict__ off,
                                             int32_t* __restrict__ cursor,
                                             uint32_t* __restrict__ bin, int64_t pair_cap,
                                             int32_t* status) {
  int64_t R = *n_rib;
  if (R > capacity) R = capacity;
  int lane = threadIdx.x & 31;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < R; base += stride) {
    int64_t r = base + threadIdx.x;
    bool act = r >= 1 && r < R && !(__ldg(tag + r) & PS_TAG_LINK_START);
    QuadFix q;
    int tx0 = 0, tx1 = -1, ty0 = 0, ty1 = -1;
    if (act) {
      if (!snap_quad(__ldg(rib + r - 1), __ldg(rib + r), q)) {
        ps_record_error(status, PS_ERR_RANGE);
      } else {
        int px0, px1, py0, py1;
        quad_pixels(q, W, H, px0, px1, py0, py1);
        if (px0 <= px1 && py0 <= py1) {
          tx0 = px0 / TILE_PX; tx1 = px1 / TILE_PX; ty0 = py0 / TILE_PX; ty1 = py1 / TILE_PX;
        }
      }
    }
    int ntx = tx1 - tx0 + 1, n = (tx1 >= tx0 && ty1 >= ty0) ? ntx * (ty1 - ty0 + 1) : 0;
    int nmax = n;
    for (int o = 16; o > 0; o >>= 1) nmax = max(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
    for (int i = 0; i < nmax; ++i) {
      int t = -1;
      if (i < n) {
        int tx = tx0 + i % ntx, ty = ty0 + i / ntx;
        // sample rectangle of the tile (1/256 px), clipped to the canvas
        int rx0 = tx * TILE_UNITS + 8, ry0 = ty * TILE_UNITS + 8;
        int rx1 = min(tx * TILE_UNITS + TILE_UNITS, W * 256) - 8;
        int ry1 = min(ty * TILE_UNITS + TILE_UNITS, H * 256) - 8;
        bool hit = n == 1 ||
                   tri_meets_rect(q.x[0], q.y[0], q.x[1], q.y[1], q.x[3], q.y[3], rx0, ry0, rx1, ry1) ||
                   tri_meets_rect(q.x[0], q.y[0], q.x[3], q.y[3], q.x[2], q.y[2], rx0, ry0, rx1, ry1);
        if (hit) t = ty * tiles_x + tx;
      }
      unsigned peers = __match_any_sync(0xffffffffu, t);
      int leader = __ffs(peers) - 1;
      int cntg = __popc(peers);
      if (t >= 0) {
        if (PASS == 0) {
          if (lane == leader) atomicAdd(count + t, cntg);
        } else {
          int basepos = 0;
          if (lane == leader) basepos = atomicAdd(cursor + t, cntg);
          basepos = __shfl_sync(peers, basepos, leader);
          int pos = basepos + __popc(peers & ((1u << lane) - 1u));
          int64_t at = (int64_t)off[t] + pos;
          if (at < pair_cap && at < off[t + 1]) bin[at] = (uint32_t)r;
          else ps_record_error(status, PS_ERR_CAPACITY);
        }
      }
    }
  }
}

// Exclusive scan of tile counts (one CTA of 1024 threads), resets cursors.
__global__ void __launch_bounds__(1024) k_tile_scan(const int32_t* __restrict__ count,
                                                    int32_t* __restrict__ off,
                                                    int32_t* __restrict__ cursor, int n_tile,
                                                    int64_t pair_cap, int32_t* status) {
  __shared__ long long warp_sums[32];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int base = 0; base < n_tile; base += 1024) {
    int i = base + threadIdx.x;
    long long v = i < n_tile ? count[i] : 0;
    long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
      long long w = warp_sums[lane];
      for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      warp_sums[lane] = w;
    }
    __syncthreads();
    long long excl = carry + x - v + (wid > 0 ? warp_sums[wid - 1] : 0);
    if (i < n_tile) {
      if (excl > 0x7fffffffLL) ps_record_error(status, PS_ERR_CAPACITY);
      off[i] = (int32_t)excl;
      cursor[i] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_sums[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    off[n_tile] = (int32_t)(carry > 0x7fffffffLL ? 0x7fffffff : carry);
    if (carry > pair_cap) ps_record_error(status, PS_ERR_CAPACITY);
  }
}

// ---------------------------------------------------------------------------
// Coverage.  One 512-thread CTA per SM, persistent over tiles.  Per tile each
// warp runs its own queue: it takes the next 32 bin entries, each lane sets one
// up (the path's mask slot from a shared hash, the edge functions relative to
// the tile, the pixel span of every pixel row the quad can reach), a warp scan
// flattens the entries' pixels so that every lane gets one pixel at a time, and
// each pixel's 16-sample mask is ORed into the path's mask in shared memory.
// Block-wide barriers only open and close a tile: per-path popcounts and the
// canvas OR are taken there.  Paths beyond SLOTS per tile take further passes.
constexpr int CV_NT = 512;
constexpr int CV_WARPS = CV_NT / 32;
constexpr int SLOTS = 224;           // per-path masks resident in shared memory
constexpr int HKEYS = 2048;          // hash of path ids (max distinct paths per tile)
constexpr int MASK_WORDS = TILE_PX * TILE_PX / 2;

struct Edge {
  int A, B;       // E(x, y) = A x + B y + C, tile-relative 1/256 px
  long long C;
};

struct EntrySetup {
  Edge e[6];               // convex quad: e[0..3]; else triangle 0: e[0..2], triangle 1: e[3..5]
  uint16_t rowpre[17];     // prefix of span widths over rows row0 ..
  uint8_t x0[16];          // first pixel of each row's span
  uint16_t slot;           // mask slot of this pass
  uint8_t valid;           // bit0 tri 0, bit1 tri 1, bit2 int64 path, bit3 convex quad
  uint8_t row0;
};

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
    long long A = (long long)ay - by, B = (long long)bx - ax;
    e[i].A = (int)A;
    e[i].B = (int)B;
    e[i].C = -(A * ax + B * ay);  // E = (bx-ax)(y-ay) - (by-ay)(x-ax)
    if (llabs(A) + llabs(B) >= (1ll << 22)) big = true;
  }
}

// x-extent of segment (ax,ay)-(bx,by) clipped to the strip y in [ylo, yhi]
__device__ __forceinline__ void seg_strip(float ax, float ay, float bx, float by, float ylo,
                                          float yhi, float& xmin, float& xmax) {
  if (ay > by) {
    float t = ax; ax = bx; bx = t;
    t = ay; ay = by; by = t;
  }
  if (by < ylo || ay > yhi) return;
  float xa = ax, xb = bx;
  if (by > ay) {
    float k = (bx - ax) / (by - ay);
    if (ay < ylo) xa = ax + k * (ylo - ay);
    if (by > yhi) xb = ax + k * (yhi - ay);
  }
  xmin = fminf(xmin, fminf(xa, xb));
  xmax = fmaxf(xmax, fmaxf(xa, xb));
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

// Set up entry r (rib id) of tile (ox, oy); returns its pixel count.
__device__ __forceinline__ int setup_entry(const float4* __restrict__ rib, uint32_t r, int slot,
                                           int ox, int oy, int tw, int th, EntrySetup& E) {
  E.slot = (uint16_t)slot;
  E.valid = 0;
  E.row0 = 0;
  E.rowpre[0] = 0;
  QuadFix q;
  if (!snap_quad(__ldg(rib + r - 1), __ldg(rib + r), q)) return 0;
  for (int v = 0; v < 4; ++v) {
    q.x[v] -= ox;
    q.y[v] -= oy;
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
        E.e[i].C = -(A * px_[a0] + B * py_[a0]);
        if (llabs(A) + llabs(B) >= (1ll << 22)) bigq = true;
      }
      big = bigq;
      flags |= 8;
    }
  }
  E.valid = flags | (big ? 4 : 0);
  // per-row pixel spans over the 5 segments bounding both triangles
  float fx[4] = {(float)q.x[0], (float)q.x[1], (float)q.x[2], (float)q.x[3]};
  float fy[4] = {(float)q.y[0], (float)q.y[1], (float)q.y[2], (float)q.y[3]};
  float ymin = fminf(fminf(fy[0], fy[1]), fminf(fy[2], fy[3]));
  float ymax = fmaxf(fmaxf(fy[0], fy[1]), fmaxf(fy[2], fy[3]));
  float mag = fmaxf(fmaxf(fabsf(fx[0]), fabsf(fx[1])), fmaxf(fabsf(fx[2]), fabsf(fx[3])));
  mag = fmaxf(mag, fmaxf(fabsf(ymin), fabsf(ymax)));
  float eps = 4.f + mag * 1e-6f;  // float error of the clipped extents, 1/256 px
  int ly0 = max(0, (int)ceilf((ymin - 248.f - eps) / 256.f));
  int ly1 = min(th - 1, (int)floorf((ymax - 8.f + eps) / 256.f));
  int first = -1, tot = 0;
  for (int ly = ly0; ly <= ly1; ++ly) {
    float ylo = 256.f * ly + 8.f - eps, yhi = 256.f * ly + 248.f + eps;
    float xmin = 3.4e38f, xmax = -3.4e38f;
    seg_strip(fx[0], fy[0], fx[1], fy[1], ylo, yhi, xmin, xmax);  // N0 P0
    seg_strip(fx[1], fy[1], fx[3], fy[3], ylo, yhi, xmin, xmax);  // P0 P1
    seg_strip(fx[3], fy[3], fx[2], fy[2], ylo, yhi, xmin, xmax);  // P1 N1
    seg_strip(fx[2], fy[2], fx[0], fy[0], ylo, yhi, xmin, xmax);  // N1 N0
    seg_strip(fx[0], fy[0], fx[3], fy[3], ylo, yhi, xmin, xmax);  // N0 P1
    int w = 0, a = 0;
    if (xmax >= xmin) {
      a = max(0, (int)ceilf((xmin - 248.f - eps) / 256.f));
      int bb = min(tw - 1, (int)floorf((xmax - 8.f + eps) / 256.f));
      if (bb >= a) w = bb - a + 1;
    }
    if (first < 0) {
      if (w == 0) continue;
      first = ly;
    }
    int k = ly - first;
    E.x0[k] = (uint8_t)a;
    tot += w;
    E.rowpre[k + 1] = (uint16_t)tot;
  }
  if (first < 0) return 0;
  E.row0 = (uint8_t)first;
  // rows after the last one repeat the final prefix: the row search below takes
  // the last row whose prefix is <= the item index, which skips empty rows
  for (int k = ly1 - first + 1; k < 16; ++k) E.rowpre[k + 1] = (uint16_t)tot;
  return tot;
}

__device__ __forceinline__ uint32_t pixel_mask(const EntrySetup& E, int lx, int ly) {
  int cx = lx * 256, cy = ly * 256;
  bool big = (E.valid & 4) != 0;
  if (E.valid & 8) {
    uint32_t m = 0xffffu;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      long long Ec = (long long)E.e[i].A * cx + (long long)E.e[i].B * cy + E.e[i].C;
      m &= edge_mask(E.e[i], Ec, big);
      if (!m) return 0u;
    }
    return m;
  }
  uint32_t m0 = 0, m1 = 0;
  if (E.valid & 1) {
    m0 = 0xffffu;
    for (int i = 0; i < 3 && m0; ++i) {
      long long Ec = (long long)E.e[i].A * cx + (long long)E.e[i].B * cy + E.e[i].C;
      m0 &= edge_mask(E.e[i], Ec, big);
    }
  }
  if ((E.valid & 2) && m0 != 0xffffu) {
    m1 = 0xffffu;
    for (int i = 3; i < 6 && m1; ++i) {
      long long Ec = (long long)E.e[i].A * cx + (long long)E.e[i].B * cy + E.e[i].C;
      m1 &= edge_mask(E.e[i], Ec, big);
    }
  }
  return m0 | m1;
}

__global__ void __launch_bounds__(CV_NT, 1) k_coverage(
    const float4* __restrict__ rib, const uint32_t* __restrict__ tag,
    const int32_t* __restrict__ off, const uint32_t* __restrict__ bin, int64_t pair_cap, int W,
    int H, int tiles_x, int n_tile, uint16_t* __restrict__ canvas,
    unsigned long long* __restrict__ covered, int n_path, int32_t* counters, int32_t* status,
    unsigned long long* __restrict__ stats) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* s_mask = reinterpret_cast<uint32_t*>(smem);                          // SLOTS*MASK_WORDS
  EntrySetup* s_ent = reinterpret_cast<EntrySetup*>(s_mask + SLOTS * MASK_WORDS);  // CV_NT
  uint32_t* s_keys = reinterpret_cast<uint32_t*>(s_ent + CV_NT);                 // HKEYS
  uint16_t* s_slot_of = reinterpret_cast<uint16_t*>(s_keys + HKEYS);             // HKEYS
  uint32_t* s_slot_path = reinterpret_cast<uint32_t*>(s_slot_of + HKEYS);        // HKEYS
  __shared__ int s_tile, s_nslot, s_next;
  __shared__ uint32_t s_pre[CV_WARPS][33];

  for (int i = threadIdx.x; i < SLOTS * MASK_WORDS; i += CV_NT) s_mask[i] = 0u;
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  EntrySetup* my = s_ent + wid * 32;
  for (;;) {
    if (threadIdx.x == 0) {
      s_tile = atomicAdd(&counters[2], 1);
      s_nslot = 0;
    }
    for (int i = threadIdx.x; i < HKEYS; i += CV_NT) {
      s_keys[i] = 0u;
      s_slot_of[i] = 0xffffu;
    }
    __syncthreads();
    int t = s_tile;
    if (t >= n_tile) return;
    int tx = t % tiles_x, ty = t / tiles_x;
    int ox = tx * TILE_UNITS, oy = ty * TILE_UNITS;
    int64_t b0 = off[t], b1 = off[t + 1];
    if (b1 > pair_cap) b1 = pair_cap;
    int n = (int)(b1 > b0 ? b1 - b0 : 0);
    int tw = min(TILE_PX, W - tx * TILE_PX), th = min(TILE_PX, H - ty * TILE_PX);
    for (int pass = 0;; ++pass) {
      int slot_lo = pass * SLOTS;
      if (threadIdx.x == 0) s_next = 0;
      __syncthreads();
      for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&s_next, 32);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n) break;
        int e = base + lane;
        int cnt = 0;
        if (e < n) {
          uint32_t r = bin[b0 + e];
          uint32_t key = (__ldg(tag + r) >> 2) + 1u;
          uint32_t h = (key * 2654435761u) & (HKEYS - 1);
          int slot = -1;
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
              do {  // the inserting lane may not have published the slot yet
                so = ((volatile uint16_t*)s_slot_of)[h];
              } while (so == 0xffffu && ++spin < (1 << 20));
              slot = so;
              break;
            }
            if (prev == 0u) break;
            h = (h + 1) & (HKEYS - 1);
          }
          if (slot >= slot_lo && slot < slot_lo + SLOTS && slot < HKEYS)
            cnt = setup_entry(rib, r, slot - slot_lo, ox, oy, tw, th, my[lane]);
        }
        // warp scan of the pixel counts
        uint32_t x = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x += y;
        }
        s_pre[wid][lane + 1] = x;
        if (lane == 0) s_pre[wid][0] = 0;
        int total = __shfl_sync(0xffffffffu, (int)x, 31);
        if (lane == 0 && stats) atomicAdd(stats, (unsigned long long)total);
        __syncwarp();
        for (int it = lane; it < total; it += 32) {
          int lo = 0, hi = 31;  // last entry with pre <= it
#pragma unroll
          for (int st = 16; st > 0; st >>= 1)
            if (lo + st <= hi && (int)s_pre[wid][lo + st] <= it) lo += st;
          const EntrySetup& E = my[lo];
          int li = it - (int)s_pre[wid][lo];
          int k = 0;  // row: the last one with rowpre[k] <= li
#pragma unroll
          for (int st = 8; st > 0; st >>= 1)
            if ((int)E.rowpre[k + st] <= li) k += st;
          int ly = E.row0 + k, lx = E.x0[k] + (li - (int)E.rowpre[k]);
          uint32_t m = pixel_mask(E, lx, ly);
          if (m) {
            int lp = ly * TILE_PX + lx;
            atomicOr(&s_mask[E.slot * MASK_WORDS + (lp >> 1)], m << (16 * (lp & 1)));
          }
        }
        __syncwarp();
      }
      __syncthreads();
      // per-path popcounts and the canvas for this pass's slots
      int nslot = min(s_nslot, HKEYS);
      int nhere = min(SLOTS, nslot - slot_lo);
      for (int s2 = wid; s2 < nhere; s2 += CV_WARPS) {
        unsigned c = 0;
        for (int w = lane; w < MASK_WORDS; w += 32) c += __popc(s_mask[s2 * MASK_WORDS + w]);
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0 && c) {
          uint32_t p = s_slot_path[slot_lo + s2];
          if ((int)p < n_path) atomicAdd(covered + p, (unsigned long long)c);
        }
      }
      for (int w = threadIdx.x; w < MASK_WORDS; w += CV_NT) {
        uint32_t v = 0;
        for (int s2 = 0; s2 < nhere; ++s2) v |= s_mask[s2 * MASK_WORDS + w];
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
      __syncthreads();
      for (int i = threadIdx.x; i < nhere * MASK_WORDS; i += CV_NT) s_mask[i] = 0u;
      if (threadIdx.x == 0 && s_nslot > HKEYS) ps_record_error(status, PS_ERR_CAPACITY);
      __syncthreads();
      if (slot_lo + SLOTS >= nslot) break;
    }
  }
}

size_t coverage_smem_bytes() {
  return sizeof(uint32_t) * SLOTS * MASK_WORDS + sizeof(EntrySetup) * CV_NT +
         sizeof(uint32_t) * HKEYS + sizeof(uint16_t) * HKEYS + sizeof(uint32_t) * HKEYS;
}

}  // namespace

extern "C" int ps_rasterize_coverage(ps_context* ctx, const float* d_rib, const uint32_t* d_tag,
                                     const int64_t* d_n_rib, int64_t capacity, int32_t n_path,
                                     int width, int height, int spp, uint16_t* d_canvas,
                                     uint64_t* d_covered, void* stream) {
  if (!ctx || !d_rib || !d_tag || !d_n_rib || !d_canvas || !d_covered) return PS_ERR_INVALID;
  if (spp != 16 || width <= 0 || height <= 0 || capacity < 0 || n_path < 0) return PS_ERR_INVALID;
  if ((int64_t)width * 256 >= COORD_LIMIT || (int64_t)height * 256 >= COORD_LIMIT)
    return PS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  ctx->last_stream = stream;
  int tiles_x = (width + TILE_PX - 1) / TILE_PX, tiles_y = (height + TILE_PX - 1) / TILE_PX;
  int64_t n_tile = (int64_t)tiles_x * tiles_y;
  if (n_tile > (1 << 26)) return PS_ERR_INVALID;
  // default bin capacity: 4 entries per rib unless reserved larger
  int64_t want_pairs = ctx->pair_cap > 0 ? ctx->pair_cap : 4 * capacity + 1024;
  int rc = ps_ensure_raster(ctx, n_tile, want_pairs);
  if (rc != PS_OK) return rc;
  size_t cov_smem = coverage_smem_bytes();
  static int attr_done = 0;
  if (!attr_done) {
    if ((rc = ps_cuda_check(cudaFuncSetAttribute((const void*)k_coverage,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)cov_smem))) != PS_OK)
      return rc;
    attr_done = 1;
  }
  int grid_cov = ps_persistent_grid(ctx, (const void*)k_coverage, CV_NT, cov_smem);
  ctx->last_n_tile = n_tile;
  cudaMemsetAsync(ctx->d_tile_count, 0, sizeof(int32_t) * (n_tile + 1), st);
  cudaMemsetAsync(ctx->d_counters, 0, sizeof(int32_t) * 16, st);
  cudaMemsetAsync(d_covered, 0, sizeof(uint64_t) * (size_t)n_path, st);
  cudaMemsetAsync(ctx->d_scratch64, 0, sizeof(int64_t), st);
  int grid_bin = ps_persistent_grid(ctx, (const void*)k_bin<0>, 256, 0);
  const float4* rib = reinterpret_cast<const float4*>(d_rib);
  { ProfScope ps_(ctx, PK_BIN_COUNT, st);
  k_bin<0><<<grid_bin, 256, 0, st>>>(rib, d_tag, d_n_rib, capacity, width, height, tiles_x,
                                      ctx->d_tile_count, ctx->d_tile_off, ctx->d_tile_cursor,
                                      ctx->d_bin, ctx->pair_cap, ctx->d_status); }
  { ProfScope ps_(ctx, PK_TILE_SCAN, st);
  k_tile_scan<<<1, 1024, 0, st>>>(ctx->d_tile_count, ctx->d_tile_off, ctx->d_tile_cursor,
                                  (int)n_tile, ctx->pair_cap, ctx->d_status); }
  { ProfScope ps_(ctx, PK_BIN_SCATTER, st);
  k_bin<1><<<grid_bin, 256, 0, st>>>(rib, d_tag, d_n_rib, capacity, width, height, tiles_x,
                                      ctx->d_tile_count, ctx->d_tile_off, ctx->d_tile_cursor,
                                      ctx->d_bin, ctx->pair_cap, ctx->d_status); }
  { ProfScope ps_(ctx, PK_COVERAGE, st);
  k_coverage<<<grid_cov, CV_NT, cov_smem, st>>>(
      rib, d_tag, ctx->d_tile_off, ctx->d_bin, ctx->pair_cap, width, height, tiles_x, (int)n_tile,
      d_canvas, reinterpret_cast<unsigned long long*>(d_covered), n_path, ctx->d_counters,
      ctx->d_status, reinterpret_cast<unsigned long long*>(ctx->d_scratch64)); }
  return ps_cuda_check(cudaGetLastError());
}

extern "C" int ps_raster_stats(ps_context* ctx, int64_t* h_pairs, int64_t* h_span_pixels) {
  if (!ctx || !h_pairs || !h_span_pixels) return PS_ERR_INVALID;
  *h_pairs = 0;
  *h_span_pixels = 0;
  if (!ctx->d_tile_off || ctx->last_n_tile <= 0) return PS_OK;
  int32_t v = 0;
  int64_t sp = 0;
  cudaStream_t st = (cudaStream_t)ctx->last_stream;
  int rc = ps_cuda_check(cudaMemcpyAsync(&v, ctx->d_tile_off + ctx->last_n_tile, sizeof(int32_t),
                                         cudaMemcpyDeviceToHost, st));
  if (rc == PS_OK)
    rc = ps_cuda_check(cudaMemcpyAsync(&sp, ctx->d_scratch64, sizeof(int64_t),
                                       cudaMemcpyDeviceToHost, st));
  if (rc == PS_OK) rc = ps_cuda_check(cudaStreamSynchronize(st));
  *h_pairs = v;
  *h_span_pixels = sp;
  return rc;
}
