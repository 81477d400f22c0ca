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

// pass 0: count (quad, tile) pairs per tile; pass 1: scatter rib ids into bins
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
  for (int64_t r = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R;
       r += (int64_t)gridDim.x * blockDim.x) {
    if (__ldg(tag + r) & PS_TAG_LINK_START) continue;
    QuadFix q;
    if (!snap_quad(__ldg(rib + r - 1), __ldg(rib + r), q)) {
      ps_record_error(status, PS_ERR_RANGE);
      continue;
    }
    int px0, px1, py0, py1;
    quad_pixels(q, W, H, px0, px1, py0, py1);
    if (px0 > px1 || py0 > py1) continue;
    int tx0 = px0 / TILE_PX, tx1 = px1 / TILE_PX, ty0 = py0 / TILE_PX, ty1 = py1 / TILE_PX;
    for (int ty = ty0; ty <= ty1; ++ty)
      for (int tx = tx0; tx <= tx1; ++tx) {
        int t = ty * tiles_x + tx;
        if (PASS == 0) {
          atomicAdd(count + t, 1);
        } else {
          int pos = atomicAdd(cursor + t, 1);
          int64_t at = (int64_t)off[t] + pos;
          if (at < pair_cap && at < off[t + 1]) bin[at] = (uint32_t)r;
          else ps_record_error(status, PS_ERR_CAPACITY);
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
// Coverage.  One CTA per tile (persistent over tiles).  Per tile:
//  A. bin entries in chunks of CHUNK: one thread per entry assigns the entry's
//     path a mask slot (shared hash), builds the two triangles' edge functions
//     relative to the tile origin and the pixel span of every pixel row of the
//     tile that the triangles can reach;
//  B. the (entry, pixel) items of the chunk are flattened with a block scan and
//     shared by all threads; each item ORs the pixel's 16-sample mask of both
//     triangles into the path's mask;
//  C. per-path popcounts, the canvas OR, and the masks are cleared.
// Paths beyond SLOTS per tile are handled in further passes over the bin.
constexpr int CV_NT = 512;
constexpr int CHUNK = 256;
constexpr int SLOTS = 256;           // per-path masks resident in shared memory
constexpr int HKEYS = 2048;          // hash of path ids (max distinct paths per tile)
constexpr int MASK_WORDS = TILE_PX * TILE_PX / 2;

struct Edge {
  int A, B;       // E(x, y) = A x + B y + C, tile-relative 1/256 px
  long long C;
};

struct EntrySetup {
  Edge e[6];               // triangle 0: e[0..2], triangle 1: e[3..5]
  uint16_t rowpre[17];     // prefix of span widths over the tile's 16 rows
  uint8_t x0[16];          // first pixel of each row's span
  uint16_t slot;           // mask slot (0xffff: not this pass)
  uint8_t valid;           // bit0 tri 0 non-degenerate, bit1 tri 1, bit2 needs int64 path
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

// 16-sample mask of one triangle at tile pixel (lx, ly)
__device__ __forceinline__ uint32_t tri_pixel_mask(const Edge* e, bool big, int lx, int ly) {
  uint32_t m = 0xffffu;
  int cx = lx * 256, cy = ly * 256;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    long long Ec = (long long)e[i].A * cx + (long long)e[i].B * cy + e[i].C;
    if (!big) {
      long long D = 248ll * (llabs((long long)e[i].A) + llabs((long long)e[i].B));
      if (Ec - D >= 0) continue;          // every sample inside this edge
      if (Ec + D < 0) return 0u;          // none
      int E0 = (int)Ec, A = e[i].A, B = e[i].B;
      uint32_t em = 0;
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        int v = E0 + A * (16 * k + 8) + B * (16 * ((5 * k) & 15) + 8);
        em |= (v >= 0 ? 1u : 0u) << k;
      }
      m &= em;
    } else {
      uint32_t em = 0;
      for (int k = 0; k < 16; ++k) {
        long long v = Ec + (long long)e[i].A * (16 * k + 8) + (long long)e[i].B * (16 * ((5 * k) & 15) + 8);
        em |= (v >= 0 ? 1u : 0u) << k;
      }
      m &= em;
    }
    if (!m) return 0u;
  }
  return m;
}

__global__ void __launch_bounds__(CV_NT, 1) k_coverage(
    const float4* __restrict__ rib, const uint32_t* __restrict__ tag,
    const int32_t* __restrict__ off, const uint32_t* __restrict__ bin, int64_t pair_cap, int W,
    int H, int tiles_x, int n_tile, uint16_t* __restrict__ canvas,
    unsigned long long* __restrict__ covered, int n_path, int32_t* counters, int32_t* status) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* s_mask = reinterpret_cast<uint32_t*>(smem);                       // SLOTS*MASK_WORDS
  EntrySetup* s_ent = reinterpret_cast<EntrySetup*>(s_mask + SLOTS * MASK_WORDS);  // CHUNK
  uint32_t* s_keys = reinterpret_cast<uint32_t*>(s_ent + CHUNK);              // HKEYS
  uint16_t* s_slot_of = reinterpret_cast<uint16_t*>(s_keys + HKEYS);          // HKEYS
  uint32_t* s_slot_path = reinterpret_cast<uint32_t*>(s_slot_of + HKEYS);     // HKEYS
  uint32_t* s_pre = s_slot_path + HKEYS;                                      // CHUNK + 1
  __shared__ int s_tile, s_nslot, s_total;
  __shared__ uint32_t s_wsum[CV_NT / 32];

  for (int i = threadIdx.x; i < SLOTS * MASK_WORDS; i += CV_NT) s_mask[i] = 0u;
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
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
    int64_t n = b1 > b0 ? b1 - b0 : 0;
    // valid pixels of this tile (canvas edge)
    int tw = min(TILE_PX, W - tx * TILE_PX), th = min(TILE_PX, H - ty * TILE_PX);
    for (int pass = 0;; ++pass) {
      int slot_lo = pass * SLOTS;
      for (int64_t c0 = 0; c0 < n; c0 += CHUNK) {
        int ne = (int)(n - c0 < (int64_t)CHUNK ? n - c0 : (int64_t)CHUNK);
        // ---- A: per-entry setup
        uint32_t cnt = 0;
        if (threadIdx.x < ne) {
          EntrySetup& E = s_ent[threadIdx.x];
          E.slot = 0xffff;
          E.valid = 0;
          uint32_t r = bin[b0 + c0 + threadIdx.x];
          uint32_t key = (__ldg(tag + r) >> 2) + 1u;
          // slot of the path (insert on the first pass)
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
              // the inserting thread may not have published the slot yet
              uint16_t so;
              int spin = 0;
              do {
                so = ((volatile uint16_t*)s_slot_of)[h];
              } while (so == 0xffffu && ++spin < (1 << 20));
              slot = so;
              break;
            }
            if (prev == 0u) break;
            h = (h + 1) & (HKEYS - 1);
          }
          QuadFix q;
          if (slot >= slot_lo && slot < slot_lo + SLOTS &&
              snap_quad(__ldg(rib + r - 1), __ldg(rib + r), q)) {
            for (int v = 0; v < 4; ++v) {
              q.x[v] -= ox;
              q.y[v] -= oy;
            }
            bool v0, v1, big = false;
            make_edges(q.x[0], q.y[0], q.x[1], q.y[1], q.x[3], q.y[3], E.e, v0, big);  // N0 P0 P1
            make_edges(q.x[0], q.y[0], q.x[3], q.y[3], q.x[2], q.y[2], E.e + 3, v1, big);  // N0 P1 N1
            E.valid = (v0 ? 1 : 0) | (v1 ? 2 : 0) | (big ? 4 : 0);
            E.slot = (uint16_t)(slot - slot_lo);
            // per-row spans over the 5 segments bounding both triangles
            float fx[4] = {(float)q.x[0], (float)q.x[1], (float)q.x[2], (float)q.x[3]};
            float fy[4] = {(float)q.y[0], (float)q.y[1], (float)q.y[2], (float)q.y[3]};
            float ymin = fminf(fminf(fy[0], fy[1]), fminf(fy[2], fy[3]));
            float ymax = fmaxf(fmaxf(fy[0], fy[1]), fmaxf(fy[2], fy[3]));
            E.rowpre[0] = 0;
            for (int ly = 0; ly < TILE_PX; ++ly) {
              int w = 0;
              if (ly < th && (v0 || v1)) {
                // sample rows of pixel row ly: y in [256 ly + 8, 256 ly + 248]; pad 1/256
                float ylo = 256.f * ly + 7.f, yhi = 256.f * ly + 249.f;
                if (!(ymax < ylo || ymin > yhi)) {
                  float xmin = 3.4e38f, xmax = -3.4e38f;
                  seg_strip(fx[0], fy[0], fx[1], fy[1], ylo, yhi, xmin, xmax);  // N0 P0
                  seg_strip(fx[1], fy[1], fx[3], fy[3], ylo, yhi, xmin, xmax);  // P0 P1
                  seg_strip(fx[3], fy[3], fx[2], fy[2], ylo, yhi, xmin, xmax);  // P1 N1
                  seg_strip(fx[2], fy[2], fx[0], fy[0], ylo, yhi, xmin, xmax);  // N1 N0
                  seg_strip(fx[0], fy[0], fx[3], fy[3], ylo, yhi, xmin, xmax);  // N0 P1
                  if (xmax >= xmin) {
                    // conservative by one pixel on each side of the float extent
                    int a = (int)floorf((xmin - 248.f) / 256.f), bb = (int)floorf((xmax - 8.f) / 256.f) + 1;
                    a = max(a, 0);
                    bb = min(bb, tw - 1);
                    if (bb >= a) {
                      w = bb - a + 1;
                      E.x0[ly] = (uint8_t)a;
                    }
                  }
                }
              }
              E.rowpre[ly + 1] = (uint16_t)(E.rowpre[ly] + w);
            }
            cnt = E.rowpre[TILE_PX];
          } else {
            E.rowpre[TILE_PX] = 0;
          }
        }
        // block exclusive scan of item counts
        uint32_t x = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x += y;
        }
        if (lane == 31) s_wsum[wid] = x;
        __syncthreads();
        if (wid == 0) {
          uint32_t v = lane < CV_NT / 32 ? s_wsum[lane] : 0u;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
          }
          if (lane < CV_NT / 32) s_wsum[lane] = v;
          if (lane == CV_NT / 32 - 1) s_total = (int)v;
        }
        __syncthreads();
        if (threadIdx.x < CHUNK) s_pre[threadIdx.x] = x - cnt + (wid > 0 ? s_wsum[wid - 1] : 0u);
        if (threadIdx.x == 0) s_pre[CHUNK] = 0x7fffffffu;
        __syncthreads();
        int total = s_total;
        // ---- B: items
        for (int it = threadIdx.x; it < total; it += CV_NT) {
          int lo = 0, hi = ne - 1;  // last entry with pre <= it
          while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if ((int)s_pre[mid] <= it) lo = mid; else hi = mid - 1;
          }
          const EntrySetup& E = s_ent[lo];
          int li = it - (int)s_pre[lo];
          int ly = 0;
          while ((int)E.rowpre[ly + 1] <= li) ++ly;
          int lx = E.x0[ly] + (li - (int)E.rowpre[ly]);
          bool big = (E.valid & 4) != 0;
          uint32_t m = 0;
          if (E.valid & 1) m |= tri_pixel_mask(E.e, big, lx, ly);
          if ((E.valid & 2) && m != 0xffffu) m |= tri_pixel_mask(E.e + 3, big, lx, ly);
          if (m) {
            int lp = ly * TILE_PX + lx;
            atomicOr(&s_mask[E.slot * MASK_WORDS + (lp >> 1)], m << (16 * (lp & 1)));
          }
        }
        __syncthreads();
      }
      // ---- C: popcounts and canvas for this pass's slots
      int nslot = min(s_nslot, HKEYS);
      int nhere = min(SLOTS, nslot - slot_lo);
      for (int s2 = wid; s2 < nhere; s2 += CV_NT / 32) {
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
        for (int s2 = 0; s2 < nhere; ++s2) {
          v |= s_mask[s2 * MASK_WORDS + w];
        }
        int lp = 2 * w;
        int py = ty * TILE_PX + lp / TILE_PX, px = tx * TILE_PX + lp % TILE_PX;
        if (py < H) {
          // later passes OR into what earlier passes wrote
          uint32_t prevv = 0;
          if (pass > 0) {
            if (px < W) prevv |= canvas[(int64_t)py * W + px];
            if (px + 1 < W) prevv |= (uint32_t)canvas[(int64_t)py * W + px + 1] << 16;
          }
          v |= prevv;
          if (px < W) canvas[(int64_t)py * W + px] = (uint16_t)(v & 0xffffu);
          if (px + 1 < W) canvas[(int64_t)py * W + px + 1] = (uint16_t)(v >> 16);
        }
      }
      __syncthreads();
      for (int i = threadIdx.x; i < nhere * MASK_WORDS; i += CV_NT) s_mask[i] = 0u;
      __syncthreads();
      if (nslot > HKEYS) {
        if (threadIdx.x == 0) ps_record_error(status, PS_ERR_CAPACITY);
      }
      if (slot_lo + SLOTS >= nslot) break;
    }
    __syncthreads();
  }
}

size_t coverage_smem_bytes() {
  return sizeof(uint32_t) * SLOTS * MASK_WORDS + sizeof(EntrySetup) * CHUNK +
         sizeof(uint32_t) * HKEYS + sizeof(uint16_t) * HKEYS + sizeof(uint32_t) * HKEYS +
         sizeof(uint32_t) * (CHUNK + 1);
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
      ctx->d_status); }
  return ps_cuda_check(cudaGetLastError());
}

extern "C" int ps_raster_pair_count(ps_context* ctx, int64_t* h_pairs) {
  if (!ctx || !h_pairs) return PS_ERR_INVALID;
  *h_pairs = 0;
  if (!ctx->d_tile_off || ctx->last_n_tile <= 0) return PS_OK;
  int32_t v = 0;
  cudaStream_t st = (cudaStream_t)ctx->last_stream;
  int rc = ps_cuda_check(cudaMemcpyAsync(&v, ctx->d_tile_off + ctx->last_n_tile, sizeof(int32_t),
                                         cudaMemcpyDeviceToHost, st));
  if (rc == PS_OK) rc = ps_cuda_check(cudaStreamSynchronize(st));
  *h_pairs = v;
  return rc;
}
