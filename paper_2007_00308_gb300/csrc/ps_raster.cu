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
constexpr int COV_NT = 256;                 // threads per coverage CTA
constexpr int COV_WARPS = COV_NT / 32;
constexpr int SMEM_SLOTS = 24;              // per-path masks kept in shared memory
constexpr int MAX_SLOTS = 512;              // per-path masks per tile (rest: global scratch)
constexpr int HASH = 1024;                  // open-addressing table of path ids
constexpr int WORDS_PER_MASK = TILE_PX * TILE_PX / 2;  // 2 pixels per 32-bit word
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

// Per-edge sample thresholds of one triangle, sorted, with cumulative masks:
// sample k passes the edge iff E(pixel) >= th[k]; with th sorted ascending,
// mask(E) = cm[c - 1] where c = #{th <= E}.
struct EdgeTab {
  int th[16];
  uint16_t cm[16];
};

struct TriSetup {
  int ax, ay;        // first vertex (1/256 px)
  int A[3], B[3];    // edge e: E = A (x - x_e) + B (y - y_e) with (x_e, y_e) its start vertex
  int ex[3], ey[3];
  bool valid;
};

__device__ __forceinline__ void tri_setup(int x0, int y0, int x1, int y1, int x2, int y2,
                                          TriSetup& T) {
  long long area = (long long)(x1 - x0) * (y2 - y0) - (long long)(y1 - y0) * (x2 - x0);
  T.valid = area != 0;
  if (area < 0) {
    int tx = x1, ty = y1;
    x1 = x2; y1 = y2; x2 = tx; y2 = ty;
  }
  int vx[3] = {x0, x1, x2}, vy[3] = {y0, y1, y2};
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    int ax = vx[e], ay = vy[e], bx = vx[(e + 1) % 3], by = vy[(e + 1) % 3];
    T.A[e] = ay - by;  // E = (bx-ax)(sy-ay) - (by-ay)(sx-ax)
    T.B[e] = bx - ax;
    T.ex[e] = ax;
    T.ey[e] = ay;
  }
}

// Build the three edge tables of a triangle cooperatively (lanes 0..15 sample k).
__device__ __forceinline__ void build_tabs(const TriSetup& T, EdgeTab* tab, int lane) {
  int k = lane & 15;
  int ox = 16 * k + 8, oy = 16 * ((5 * k) & 15) + 8;
  for (int e = 0; e < 3; ++e) {
    // threshold on E(pixel corner): E(sample) = E(corner) + A ox + B oy >= 0
    int th = -(T.A[e] * ox + T.B[e] * oy);
    uint32_t bit = 1u << k;
    // bitonic sort of (th, bit) over the 16-lane groups
#pragma unroll
    for (int size = 2; size <= 16; size <<= 1) {
#pragma unroll
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        int oth = __shfl_xor_sync(0xffffffffu, th, stride);
        uint32_t obit = __shfl_xor_sync(0xffffffffu, bit, stride);
        bool up = ((k & size) == 0);
        bool lower = (k & stride) == 0;
        bool take_min = (lower == up);
        bool swap = take_min ? (oth < th || (oth == th && obit < bit))
                             : (oth > th || (oth == th && obit > bit));
        if (swap) {
          th = oth;
          bit = obit;
        }
      }
    }
    // inclusive OR-prefix of bits in sorted order
    uint32_t cm = bit;
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, cm, o, 16);
      if (k >= o) cm |= y;
    }
    if (lane < 16) {
      tab[e].th[k] = th;
      tab[e].cm[k] = (uint16_t)cm;
    }
  }
}

__device__ __forceinline__ uint32_t edge_mask(const EdgeTab& t, long long E) {
  if (E < (long long)t.th[0]) return 0u;
  if (E >= (long long)t.th[15]) return 0xffffu;
  int e = (int)E;  // within [th[0], th[15]) so it fits
  int c = 0;       // c = #{th <= e} - 1 via binary search
#pragma unroll
  for (int s = 8; s > 0; s >>= 1)
    if (t.th[c + s] <= e) c += s;
  return t.cm[c];
}

__device__ __forceinline__ uint32_t tri_mask(const TriSetup& T, const EdgeTab* tab, int bx, int by) {
  uint32_t m = 0xffffu;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    long long E = (long long)T.A[e] * (bx - T.ex[e]) + (long long)T.B[e] * (by - T.ey[e]);
    m &= edge_mask(tab[e], E);
    if (!m) break;
  }
  return m;
}

__device__ __forceinline__ int hash_find(const uint32_t* keys, uint32_t key) {
  uint32_t h = (key * 2654435761u) & (HASH - 1);
  for (int i = 0; i < HASH; ++i) {
    uint32_t k = keys[h];
    if (k == key) return (int)h;
    if (k == 0u) return -1;
    h = (h + 1) & (HASH - 1);
  }
  return -1;
}

__global__ void __launch_bounds__(COV_NT) k_coverage(
    const float4* __restrict__ rib, const uint32_t* __restrict__ tag,
    const int32_t* __restrict__ off, const uint32_t* __restrict__ bin, int64_t pair_cap, int W,
    int H, int tiles_x, int n_tile, uint16_t* __restrict__ canvas,
    unsigned long long* __restrict__ covered, int n_path, uint32_t* __restrict__ gscratch,
    int32_t* counters, int32_t* status) {
  __shared__ uint32_t s_keys[HASH];
  __shared__ uint16_t s_slot_of[HASH];
  __shared__ uint32_t s_slot_path[MAX_SLOTS];
  __shared__ uint32_t s_masks[SMEM_SLOTS * WORDS_PER_MASK];
  __shared__ EdgeTab s_tab[COV_WARPS][2][3];
  __shared__ int s_nslot, s_tile;
  uint32_t* g_masks = gscratch + (size_t)blockIdx.x * MAX_SLOTS * WORDS_PER_MASK;
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(&counters[2], 1);
    for (int i = threadIdx.x; i < HASH; i += COV_NT) s_keys[i] = 0u;
    if (threadIdx.x == 0) s_nslot = 0;
    __syncthreads();
    int t = s_tile;
    if (t >= n_tile) return;
    int tx = t % tiles_x, ty = t / tiles_x;
    int64_t b0 = off[t], b1 = off[t + 1];
    if (b1 > pair_cap) b1 = pair_cap;
    int64_t n = b1 > b0 ? b1 - b0 : 0;
    // phase A: distinct paths of the tile -> slots
    for (int64_t i = threadIdx.x; i < n; i += COV_NT) {
      uint32_t r = bin[b0 + i];
      uint32_t key = (__ldg(tag + r) >> 2) + 1u;
      uint32_t h = (key * 2654435761u) & (HASH - 1);
      for (int it = 0; it < HASH; ++it) {
        uint32_t prev = atomicCAS(&s_keys[h], 0u, key);
        if (prev == 0u) {
          int s = atomicAdd(&s_nslot, 1);
          if (s < MAX_SLOTS) s_slot_path[s] = key - 1u;
          s_slot_of[h] = (uint16_t)(s < MAX_SLOTS ? s : 0xffff);
          break;
        }
        if (prev == key) break;
        h = (h + 1) & (HASH - 1);
      }
    }
    __syncthreads();
    int nslot = s_nslot;
    if (nslot > MAX_SLOTS) {
      if (threadIdx.x == 0) ps_record_error(status, PS_ERR_CAPACITY);
      nslot = MAX_SLOTS;
    }
    uint32_t* masks = nslot <= SMEM_SLOTS ? s_masks : g_masks;
    for (int i = threadIdx.x; i < nslot * WORDS_PER_MASK; i += COV_NT) masks[i] = 0u;
    __syncthreads();
    // phase B: every quad of the bin ORs its samples into its path's mask
    int tpx0 = tx * TILE_PX, tpy0 = ty * TILE_PX;
    for (int64_t i = wid; i < n; i += COV_WARPS) {
      uint32_t r = bin[b0 + i];
      uint32_t key = (__ldg(tag + r) >> 2) + 1u;
      int h = hash_find(s_keys, key);
      int slot = h >= 0 ? s_slot_of[h] : 0xffff;
      if (slot >= nslot) continue;
      QuadFix q;
      if (!snap_quad(__ldg(rib + r - 1), __ldg(rib + r), q)) continue;
      int px0, px1, py0, py1;
      quad_pixels(q, W, H, px0, px1, py0, py1);
      px0 = max(px0, tpx0);
      px1 = min(px1, tpx0 + TILE_PX - 1);
      py0 = max(py0, tpy0);
      py1 = min(py1, tpy0 + TILE_PX - 1);
      if (px0 > px1 || py0 > py1) continue;
      TriSetup T0, T1;
      tri_setup(q.x[0], q.y[0], q.x[1], q.y[1], q.x[3], q.y[3], T0);  // N0 P0 P1
      tri_setup(q.x[0], q.y[0], q.x[3], q.y[3], q.x[2], q.y[2], T1);  // N0 P1 N1
      __syncwarp();
      if (T0.valid) build_tabs(T0, s_tab[wid][0], lane);
      if (T1.valid) build_tabs(T1, s_tab[wid][1], lane);
      __syncwarp();
      int wpx = px1 - px0 + 1, npx = wpx * (py1 - py0 + 1);
      for (int pi = lane; pi < npx; pi += 32) {
        int px = px0 + pi % wpx, py = py0 + pi / wpx;
        int bx = px * 256, by = py * 256;
        uint32_t m = 0;
        if (T0.valid) m |= tri_mask(T0, s_tab[wid][0], bx, by);
        if (T1.valid && m != 0xffffu) m |= tri_mask(T1, s_tab[wid][1], bx, by);
        if (m) {
          int lp = (py - tpy0) * TILE_PX + (px - tpx0);
          atomicOr(&masks[slot * WORDS_PER_MASK + (lp >> 1)], m << (16 * (lp & 1)));
        }
      }
    }
    __syncthreads();
    // phase C: per-path popcounts and the canvas OR
    for (int s = wid; s < nslot; s += COV_WARPS) {
      unsigned cnt = 0;
      for (int w = lane; w < WORDS_PER_MASK; w += 32) cnt += __popc(masks[s * WORDS_PER_MASK + w]);
      for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
      if (lane == 0 && cnt) {
        uint32_t p = s_slot_path[s];
        if ((int)p < n_path) atomicAdd(covered + p, (unsigned long long)cnt);
      }
    }
    for (int w = threadIdx.x; w < WORDS_PER_MASK; w += COV_NT) {
      uint32_t v = 0;
      for (int s = 0; s < nslot; ++s) v |= masks[s * WORDS_PER_MASK + w];
      int lp = 2 * w;
      int py = tpy0 + lp / TILE_PX, px = tpx0 + lp % TILE_PX;
      if (py < H) {
        if (px < W) canvas[(int64_t)py * W + px] = (uint16_t)(v & 0xffffu);
        if (px + 1 < W) canvas[(int64_t)py * W + px + 1] = (uint16_t)(v >> 16);
      }
    }
    __syncthreads();
  }
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
  int grid_cov = ps_persistent_grid(ctx, (const void*)k_coverage, COV_NT, 0);
  size_t scratch_words = (size_t)grid_cov * MAX_SLOTS * WORDS_PER_MASK;
  if (ctx->d_scratch_words < scratch_words) {
    if (ctx->d_mask_scratch) cudaFree(ctx->d_mask_scratch);
    ctx->d_mask_scratch = nullptr;
    if ((rc = ps_cuda_check(cudaMalloc((void**)&ctx->d_mask_scratch,
                                       scratch_words * sizeof(uint32_t)))) != PS_OK)
      return rc;
    ctx->d_scratch_words = scratch_words;
  }
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
  k_coverage<<<grid_cov, COV_NT, 0, st>>>(rib, d_tag, ctx->d_tile_off, ctx->d_bin, ctx->pair_cap,
                                          width, height, tiles_x, (int)n_tile, d_canvas,
                                          reinterpret_cast<unsigned long long*>(d_covered),
                                          n_path, ctx->d_mask_scratch, ctx->d_counters,
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
