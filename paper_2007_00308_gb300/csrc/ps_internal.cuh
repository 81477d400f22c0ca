// Internal declarations of the GB300 polar stroking library.
//
// Device-side geometry is FP32; FP64 appears only in the predicated islands of
// the PS_PREC_MIXED variant (GB300 issues FP64 FMAs ~57x slower than FP32).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/polarstroke.h"
#include "ps_df.cuh"

#define PS_PI_F 3.14159265358979323846f
#define PS_TWO_PI_F 6.28318530717958647692f
#define PS_PI_D 3.14159265358979323846
#define PS_TWO_PI_D 6.28318530717958647692

// Bounded spin for inter-CTA waits: after this many polls a wait gives up,
// records PS_ERR_TIMEOUT and proceeds (results of that launch are invalid).
#define PS_SPIN_LIMIT (1 << 22)

// Link kinds stored in LinkRec::meta bits 0-1.
enum { LK_EMPTY = 0, LK_SEG = 1, LK_JOIN = 2, LK_CAP = 3 };

// Per-link interval record written by the setup pass and read by the rib pass.
// 240 bytes; at most 6 intervals (3 curvature-monotone intervals of a cubic,
// each split once at pi -- Sec. 3.3.5), boundaries k = 0..M.  The *_lo fields
// complete psi, p and step to double-float pairs (hi + lo) in PS_PREC_MIXED;
// they are zero in PS_PREC_FP32.
struct __align__(16) LinkRec {
  float2 P[4];        // control points (segment) / P[0] = pivot point (join, cap)
  float w;            // conic weight
  float rN, rP;       // radii of the N and P sides (Eq. 16-17)
  uint32_t meta;      // kind | type<<2 | M<<4 | pivot mask<<8 | style<<16 | flags<<20
  float psi[7];       // Psi_k at interval boundaries (Eq. 5)
  float p[7];         // p_k (Eq. 4)
  float step[6];      // delta_k / Delta_k (Eq. 12, psi(j) of Sec. 4.2.1)
  uint16_t dsum[7];   // Delta_Sigma(k) (Eq. 13)
  uint16_t pad;
  float2 v1, v2;      // miter override vertices for ribs 1 and 2
  float psi_lo[7];
  float p_lo[7];
  float step_lo[6];
};
static_assert(sizeof(LinkRec) == 240, "LinkRec layout");

#define META_KIND(m) ((m) & 3u)
#define META_TYPE(m) (((m) >> 2) & 3u)
#define META_M(m) (((m) >> 4) & 15u)
#define META_PIVOT(m, k) (((m) >> (8 + (k))) & 1u)
#define META_STYLE(m) (((m) >> 16) & 15u)
#define META_FLAG_OVERRIDE (1u << 20)  // ribs 1,2 outer vertex = v1, v2 (miter)
#define META_FLAG_SQUARE (1u << 21)    // square cap: ribs 1,3 outer radius * sqrt(2)
// interior boundary k (1..6) is a split point (Sec. 3.3.5) rather than an inflection
#define META_SPLIT_BIT(k) (1u << (21 + (k)))
#define META_SPLIT(m, k) (((m) >> (21 + (k))) & 1u)

// Profiling slots (one per kernel).
enum {
  PK_LINK_PATH = 0, PK_LINK_SETUP, PK_EMIT, PK_ARCLEN, PK_MIDCHORD, PK_BIN_COUNT, PK_TILE_SCAN,
  PK_BIN_SCATTER, PK_COVERAGE, PK_DASH, PK_COUNT
};
static_assert(PK_COUNT == PS_PROF_SLOTS, "profile slots");

// Host-side context.
struct ps_context {
  int prof_on;
  cudaEvent_t prof_ev[PK_COUNT][2];
  int prof_recorded[PK_COUNT];
  int device;
  int cov_attr_done[2];  // coverage kernels' shared-memory attribute set on this device
  void* last_stream;
  int32_t* d_status;        // first error recorded by a kernel
  // scan tile states (shared by the passes of one call; calls on one context
  // are serialized on the stream they are issued to)
  uint32_t* d_tile_flag;
  long long* d_tile_agg;
  long long* d_tile_incl;
  double* d_tile_aggd;
  double* d_tile_incld;
  int64_t tile_cap;
  int32_t* d_counters;      // ticket counters, 16 ints
  LinkRec* d_recs;
  int64_t rec_cap;
  // raster workspace
  int32_t* d_tile_count;    // [n_tile + 1]
  int32_t* d_tile_off;      // [n_tile + 1]
  int32_t* d_tile_cursor;   // [2 (n_tile + 1)]: scatter cursors from the front, then from the back
  int32_t* d_tile_list;     // tiles with bin entries, then their count
  int64_t raster_tile_cap;
  uint32_t* d_bin;          // [pair_cap]
  uint32_t* d_quad_hits;    // [2 quad_hits_cap] per-rib {hits, box} words of the binning passes
  int64_t quad_hits_cap;
  int64_t pair_cap;
  int64_t* d_scratch64;     // 16 int64 of per-call scalars
  int64_t last_n_tile;      // tiles of the most recent raster call
  uint32_t* d_mask_scratch; // per-CTA per-path tile masks beyond shared memory
  size_t d_scratch_words;
  void* d_adj;              // adjoint workspace
  size_t adj_bytes;
  int num_sms;
  int tune[PS_TUNE_COUNT];  // launch parameters (ps_set_tuning)
  float pixel_tol;          // pixel tolerance of the per-link step boost (0: off)
};

// ---- status -----------------------------------------------------------------
__device__ __forceinline__ void ps_record_error(int32_t* status, int code) {
  // read first: a launch where many threads fail would otherwise serialize on
  // one atomic per failure
  if (status && *(volatile int32_t*)status == 0) atomicCAS(status, 0, code);
}

// ---- release / acquire ------------------------------------------------------
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_s64(long long* p, long long v) {
  asm volatile("st.relaxed.gpu.global.s64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ long long ld_relaxed_s64(const long long* p) {
  long long v;
  asm volatile("ld.relaxed.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_f64(double* p, double v) {
  asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ double ld_relaxed_f64(const double* p) {
  double v;
  asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
  return v;
}

// Tile flags of the single-pass scans (decoupled look-back, Merrill & Garland
// 2016): 0 = not ready, 1 = aggregate published, 2 = inclusive prefix published.
// Bit 2 marks a segment head (segmented scans).
#define TF_AGG 1u
#define TF_INCL 2u
#define TF_HEAD 4u

// Exclusive prefix of tile t for an int64 sum, with the walk spread over one
// warp (all 32 lanes call it): lane k reads the state of tile i - k, so one
// round covers 32 predecessors.  The walk ends at the nearest tile with an
// inclusive prefix; that tile and every nearer one must have published before
// the round is summed, else the round is read again (bounded by
// PS_SPIN_LIMIT).
__device__ __forceinline__ long long lookback_sum_warp(uint32_t* flag, long long* agg,
                                                       long long* incl, long long tile_agg,
                                                       int64_t t, int32_t* status) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) {
    if (t == 0) {
      st_relaxed_s64(&incl[0], tile_agg);
      st_release_u32(&flag[0], TF_INCL);
    } else {
      st_relaxed_s64(&agg[t], tile_agg);
      st_release_u32(&flag[t], TF_AGG);
    }
  }
  if (t == 0) return 0;
  long long prefix = 0;
  int64_t i = t - 1;
  int spins = 0;
  for (;;) {
    int64_t j = i - lane;
    uint32_t f = j >= 0 ? ld_acquire_u32(&flag[j]) : TF_INCL;  // before tile 0: zero
    unsigned stop_m = __ballot_sync(0xffffffffu, (f & TF_INCL) != 0u);
    unsigned unready = __ballot_sync(0xffffffffu, (f & (TF_INCL | TF_AGG)) == 0u);
    int first = stop_m ? __ffs(stop_m) - 1 : 31;
    unsigned need = first == 31 ? 0xffffffffu : ((2u << first) - 1u);
    if (unready & need) {
      if (++spins > PS_SPIN_LIMIT) {
        if (lane == 0) ps_record_error(status, PS_ERR_TIMEOUT);
        break;
      }
      __nanosleep(32);
      continue;
    }
    long long v = 0;
    if (lane <= first && j >= 0) v = (f & TF_INCL) ? ld_relaxed_s64(&incl[j]) : ld_relaxed_s64(&agg[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    prefix += v;
    if (stop_m) break;
    i -= 32;
  }
  if (lane == 0) {
    st_relaxed_s64(&incl[t], prefix + tile_agg);
    st_release_u32(&flag[t], TF_INCL);
  }
  return prefix;
}

// Tile states of the arc-length look-backs: a double-float pair packed in 64
// bits (hi in the low word), stored and loaded relaxed.
__device__ __forceinline__ void st_relaxed_df(unsigned long long* p, ps::DF v) {
  const unsigned long long w =
      ((unsigned long long)__float_as_uint(v.lo) << 32) | (unsigned long long)__float_as_uint(v.hi);
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}
__device__ __forceinline__ ps::DF ld_relaxed_df(const unsigned long long* p) {
  unsigned long long w;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
  return ps::DF{__uint_as_float((uint32_t)w), __uint_as_float((uint32_t)(w >> 32))};
}

// Segmented (by path) sum of the tiles (chunks) before tile t: the carry into
// the tile's elements that precede its first segment head (path start).  A chunk that holds a path
// start publishes its inclusive value at once (it does not depend on the
// carry); the walk, one warp reading 32 predecessors per round, ends at the
// nearest chunk with an inclusive value or a path start, once that chunk and
// every nearer one have published (bounded by PS_SPIN_LIMIT; PS_ERR_TIMEOUT
// after it).  Sums are double-float pairs.
__device__ __forceinline__ ps::DF lookback_segsum_df(uint32_t* flag, unsigned long long* agg,
                                                 unsigned long long* incl, ps::DF tile_agg,
                                                 bool tile_head, int64_t t, int32_t* status) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) {
    if (t == 0 || tile_head) {
      st_relaxed_df(&incl[t], tile_agg);
      st_release_u32(&flag[t], TF_INCL | (tile_head ? TF_HEAD : 0u));
    } else {
      st_relaxed_df(&agg[t], tile_agg);
      st_release_u32(&flag[t], TF_AGG);
    }
  }
  ps::DF carry{0.f, 0.f};
  if (t == 0) return carry;
  int64_t i = t - 1;
  int spins = 0;
  for (;;) {
    const int64_t j = i - lane;
    const uint32_t f = j >= 0 ? ld_acquire_u32(&flag[j]) : TF_INCL;  // before chunk 0: zero
    const unsigned stop_m = __ballot_sync(0xffffffffu, (f & TF_INCL) != 0u);
    const unsigned unready = __ballot_sync(0xffffffffu, (f & (TF_INCL | TF_AGG)) == 0u);
    const int first = stop_m ? __ffs(stop_m) - 1 : 31;
    const unsigned need = first == 31 ? 0xffffffffu : ((2u << first) - 1u);
    if (unready & need) {
      if (++spins > PS_SPIN_LIMIT) {
        if (lane == 0) ps_record_error(status, PS_ERR_TIMEOUT);
        break;
      }
      __nanosleep(32);
      continue;
    }
    ps::DF v{0.f, 0.f};
    if (lane <= first && j >= 0) v = (f & TF_INCL) ? ld_relaxed_df(&incl[j]) : ld_relaxed_df(&agg[j]);
    if (first == 0) {  // the nearest predecessor holds the prefix: no reduction
      v = ps::DF{__shfl_sync(0xffffffffu, v.hi, 0), __shfl_sync(0xffffffffu, v.lo, 0)};
    } else {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
        v = ps::df_add(v, ps::DF{__shfl_xor_sync(0xffffffffu, v.hi, o),
                                 __shfl_xor_sync(0xffffffffu, v.lo, o)});
    }
    carry = ps::df_add(carry, v);
    if (stop_m) break;
    i -= 32;
  }
  if (lane == 0 && !tile_head) {
    st_relaxed_df(&incl[t], ps::df_add(carry, tile_agg));
    st_release_u32(&flag[t], TF_INCL);
  }
  return carry;
}

// ---- host helpers -------------------------------------------------------------
int ps_ensure_tiles(ps_context* ctx, int64_t n_tile);
int ps_ensure_recs(ps_context* ctx, int64_t n_link);
int ps_ensure_raster(ps_context* ctx, int64_t n_tile, int64_t n_pair);
int ps_ensure_quad_hits(ps_context* ctx, int64_t n_rib);
int ps_cuda_check(cudaError_t e);
int ps_persistent_grid(ps_context* ctx, const void* kernel, int block, size_t smem);
// Link setup (records in ctx->d_recs, link path indices after them) into the given
// offset arrays; used by the adjoint to rebuild the forward's interval records.
int ps_run_link_setup(ps_context* ctx, const ps_segments* seg, const ps_paths* paths, float dtheta,
                      int precision, int32_t* d_link_off, int32_t* d_path_off, int64_t* d_n_rib,
                      cudaStream_t st);
// Segmented (by path) inclusive prefix of per-rib values, in place, with per-path totals.
int ps_run_segmented_prefix(ps_context* ctx, float* d_vals, const uint32_t* d_tag,
                            const int64_t* d_n_rib, int64_t capacity, float* d_path_tot,
                            int32_t n_path, cudaStream_t st);
void ps_prof_mark(ps_context* ctx, int slot, int end, cudaStream_t st);
struct ProfScope {
  ps_context* c;
  int slot;
  cudaStream_t st;
  ProfScope(ps_context* c_, int s_, cudaStream_t st_) : c(c_), slot(s_), st(st_) {
    ps_prof_mark(c, slot, 0, st);
  }
  ~ProfScope() { ps_prof_mark(c, slot, 1, st); }
};
