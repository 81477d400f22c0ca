#include <cmath>
// Context, workspace and status handling of the C ABI.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "ps_internal.cuh"

int ps_cuda_check(cudaError_t e) { return e == cudaSuccess ? PS_OK : PS_ERR_CUDA; }

static int grow(void** p, size_t bytes) {
  if (*p) cudaFree(*p);
  *p = nullptr;
  if (bytes == 0) return PS_OK;
  return ps_cuda_check(cudaMalloc(p, bytes));
}

int ps_ensure_tiles(ps_context* ctx, int64_t n) {
  if (n <= ctx->tile_cap) return PS_OK;
  int64_t cap = n + n / 4 + 64;
  int rc;
  if ((rc = grow((void**)&ctx->d_tile_flag, sizeof(uint32_t) * cap)) != PS_OK) return rc;
  if ((rc = grow((void**)&ctx->d_tile_agg, sizeof(long long) * cap)) != PS_OK) return rc;
  if ((rc = grow((void**)&ctx->d_tile_incl, sizeof(long long) * cap)) != PS_OK) return rc;
  if ((rc = grow((void**)&ctx->d_tile_aggd, sizeof(double) * cap)) != PS_OK) return rc;
  if ((rc = grow((void**)&ctx->d_tile_incld, sizeof(double) * cap)) != PS_OK) return rc;
  ctx->tile_cap = cap;
  return PS_OK;
}

int ps_ensure_recs(ps_context* ctx, int64_t n_link) {
  if (n_link <= ctx->rec_cap) return PS_OK;
  int64_t cap = n_link + n_link / 4 + 64;
  // records followed by one int32 path index per link
  int rc = grow((void**)&ctx->d_recs, (sizeof(LinkRec) + sizeof(int32_t)) * cap);
  if (rc != PS_OK) return rc;
  ctx->rec_cap = cap;
  return PS_OK;
}

int ps_ensure_raster(ps_context* ctx, int64_t n_tile, int64_t n_pair) {
  int rc;
  if (n_tile > ctx->raster_tile_cap) {
    int64_t cap = n_tile + 64;
    if ((rc = grow((void**)&ctx->d_tile_count, sizeof(int32_t) * (cap + 1))) != PS_OK) return rc;
    if ((rc = grow((void**)&ctx->d_tile_off, sizeof(int32_t) * (cap + 1))) != PS_OK) return rc;
    if ((rc = grow((void**)&ctx->d_tile_cursor, 2 * sizeof(int32_t) * (cap + 1))) != PS_OK) return rc;
    if ((rc = grow((void**)&ctx->d_tile_list, sizeof(int32_t) * (cap + 1))) != PS_OK) return rc;
    ctx->raster_tile_cap = cap;
  }
  if (n_pair > ctx->pair_cap) {
    int64_t cap = n_pair + n_pair / 8 + 1024;
    if ((rc = grow((void**)&ctx->d_bin, sizeof(uint32_t) * cap)) != PS_OK) return rc;
    ctx->pair_cap = cap;
  }
  return PS_OK;
}

int ps_ensure_quad_hits(ps_context* ctx, int64_t n_rib) {
  if (n_rib <= ctx->quad_hits_cap) return PS_OK;
  int64_t cap = n_rib + n_rib / 8 + 1024;
  int rc = grow((void**)&ctx->d_quad_hits, 2 * sizeof(uint32_t) * cap);
  if (rc != PS_OK) return rc;
  ctx->quad_hits_cap = cap;
  return PS_OK;
}

int ps_persistent_grid(ps_context* ctx, const void* kernel, int block, size_t smem) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return ctx->num_sms * per_sm;
}

extern "C" int ps_create(ps_context** out) {
  if (!out) return PS_ERR_INVALID;
  ps_context* ctx = (ps_context*)calloc(1, sizeof(ps_context));
  if (!ctx) return PS_ERR_INVALID;
  if (cudaGetDevice(&ctx->device) != cudaSuccess) {
    free(ctx);
    return PS_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (ctx->num_sms <= 0) ctx->num_sms = 1;
  if (cudaMalloc((void**)&ctx->d_status, 64) != cudaSuccess ||
      cudaMalloc((void**)&ctx->d_counters, sizeof(int32_t) * 16) != cudaSuccess ||
      cudaMalloc((void**)&ctx->d_scratch64, sizeof(int64_t) * 16) != cudaSuccess) {
    ps_destroy(ctx);
    return PS_ERR_CUDA;
  }
  cudaMemset(ctx->d_status, 0, 64);
  cudaMemset(ctx->d_counters, 0, sizeof(int32_t) * 16);
  ctx->tune[PS_TUNE_EMIT_SLABS] = 32;
  ctx->tune[PS_TUNE_SETUP_LINKS] = 2;
  ctx->tune[PS_TUNE_BIN_BLOCKS] = 0;
  ctx->pixel_tol = 0.f;
  *out = ctx;
  return PS_OK;
}

extern "C" int ps_set_tuning(ps_context* ctx, int key, int value) {
  if (!ctx) return PS_ERR_INVALID;
  switch (key) {
    case PS_TUNE_EMIT_SLABS:
      if (value != 4 && value != 8 && value != 16 && value != 32 && value != 64)
        return PS_ERR_INVALID;
      break;
    case PS_TUNE_SETUP_LINKS:
      if (value != 1 && value != 2 && value != 4) return PS_ERR_INVALID;
      break;
    case PS_TUNE_BIN_BLOCKS:
      if (value < 0 || value > 16) return PS_ERR_INVALID;
      break;
    default:
      return PS_ERR_INVALID;
  }
  ctx->tune[key] = value;
  return PS_OK;
}

extern "C" int ps_get_tuning(ps_context* ctx, int key, int* value) {
  if (!ctx || !value || key < 0 || key >= PS_TUNE_COUNT) return PS_ERR_INVALID;
  *value = ctx->tune[key];
  return PS_OK;
}

extern "C" int ps_set_pixel_tolerance(ps_context* ctx, float tau) {
  if (!ctx || !(tau >= 0.f) || !(tau < INFINITY)) return PS_ERR_INVALID;
  ctx->pixel_tol = tau;
  return PS_OK;
}

extern "C" int ps_get_pixel_tolerance(ps_context* ctx, float* tau) {
  if (!ctx || !tau) return PS_ERR_INVALID;
  *tau = ctx->pixel_tol;
  return PS_OK;
}

extern "C" void ps_destroy(ps_context* ctx) {
  if (!ctx) return;
  if (ctx->prof_on) ps_profile_enable(ctx, 0);
  void* ptrs[] = {ctx->d_status, ctx->d_tile_flag, ctx->d_tile_agg, ctx->d_tile_incl,
                  ctx->d_tile_aggd, ctx->d_tile_incld, ctx->d_counters, ctx->d_recs,
                  ctx->d_tile_count, ctx->d_tile_off, ctx->d_tile_cursor, ctx->d_bin,
                  ctx->d_scratch64, ctx->d_mask_scratch, ctx->d_adj, ctx->d_quad_hits,
                  ctx->d_tile_list};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  free(ctx);
}

extern "C" int ps_reserve(ps_context* ctx, int64_t n_link, int64_t n_rib, int64_t n_tile,
                          int64_t n_pair) {
  if (!ctx || n_link < 0 || n_rib < 0 || n_tile < 0 || n_pair < 0) return PS_ERR_INVALID;
  int rc;
  if (n_link && (rc = ps_ensure_recs(ctx, n_link)) != PS_OK) return rc;
  int64_t tiles = (n_link + 511) / 512 + (n_rib + 2047) / 2048 + 4 + n_rib / 512;
  if ((rc = ps_ensure_tiles(ctx, tiles)) != PS_OK) return rc;
  if ((n_tile || n_pair) && (rc = ps_ensure_raster(ctx, n_tile, n_pair)) != PS_OK) return rc;
  return PS_OK;
}

extern "C" int ps_max_ribs(int64_t n_seg, int32_t n_path, float dtheta, int64_t* h_bound) {
  if (!h_bound || n_seg < 0 || n_path < 0 || !(dtheta > 0.f)) return PS_ERR_INVALID;
  double q = dtheta;
  int64_t per_seg = (int64_t)ceil(2.0 * 3.14159265358979323846 / q) + 7;
  int64_t half = (int64_t)ceil(3.14159265358979323846 / q);
  int64_t per_pivot = (half > 4 ? half : 4) + 1;
  *h_bound = n_seg * per_seg + (n_seg + (int64_t)n_path) * per_pivot;
  return PS_OK;
}

extern "C" int ps_get_status(ps_context* ctx, int* h_status) {
  if (!ctx || !h_status) return PS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)ctx->last_stream;
  int32_t v = 0;
  int rc = ps_cuda_check(cudaMemcpyAsync(&v, ctx->d_status, sizeof(int32_t),
                                         cudaMemcpyDeviceToHost, st));
  if (rc == PS_OK) rc = ps_cuda_check(cudaStreamSynchronize(st));
  if (rc != PS_OK) return rc;
  *h_status = v;
  cudaMemsetAsync(ctx->d_status, 0, sizeof(int32_t), st);
  return ps_cuda_check(cudaStreamSynchronize(st));
}

// One warp takes the part of tile 1 of a look-back whose tile 0 never
// publishes: its wait runs to the poll limit, records PS_ERR_TIMEOUT and ends.
// It touches tiles 0 and 1 only.
__global__ void k_wait_check(uint32_t* flag, long long* agg, long long* incl, double* aggd,
                             double* incld, int which, int32_t* status) {
  if (which == 0)
    lookback_sum_warp(flag, agg, incl, 1, 1, status);
  else
    lookback_segsum_df(flag, reinterpret_cast<unsigned long long*>(aggd),
                       reinterpret_cast<unsigned long long*>(incld), ps::DF{1.f, 0.f}, false, 1,
                       status);
}

extern "C" int ps_check_wait_timeout(ps_context* ctx, int which, void* stream) {
  if (!ctx || (which != 0 && which != 1)) return PS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  // flags at 0, int64 values at 64 and 96, doubles at 128 and 160 (2 tiles each)
  char* buf = nullptr;
  int rc = ps_cuda_check(cudaMalloc((void**)&buf, 256));
  if (rc != PS_OK) return rc;
  rc = ps_cuda_check(cudaMemsetAsync(buf, 0, 256, st));
  if (rc == PS_OK) {
    k_wait_check<<<1, 32, 0, st>>>((uint32_t*)buf, (long long*)(buf + 64),
                                   (long long*)(buf + 96), (double*)(buf + 128),
                                   (double*)(buf + 160), which, ctx->d_status);
    rc = ps_cuda_check(cudaGetLastError());
  }
  if (rc == PS_OK) rc = ps_cuda_check(cudaStreamSynchronize(st));
  cudaFree(buf);
  ctx->last_stream = stream;
  return rc;
}

void ps_prof_mark(ps_context* ctx, int slot, int end, cudaStream_t st) {
  if (!ctx->prof_on) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  if (cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(ctx->prof_ev[slot][end], st, cudaEventRecordExternal);
  else
    cudaEventRecord(ctx->prof_ev[slot][end], st);
  if (end) ctx->prof_recorded[slot] = 1;
}

extern "C" int ps_profile_enable(ps_context* ctx, int enable) {
  if (!ctx) return PS_ERR_INVALID;
  if (enable && !ctx->prof_on) {
    for (int s = 0; s < PK_COUNT; ++s)
      for (int e = 0; e < 2; ++e)
        if (cudaEventCreate(&ctx->prof_ev[s][e]) != cudaSuccess) return PS_ERR_CUDA;
  }
  if (!enable && ctx->prof_on) {
    cudaDeviceSynchronize();
    for (int s = 0; s < PK_COUNT; ++s)
      for (int e = 0; e < 2; ++e) cudaEventDestroy(ctx->prof_ev[s][e]);
  }
  for (int s = 0; s < PK_COUNT; ++s) ctx->prof_recorded[s] = 0;
  ctx->prof_on = enable ? 1 : 0;
  return PS_OK;
}

extern "C" int ps_profile_read(ps_context* ctx, float* h_ms) {
  if (!ctx || !h_ms) return PS_ERR_INVALID;
  for (int s = 0; s < PK_COUNT; ++s) {
    h_ms[s] = -1.f;
    if (!ctx->prof_on || !ctx->prof_recorded[s]) continue;
    if (cudaEventSynchronize(ctx->prof_ev[s][1]) != cudaSuccess) return PS_ERR_CUDA;
    float ms = -1.f;
    if (cudaEventElapsedTime(&ms, ctx->prof_ev[s][0], ctx->prof_ev[s][1]) == cudaSuccess) h_ms[s] = ms;
  }
  return PS_OK;
}

extern "C" const char* ps_profile_slot_name(int slot) {
  static const char* names[PK_COUNT] = {"k_link_path", "k_link_setup", "k_emit", "k_arclen_scan",
                                        "k_midpoint_chords", "k_bin_count", "k_tile_scan",
                                        "k_bin_scatter", "k_coverage", "k_dash"};
  return (slot >= 0 && slot < PK_COUNT) ? names[slot] : "";
}

extern "C" const char* ps_error_string(int code) {
  switch (code) {
    case PS_OK: return "ok";
    case PS_ERR_INVALID: return "invalid argument";
    case PS_ERR_CAPACITY: return "capacity exceeded";
    case PS_ERR_TIMEOUT: return "bounded inter-CTA wait timed out";
    case PS_ERR_CUDA: return "CUDA runtime error";
    case PS_ERR_RANGE: return "vertex coordinate out of the rasterizer's range";
    default: return "unknown error";
  }
}

// ---------------------------------------------------------------------------
// SVG elliptical arc (endpoint parameterization) -> conic segments.  Host code.
// Steps (SVG 1.1 arc implementation notes, restated): move the chord midpoint
// to the origin and undo the rotation phi; scale the radii up when the
// endpoints are too far apart for them; the centre follows from the chord and
// the radii, on the side the two flags select; the start angle and the signed
// sweep are taken on the unit circle of the ellipse's own axes.  The sweep is
// cut into n <= 4 equal pieces of at most 90 degrees; a piece [a, b] of the
// unit circle is the rational quadratic with end points at angles a and b,
// middle control point at angle (a+b)/2 and distance 1/cos h (h = (b-a)/2, where
// the end tangents meet), and weight cos h.  An affine map (scale by rx, ry,
// rotate by phi, translate to the centre) keeps the weight.
extern "C" int ps_svg_arc_to_conics(float x0, float y0, float rx, float ry, float phi_deg,
                                    int large_arc, int sweep, float x1, float y1,
                                    float* h_pts, float* h_w) {
  if (!h_pts || !h_w) return PS_ERR_INVALID;
  if (!(std::isfinite(x0) && std::isfinite(y0) && std::isfinite(x1) && std::isfinite(y1) &&
        std::isfinite(rx) && std::isfinite(ry) && std::isfinite(phi_deg)))
    return PS_ERR_INVALID;
  if (x0 == x1 && y0 == y1) return 0;  // no arc at all
  double Rx = std::fabs((double)rx), Ry = std::fabs((double)ry);
  auto put = [&](int i, double ax, double ay, double bx, double by, double dx, double dy,
                 double w) {
    float* o = h_pts + 8 * i;
    o[0] = (float)ax; o[1] = (float)ay; o[2] = (float)bx; o[3] = (float)by;
    o[4] = (float)bx; o[5] = (float)by; o[6] = (float)dx; o[7] = (float)dy;
    h_w[i] = (float)w;
  };
  if (Rx == 0.0 || Ry == 0.0) {  // a straight segment: a flat conic
    put(0, x0, y0, 0.5 * ((double)x0 + x1), 0.5 * ((double)y0 + y1), x1, y1, 1.0);
    return 1;
  }
  const double PI = 3.14159265358979323846;
  double phi = (double)phi_deg * PI / 180.0, cp = std::cos(phi), sp = std::sin(phi);
  double hx = 0.5 * ((double)x0 - x1), hy = 0.5 * ((double)y0 - y1);
  double xp = cp * hx + sp * hy, yp = -sp * hx + cp * hy;
  double lam = (xp * xp) / (Rx * Rx) + (yp * yp) / (Ry * Ry);
  if (lam > 1.0) {
    double k = std::sqrt(lam);
    Rx *= k;
    Ry *= k;
  }
  double num = Rx * Rx * Ry * Ry - Rx * Rx * yp * yp - Ry * Ry * xp * xp;
  double den = Rx * Rx * yp * yp + Ry * Ry * xp * xp;
  double f = (num > 0.0 && den > 0.0) ? std::sqrt(num / den) : 0.0;
  if ((large_arc != 0) == (sweep != 0)) f = -f;
  double cxp = f * Rx * yp / Ry, cyp = -f * Ry * xp / Rx;
  double cx = cp * cxp - sp * cyp + 0.5 * ((double)x0 + x1);
  double cy = sp * cxp + cp * cyp + 0.5 * ((double)y0 + y1);
  double ux = (xp - cxp) / Rx, uy = (yp - cyp) / Ry, vx = (-xp - cxp) / Rx, vy = (-yp - cyp) / Ry;
  double th0 = std::atan2(uy, ux);
  double dth = std::atan2(ux * vy - uy * vx, ux * vx + uy * vy);
  if (!sweep && dth > 0.0) dth -= 2.0 * PI;
  if (sweep && dth < 0.0) dth += 2.0 * PI;
  int n = (int)std::ceil(std::fabs(dth) / (0.5 * PI) - 1e-12);
  if (n < 1) n = 1;
  if (n > 4) n = 4;
  auto map = [&](double px, double py, double& X, double& Y) {
    double ex = Rx * px, ey = Ry * py;
    X = cx + cp * ex - sp * ey;
    Y = cy + sp * ex + cp * ey;
  };
  double step = dth / n, hh = 0.5 * step, wv = std::cos(hh);
  double px = (double)x0, py = (double)y0;
  for (int i = 0; i < n; ++i) {
    double a = th0 + step * i, m = a + hh, b = a + step;
    double bx, by, dx, dy;
    map(std::cos(m) / wv, std::sin(m) / wv, bx, by);
    if (i == n - 1) {
      dx = x1;
      dy = y1;
    } else {
      map(std::cos(b), std::sin(b), dx, dy);
    }
    put(i, px, py, bx, by, dx, dy, wv);
    px = dx;
    py = dy;
  }
  return n;
}
