/*
 * polarstroke.h — C ABI of the GB300 polar stroking library (libpolarstroke.so).
 *
 * The library implements the data-parallel hot path of polar stroking
 * (M. J. Kilgard, "Polar Stroking: New Theory and Methods for Stroking
 * Paths", ACM TOG 39(4), 2020) as sm_103a CUDA kernels:
 *
 *   ps_tessellate_strokes   per-link intervals and step counts (Sec. 3.3-3.4,
 *                           Eq. 4-6, 12-13), rib offsets, the t(psi) solve
 *                           (Eq. 11), rib vertices (Eq. 14-17), joins and caps
 *                           (Sec. 4.3) and cumulative arc length (Eq. 18, Sec. 5.1)
 *   ps_arclength_scan       cumulative arc length of a rib stream (Eq. 18)
 *   ps_dash                 dashing by cumulative arc length (Sec. 5.2)
 *   ps_rasterize_coverage   16-sample coverage of the stroked quads, binned into
 *                           16x16-pixel tiles (Sec. 4.1: quads drawn as two
 *                           triangles; Sec. 3.3.6: per-path union)
 *   ps_rasterize_coverage_rows, ps_route_quads   the same on a window of rows,
 *                           and the routing of quads to the owners of a canvas
 *                           split by rows over several GPUs
 *
 * Conventions shared by every call
 *   - Pointers named d_* are DEVICE pointers owned by the caller; h_* are host
 *     pointers.  The library never frees caller memory.
 *   - Every call is asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL = legacy default stream) and never synchronizes the host, except
 *     ps_get_status and ps_count_ribs_sync, which say so.
 *   - Sizes that depend on the data (rib count, bin entries) live in device
 *     memory; kernels read them there, so a sequence of calls can be captured
 *     in a CUDA graph once the context's workspace has been reserved (the first
 *     call with given sizes may cudaMalloc; capture the second).
 *   - Return codes: PS_OK or a negative PS_ERR_* for argument errors detected on
 *     the host.  Errors found by kernels (capacity exceeded, a bounded wait that
 *     gave up, out-of-range coordinates) are recorded in the context's device
 *     status word, read by ps_get_status.
 *
 * Input layout (structure of arrays)
 *   segment i:  d_seg_type[i]   uint8   PS_LINE / PS_QUAD / PS_CUBIC / PS_CONIC
 *               d_seg_pts[8i..8i+7]  float32  A.x A.y B.x B.y C.x C.y D.x D.y
 *                           (Table 1's control points; quadratic and conic use
 *                            A, B, D; a line uses A, D)
 *               d_seg_w[i]      float32 conic weight w_B (must be > -1)
 *   path p:     segments [d_path_seg_off[p], d_path_seg_off[p+1]) (non-decreasing,
 *               d_path_seg_off[0] = 0), d_path_width[p] (> 0), d_path_join[p],
 *               d_path_cap[p], d_path_miter[p] (miter limit, ratio of miter length
 *               to stroke width), d_path_closed[p] (0/1)
 *
 * Link order: path p owns links [2*seg_off[p] + p, 2*seg_off[p+1] + p + 1) in the
 * order start cap, segment 0, join 0/1, segment 1, ..., segment n-1, end cap (an
 * open path) or closing join (a closed path) (Sec. 4.4: a path is divided into
 * links, one per segment, join and cap).  Links with no ribs are empty.
 *
 * Output layout
 *   rib r:  d_rib[4r..4r+3] = N.x N.y P.x P.y (Eq. 16-17; N = g - r_N n,
 *           P = g + r_P n with n = <-sin psi, cos psi>)
 *           d_tag[r] = (path << 2) | (is segment link << 1) | (first rib of link)
 *           d_s[r] cumulative arc length of the path at the rib (Eq. 18)
 *   quad:   ribs r-1, r with d_tag[r] & 1 == 0 form one quad (Sec. 4.1)
 */
#ifndef POLARSTROKE_H
#define POLARSTROKE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return / status codes ----------------------------------------------- */
#define PS_OK 0
#define PS_ERR_INVALID (-1)   /* bad argument (null pointer, bad size, bad enum) */
#define PS_ERR_CAPACITY (-2)  /* an output or workspace capacity was too small */
#define PS_ERR_TIMEOUT (-3)   /* a bounded inter-CTA wait gave up */
#define PS_ERR_CUDA (-4)      /* a CUDA runtime call failed */
#define PS_ERR_RANGE (-5)     /* a vertex outside +-2^21 px reached the rasterizer */

/* ---- enums ---------------------------------------------------------------- */
#define PS_LINE 0
#define PS_QUAD 1
#define PS_CUBIC 2
#define PS_CONIC 3

#define PS_JOIN_NONE 0
#define PS_JOIN_BEVEL 1
#define PS_JOIN_MITER 2          /* miter; reverts to bevel above the limit */
#define PS_JOIN_MITER_TRUNCATE 3 /* miter clipped at limit * w/2 */
#define PS_JOIN_ROUND 4
#define PS_JOIN_TRIANGLE 5

#define PS_CAP_BUTT 0
#define PS_CAP_SQUARE 1
#define PS_CAP_ROUND 2
#define PS_CAP_TRIANGLE 3

#define PS_PREC_FP32 0  /* all-FP32 arithmetic */
#define PS_PREC_MIXED 1 /* FP32 pipe: angles, normals, t and vertices as
                           double-float pairs (each vertex rounded once), FP64
                           only in the inflection discriminant and near-double-root
                           t(psi) solves */

/* ps_tessellate_strokes flags */
#define PS_TESS_ARCLENGTH 1u  /* also write d_s and d_path_len */
#define PS_TESS_COUNT_ONLY 2u /* only per-link offsets, path offsets and *d_n_rib */

#define PS_TAG_LINK_START 1u
#define PS_TAG_SEGMENT 2u

typedef struct ps_context ps_context;

typedef struct {
  const uint8_t* d_type; /* [n_seg] */
  const float* d_pts;    /* [n_seg * 8] */
  const float* d_w;      /* [n_seg] */
  int64_t n_seg;
} ps_segments;

typedef struct {
  const int32_t* d_seg_off; /* [n_path + 1] */
  const float* d_width;     /* [n_path] */
  const uint8_t* d_join;    /* [n_path] */
  const uint8_t* d_cap;     /* [n_path] */
  const float* d_miter;     /* [n_path] */
  const uint8_t* d_closed;  /* [n_path] */
  int32_t n_path;
} ps_paths;

typedef struct {
  float* d_rib;             /* [capacity * 4] */
  uint32_t* d_tag;          /* [capacity] */
  float* d_s;               /* [capacity]; NULL unless PS_TESS_ARCLENGTH */
  float* d_t;               /* [capacity]; optional t(j) per rib, may be NULL */
  int32_t* d_link_rib_off;  /* [n_link + 1], n_link = 2 n_seg + n_path */
  int32_t* d_path_rib_off;  /* [n_path + 1] */
  float* d_path_len;        /* [n_path]; NULL unless PS_TESS_ARCLENGTH */
  int64_t* d_n_rib;         /* [1]: total ribs R (written even when R > capacity) */
  int64_t capacity;         /* rib capacity of d_rib / d_tag / d_s / d_t */
} ps_tess_out;

/* ---- context ---------------------------------------------------------------
 * A context owns device workspace (tile states for the single-pass scans, the
 * per-link interval records, raster bins) and a device status word.  It is
 * bound to the device that is current at ps_create.  Not thread-safe: use one
 * context per host thread / stream. */
int ps_create(ps_context** ctx);
void ps_destroy(ps_context* ctx);

/* Reserve workspace for up to n_link links, n_rib ribs, n_tile raster tiles
 * and n_pair raster bin entries (any may be 0 = keep).  Allocates with
 * cudaMalloc (synchronous); call before capturing a graph. */
int ps_reserve(ps_context* ctx, int64_t n_link, int64_t n_rib, int64_t n_tile, int64_t n_pair);

/* Host-only static bound on the rib count of n_seg segments in n_path paths
 * at step dtheta (radians): a segment turns < 2 pi in at most 6 intervals
 * (Sec. 3.3.5), a join or cap pivots at most pi (Sec. 4.3). */
int ps_max_ribs(int64_t n_seg, int32_t n_path, float dtheta, int64_t* h_bound);

/* Read and clear the device status word.  SYNCHRONIZES the context's last
 * stream.  *h_status receives PS_OK or the first PS_ERR_* a kernel recorded. */
int ps_get_status(ps_context* ctx, int* h_status);

const char* ps_error_string(int code);

/* Failure-detection self-check of the bounded inter-CTA wait (the paper has
 * no counterpart).  Every single-pass scan of the library waits for its
 * predecessor tiles (decoupled look-back) for at most 2^22 polls, then records
 * PS_ERR_TIMEOUT in the status word and carries on, so that a lost tile ends
 * the launch with an error instead of a hang.  This call launches one warp on
 * `stream` that waits, through that same wait, on a predecessor tile whose
 * flag nothing ever sets: which = 0 takes the int64 sum (rib offsets, raster
 * tile offsets, dash output offsets), which = 1 the segmented double-float
 * sum (arc length).  The wait gives up after a second or a few and the kernel returns;
 * the context stays usable.  Uses a 256-byte scratch allocation of its own.
 * SYNCHRONIZES.  Returns PS_OK once the kernel has finished, PS_ERR_INVALID
 * for a null context or another `which`; ps_get_status then reads
 * PS_ERR_TIMEOUT. */
int ps_check_wait_timeout(ps_context* ctx, int which, void* stream);

/* ---- the hot path ------------------------------------------------------------ */

/* Tessellate every path (Sec. 4.4's complete algorithm, all links in parallel).
 *   dtheta     q, the tangent-angle step in radians (Sec. 4.2), > 0
 *   precision  PS_PREC_FP32 or PS_PREC_MIXED
 *   flags      PS_TESS_ARCLENGTH, PS_TESS_COUNT_ONLY
 * Writes out->d_link_rib_off, d_path_rib_off, *d_n_rib, and (unless COUNT_ONLY)
 * the first min(R, capacity) ribs.  R > capacity records PS_ERR_CAPACITY.
 * Ribs of path p are [path_rib_off[p], path_rib_off[p+1]); ribs of link l are
 * [link_rib_off[l], link_rib_off[l+1]).  Offsets are int32: R < 2^31.
 * n_path = 0 with n_seg = 0 is an empty batch: R = 0, link_rib_off[0] =
 * path_rib_off[0] = 0, no kernel runs and the other pointers may be NULL;
 * n_path = 0 with segments, or n_path < 0, is PS_ERR_INVALID.  (The same
 * holds for the allocation-free variant; the adjoint and the uniform
 * comparison return PS_OK at once on an empty batch.) */
int ps_tessellate_strokes(ps_context* ctx, const ps_segments* seg, const ps_paths* paths,
                          float dtheta, int precision, uint32_t flags, ps_tess_out* out,
                          void* stream);

/* Tessellate the links [link_begin, link_end) of the batch only: one rank's
 * share when a batch (or a single long path) is split over several GPUs by
 * links (Sec. 4.4: links are independent; Eq. 13 and Eq. 18: offsets and arc
 * length are prefix sums, fixed up afterwards from the ranks' totals).  Links
 * are numbered over the batch as in ps_tessellate_strokes (path p's links are
 * 2 seg_off[p] + p ... 2 seg_off[p+1] + p).  Arguments as ps_tessellate_strokes,
 * with the outputs local to the range:
 *   out->d_link_rib_off  [link_end - link_begin + 1] rib offsets from 0;
 *   out->d_path_rib_off  [n_path + 1]: for a path whose first link lies in the
 *                        range its first rib, -1 otherwise (the call fills it),
 *                        and for the path whose last link is the range's last
 *                        link its end;
 *   ribs, tags (global path indices), t, and s: s restarts at 0 at the start of
 *                        every path that begins in the range, and for the path
 *                        running into the range (begun on an earlier range) at
 *                        the range's first rib -- add its carry with
 *                        ps_add_s_carry;
 *   path_len             for the paths that end in the range (the running-in
 *                        one: its length within the range).
 * 0 <= link_begin < link_end <= 2 n_seg + n_path, else PS_ERR_INVALID. */
int ps_tessellate_links(ps_context* ctx, const ps_segments* seg, const ps_paths* paths,
                        float dtheta, int precision, uint32_t flags, int64_t link_begin,
                        int64_t link_end, ps_tess_out* out, void* stream);

/* s[r] += carry for the leading ribs of a rib stream whose tag's path is
 * `path` (the path that runs into a link range), and path_len[path] += carry
 * when with_len is set (the path ends in the range).  carry is the path's
 * length on the ranges before (double, added as a double-float pair).
 * Asynchronous on `stream`.  PS_ERR_INVALID on null pointers, capacity < 0 or
 * path < 0. */
int ps_add_s_carry(ps_context* ctx, float* d_s, const uint32_t* d_tag, const int64_t* d_n_rib,
                   int64_t capacity, int32_t path, double carry, float* d_path_len, int with_len,
                   void* stream);

/* Allocation-free variant of ps_tessellate_strokes (the paper has no
 * counterpart; this is an interface for callers that cannot allocate device
 * memory when they stroke -- for example code running under an allocator that
 * owns the device's memory budget, or code that must not block on, or fail
 * in, an allocation partway through its work).
 * Same arguments, outputs and semantics as ps_tessellate_strokes, except:
 *   - no context: the workspace is a fixed array inside the library image
 *     (about 4.0 MB on every device that loads the library, kept until exit);
 *     the call makes no cudaMalloc, cudaFree or other allocating call;
 *   - d_status: caller-owned device int32 that kernels set to the first
 *     PS_ERR_* they meet (the caller zeroes it and reads it back);
 *   - limits: at most 16384 links (2 n_seg + n_path) and, with
 *     PS_TESS_ARCLENGTH, a rib capacity of at most 4194304; larger problems
 *     return PS_ERR_CAPACITY before any launch;
 *   - PS_TESS_ARCLENGTH with d_s == NULL returns PS_ERR_INVALID (the
 *     regular call then skips arc length and writes no d_s);
 *   - the first call on a device looks up the array's device address (with
 *     that device current); make that first call outside any stream capture;
 *   - every call uses the same array, which keeps the previous call's
 *     contents (the call clears what must start at zero): calls that may run
 *     at the same time on the GPU -- on different streams, or different host
 *     threads -- race and must be serialized by the caller. */
int ps_tessellate_strokes_noalloc(const ps_segments* seg, const ps_paths* paths, float dtheta,
                                  int precision, uint32_t flags, ps_tess_out* out,
                                  int32_t* d_status, void* stream);

/* Adjoint of ps_tessellate_strokes at the forward pass's fixed step counts.
 * Given dL/d(rib vertices) (d_grad_rib, [R*4]) and optionally dL/ds
 * (d_grad_s, [R]), writes dL/d(control points) (d_grad_pts, [n_seg*8], zeroed
 * by the call; a quadratic's or conic's middle point gets its gradient in the B
 * slot) and dL/d(stroke width) (d_grad_width, [n_path]).  `fwd` is the forward
 * call's output with d_t filled (the forward must request t).  Each rib's t(j)
 * solves Eq. 11 and is differentiated implicitly; normal angles interpolate
 * their interval's boundary angles; arc length is the chord sum of Eq. 18.
 * Not followed (gradient contribution omitted): conic weights, miter tips
 * (their vertices move with the join point only), collinear pivots.  The
 * paper has no differentiation; this is the library's extension. */
int ps_tessellate_backward(ps_context* ctx, const ps_segments* seg, const ps_paths* paths,
                           float dtheta, int precision, const ps_tess_out* fwd,
                           const float* d_grad_rib, const float* d_grad_s, float* d_grad_pts,
                           float* d_grad_width, void* stream);

/* Convenience: run the count phase and return R on the host.  SYNCHRONIZES. */
int ps_count_ribs_sync(ps_context* ctx, const ps_segments* seg, const ps_paths* paths,
                       float dtheta, int precision, ps_tess_out* out, void* stream,
                       int64_t* h_n_rib);

/* Cumulative arc length of an existing rib stream (Eq. 18): the centreline
 * point of a segment rib is its midpoint (N + P)/2 (exact when r_N = r_P, as in
 * segment links); joins and caps add 0; s restarts at 0 at every path's first
 * rib.  d_n_rib: device rib count; capacity bounds it.  d_path_len may be NULL. */
int ps_arclength_scan(ps_context* ctx, const float* d_rib, const uint32_t* d_tag,
                      const int64_t* d_n_rib, int64_t capacity, float* d_s,
                      float* d_path_len, int32_t n_path, void* stream);

/* Dash a rib stream by its cumulative arc length (Sec. 5.2).  h_pattern holds
 * n_pattern (1..32) non-negative lengths, on/off alternating (an odd count is
 * repeated twice), restarting at s = 0 of every path, shifted by `offset`.
 * Each quad is clipped to the "on" stretches [a, b) by interpolating both rib
 * vertices; every piece is emitted as an independent 2-rib strip; a zero-length
 * quad (join, cap, cusp pivot) is kept whole iff its s is "on".
 * Outputs: d_out_rib[4 cap], d_out_s[cap], d_out_tag[cap], d_out_src[cap]
 * (index of the source quad's end rib, may be NULL), *d_n_out (device).  More
 * than out_capacity ribs records PS_ERR_CAPACITY. */
int ps_dash(ps_context* ctx, const float* d_rib, const float* d_s, const uint32_t* d_tag,
            const int64_t* d_n_rib, int64_t capacity, const float* h_pattern, int n_pattern,
            float offset, float* d_out_rib, float* d_out_s, uint32_t* d_out_tag,
            int32_t* d_out_src, int64_t* d_n_out, int64_t out_capacity, void* stream);

/* ps_dash with capped dash ends (Sec. 5.2; the paper leaves their form open):
 * every on-stretch also gets its path's cap style (d_path_cap[p], PS_CAP_*;
 * butt adds nothing) at its ends inside the path -- a start cap where the
 * stretch begins at 0 < a inside a segment quad [s_{r-1}, s_r), an end cap
 * where it ends at b in (s_{r-1}, s_r].  A cap is the path cap of Sec. 4.3.5
 * (pivot through +pi, outer side N, inner radius 0; round caps step by at most
 * dtheta) about the boundary rib: centre the rib's midpoint, radius half its
 * length, tangent the rib turned clockwise.  Its J+1 ribs form a strip of their
 * own (link-start tag on the first, segment bit clear) at the boundary's s,
 * written right before the stretch's first piece (start cap) or right after its
 * last piece (end cap).  Counts, offsets and errors as ps_dash; the output
 * count includes the cap ribs. */
int ps_dash_capped(ps_context* ctx, const float* d_rib, const float* d_s, const uint32_t* d_tag,
                   const int64_t* d_n_rib, int64_t capacity, const float* h_pattern, int n_pattern,
                   float offset, const uint8_t* d_path_cap, int32_t n_path, float dtheta,
                   float* d_out_rib, float* d_out_s, uint32_t* d_out_tag, int32_t* d_out_src,
                   int64_t* d_n_out, int64_t out_capacity, void* stream);

/* Coverage of the quads of a rib stream on a width x height canvas with 16
 * samples per pixel (spp must be 16).  Vertices snap to round-half-even(v*256);
 * sample k of pixel (x, y) sits at (x + (16k+8)/256, y + (16((5k) mod 16)+8)/256);
 * a sample is covered by a triangle iff its three edge functions are >= 0 with
 * the triangle oriented counter-clockwise (zero-area triangles cover nothing);
 * quad (r-1, r) is the triangles (N_{r-1}, P_{r-1}, P_r), (N_{r-1}, P_r, N_r).
 *   d_canvas[y*width + x]   uint16 sample mask, OR over all paths (overwritten)
 *   d_covered[p]            uint64 samples covered by path p (union of its
 *                           quads; overwritten)
 * Quads with a vertex beyond +-2^21 px are skipped and record PS_ERR_RANGE.  A
 * 16x16-pixel tile met by more than 1024 distinct paths records
 * PS_ERR_CAPACITY (its coverage is then incomplete).  Returns PS_ERR_INVALID
 * (before any launch) for a NULL pointer, spp != 16, a non-positive size, a
 * width or height of 2^21 px or more, or more than 2^26 tiles (the binning
 * words hold a tile index in 26 bits). */
int ps_rasterize_coverage(ps_context* ctx, const float* d_rib, const uint32_t* d_tag,
                          const int64_t* d_n_rib, int64_t capacity, int32_t n_path,
                          int width, int height, int spp, uint16_t* d_canvas,
                          uint64_t* d_covered, void* stream);

/* ps_rasterize_coverage with every quad filled as its polygon N_{r-1} ->
 * P_{r-1} -> P_r -> N_r -> N_{r-1} instead of as two triangles (Sec. 4.1:
 * quads rasterized as quads, bow-tie quads as bow-ties; Sec. 7: two
 * overlapping triangles exaggerate a bow-tie's coverage).  A sample is covered
 * by a quad iff the ray from it towards +x crosses an odd number of the
 * polygon's edges, edge a -> b being crossed iff a.y <= y < b.y with the sample
 * strictly left of a -> b, or b.y <= y < a.y with it strictly right (integer
 * edge functions on the same snapped vertices).  Arguments, union and counts as
 * ps_rasterize_coverage. */
int ps_rasterize_coverage_exact(ps_context* ctx, const float* d_rib, const uint32_t* d_tag,
                                const int64_t* d_n_rib, int64_t capacity, int32_t n_path,
                                int width, int height, int spp, uint16_t* d_canvas,
                                uint64_t* d_covered, void* stream);

/* Coverage of the pixel rows [row_begin, row_begin + height) of a picture
 * (a window of a canvas split by tile rows over several GPUs; row_begin >= 0 a
 * multiple of 16, the tile size).  Quads are snapped in picture coordinates
 * (Sec. 4.1, as ps_rasterize_coverage) and moved to the window's origin after
 * snapping, in 1/256-px integers, so every pixel of the window gets the same
 * mask as in ps_rasterize_coverage of the whole picture; quads outside the
 * window are clipped away.
 *   d_canvas[y*width + x]   uint16 mask of picture pixel (x, row_begin + y),
 *                           height x width (overwritten)
 *   d_covered[p]            uint64 samples of path p inside the window
 *                           (overwritten); summed over windows that partition
 *                           the picture's rows they equal ps_rasterize_coverage's
 * exact != 0 selects the crossing rule of ps_rasterize_coverage_exact.
 * Returns PS_ERR_INVALID for a negative or unaligned row_begin; other arguments
 * and errors as ps_rasterize_coverage. */
int ps_rasterize_coverage_rows(ps_context* ctx, const float* d_rib, const uint32_t* d_tag,
                               const int64_t* d_n_rib, int64_t capacity, int32_t n_path,
                               int width, int row_begin, int height, int spp,
                               uint16_t* d_canvas, uint64_t* d_covered, int exact, void* stream);

/* Routes the quads of a rib stream to the owners of a canvas split by pixel
 * rows (the raster half of splitting one batch over several GPUs; Sec. 4.4
 * makes links independent, Sec. 3.3.6 makes coverage a per-path union, so the
 * owner of a row must see every quad of every path that reaches it).
 * Destination d owns rows [row_begin[d], row_begin[d+1]) of a width x height
 * canvas; d_row_begin is a DEVICE int32 array of n_dest + 1 non-decreasing
 * multiples of 16 (row_begin[0] = 0, row_begin[n_dest] = height; 1 <= n_dest
 * <= 4096; an empty window receives nothing).  Quad (r-1, r) (tag r without
 * PS_TAG_LINK_START) goes to every owner of a pixel row that its snapped
 * bounding box reaches, in the same rows the binning would test it against.
 * Output, grouped by destination (block d = quads [dest_off[d], dest_off[d+1])):
 *   d_out_rib[2i], d_out_rib[2i+1]   float4 x 2: ribs r-1 and r of quad i
 *                                     (2 * out_capacity float4 of room)
 *   d_out_tag[2i], d_out_tag[2i+1]   tag r with PS_TAG_LINK_START set, tag r
 *                                     (2 * out_capacity uint32 of room)
 *   d_dest_count[d]                  int64 quads of destination d
 *   d_dest_off[d]                    int64 exclusive prefix, n_dest + 1 entries
 * so that a destination's block, and any concatenation of blocks from several
 * ranks, is itself a rib stream whose quads are exactly the routed ones; it
 * goes to ps_rasterize_coverage_rows with the destination's window.  Counts
 * and offsets are written even when the quads do not fit: the device status
 * then records PS_ERR_CAPACITY and only quads below out_capacity are written.
 * With d_out_rib and d_out_tag NULL and out_capacity 0 the call only counts
 * (d_dest_count, d_dest_off), so that the caller can size the output.
 * Quads with a vertex beyond +-2^21 px record PS_ERR_RANGE and go nowhere. */
int ps_route_quads(ps_context* ctx, const float* d_rib, const uint32_t* d_tag,
                   const int64_t* d_n_rib, int64_t capacity, int32_t width, int32_t height,
                   int32_t n_dest, const int32_t* d_row_begin, float* d_out_rib,
                   uint32_t* d_out_tag, int64_t out_capacity, int64_t* d_dest_count,
                   int64_t* d_dest_off, void* stream);

/* ---- kernel timing (measurement hooks) ------------------------------------------
 * With profiling enabled the library records a CUDA event pair around each of its
 * kernel launches on the launching stream (as external event-record nodes when
 * the stream is being captured into a graph, so graph replays are timed too).
 * Slot s names one kernel (ps_profile_slot_name).  ps_profile_read waits for the
 * events and returns, per slot, the duration in ms of the most recent launch,
 * or -1 if the slot has not been recorded since profiling was enabled. */
#define PS_PROF_SLOTS 10
int ps_profile_enable(ps_context* ctx, int enable);
int ps_profile_read(ps_context* ctx, float* h_ms /* [PS_PROF_SLOTS] */);
const char* ps_profile_slot_name(int slot);

/* Uniform parametric comparison (Sec. 8.1).  For every segment link of the
 * polar tessellation fwd (made from the same seg and paths), writes the same
 * number of ribs N+1 at uniform parameters t_j = j/N: g(t_j) -+ (w/2) n(t_j)
 * with n the unit left normal of g'(t_j) (Eq. 1 sampled uniformly; at an exact
 * cusp the direction of g''(t) stands in for the tangent).  Join and cap links
 * keep the polar ribs, so fwd's tags, offsets and counts describe the output
 * too (equal quad counts, as the paper compares).
 *   d_rib_out  float4[fwd->capacity] (N.x, N.y, P.x, P.y), caller-owned.
 * Returns PS_ERR_INVALID for null or inconsistent arguments. */
int ps_uniform_tessellate(ps_context* ctx, const ps_segments* seg, const ps_paths* paths,
                          const ps_tess_out* fwd, float* d_rib_out, void* stream);

/* Facet-angle statistics of a rib stream (Sec. 4.2, 8.1).  A facet is where one
 * quad's boundary edge meets the next: at every interior rib of a segment link,
 * on the N and P sides, the angle in [0, pi] between the edges before and after
 * it.  Only ordinary facets count: each of the two edges points between the
 * tangents of its end ribs (a rib P - N turned clockwise) within `slack`
 * (cross products of unit vectors; ~1e-5 suits FP32 ribs), which leaves out
 * the facets next to offset cusps; ribs of zero length use the centreline.
 *   d_stats[4 l .. 4 l + 3] = max, sum, sum of squares, count of the ordinary
 *   facet angles (radians) of link l; zeros for links without any.
 * The ribs' link structure comes from d_tag and d_link_rib_off[n_link + 1]. */
int ps_facet_stats(ps_context* ctx, const float* d_rib, const uint32_t* d_tag,
                   const int32_t* d_link_rib_off, int64_t n_link, const int64_t* d_n_rib,
                   int64_t capacity, float slack, float* d_stats, void* stream);

/* SVG elliptical arc -> conic segments (host function, no device work).
 * The arc runs from (x0, y0) to (x1, y1) on the ellipse with radii rx, ry whose
 * x axis is rotated by phi_deg, the large-arc and sweep flags choosing among the
 * four candidate arcs as in SVG 1.1 (radii too small for the chord are scaled
 * up; negative radii count as their absolute values).  The paper takes arcs in
 * through its rational conic form (Table 1): each output piece spans at most 90
 * degrees of the ellipse and is written as a PS_CONIC segment, h_pts[8 i .. 8 i
 * + 7] = A, B, B, D (the layout of d_pts) and h_w[i] = w_B.  The first A and
 * the last D are the given end points exactly.
 * Returns the number of pieces (0 when the end points coincide, 1 flat piece
 * when a radius is zero, else 1..4), or PS_ERR_INVALID (null pointers,
 * non-finite input).  h_pts holds 32 floats, h_w 4. */
int ps_svg_arc_to_conics(float x0, float y0, float rx, float ry, float phi_deg, int large_arc,
                         int sweep, float x1, float y1, float* h_pts, float* h_w);

/* Launch parameters of a context, for autotuning.  They change how work is
 * split over threads, never what is computed.
 *   PS_TUNE_EMIT_SLABS   ribs per warp task in the rib kernel, in slabs of 32:
 *                        4, 8, 16, 32 (default) or 64
 *   PS_TUNE_SETUP_LINKS  links per thread in the link-setup kernel: 1, 2
 *                        (default) or 4
 *   PS_TUNE_BIN_BLOCKS   CTAs per SM of the two binning passes: 0 (default: as
 *                        many as fit) or 1..16
 * ps_set_tuning returns PS_ERR_INVALID for an unknown key or value; the
 * allocation-free entry point always uses the defaults. */
enum {
  PS_TUNE_EMIT_SLABS = 0,
  PS_TUNE_SETUP_LINKS = 1,
  PS_TUNE_BIN_BLOCKS = 2,
  PS_TUNE_COUNT = 3
};
int ps_set_tuning(ps_context* ctx, int key, int value);
int ps_get_tuning(ps_context* ctx, int key, int* value);

/* Pixel-scale boost of the angle step (Sec. 7 suggests boosting q for
 * segments, joins and caps near the scale of pixels; the rule is this
 * library's).  With tau > 0 (px) every later tessellation, count and adjoint
 * call of the context steps each link by its own q_link >= dtheta:
 *   round join / round cap:  max(dtheta, 2 acos(1 - tau/r)), pi once tau >= r
 *                            (r = width/2; the largest step whose arc-to-chord
 *                            gap on the circular boundary is <= tau);
 *   segment:                 max(dtheta, min(2 atan(tau/L_g), sqrt(pi tau/(2r)),
 *                            pi/2)), L_g the length of its control polygon
 *                            (keeps every step's boundary edge within tau of
 *                            the offset curve on sides that do not fold);
 *   conic with w_B <= 0, other join and cap styles:  dtheta.
 * Counts only ever decrease, so ps_max_ribs stays a bound.  tau = 0 (the
 * default) turns the boost off; the allocation-free entry point never applies
 * it.  PS_ERR_INVALID for tau < 0 or not finite. */
int ps_set_pixel_tolerance(ps_context* ctx, float tau);
int ps_get_pixel_tolerance(ps_context* ctx, float* tau);

/* Work counts of the context's most recent ps_rasterize_coverage call, read from
 * its device workspace into h_counts[0 .. n_counts-1] (entries past
 * PS_RSTAT_COUNT are zeroed):
 *   PS_RSTAT_PAIRS          (quad, tile) bin entries
 *   PS_RSTAT_SPAN_PIXELS    pixels of the per-row spans the coverage kernel
 *                           tested (16 samples each), the sum of the next three
 *   PS_RSTAT_CONVEX_PIXELS  ... of quads that are convex (or one triangle)
 *   PS_RSTAT_TWO_TRI_PIXELS ... of non-convex quads (two triangles)
 *   PS_RSTAT_GENERAL_PIXELS ... of quads with an edge longer than 1024 px
 *   PS_RSTAT_TILE_PATHS     sum over tiles of the distinct paths met there
 *   PS_RSTAT_TILE_PASSES    sum over tiles with bin entries of the passes over
 *                           the tile's bin (one per 96 distinct paths)
 *   PS_RSTAT_SPAN_ROWS      (bin entry, pixel row) pairs whose span was computed
 * SYNCHRONIZES. */
enum {
  PS_RSTAT_PAIRS = 0,
  PS_RSTAT_SPAN_PIXELS = 1,
  PS_RSTAT_CONVEX_PIXELS = 2,
  PS_RSTAT_TWO_TRI_PIXELS = 3,
  PS_RSTAT_GENERAL_PIXELS = 4,
  PS_RSTAT_TILE_PATHS = 5,
  PS_RSTAT_TILE_PASSES = 6,
  PS_RSTAT_SPAN_ROWS = 7,
  PS_RSTAT_COUNT = 8
};
int ps_raster_stats(ps_context* ctx, int64_t* h_counts, int n_counts);

#ifdef __cplusplus
}
#endif
#endif /* POLARSTROKE_H */
