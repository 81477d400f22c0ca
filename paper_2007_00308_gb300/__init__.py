"""GB300 polar stroking: Python binding of libpolarstroke.so.

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels (see ``include/polarstroke.h``).  PyTorch supplies device memory
and streams.  There is no CPU fallback: if the compiled library is missing the
import of any entry point raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpolarstroke.so")

PS_OK, PS_ERR_INVALID, PS_ERR_CAPACITY, PS_ERR_TIMEOUT, PS_ERR_CUDA, PS_ERR_RANGE = 0, -1, -2, -3, -4, -5
PS_PREC_FP32, PS_PREC_MIXED = 0, 1
PS_TESS_ARCLENGTH, PS_TESS_COUNT_ONLY = 1, 2
TAG_LINK_START, TAG_SEGMENT = 1, 2

EXPORTS = ["ps_create", "ps_destroy", "ps_reserve", "ps_max_ribs", "ps_get_status",
           "ps_error_string", "ps_tessellate_strokes", "ps_count_ribs_sync", "ps_arclength_scan",
           "ps_dash", "ps_rasterize_coverage", "ps_profile_enable", "ps_profile_read",
           "ps_profile_slot_name", "ps_raster_stats", "ps_tessellate_strokes_noalloc",
           "ps_tessellate_backward", "ps_set_tuning", "ps_get_tuning", "ps_svg_arc_to_conics",
           "ps_uniform_tessellate", "ps_facet_stats", "ps_dash_capped",
           "ps_rasterize_coverage_exact", "ps_set_pixel_tolerance", "ps_get_pixel_tolerance",
           "ps_check_wait_timeout", "ps_tessellate_links", "ps_add_s_carry",
           "ps_rasterize_coverage_rows", "ps_route_quads"]
PS_PROF_SLOTS = 10
PS_TUNE_EMIT_SLABS, PS_TUNE_SETUP_LINKS, PS_TUNE_BIN_BLOCKS = 0, 1, 2
TUNE_CANDIDATES = {PS_TUNE_EMIT_SLABS: (4, 8, 16, 32, 64), PS_TUNE_SETUP_LINKS: (1, 2, 4),
                   PS_TUNE_BIN_BLOCKS: (0, 2, 4, 8)}
TUNE_NAMES = {PS_TUNE_EMIT_SLABS: "emit_slabs", PS_TUNE_SETUP_LINKS: "setup_links",
              PS_TUNE_BIN_BLOCKS: "bin_blocks"}


class PolarStrokeError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {error_string(code)} ({code})")


class _Segments(ctypes.Structure):
    _fields_ = [("d_type", ctypes.c_void_p), ("d_pts", ctypes.c_void_p), ("d_w", ctypes.c_void_p),
                ("n_seg", ctypes.c_int64)]


class _Paths(ctypes.Structure):
    _fields_ = [("d_seg_off", ctypes.c_void_p), ("d_width", ctypes.c_void_p),
                ("d_join", ctypes.c_void_p), ("d_cap", ctypes.c_void_p),
                ("d_miter", ctypes.c_void_p), ("d_closed", ctypes.c_void_p),
                ("n_path", ctypes.c_int32)]


class _TessOut(ctypes.Structure):
    _fields_ = [("d_rib", ctypes.c_void_p), ("d_tag", ctypes.c_void_p), ("d_s", ctypes.c_void_p),
                ("d_t", ctypes.c_void_p), ("d_link_rib_off", ctypes.c_void_p),
                ("d_path_rib_off", ctypes.c_void_p), ("d_path_len", ctypes.c_void_p),
                ("d_n_rib", ctypes.c_void_p), ("capacity", ctypes.c_int64)]


_lib = None


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        L.ps_create.argtypes = [ctypes.POINTER(ctypes.c_void_p)]
        L.ps_destroy.argtypes = [P]
        L.ps_destroy.restype = None
        L.ps_reserve.argtypes = [P, I64, I64, I64, I64]
        L.ps_max_ribs.argtypes = [I64, I32, ctypes.c_float, ctypes.POINTER(I64)]
        L.ps_get_status.argtypes = [P, ctypes.POINTER(ctypes.c_int)]
        L.ps_error_string.argtypes = [ctypes.c_int]
        L.ps_error_string.restype = ctypes.c_char_p
        L.ps_tessellate_strokes.argtypes = [P, ctypes.POINTER(_Segments), ctypes.POINTER(_Paths),
                                            ctypes.c_float, ctypes.c_int, ctypes.c_uint32,
                                            ctypes.POINTER(_TessOut), P]
        L.ps_count_ribs_sync.argtypes = [P, ctypes.POINTER(_Segments), ctypes.POINTER(_Paths),
                                         ctypes.c_float, ctypes.c_int, ctypes.POINTER(_TessOut), P,
                                         ctypes.POINTER(I64)]
        L.ps_arclength_scan.argtypes = [P, P, P, P, I64, P, P, I32, P]
        L.ps_dash.argtypes = [P, P, P, P, P, I64, P, ctypes.c_int, ctypes.c_float, P, P, P, P, P,
                              I64, P]
        L.ps_rasterize_coverage.argtypes = [P, P, P, P, I64, I32, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, P, P, P]
        L.ps_rasterize_coverage_exact.argtypes = [P, P, P, P, I64, I32, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, P, P, P]
        L.ps_profile_enable.argtypes = [P, ctypes.c_int]
        L.ps_profile_read.argtypes = [P, P]
        L.ps_profile_slot_name.argtypes = [ctypes.c_int]
        L.ps_profile_slot_name.restype = ctypes.c_char_p
        L.ps_raster_stats.argtypes = [P, P, ctypes.c_int]
        L.ps_set_tuning.argtypes = [P, ctypes.c_int, ctypes.c_int]
        F = ctypes.c_float
        L.ps_svg_arc_to_conics.argtypes = [F, F, F, F, F, ctypes.c_int, ctypes.c_int, F, F, P, P]
        L.ps_dash_capped.argtypes = [P, P, P, P, P, I64, P, ctypes.c_int, F, P, I32, F, P, P, P,
                                     P, P, I64, P]
        L.ps_uniform_tessellate.argtypes = [P, ctypes.POINTER(_Segments), ctypes.POINTER(_Paths),
                                            ctypes.POINTER(_TessOut), P, P]
        L.ps_facet_stats.argtypes = [P, P, P, P, I64, P, I64, F, P, P]
        L.ps_get_tuning.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.ps_set_pixel_tolerance.argtypes = [P, ctypes.c_float]
        L.ps_get_pixel_tolerance.argtypes = [P, ctypes.POINTER(ctypes.c_float)]
        L.ps_check_wait_timeout.argtypes = [P, ctypes.c_int, P]
        L.ps_tessellate_backward.argtypes = [P, ctypes.POINTER(_Segments), ctypes.POINTER(_Paths),
                                             ctypes.c_float, ctypes.c_int,
                                             ctypes.POINTER(_TessOut), P, P, P, P, P]
        L.ps_tessellate_links.argtypes = [P, ctypes.POINTER(_Segments), ctypes.POINTER(_Paths),
                                          ctypes.c_float, ctypes.c_int, ctypes.c_uint32, I64, I64,
                                          ctypes.POINTER(_TessOut), P]
        L.ps_add_s_carry.argtypes = [P, P, P, P, I64, I32, ctypes.c_double, P, ctypes.c_int, P]
        L.ps_rasterize_coverage_rows.argtypes = [P, P, P, P, I64, I32, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, P]
        L.ps_route_quads.argtypes = [P, P, P, P, I64, I32, I32, I32, P, P, P, I64, P, P, P]
        L.ps_tessellate_strokes_noalloc.argtypes = [ctypes.POINTER(_Segments),
                                                    ctypes.POINTER(_Paths), ctypes.c_float,
                                                    ctypes.c_int, ctypes.c_uint32,
                                                    ctypes.POINTER(_TessOut), P, P]
        _lib = L
    return _lib


def error_string(code: int) -> str:
    return lib().ps_error_string(int(code)).decode()


def _check(rc, what):
    if rc != PS_OK:
        raise PolarStrokeError(rc, what)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """Owns a ps_context (device workspace + status word) on the current device."""

    def __init__(self):
        h = ctypes.c_void_p()
        _check(lib().ps_create(ctypes.byref(h)), "ps_create")
        self.handle = h

    def close(self):
        if self.handle:
            lib().ps_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reserve(self, n_link=0, n_rib=0, n_tile=0, n_pair=0):
        _check(lib().ps_reserve(self.handle, n_link, n_rib, n_tile, n_pair), "ps_reserve")

    def profile(self, enable: bool = True):
        """Record a CUDA event pair around every library kernel launch."""
        _check(lib().ps_profile_enable(self.handle, int(bool(enable))), "ps_profile_enable")

    def profile_read(self) -> dict:
        """Duration (ms) of the most recent launch of each kernel (waits for it)."""
        ms = (ctypes.c_float * PS_PROF_SLOTS)()
        _check(lib().ps_profile_read(self.handle, ctypes.cast(ms, ctypes.c_void_p)), "ps_profile_read")
        return {lib().ps_profile_slot_name(i).decode(): ms[i] for i in range(PS_PROF_SLOTS)
                if ms[i] >= 0}

    def set_tuning(self, key: int, value: int):
        _check(lib().ps_set_tuning(self.handle, int(key), int(value)), "ps_set_tuning")

    def get_tuning(self, key: int) -> int:
        v = ctypes.c_int(0)
        _check(lib().ps_get_tuning(self.handle, int(key), ctypes.byref(v)), "ps_get_tuning")
        return v.value

    def set_pixel_tolerance(self, tau: float):
        """Pixel-scale boost of the angle step for later tessellations (0: off)."""
        _check(lib().ps_set_pixel_tolerance(self.handle, float(tau)), "ps_set_pixel_tolerance")

    def get_pixel_tolerance(self) -> float:
        v = ctypes.c_float(0.0)
        _check(lib().ps_get_pixel_tolerance(self.handle, ctypes.byref(v)),
               "ps_get_pixel_tolerance")
        return v.value

    def status(self) -> int:
        """Read and clear the device status word (synchronizes)."""
        v = ctypes.c_int(0)
        _check(lib().ps_get_status(self.handle, ctypes.byref(v)), "ps_get_status")
        return v.value


class DeviceBatch:
    """A stroke batch's input arrays on the GPU (torch tensors)."""

    def __init__(self, batch, device="cuda"):
        import torch
        t = lambda a, dt: torch.from_numpy(np.array(a, dtype=dt, order="C")).to(device)
        self.seg_type = t(batch.seg_type, np.uint8)
        self.seg_pts = t(np.asarray(batch.seg_pts, np.float32).reshape(-1), np.float32)
        self.seg_w = t(batch.seg_w, np.float32)
        self.path_seg_off = t(batch.path_seg_off, np.int32)
        self.path_width = t(batch.path_width, np.float32)
        self.path_join = t(batch.path_join, np.uint8)
        self.path_cap = t(batch.path_cap, np.uint8)
        self.path_miter = t(batch.path_miter, np.float32)
        self.path_closed = t(batch.path_closed, np.uint8)
        self.n_seg = int(batch.seg_type.shape[0])
        self.n_path = int(batch.path_width.shape[0])
        self.dtheta = float(np.float32(batch.dtheta))

    @property
    def n_link(self):
        return 2 * self.n_seg + self.n_path

    def _structs(self):
        seg = _Segments(_ptr(self.seg_type).value, _ptr(self.seg_pts).value, _ptr(self.seg_w).value,
                        self.n_seg)
        paths = _Paths(_ptr(self.path_seg_off).value, _ptr(self.path_width).value,
                       _ptr(self.path_join).value, _ptr(self.path_cap).value,
                       _ptr(self.path_miter).value, _ptr(self.path_closed).value, self.n_path)
        return seg, paths


class TessOutput:
    """Caller-owned output buffers of ps_tessellate_strokes."""

    def __init__(self, n_link, n_path, capacity, arclength=True, want_t=False, device="cuda"):
        import torch
        self.capacity = int(capacity)
        self.rib = torch.empty((self.capacity, 4), dtype=torch.float32, device=device)
        self.tag = torch.empty(self.capacity, dtype=torch.int32, device=device)
        self.s = torch.empty(self.capacity, dtype=torch.float32, device=device) if arclength else None
        self.t = torch.empty(self.capacity, dtype=torch.float32, device=device) if want_t else None
        self.link_rib_off = torch.empty(n_link + 1, dtype=torch.int32, device=device)
        self.path_rib_off = torch.empty(n_path + 1, dtype=torch.int32, device=device)
        self.path_len = torch.empty(n_path, dtype=torch.float32, device=device) if arclength else None
        self.n_rib = torch.zeros(1, dtype=torch.int64, device=device)

    def _struct(self):
        p = lambda x: None if x is None else x.data_ptr()
        return _TessOut(p(self.rib), p(self.tag), p(self.s), p(self.t), p(self.link_rib_off),
                        p(self.path_rib_off), p(self.path_len), p(self.n_rib), self.capacity)


RSTAT_NAMES = ("pairs", "span_pixels", "convex_pixels", "two_triangle_pixels", "general_pixels",
               "tile_paths", "tile_passes", "span_rows")


def ps_raster_stats(ctx: Context) -> dict:
    """Work counts of the context's most recent raster call (``RSTAT_NAMES``)."""
    buf = (ctypes.c_int64 * len(RSTAT_NAMES))()
    _check(lib().ps_raster_stats(ctx.handle, ctypes.cast(buf, ctypes.c_void_p), len(RSTAT_NAMES)),
           "ps_raster_stats")
    return dict(zip(RSTAT_NAMES, (int(v) for v in buf)))


def ps_uniform_tessellate(ctx: Context, db: DeviceBatch, fwd: TessOutput, out_rib, stream=None):
    """Uniform parametric ribs with the polar tessellation fwd's per-link counts."""
    seg, paths = db._structs()
    o = fwd._struct()
    _check(lib().ps_uniform_tessellate(ctx.handle, ctypes.byref(seg), ctypes.byref(paths),
                                       ctypes.byref(o), _ptr(out_rib), _stream(stream)),
           "ps_uniform_tessellate")


def ps_facet_stats(ctx: Context, rib, tag, link_rib_off, n_rib, capacity, stats, slack=1e-5,
                   stream=None):
    """Per-link (max, sum, sum of squares, count) of ordinary facet angles into
    stats float32[n_link, 4]."""
    n_link = int(link_rib_off.numel()) - 1
    _check(lib().ps_facet_stats(ctx.handle, _ptr(rib), _ptr(tag), _ptr(link_rib_off), n_link,
                                _ptr(n_rib), int(capacity), float(slack), _ptr(stats),
                                _stream(stream)), "ps_facet_stats")


def svg_arc_to_conics(x0, y0, rx, ry, phi_deg, large_arc, sweep, x1, y1):
    """SVG elliptical arc -> conic segments: (pts float32[n, 4, 2] as A, B, B, D;
    w float32[n]).  Host only."""
    import numpy as np
    pts = np.zeros(32, np.float32)
    w = np.zeros(4, np.float32)
    n = lib().ps_svg_arc_to_conics(float(x0), float(y0), float(rx), float(ry), float(phi_deg),
                                   int(bool(large_arc)), int(bool(sweep)), float(x1), float(y1),
                                   pts.ctypes.data_as(ctypes.c_void_p),
                                   w.ctypes.data_as(ctypes.c_void_p))
    if n < 0:
        _check(n, "ps_svg_arc_to_conics")
    return pts[:8 * n].reshape(n, 4, 2), w[:n]


def ps_max_ribs(n_seg, n_path, dtheta) -> int:
    b = ctypes.c_int64(0)
    _check(lib().ps_max_ribs(int(n_seg), int(n_path), float(dtheta), ctypes.byref(b)), "ps_max_ribs")
    return b.value


def ps_tessellate_strokes(ctx: Context, db: DeviceBatch, out: TessOutput, precision=PS_PREC_FP32,
                          flags=PS_TESS_ARCLENGTH, dtheta=None, stream=None):
    seg, paths = db._structs()
    o = out._struct()
    q = db.dtheta if dtheta is None else float(dtheta)
    rc = lib().ps_tessellate_strokes(ctx.handle, ctypes.byref(seg), ctypes.byref(paths), q,
                                     int(precision), int(flags), ctypes.byref(o), _stream(stream))
    _check(rc, "ps_tessellate_strokes")


def ps_tessellate_links(ctx: Context, db: DeviceBatch, out: TessOutput, link_begin: int,
                        link_end: int, precision=PS_PREC_FP32, flags=PS_TESS_ARCLENGTH,
                        dtheta=None, stream=None):
    """Tessellate the links [link_begin, link_end) of the batch (one rank's
    share); ``out`` is sized for link_end - link_begin links."""
    seg, paths = db._structs()
    o = out._struct()
    q = db.dtheta if dtheta is None else float(dtheta)
    rc = lib().ps_tessellate_links(ctx.handle, ctypes.byref(seg), ctypes.byref(paths), q,
                                   int(precision), int(flags), int(link_begin), int(link_end),
                                   ctypes.byref(o), _stream(stream))
    _check(rc, "ps_tessellate_links")


def ps_add_s_carry(ctx: Context, out: TessOutput, path: int, carry: float, with_len: bool,
                   stream=None):
    """Add a path's arc-length carry to the leading ribs of ``out`` that belong to it."""
    rc = lib().ps_add_s_carry(ctx.handle, _ptr(out.s), _ptr(out.tag), _ptr(out.n_rib),
                              int(out.capacity), int(path), float(carry), _ptr(out.path_len),
                              int(bool(with_len)), _stream(stream))
    _check(rc, "ps_add_s_carry")


def ps_tessellate_strokes_noalloc(db: DeviceBatch, out: TessOutput, status, precision=PS_PREC_FP32,
                                  flags=PS_TESS_ARCLENGTH, dtheta=None, stream=None):
    """Allocation-free tessellation: workspace from the library's fixed device
    array; ``status`` is a caller-owned int32 device tensor for kernel errors.
    Returns the host return code (0, or PS_ERR_* without raising)."""
    seg, paths = db._structs()
    o = out._struct()
    q = db.dtheta if dtheta is None else float(dtheta)
    return lib().ps_tessellate_strokes_noalloc(ctypes.byref(seg), ctypes.byref(paths), q,
                                               int(precision), int(flags), ctypes.byref(o),
                                               _ptr(status), _stream(stream))


def ps_tessellate_backward(ctx: Context, db: DeviceBatch, fwd: TessOutput, grad_rib, grad_s,
                           grad_pts, grad_width, precision=PS_PREC_MIXED, dtheta=None,
                           stream=None):
    """Adjoint of a forward call (which must have requested t)."""
    seg, paths = db._structs()
    o = fwd._struct()
    q = db.dtheta if dtheta is None else float(dtheta)
    rc = lib().ps_tessellate_backward(ctx.handle, ctypes.byref(seg), ctypes.byref(paths), q,
                                      int(precision), ctypes.byref(o), _ptr(grad_rib),
                                      _ptr(grad_s), _ptr(grad_pts), _ptr(grad_width),
                                      _stream(stream))
    _check(rc, "ps_tessellate_backward")


def ps_count_ribs_sync(ctx: Context, db: DeviceBatch, out: TessOutput, precision=PS_PREC_FP32,
                       dtheta=None, stream=None) -> int:
    seg, paths = db._structs()
    o = out._struct()
    n = ctypes.c_int64(0)
    q = db.dtheta if dtheta is None else float(dtheta)
    rc = lib().ps_count_ribs_sync(ctx.handle, ctypes.byref(seg), ctypes.byref(paths), q,
                                  int(precision), ctypes.byref(o), _stream(stream), ctypes.byref(n))
    _check(rc, "ps_count_ribs_sync")
    return n.value


def ps_check_wait_timeout(ctx: Context, which: int, stream=None):
    """Run the bounded-wait self-check (synchronizes); the status word then
    holds PS_ERR_TIMEOUT."""
    _check(lib().ps_check_wait_timeout(ctx.handle, int(which), _stream(stream)),
           "ps_check_wait_timeout")


def ps_arclength_scan(ctx: Context, rib, tag, n_rib, capacity, s, path_len, n_path, stream=None):
    rc = lib().ps_arclength_scan(ctx.handle, _ptr(rib), _ptr(tag), _ptr(n_rib), int(capacity),
                                 _ptr(s), _ptr(path_len), int(n_path), _stream(stream))
    _check(rc, "ps_arclength_scan")


def ps_dash(ctx: Context, rib, s, tag, n_rib, capacity, pattern, offset, out_rib, out_s, out_tag,
            out_src, n_out, out_capacity, stream=None):
    pat = (ctypes.c_float * len(pattern))(*[float(v) for v in pattern])
    rc = lib().ps_dash(ctx.handle, _ptr(rib), _ptr(s), _ptr(tag), _ptr(n_rib), int(capacity),
                       ctypes.cast(pat, ctypes.c_void_p), len(pattern), float(offset), _ptr(out_rib),
                       _ptr(out_s), _ptr(out_tag), _ptr(out_src), _ptr(n_out), int(out_capacity),
                       _stream(stream))
    _check(rc, "ps_dash")


def ps_dash_capped(ctx: Context, rib, s, tag, n_rib, capacity, pattern, offset, path_cap, dtheta,
                   out_rib, out_s, out_tag, out_src, n_out, out_capacity, stream=None):
    """ps_dash with the paths' cap styles (uint8 device tensor path_cap[P]) at
    every dash end inside a path."""
    pat = (ctypes.c_float * len(pattern))(*[float(v) for v in pattern])
    rc = lib().ps_dash_capped(ctx.handle, _ptr(rib), _ptr(s), _ptr(tag), _ptr(n_rib),
                              int(capacity), ctypes.cast(pat, ctypes.c_void_p), len(pattern),
                              float(offset), _ptr(path_cap), int(path_cap.numel()), float(dtheta),
                              _ptr(out_rib), _ptr(out_s), _ptr(out_tag), _ptr(out_src), _ptr(n_out),
                              int(out_capacity), _stream(stream))
    _check(rc, "ps_dash_capped")


def ps_rasterize_coverage(ctx: Context, rib, tag, n_rib, capacity, n_path, width, height, canvas,
                          covered, spp=16, stream=None, exact=False):
    fn = lib().ps_rasterize_coverage_exact if exact else lib().ps_rasterize_coverage
    rc = fn(ctx.handle, _ptr(rib), _ptr(tag), _ptr(n_rib), int(capacity),
                                     int(n_path), int(width), int(height), int(spp), _ptr(canvas),
                                     _ptr(covered), _stream(stream))
    _check(rc, "ps_rasterize_coverage")


def ps_rasterize_coverage_rows(ctx: Context, rib, tag, n_rib, capacity, n_path, width, row_begin,
                               height, canvas, covered, spp=16, stream=None, exact=False):
    """Coverage of picture rows [row_begin, row_begin + height) into ``canvas``
    (height x width) and the per-path samples inside them into ``covered``."""
    rc = lib().ps_rasterize_coverage_rows(ctx.handle, _ptr(rib), _ptr(tag), _ptr(n_rib),
                                          int(capacity), int(n_path), int(width), int(row_begin),
                                          int(height), int(spp), _ptr(canvas), _ptr(covered),
                                          int(bool(exact)), _stream(stream))
    _check(rc, "ps_rasterize_coverage_rows")


def ps_route_quads(ctx: Context, rib, tag, n_rib, capacity, width, height, row_begin, out_rib,
                   out_tag, out_capacity, dest_count, dest_off, stream=None):
    """Group the quads of a rib stream by the owners of the canvas rows they reach
    (``row_begin``: device int32 [n_dest + 1]); see the C header for the layout."""
    rc = lib().ps_route_quads(ctx.handle, _ptr(rib), _ptr(tag), _ptr(n_rib), int(capacity),
                              int(width), int(height), int(row_begin.numel() - 1), _ptr(row_begin),
                              _ptr(out_rib), _ptr(out_tag), int(out_capacity), _ptr(dest_count),
                              _ptr(dest_off), _stream(stream))
    _check(rc, "ps_route_quads")


def tessellate(ctx: Context, db: DeviceBatch, precision=PS_PREC_FP32, arclength=True,
               want_t=False, capacity=None, stream=None) -> TessOutput:
    """Allocate exact-size outputs (one host sync for the count) and tessellate."""
    if capacity is None:
        probe = TessOutput(db.n_link, db.n_path, 0, arclength=False)
        capacity = ps_count_ribs_sync(ctx, db, probe, precision, stream=stream)
    out = TessOutput(db.n_link, db.n_path, max(int(capacity), 1), arclength=arclength, want_t=want_t)
    ps_tessellate_strokes(ctx, db, out, precision,
                          PS_TESS_ARCLENGTH if arclength else 0, stream=stream)
    return out
