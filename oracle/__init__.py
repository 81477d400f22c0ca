"""FP64 CPU oracle for polar stroking — TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package.  It shares no code with the CUDA
library (``paper_2007_00308_gb300``) and imports nothing from it; batches are
taken by attribute (any object with the input arrays of the library's layout).

The C source ``polar_oracle.c`` restates the paper step by step in FP64; this
module only compiles it with gcc and marshals numpy arrays.

Parity status per function (see the tests under ``tests/test_oracle_*.py``):
  tessellate       pinned (closed forms: line, circle-arc conic, parabola, cusp
                   structure, per-step turn, total turning, chord error, joins,
                   caps; coverage against brute force; negative-weight conics
                   as complementary arcs); tau > 0 pinned (closed-form
                   sagittas and minimal counts of joins and caps, quarter-circle
                   counts, densely sampled offset curves of small cubics)
  dash             pinned (straight line against the analytic dash pieces)
  dash_capped      pinned (straight line: caps against the analytic cap shapes;
                   coverage of a capped dashed line against brute force)
  raster           pinned (axis-aligned rectangles and triangles against a
                   point-in-polygon count written with a different predicate);
                   exact=True pinned (convex quads equal the two-triangle raster
                   off the boundary, bow-tie lobes against rational geometry)
  centreline_distance  pinned (distance to a line and a circle in closed form)
  uniform_ribs     pinned (parabola chords against the midpoint tangent, closed form)
  facet_angles     pinned (circle arc: every facet equals the polar step)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "polar_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

FRAGILE64 = 1
FRAGILE32 = 2
TAG_LINK_START = 1
TAG_SEGMENT = 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-adds)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I64, I32, D = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
            _lib.orc_tessellate.argtypes = [I64, P, P, P, I32, P, P, P, P, P, P, D, D, P, P, I64, P,
                                            P, P, P, P, P, P, P]
            _lib.orc_tessellate.restype = ctypes.c_int
            _lib.orc_tessellate_f64.argtypes = [I64, P, P, P, I32, P, P, P, P, P, P, D, D, P, P,
                                                I64, P, P, P, P, P, P, P, P]
            _lib.orc_tessellate_f64.restype = ctypes.c_int
            _lib.orc_segment_intervals.argtypes = [ctypes.c_int, P, ctypes.c_float, D, P, P, P, P, P, P]
            _lib.orc_segment_intervals.restype = ctypes.c_int
            _lib.orc_segment_probe.argtypes = [ctypes.c_int, P, ctypes.c_float, ctypes.c_int, ctypes.c_int, P, P]
            _lib.orc_segment_probe.restype = None
            _lib.orc_dash.argtypes = [I64, P, P, P, P, ctypes.c_int, D, I64, P, P, P, P, P]
            _lib.orc_dash.restype = ctypes.c_int
            _lib.orc_raster.argtypes = [I64, P, P, ctypes.c_int, ctypes.c_int, I32, P, P]
            _lib.orc_raster.restype = ctypes.c_int
            _lib.orc_raster_exact.argtypes = [I64, P, P, ctypes.c_int, ctypes.c_int, I32, P, P]
            _lib.orc_raster_exact.restype = ctypes.c_int
            _lib.orc_centreline_distance.argtypes = [I64, P, P, P, ctypes.c_int, ctypes.c_int,
                                                     ctypes.c_int, P]
            _lib.orc_centreline_distance.restype = ctypes.c_int
            _lib.orc_dash_capped.argtypes = [I64, P, P, P, P, ctypes.c_int, D, P, I64, D, I64, P,
                                             P, P, P, P]
            _lib.orc_dash_capped.restype = ctypes.c_int
            _lib.orc_uniform_ribs.argtypes = [ctypes.c_int, P, D, ctypes.c_int, D, P]
            _lib.orc_uniform_ribs.restype = ctypes.c_int
            _lib.orc_facet_angles.argtypes = [I64, P, D, P, P]
            _lib.orc_facet_angles.restype = ctypes.c_int
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class OracleError(RuntimeError):
    pass


def tessellate(batch, dtheta=None, seg_pts64=None, width64=None, tau=0.0):
    """Tessellate every path of ``batch`` (FP64).  Returns a dict of numpy arrays:
    link_nrib[L], link_info[L], rib[R,4], s[R], t[R], psi[R], rho[R], tag[R],
    path_len[P], link_rib_off[L+1], path_rib_off[P+1].
    seg_pts64 / width64 (optional) replace the batch's FP32 control points /
    widths with FP64 values (finite differences).  tau > 0 is the pixel
    tolerance of the per-link step boost (reading R21; taken as FP32 like q)."""
    lib = _load()
    q = float(np.float32(batch.dtheta if dtheta is None else dtheta))
    tau = float(np.float32(tau))
    st = _c(batch.seg_type, np.uint8)
    sp = _c(batch.seg_pts if seg_pts64 is None else seg_pts64, np.float64).reshape(-1)
    sw = _c(batch.seg_w, np.float64)
    off = _c(batch.path_seg_off, np.int32)
    pw = _c(batch.path_width if width64 is None else width64, np.float64)
    pj = _c(batch.path_join, np.uint8)
    pc = _c(batch.path_cap, np.uint8)
    pm = _c(batch.path_miter, np.float64)
    pcl = _c(batch.path_closed, np.uint8)
    S, P = len(st), len(pw)
    L = 2 * S + P
    link_nrib = np.zeros(L, np.int64)
    link_info = np.zeros(L, np.uint8)
    total = ctypes.c_int64(0)
    args = (S, _p(st), _p(sp), _p(sw), P, _p(off), _p(pw), _p(pj), _p(pc), _p(pm), _p(pcl), q, tau)
    rc = lib.orc_tessellate_f64(*args, _p(link_nrib), _p(link_info), 0, None, None, None, None,
                                None, None, None, ctypes.byref(total))
    if rc not in (0, -2):
        raise OracleError(f"orc_tessellate count failed: {rc}")
    R = int(total.value)
    rib = np.zeros((R, 4), np.float64)
    s = np.zeros(R, np.float64)
    t = np.zeros(R, np.float64)
    psi = np.zeros(R, np.float64)
    rho = np.zeros(R, np.float64)
    tag = np.zeros(R, np.uint32)
    plen = np.zeros(P, np.float64)
    rc = lib.orc_tessellate_f64(*args, _p(link_nrib), _p(link_info), R, _p(rib), _p(s), _p(t),
                                _p(psi), _p(rho), _p(tag), _p(plen), ctypes.byref(total))
    if rc != 0:
        raise OracleError(f"orc_tessellate failed: {rc}")
    link_off = np.zeros(L + 1, np.int64)
    link_off[1:] = np.cumsum(link_nrib)
    lbase = 2 * off[:-1].astype(np.int64) + np.arange(P)
    path_off = np.zeros(P + 1, np.int64)
    path_off[:-1] = link_off[lbase]
    path_off[-1] = R
    return dict(link_nrib=link_nrib, link_info=link_info, rib=rib, s=s, t=t, psi=psi, rho=rho,
                tag=tag, path_len=plen, link_rib_off=link_off, path_rib_off=path_off)


def segment_intervals(seg_type, pts, w=1.0, dtheta=np.radians(2.0)):
    """Interval table of one segment: dict(M, p, Psi, delta, Delta, pivot, flags)."""
    lib = _load()
    pts = _c(np.asarray(pts, np.float64).reshape(8), np.float32)
    n = 16
    p = np.zeros(n); Psi = np.zeros(n); delta = np.zeros(n)
    Delta = np.zeros(n, np.int32); pivot = np.zeros(n, np.int32); flags = np.zeros(1, np.int32)
    M = lib.orc_segment_intervals(int(seg_type), _p(pts), float(w), float(np.float32(dtheta)),
                                  _p(p), _p(Psi), _p(delta), _p(Delta), _p(pivot), _p(flags))
    return dict(M=M, p=p[:M + 1], Psi=Psi[:M + 1], delta=delta[:M], Delta=Delta[:M],
                pivot=pivot[:M], flags=int(flags[0]), N=int(Delta[:M].sum()))


def probe(seg_type, pts, w, what, t):
    """Evaluate g (what=0), H (1), H' (2), c (3) or C (4) at parameters t."""
    lib = _load()
    pts = _c(np.asarray(pts, np.float64).reshape(8), np.float32)
    t = _c(np.atleast_1d(t), np.float64)
    out = np.zeros((len(t), 2))
    lib.orc_segment_probe(int(seg_type), _p(pts), float(w), int(what), len(t), _p(t), _p(out))
    return out


def dash(rib, s, tag, pattern, offset=0.0):
    """Dash a rib stream (Sec. 5.2).  Returns dict(rib[n,4], s[n], tag[n], src[n])."""
    lib = _load()
    rib = _c(rib, np.float64).reshape(-1)
    s = _c(s, np.float64)
    tag = _c(tag, np.uint32)
    pat = _c(pattern, np.float64)
    R = len(s)
    n = ctypes.c_int64(0)
    rc = lib.orc_dash(R, _p(rib), _p(s), _p(tag), _p(pat), len(pat), float(offset), 0, None, None,
                      None, None, ctypes.byref(n))
    if rc not in (0, -2):
        raise OracleError(f"orc_dash count failed: {rc}")
    m = int(n.value)
    orib = np.zeros((m, 4)); os_ = np.zeros(m); otag = np.zeros(m, np.uint32)
    osrc = np.zeros(m, np.int64)
    rc = lib.orc_dash(R, _p(rib), _p(s), _p(tag), _p(pat), len(pat), float(offset), m, _p(orib),
                      _p(os_), _p(otag), _p(osrc), ctypes.byref(n))
    if rc != 0:
        raise OracleError(f"orc_dash failed: {rc}")
    return dict(rib=orib, s=os_, tag=otag, src=osrc)


def dash_capped(rib, s, tag, pattern, offset, path_cap, dtheta):
    """Dashing with capped dash ends (Sec. 5.2, reading R18): as ``dash`` plus the
    path's cap style (path_cap[p]) at every stretch end inside the path.
    Returns dict(rib[n,4], s[n], tag[n], src[n])."""
    lib = _load()
    rib = _c(rib, np.float64).reshape(-1)
    s = _c(s, np.float64)
    tag = _c(tag, np.uint32)
    pat = _c(pattern, np.float64)
    pc = _c(path_cap, np.uint8)
    q = float(np.float32(dtheta))
    R = len(s)
    n = ctypes.c_int64(0)
    args = (R, _p(rib), _p(s), _p(tag), _p(pat), len(pat), float(offset), _p(pc), len(pc), q)
    rc = lib.orc_dash_capped(*args, 0, None, None, None, None, ctypes.byref(n))
    if rc not in (0, -2):
        raise OracleError(f"orc_dash_capped count failed: {rc}")
    m = int(n.value)
    orib = np.zeros((m, 4)); os_ = np.zeros(m); otag = np.zeros(m, np.uint32)
    osrc = np.zeros(m, np.int64)
    rc = lib.orc_dash_capped(*args, m, _p(orib), _p(os_), _p(otag), _p(osrc), ctypes.byref(n))
    if rc != 0:
        raise OracleError(f"orc_dash_capped failed: {rc}")
    return dict(rib=orib, s=os_, tag=otag, src=osrc)


def raster(rib, tag, width, height, n_path, exact=False):
    """16-sample coverage of a rib stream.  Returns (canvas uint16[H,W], covered uint64[P]).
    exact: quads filled as polygons by the crossing rule (reading R19) instead of as
    two triangles."""
    lib = _load()
    rib = _c(rib, np.float64).reshape(-1)
    tag = _c(tag, np.uint32)
    canvas = np.zeros((height, width), np.uint16)
    covered = np.zeros(max(int(n_path), 1), np.uint64)
    fn = lib.orc_raster_exact if exact else lib.orc_raster
    rc = fn(len(tag), _p(rib), _p(tag), int(width), int(height), int(n_path), _p(canvas),
            _p(covered))
    if rc != 0:
        raise OracleError(f"orc_raster failed: {rc}")
    return canvas, covered[:n_path]


def centreline_distance(batch, width, height, n_dense=2000):
    """Distance from each sample of a width x height canvas to the union of the
    batch's generator curves: float64[H, W, 16]."""
    lib = _load()
    st = _c(batch.seg_type, np.uint8)
    sp = _c(batch.seg_pts, np.float32).reshape(-1)
    sw = _c(batch.seg_w, np.float32)
    out = np.zeros((height, width, 16))
    rc = lib.orc_centreline_distance(len(st), _p(st), _p(sp), _p(sw), int(width), int(height),
                                     int(n_dense), _p(out))
    if rc != 0:
        raise OracleError(f"orc_centreline_distance failed: {rc}")
    return out


def uniform_ribs(seg_type, pts, w, n_quads, width):
    """Uniform parametric ribs of one segment (Sec. 8.1): float64[n_quads + 1, 4]."""
    lib = _load()
    p = _c(np.asarray(pts, np.float64).reshape(8), np.float64)
    rib = np.zeros((int(n_quads) + 1, 4))
    rc = lib.orc_uniform_ribs(int(seg_type), _p(p), float(w), int(n_quads), 0.5 * float(width),
                              _p(rib))
    if rc != 0:
        raise OracleError(f"orc_uniform_ribs failed: {rc}")
    return rib


def facet_angles(rib, slack=1e-12):
    """Facet angles of one segment's rib run: (angle float64[n, 2] (-1 where
    undefined), ordinary bool[n, 2]); columns are the N and P sides.  slack:
    tolerance of the tangent-range test (1e-12 for FP64 ribs)."""
    lib = _load()
    rib = _c(rib, np.float64).reshape(-1, 4)
    n = len(rib)
    ang = np.zeros((n, 2))
    ordn = np.zeros((n, 2), np.uint8)
    rc = lib.orc_facet_angles(n, _p(rib), float(slack), _p(ang), _p(ordn))
    if rc != 0:
        raise OracleError(f"orc_facet_angles failed: {rc}")
    return ang, ordn.astype(bool)


def sample_positions(width, height):
    """Sample coordinates (px) of the 16-sample pattern: float64[H, W, 16, 2]."""
    k = np.arange(16)
    ox = (16 * k + 8) / 256.0
    oy = (16 * ((5 * k) % 16) + 8) / 256.0
    ys, xs = np.mgrid[0:height, 0:width]
    return np.stack([xs[..., None] + ox, ys[..., None] + oy], axis=-1)
