"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI and
compare it with the FP64 oracle."""
import numpy as np

import oracle

F32_EPS = 2.0 ** -24


def gpu_tessellate(batch, precision, want_t=True, tau=0.0):
    import torch
    import paper_2007_00308_gb300 as ps
    ctx = ps.Context()
    if tau:
        ctx.set_pixel_tolerance(tau)
    db = ps.DeviceBatch(batch)
    out = ps.tessellate(ctx, db, precision, arclength=True, want_t=want_t)
    torch.cuda.synchronize()
    R = int(out.n_rib.item())
    res = dict(
        R=R,
        rib=out.rib[:R].cpu().numpy().astype(np.float64),
        tag=out.tag[:R].cpu().numpy().view(np.uint32),
        s=out.s[:R].cpu().numpy().astype(np.float64),
        t=out.t[:R].cpu().numpy().astype(np.float64) if want_t else None,
        link_rib_off=out.link_rib_off.cpu().numpy().astype(np.int64),
        path_rib_off=out.path_rib_off.cpu().numpy().astype(np.int64),
        path_len=out.path_len.cpu().numpy().astype(np.float64),
        status=ctx.status(), ctx=ctx, out=out)
    return res


def ulp32(x):
    x = np.abs(np.asarray(x, np.float64))
    e = np.floor(np.log2(np.maximum(x, 1e-30)))
    return np.where(x > 0, 2.0 ** (e - 23), 2.0 ** -149)


def vertex_tolerance(o_rib, rho, r, eps_ang):
    """Diagnostic bound of the all-FP32 kernel (not the contract): 1e-4 px, plus
    FP32 representation (2 ulp of the coordinate), plus the along-curve shift of
    a rib whose angle is off by eps_ang (radius of curvature rho) and the
    normal's rotation (r eps_ang)."""
    mag = np.abs(o_rib)
    return 1e-4 + 2.0 * ulp32(mag) + ((np.minimum(rho, 1e12) + r) * eps_ang)[:, None]


# Computational allowance of the contract bar, relative to the coordinate (see
# contract_tolerance).
REL_ALLOW = 2.0 ** -30


def contract_tolerance(o_rib, g_rib):
    """The vertex bar of the mixed-precision path: per coordinate
    max(1e-4 px, ulp32(m)/2 + 2^-30 m), m = max(|x_oracle|, |x_gpu|).

    1e-4 px absolute is the bar up to |x| = 2048, where half an FP32 ulp is
    6.1e-5.  Above it the FP32 output's own rounding (half an ulp) is the
    floor; no computation can meet half an ulp exactly, because an exact value
    within e of a rounding midpoint rounds either way for any error e > 0, so
    the bar adds an allowance of 2^-30 m (3.8e-6 px at 4096 px) for the value
    before its single final rounding."""
    m = np.maximum(np.abs(o_rib), np.abs(g_rib))
    return np.maximum(1e-4, 0.5 * ulp32(m) + REL_ALLOW * m)


def compare_tess(o, g, batch, fragile_bit, eps_ang=None, s_rel=1e-5, check_s=True):
    """Compare GPU output g with oracle output o.  Returns (stats, failures).

    Counts: exact on every link the oracle does not flag fragile for this
    precision.  Vertices (non-fragile links): eps_ang None is the contract bar
    of the mixed-precision path, contract_tolerance; otherwise the FP32
    kernel's diagnostic bound vertex_tolerance with that angle error.  Arc
    length (paths without fragile links): |ds| <= s_rel * max(s, 1 px) under
    the contract; the diagnostic bound adds 2 m, m the running maximum of the
    vertex bound along the path (a rib displaced by e along the curve changes
    the two chords beside it by about +e and -e, so the sum telescopes to the
    end displacements).  stats carries the absolute vertex error (max, p99,
    median) and the relative s error (max, p99)."""
    contract = eps_ang is None
    fails = []
    stats = {}
    g_n = np.diff(g["link_rib_off"])
    o_n = o["link_nrib"]
    frag = (o["link_info"] & fragile_bit) != 0
    mism = g_n != o_n
    stats["links"] = len(o_n)
    stats["count_mismatch_nonfragile"] = int((mism & ~frag).sum())
    stats["count_mismatch_fragile"] = int((mism & frag).sum())
    stats["fragile_links"] = int(frag.sum())
    if stats["count_mismatch_nonfragile"]:
        bad = np.where(mism & ~frag)[0][:5]
        fails.append(f"count mismatch on non-fragile links {bad.tolist()}: gpu {g_n[bad].tolist()} "
                     f"oracle {o_n[bad].tolist()}")
    o_off = o["link_rib_off"]
    g_off = g["link_rib_off"]
    ok = ~mism & ~frag & (o_n > 0)
    sel_links = np.where(ok)[0]
    idx_o = np.concatenate([np.arange(o_off[l], o_off[l + 1]) for l in sel_links]) if len(sel_links) else np.zeros(0, np.int64)
    idx_g = np.concatenate([np.arange(g_off[l], g_off[l + 1]) for l in sel_links]) if len(sel_links) else np.zeros(0, np.int64)
    P = batch.n_path
    r_path = 0.5 * batch.path_width.astype(np.float64)
    if len(idx_o):
        r_rib = r_path[(o["tag"][idx_o] >> 2).astype(np.int64)]
        if not np.array_equal(g["tag"][idx_g], o["tag"][idx_o]):
            fails.append("tag mismatch")
        err = np.abs(g["rib"][idx_g] - o["rib"][idx_o])
        if contract:
            tol = contract_tolerance(o["rib"][idx_o], g["rib"][idx_g])
        else:
            tol = vertex_tolerance(o["rib"][idx_o], o["rho"][idx_o], r_rib, eps_ang)
        ratio = err / tol
        stats["vertex_err_max"] = float(err.max())
        stats["vertex_err_p99"] = float(np.quantile(err, 0.99))
        stats["vertex_err_p50"] = float(np.median(err))
        stats["vertex_ratio_max"] = float(ratio.max())
        stats["vertex_over_tol"] = int((ratio > 1).any(axis=1).sum())
        if ratio.max() > 1.0:
            w = np.unravel_index(np.argmax(ratio), ratio.shape)
            fails.append(f"{stats['vertex_over_tol']} ribs beyond tolerance; worst {err[w]:.3e} > "
                         f"tol {tol[w]:.3e} at oracle rib {idx_o[w[0]]} (rho {o['rho'][idx_o[w[0]]]:.3g}, "
                         f"coord {o['rib'][idx_o[w[0]], w[1]]:.6g})")
    # arc length on paths with no fragile or mismatched link
    lbase = 2 * batch.path_seg_off[:-1].astype(np.int64) + np.arange(P)
    link_path = np.repeat(np.arange(P), np.diff(np.r_[lbase, len(o_n)]))
    bad_path = np.zeros(P, bool)
    bad_path[link_path[mism | frag]] = True
    good = ~bad_path
    if check_s and good.any() and len(idx_o):
        rib_path = (o["tag"][idx_o] >> 2).astype(np.int64)
        sel = good[rib_path]
        so, sg = o["s"][idx_o][sel], g["s"][idx_g][sel]
        vt = tol.max(axis=1)[sel]
        rp = rib_path[sel]
        # running maximum of the vertex tolerance within each path (ribs are path-ordered)
        run = np.empty_like(vt)
        cur, prev = 0.0, -1
        for i in range(len(vt)):
            if rp[i] != prev:
                cur, prev = 0.0, rp[i]
            cur = max(cur, vt[i])
            run[i] = cur
        serr = np.abs(sg - so)
        stol = s_rel * np.maximum(so, 1.0) + (0.0 if contract else 2.0 * run)
        srel = serr / np.maximum(so, 1.0)
        stats["s_err_max"] = float(serr.max()) if len(serr) else 0.0
        stats["s_rel_max"] = float(srel.max()) if len(serr) else 0.0
        stats["s_rel_p99"] = float(np.quantile(srel, 0.99)) if len(serr) else 0.0
        stats["s_ratio_max"] = float((serr / stol).max()) if len(serr) else 0.0
        if len(serr) and (serr > stol).any():
            w = np.argmax(serr / stol)
            fails.append(f"s error {serr[w]:.3e} > {stol[w]:.3e} (s={so[w]:.4g})")
        last = np.r_[np.diff(rp) != 0, True]
        lerr = np.abs(sg[last] - so[last])
        if (lerr > stol[last]).any():
            fails.append(f"path length error {lerr.max():.3e}")
    return stats, fails
