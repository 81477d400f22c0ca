"""torch.autograd.Function over the tessellation: (control points, widths) ->
(rib vertices, cumulative arc length), with the library's adjoint kernel for
the backward pass.  Step counts are those of the forward pass."""
from __future__ import annotations

import torch

from . import (PS_PREC_MIXED, Context, DeviceBatch, ps_tessellate_backward, tessellate)


class PolarStroke(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pts, width, batch, precision=PS_PREC_MIXED, psctx=None):
        """pts: float32 [S, 4, 2] on the GPU; width: float32 [P]; batch: the
        StrokeBatch giving types, weights, path structure, joins, caps and dtheta.
        Returns rib [R, 4] (N.x N.y P.x P.y) and s [R]."""
        c = psctx or Context()
        db = DeviceBatch(batch, device=pts.device)
        db.seg_pts = pts.detach().contiguous().reshape(-1)
        db.path_width = width.detach().contiguous()
        out = tessellate(c, db, precision, arclength=True, want_t=True)
        R = int(out.n_rib.item())
        ctx.state = (c, db, out, precision)
        ctx.shapes = (pts.shape, width.shape)
        return out.rib[:R], out.s[:R]

    @staticmethod
    def backward(ctx, grad_rib, grad_s):
        c, db, out, precision = ctx.state
        R = grad_rib.shape[0] if grad_rib is not None else grad_s.shape[0]
        g_rib = torch.zeros((out.capacity, 4), dtype=torch.float32, device=out.rib.device)
        g_s = torch.zeros(out.capacity, dtype=torch.float32, device=out.rib.device)
        if grad_rib is not None:
            g_rib[:R] = grad_rib
        if grad_s is not None:
            g_s[:R] = grad_s
        g_pts = torch.empty(db.n_seg * 8, dtype=torch.float32, device=out.rib.device)
        g_w = torch.empty(db.n_path, dtype=torch.float32, device=out.rib.device)
        ps_tessellate_backward(c, db, out, g_rib, g_s, g_pts, g_w, precision)
        return g_pts.reshape(ctx.shapes[0]), g_w.reshape(ctx.shapes[1]), None, None, None
