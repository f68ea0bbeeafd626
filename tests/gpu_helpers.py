"""Shared helpers of the GPU parity tests (test-side code only)."""
from __future__ import annotations

import math

import numpy as np

import oracle

LOG2E = 1.0 / math.log(2.0)


def gpu_render(rctx, scene_id, cams, want_state=True):
    import torch
    flat, state, st = rctx.render(scene_id, cams, want_state=want_state, stats=True)
    torch.cuda.synchronize()
    return flat, state, st


def per_view_offsets(cams, tile=16):
    """Global tile base and pixel base of each view, as the chain numbers them."""
    tb, pb, out = 0, 0, []
    for c in cams:
        W, H, Tx, Ty = oracle.grid(c.as_array(), tile)
        out.append((tb, pb, W, H, Tx, Ty))
        tb += Tx * Ty
        pb += W * H
    return out


def read_state(rctx, state, scene, cams):
    from paper_2508_03180_gb300 import _lib as L
    V = len(cams)
    offs = per_view_offsets(cams)
    T = offs[-1][0] + offs[-1][4] * offs[-1][5]
    P = offs[-1][1] + offs[-1][2] * offs[-1][3]
    d = dict(
        rect=rctx.read(state, L.DGS_BUF_CELL_RECT, np.int32, (V, scene.N, 4)),
        depth=rctx.read(state, L.DGS_BUF_CELL_DEPTH, np.float32, (V, scene.N)),
        cells=rctx.read(state, L.DGS_BUF_TILE_CELLS, np.uint32),
        ranges=rctx.read(state, L.DGS_BUF_TILE_RANGES, np.uint32, (T, 2)),
        rec=rctx.read(state, L.DGS_BUF_GAUSS_REC, np.float32, (V, scene.G, 12)),
        D=rctx.read(state, L.DGS_BUF_PIX_D, np.float32, (P,)),
        nd=rctx.read(state, L.DGS_BUF_PIX_NDONE, np.int32, (P,)),
        offs=offs,
    )
    return d


def view_slices(gs, v):
    tb, pb, W, H, Tx, Ty = gs["offs"][v]
    rng = gs["ranges"][tb:tb + Tx * Ty].astype(np.int64)
    return dict(rect=gs["rect"][v], depth=gs["depth"][v], ranges=rng, rec=gs["rec"][v],
                D=gs["D"][pb:pb + W * H].reshape(H, W), nd=gs["nd"][pb:pb + W * H].reshape(H, W), W=W, H=H,
                Tx=Tx, Ty=Ty)


def tile_lists_equal(gv, cells_all, ocells, orng):
    """Per tile, the GPU list equals the oracle list (bit-exact)."""
    bad = 0
    for t in range(orng.shape[0]):
        o = ocells[orng[t, 0]:orng[t, 1]]
        a, b = gv["ranges"][t]
        g = cells_all[a:b].astype(np.int64) if b > a else np.zeros(0, np.int64)
        if not np.array_equal(g, o):
            bad += 1
    return bad
