"""The renderer's variant flags on the GPU against the oracle with the same
options: images under the termination-count protocol and the parameter
gradients (gradient tolerance as for the default renderer), for a
background weight, the numerator output, the 1/255 alpha skip, the 3DGS
termination rule, the square AABB and a combination; and a served request
with flags equals the direct render.  The near-plane footprint variant is
checked with a camera inside the scene, its binning bit for bit.

The alpha skip is decided in FP32 on the GPU and in FP64 in the oracle; the
scene used for it keeps every alpha at least 1e-4 (relative) away from 1/255,
checked here, so both sides take the same decisions."""
import numpy as np
import pytest
import torch

import oracle
from paper_2508_03180_gb300 import synth
from tests.gpu_helpers import read_state, tile_lists_equal, view_slices
from tests.test_gpu_grad import assert_close_group

pytestmark = pytest.mark.gpu

BG = (0.3, 0.1, 0.6)
VARIANTS = {
    "w_bg": (dict(w_bg=0.4, bg=BG), oracle.Options(bg=BG, w_bg=0.4)),
    "numerator": (dict(flags=8), oracle.Options(out_numerator=True)),
    "alpha_skip": (dict(flags=1), oracle.Options(alpha_skip=True)),
    "term_exclude": (dict(flags=2), oracle.Options(term_exclude=True)),
    "aabb_square": (dict(flags=4), oracle.Options(aabb_square=True)),
    "combined": (dict(flags=1 | 2 | 4, w_bg=0.25, bg=BG),
                 oracle.Options(bg=BG, w_bg=0.25, alpha_skip=True, term_exclude=True, aabb_square=True)),
}


def _alpha_margin(sc, cam, opt):
    """min over (pixel, Gaussian) pairs inside the AABB of |255 alpha - 1| (FP64)."""
    pv = oracle.prepare_view(sc, cam, opt)
    pr, mu2f, extf, valid = pv["proj"], pv["mu2f"], pv["extf"], pv["valid"]
    W, H = int(cam[0]), int(cam[1])
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float32) + np.float32(0.5)
    worst = np.inf
    for g in np.nonzero(valid)[0]:
        m = (np.abs(xs - mu2f[g, 0]) <= extf[g, 0]) & (np.abs(ys - mu2f[g, 1]) <= extf[g, 1])
        if m.any():
            dx = xs[m].astype(np.float64) - pr["mu2"][g, 0]
            dy = ys[m].astype(np.float64) - pr["mu2"][g, 1]
            a, b, c = pr["conic"][g]
            al = pr["opac"][g] * np.exp(-0.5 * (a * dx * dx + 2 * b * dx * dy + c * dy * dy))
            worst = min(worst, float(np.min(np.abs(al * 255.0 - 1.0))))
    return worst


def _variant_scene():
    sc = synth.make_scene(60, 4, synth._box(-0.5, 0.5), 0.15, 0.4, 1, seed=22)
    sc.cell_v[:] = np.random.default_rng(4).uniform(0.3, 1.0, sc.N).astype(np.float32)
    return sc


@pytest.mark.parametrize("name", list(VARIANTS))
def test_variant_render_and_gradients(name):
    cfg, opt = VARIANTS[name]
    sc = _variant_scene()
    cams = synth.sphere_cameras(2, 3.0, 48, 40, seed0=5)
    if opt.alpha_skip:
        assert min(_alpha_margin(sc, c.as_array(), opt) for c in cams) > 1e-4
    _check_variant(name, sc, cams, cfg, opt)


def test_near_full_binning_render_and_gradients():
    """DGS_FLAG_NEAR_FULL with a camera inside the scene: cells straddling
    the near plane cover every tile; rectangles, depths and tile lists bit for
    bit, then the image and gradients as for the other variants."""
    sc = _variant_scene()
    cams = [synth.look_at((0.05, -0.42, 0.03), (0.0, 0.6, 0.0), 48, 40)]
    opt = oracle.Options(near_full=True)
    cam = cams[0].as_array()
    rect0, _ = oracle.cell_rects(sc, cam)
    rect, depth = oracle.cell_rects(sc, cam, opt)
    assert ((rect0[:, 0] < 0) & (rect[:, 0] >= 0)).sum() >= 2  # the camera sits among the cells
    gv = _check_variant("near_full", sc, cams, dict(flags=16), opt, keep_state=True)
    assert np.array_equal(gv["rect"], rect)
    vis = rect[:, 0] >= 0
    assert np.array_equal(gv["depth"][vis].view(np.uint32), depth[vis].view(np.uint32))
    ocells, orng = oracle.tile_lists(rect, depth, cam, opt)
    assert tile_lists_equal(gv, gv["cells"], ocells, orng) == 0


def _check_variant(name, sc, cams, cfg, opt, keep_state=False):
    from paper_2508_03180_gb300.renderer import Context
    ctx = Context(**cfg)
    try:
        sid = ctx.upload_scene(sc)
        flat, state, _ = ctx.render(sid, cams, want_state=True)
        dl = torch.randn(flat.numel(), generator=torch.Generator().manual_seed(1)).cuda()
        G, N = sc.G, sc.N
        gr = dict(g_mean=torch.zeros(G, 3, device="cuda"), g_scale=torch.zeros(G, 3, device="cuda"),
                  g_quat=torch.zeros(G, 4, device="cuda"), g_logit=torch.zeros(G, device="cuda"),
                  g_sh=torch.zeros(G, 4, 3, device="cuda"), g_cell_v=torch.zeros(N, device="cuda"))
        ctx.backward(state, dl, gr)
        torch.cuda.synchronize()
        gs = read_state(ctx, state, sc, cams)
        imgs = [i.cpu().numpy() for i in ctx.split(flat, cams)]
        dlh = dl.cpu().numpy()
        tot, o = None, 0
        for v, cam in enumerate(cams):
            gv = view_slices(gs, v)
            r = oracle.render_view(sc, cam.as_array(), opt, forced_ndone=gv["nd"])
            assert r["bad"] == 0, (name, v)
            assert np.abs(imgs[v].reshape(r["C"].shape) - r["C"]).max() <= 1e-4, name
            n = 3 * cam.H * cam.W
            g = dlh[o:o + n].reshape(3, cam.H, cam.W).astype(np.float64)
            o += n
            img, _, pg = oracle.render_and_grad(sc, cam.as_array(), g, opt, ndone=gv["nd"])
            tot = pg if tot is None else {k: tot[k] + pg[k] for k in tot}
        for k in ("mean", "scale", "quat", "logit", "sh"):
            assert_close_group(f"{name} {k}", gr[f"g_{k}"].cpu(), tot[k])
        assert_close_group(f"{name} cell_v", gr["g_cell_v"].cpu(), tot["cell_v"])
        ctx.release_state(state)
        ctx.release_scene(sid)
        return view_slices(gs, 0) | {"cells": gs["cells"]} if keep_state else None
    finally:
        ctx.close()


def test_variants_change_the_result():
    """Each flag changes the image of the test scene (so the tests above test it)."""
    from paper_2508_03180_gb300.renderer import Context
    sc = synth.make_scene(60, 4, synth._box(-0.5, 0.5), 0.15, 0.4, 1, seed=22)
    sc.cell_v[:] = np.random.default_rng(4).uniform(0.3, 1.0, sc.N).astype(np.float32)
    cam = synth.sphere_cameras(1, 3.0, 48, 40, seed0=5)
    out = {}
    for name, (cfg, _) in [("default", ({}, None))] + list(VARIANTS.items()):
        ctx = Context(**cfg)
        try:
            sid = ctx.upload_scene(sc)
            flat, _, _ = ctx.render(sid, cam)
            out[name] = flat.cpu().numpy()
            ctx.release_scene(sid)
        finally:
            ctx.close()
    for name in VARIANTS:
        assert np.abs(out[name] - out["default"]).max() > 1e-5, name


def test_served_request_with_flags_equals_direct_render():
    from paper_2508_03180_gb300.renderer import Context
    sc = synth.make_scene(200, 4, synth._box(-0.6, 0.6), 0.1, 0.3, 1, seed=3)
    cam = synth.sphere_cameras(1, 3.0, 96, 64, seed0=2)[0]
    ctx = Context(flags=1 | 2 | 4, w_bg=0.3, bg=BG)
    try:
        sid = ctx.upload_scene(sc)
        direct, _, _ = ctx.render(sid, [cam])
        ctx.serve_start(max_batch=4)
        try:
            out = torch.zeros(3 * 96 * 64, device="cuda")
            assert ctx.poll(ctx.submit(sid, cam, out), -1).status == 0
        finally:
            ctx.serve_stop()
        torch.cuda.synchronize()
        assert torch.equal(out, direct)
        ctx.release_scene(sid)
    finally:
        ctx.close()
