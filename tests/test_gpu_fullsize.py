"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times, on sampled outputs the oracle computes in seconds:

* the multi-scale scene (1M Gaussians) rendered from the bench's 8 cameras
  at 1920x1080 in one chain: cell rectangles, depths and every tile list
  bit-exact for sampled views; images on a band of tile rows of every view;
  parameter gradients of a loss supported on a band of one view;
* the large-scale scene (10M Gaussians) at 1920x1080 and 3840x2160 from
  street-level cameras: binning bit-exact, image band.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2508_03180_gb300 import synth
from tests.gpu_helpers import read_state, tile_lists_equal, view_slices

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4


@pytest.fixture(scope="module")
def rctx():
    from paper_2508_03180_gb300.renderer import Context
    c = Context()
    yield c
    c.close()


def _check_binning(scene, cam, gv, cells_all):
    rect, depth = oracle.cell_rects(scene, cam)
    assert np.array_equal(gv["rect"], rect)
    vis = rect[:, 0] >= 0
    assert np.array_equal(gv["depth"][vis].view(np.uint32), depth[vis].view(np.uint32))
    ocells, orng = oracle.tile_lists(rect, depth, cam)
    assert tile_lists_equal(gv, cells_all, ocells, orng) == 0
    mu2f, extf, valid = oracle.gauss_decisions(scene, cam)
    ok = np.repeat(vis, scene.K) & (valid != 0)
    assert np.array_equal(gv["rec"][ok, 0:4].view(np.uint32),
                          np.concatenate([mu2f, extf], 1)[ok].view(np.uint32))


# Pixels whose FP64 stopping cell differs from the GPU's (both valid within
# the slack): at most 0.01% of a band, except on the large-scale scene, whose
# street-level views cross eps after long chains of cells, each carrying the
# FP32 rounding of its Gaussians' alphas into T: there at most 0.05%.
DIFF_FRAC = 1e-4
DIFF_FRAC_LARGE = 5e-4


def _check_band(scene, cam, gv, img, rows, diff_frac=DIFF_FRAC):
    r = oracle.render_view(scene, cam, forced_ndone=gv["nd"], tile_rows=rows)
    H, W = gv["H"], gv["W"]
    y0, y1 = rows[0] * 16, min(rows[1] * 16, H)
    assert r["bad"] == 0
    n_px = (y1 - y0) * W
    # pixels where the FP64 oracle's own stopping cell differs from the GPU's
    # (both valid within the relative slack on T): a rounding statistic
    diff = int((r["ndone"][y0:y1] != gv["nd"][y0:y1]).sum())
    print(f"band rows {rows}: {diff} of {n_px} pixels stop at a different cell in the oracle's own rule")
    assert diff <= max(1, int(diff_frac * n_px)), (diff, n_px)
    err = float(np.abs(img.reshape(3, H, W)[:, y0:y1] - r["C"][:, y0:y1]).max())
    assert err <= IMG_TOL, err
    return err


def test_bench_configuration_sampled(rctx):
    scene = synth.scene_multiscale()
    cams = synth.sphere_cameras(8, 15.0, 1920, 1080, seed0=0)
    sid = rctx.upload_scene(scene)
    flat, state, st = rctx.render(sid, cams, want_state=True, stats=True)
    torch.cuda.synchronize()
    try:
        gs = read_state(rctx, state, scene, cams)
        imgs = [i.cpu().numpy() for i in rctx.split(flat, cams)]
        for v in (0, 5):
            _check_binning(scene, cams[v].as_array(), view_slices(gs, v), gs["cells"])
        for v, cam in enumerate(cams):
            band = (4 + 7 * v, 6 + 7 * v)  # two tile rows per view, a different band each
            _check_band(scene, cam.as_array(), view_slices(gs, v), imgs[v], band)
        # gradients of a loss supported on one band of view 3
        G, C = scene.G, 16
        band = (30, 32)
        sizes = [3 * 1080 * 1920] * 8
        dl = torch.zeros(sum(sizes))
        g = torch.Generator().manual_seed(5)
        o3 = 3 * sizes[0]
        view3 = dl[o3:o3 + sizes[0]].view(3, 1080, 1920)
        view3[:, band[0] * 16:band[1] * 16] = torch.randn(3, 32, 1920, generator=g) * 1e-3
        gr = dict(g_mean=torch.zeros(G, 3, device="cuda"), g_log_scale=torch.zeros(G, 3, device="cuda"),
                  g_quat=torch.zeros(G, 4, device="cuda"), g_logit=torch.zeros(G, device="cuda"),
                  g_sh=torch.zeros(G, C, 3, device="cuda"))
        rctx.backward(state, dl.cuda(), gr)
        torch.cuda.synchronize()
        from paper_2508_03180_gb300 import _lib as L
        g2d = rctx.read(state, L.DGS_BUF_GRAD2D, np.float32, (8, G, 12))[3].astype(np.float64)
        gv3 = view_slices(gs, 3)
        _, ref2d, ref = oracle.render_and_grad(scene, cams[3].as_array(), view3.numpy().astype(np.float64),
                                               ndone=gv3["nd"], tile_rows=band)
        for name, cols in (("mu2", slice(0, 2)), ("conic", slice(2, 5)), ("opac", slice(5, 6)), ("rgb", slice(6, 9))):
            r2 = ref2d[name].reshape(G, -1)
            rel2 = np.linalg.norm(g2d[:, cols] - r2) / np.linalg.norm(r2)
            print(f"screen-space {name}: relative error {rel2:.2e}")
            assert rel2 <= 1e-3, (name, rel2)
        for kg, kr in (("g_mean", "mean"), ("g_log_scale", "log_scale"), ("g_quat", "quat"), ("g_logit", "logit"),
                       ("g_sh", "sh")):
            got = gr[kg].cpu().numpy().astype(np.float64).reshape(ref[kr].shape)
            rel = np.linalg.norm(got - ref[kr]) / np.linalg.norm(ref[kr])
            print(f"{kg}: relative error {rel:.2e}")
            assert rel <= 1e-3, (kg, rel)
            assert np.abs(got - ref[kr]).max() <= 1e-3 * np.abs(ref[kr]).max() + 1e-6
    finally:
        rctx.release_state(state)
        rctx.release_scene(sid)


@pytest.mark.parametrize("W,H", [(1920, 1080), (3840, 2160)])
def test_large_scale_sampled(rctx, W, H):
    scene = _large_scene()
    cams = synth.street_cameras(2, W, H, seed0=3)
    sid = rctx.upload_scene(scene)
    flat, state, st = rctx.render(sid, cams, want_state=True, stats=True)
    torch.cuda.synchronize()
    try:
        gs = read_state(rctx, state, scene, cams)
        imgs = [i.cpu().numpy() for i in rctx.split(flat, cams)]
        Ty = (H + 15) // 16
        for v, cam in enumerate(cams):
            gv = view_slices(gs, v)
            if v == 0:
                _check_binning(scene, cam.as_array(), gv, gs["cells"])
            mid = Ty // 2 - 1
            _check_band(scene, cam.as_array(), gv, imgs[v], (mid, mid + 2), DIFF_FRAC_LARGE)
        assert st.sort_length > 0
    finally:
        rctx.release_state(state)
        rctx.release_scene(sid)


_LARGE = {}


def _large_scene():
    if "s" not in _LARGE:
        _LARGE["s"] = synth.scene_large()
    return _LARGE["s"]
