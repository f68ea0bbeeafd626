"""Pins of the comparator oracles (per-Gaussian alpha-blending, Eq. 2-3;
weighted-sum rendering, Eq. 4-6) against the hybrid-renderer oracle, which
is itself pinned to alpha-blending closed forms, and against invariants of
the LC-WSR weight.

* K = 1 with every cell centred on its Gaussian and large enough to contain
  the Gaussian's footprint: the hybrid numerator N of Eq. 12 is exactly
  front-to-back alpha-blending, so it must equal the alpha-blend comparator
  (same depth order, same stopping rule: T_n < eps before entry n).
* One cell holding every Gaussian, v = 1: the hybrid renderer reduces to
  sum alpha c / sum alpha, which is weighted-sum rendering with w = 1 and
  no background weight.
* LC-WSR: equal depths make w constant, which cancels (the result is the
  tau = inf result); Gaussians at depth >= tau carry w = 0 and are the same
  as removed; with one Gaussian, the background weight enters as
  (c_B w_B + w alpha c) / (w_B + w alpha), alpha c taken from the
  alpha-blend oracle.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2508_03180_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _k1_scene(seed, n, scale_mul=6.0, logit_add=4.0):
    # cells of semi-axis 2 contain their Gaussian's 3-sigma ellipsoid (scales
    # below 0.45 here) with room for the EWA box; seen from 6 units away
    s = synth.scene_small(seed=seed, n_cells=n, K=1)
    return dataclasses.replace(
        s, cell_center=s.g_mean.copy(), cell_axes=np.full_like(s.cell_axes, 2.0),
        cell_v=np.ones_like(s.cell_v), g_scale=(s.g_scale * scale_mul).astype(np.float32),
        g_logit=(s.g_logit + logit_add).astype(np.float32))


def _far_camera(W=48, H=40):
    return synth.look_at((0.0, -6.0, 0.0), (0.0, 0.0, 0.0), W, H).as_array()


def test_alpha_blend_equals_hybrid_numerator_at_K1():
    scene = _k1_scene(seed=11, n=400)
    assert float(scene.g_scale.max()) < 0.6
    cam = _far_camera()
    a = oracle.render_alpha(scene, cam)
    h = oracle.render_view(scene, cam)
    assert (a["T"] < 1e-4).any(), "the scene must be opaque enough for termination to matter"
    assert np.abs(a["C"]).max() > 0.1
    np.testing.assert_allclose(a["C"], h["N"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(a["T"], h["T"], rtol=0, atol=1e-12)
    # the per-Gaussian lists are shorter than the cell lists (tight boxes)
    assert a["L"] < oracle.sort_length(scene, cam)


def test_alpha_blend_background_and_forced_counts():
    scene = _k1_scene(seed=12, n=300)
    cam = _far_camera()
    opt = oracle.Options(bg=(0.2, 0.4, 0.6))
    a = oracle.render_alpha(scene, cam, opt)
    a0 = oracle.render_alpha(scene, cam)
    bg = np.array(opt.bg)[:, None, None]
    np.testing.assert_allclose(a["C"], a0["C"] + a0["T"][None] * bg, rtol=0, atol=1e-12)
    # its own counts are valid outcomes; with no slack on T (delta = 0), one
    # entry fewer where it stopped early is not
    exact = oracle.Options(delta=0.0)
    assert oracle.render_alpha(scene, cam, exact, forced_ndone=a0["ndone"])["bad"] == 0
    stopped = a0["T"] < 1e-4
    assert stopped.sum() > 20
    fewer = a0["ndone"] - stopped.astype(np.int32)
    assert oracle.render_alpha(scene, cam, exact, forced_ndone=fewer)["bad"] == int(stopped.sum())


def _one_cell_scene(seed, n):
    s = synth.scene_small(seed=seed, n_cells=n, K=1)
    return synth.Scene(n, 0, np.zeros((1, 3), np.float32), np.full((1, 3), 2.5, np.float32),
                       np.array([[1, 0, 0, 0]], np.float32), np.ones(1, np.float32),
                       s.g_mean.copy(), (s.g_scale * 25).astype(np.float32), s.g_quat.copy(),
                       s.g_logit.copy(), s.g_sh.copy(), name="one-cell")


def test_wsr_equals_hybrid_with_one_cell():
    scene = _one_cell_scene(seed=13, n=32)
    cam = synth.look_at((0.0, -6.0, 0.0), (0.0, 0.0, 0.0), 64, 48).as_array()
    h = oracle.render_view(scene, cam)
    w = oracle.render_wsr(scene, cam)
    assert (h["D"] > 1e-3).mean() > 0.2
    np.testing.assert_allclose(w["C"], h["C"], rtol=0, atol=1e-12)


def _flat_camera(W=48, H=40):
    # view = world + (0, 0, 5): R = I, so depth = z_world + 5
    fy = np.float32((H / 2) / np.tan(np.radians(30.0)))
    return np.array([W, H, fy, fy, W / 2, H / 2, 0.2, 1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 5, 0, 0, -5],
                    dtype=np.float32)


def test_lc_wsr_constant_depth_cancels():
    s = _k1_scene(seed=14, n=50, logit_add=0.0)
    mean = s.g_mean.copy()
    mean[:, 2] = 0.0  # every Gaussian at view depth 5
    scene = dataclasses.replace(s, g_mean=mean, cell_center=mean.copy())
    cam = _flat_camera()
    inf = oracle.render_wsr(scene, cam)
    fin = oracle.render_wsr(scene, cam, tau=7.0)
    assert np.abs(inf["C"]).max() > 0.1
    np.testing.assert_allclose(fin["C"], inf["C"], rtol=0, atol=1e-12)
    # a background weight breaks the cancellation: the same tau must now matter
    wb_inf = oracle.render_wsr(scene, cam, w_bg=0.05)
    wb_fin = oracle.render_wsr(scene, cam, tau=7.0, w_bg=0.05)
    assert np.abs(wb_fin["C"] - wb_inf["C"]).max() > 1e-3


def test_lc_wsr_beyond_tau_is_removed():
    s = _k1_scene(seed=15, n=80, logit_add=0.0)
    cam = _flat_camera()
    depth = s.g_mean[:, 2].astype(np.float64) + 5.0
    tau = float(np.median(depth))
    near = np.nonzero(depth < tau)[0]
    full = oracle.render_wsr(s, cam, tau=tau)
    sub = oracle.render_wsr(s.subset_cells(near), cam, tau=tau)
    assert np.abs(full["C"]).max() > 0.1
    np.testing.assert_allclose(full["C"], sub["C"], rtol=0, atol=1e-12)
    # and tau does change the image when Gaussians straddle it
    assert np.abs(oracle.render_wsr(s, cam)["C"] - full["C"]).max() > 1e-3


def test_wsr_background_weight_single_gaussian():
    s = _k1_scene(seed=16, n=1, logit_add=0.0)
    scene = dataclasses.replace(s, g_mean=np.zeros((1, 3), np.float32), cell_center=np.zeros((1, 3), np.float32),
                                cell_v=np.full(1, 0.7, np.float32))
    cam = synth.small_camera(32, 32).as_array()
    ac = oracle.render_alpha(scene, cam)["C"]          # alpha c (background 0)
    rgb = oracle.project64(scene, cam)[0]["rgb"][0]
    ch = int(np.argmax(rgb))
    alpha = ac[ch] / rgb[ch]
    bg = (0.1, 0.3, 0.9)
    w = oracle.render_wsr(scene, cam, w_bg=0.3, opt=oracle.Options(bg=bg))["C"]
    hit = alpha > 1e-6
    assert hit.sum() > 10
    v = float(np.float32(0.7))  # the scene stores v in FP32
    for c in range(3):
        want = (bg[c] * 0.3 + v * ac[c]) / (0.3 + v * alpha)
        np.testing.assert_allclose(w[c][hit], want[hit], rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(w[c][~hit], np.where(alpha[~hit] > 0, w[c][~hit], bg[c]), atol=1e-6)
