"""Pins of the oracle's blending variants (off by default; each a renderer
config flag with the same meaning):

* term_exclude: closed form on the halving stack
  (`tests/golden/termination_halving_exclude.json`), and the count check;
* w_bg (background weight in the normalisation, Eq. 4's term): the output
  is (N + w_bg bg) / (D + w_bg) of the unweighted run's N and D, w_bg = 0 is
  the default, a large weight tends to the background;
* out_numerator: the output is the numerator N; for K = 1, v = 1 it is
  front-to-back alpha-blending (Eq. 2-3) with a zero background;
* alpha_skip: for K = 1 and v = 1, D = alpha, so the skipped run's D is the
  default D where it is >= 1/255 and 0 elsewhere;
* aabb_square: the radius is ceil(3 sqrt(lambda_max)) of the screen
  covariance (NumPy's eigvalsh of the FP64 covariance, to one unit of the
  ceiling) and the square contains the per-axis box;
* the adjoint under every variant matches FP64 central differences.
"""
import dataclasses
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle
from oracle import project as oproject
from paper_2508_03180_gb300 import synth
from tests.test_oracle_blend import _halving_stack

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _scene(seed=3, n_cells=14, K=4):
    sc = synth.make_scene(n_cells, K, synth._box(-0.5, 0.5), 0.15, 0.4, 0, seed=seed)
    sc.cell_v[:] = np.random.default_rng(seed).uniform(0.3, 1.0, n_cells).astype(np.float32)
    return sc


def test_termination_exclude_closed_form():
    gold = json.load(open(os.path.join(GOLDEN, "termination_halving_exclude.json")))
    sc, rgb = _halving_stack(gold["n_cells_stack"])
    cam = synth.small_camera(9, 9).as_array()
    opt = oracle.Options(term_exclude=True)
    r = oracle.render_view(sc, cam, opt)
    n = gold["expected_ndone"]
    assert r["ndone"][4, 4] == n
    assert r["T"][4, 4] == gold["expected_T_after"]
    assert abs(r["D"][4, 4] - gold["expected_D"]) <= 1e-15
    w = 2.0 ** -np.arange(n)
    np.testing.assert_allclose(r["C"][:, 4, 4], (w[:, None] * rgb[:n]).sum(0) / w.sum(), rtol=1e-12)
    forced = r["ndone"].copy()
    assert oracle.render_view(sc, cam, opt, forced_ndone=forced)["bad"] == 0
    for wrong in (n - 1, n + 1):
        forced[4, 4] = wrong
        assert oracle.render_view(sc, cam, opt, forced_ndone=forced)["bad"] == 1


def test_background_weight():
    sc = _scene()
    cam = synth.small_camera(32, 32).as_array()
    bg = (0.2, 0.5, 0.9)
    base = oracle.render_view(sc, cam, oracle.Options(bg=bg))
    nd = base["ndone"]
    same = oracle.render_view(sc, cam, oracle.Options(bg=bg, w_bg=0.0), forced_ndone=nd)
    np.testing.assert_array_equal(same["C"], base["C"])
    w = 0.35
    r = oracle.render_view(sc, cam, oracle.Options(bg=bg, w_bg=w), forced_ndone=nd)
    want = (base["N"] + w * np.asarray(bg)[:, None, None]) / (base["D"] + w)[None]
    np.testing.assert_allclose(r["C"], want, rtol=0, atol=1e-13)
    assert np.abs(r["C"] - base["C"]).max() > 1e-3
    far = oracle.render_view(sc, cam, oracle.Options(bg=bg, w_bg=1e9), forced_ndone=nd)
    np.testing.assert_allclose(far["C"], np.broadcast_to(np.asarray(bg)[:, None, None], far["C"].shape), atol=1e-8)


def test_numerator_output():
    sc = _scene(seed=5)
    cam = synth.small_camera(32, 32).as_array()
    base = oracle.render_view(sc, cam)
    r = oracle.render_view(sc, cam, oracle.Options(out_numerator=True), forced_ndone=base["ndone"])
    np.testing.assert_array_equal(r["C"], base["N"])
    # K = 1, v = 1, every Gaussian at its cell's centre (so cell and Gaussian depth
    # orders agree): the output is alpha-blending with a zero background (Eq. 2-3)
    from tests.test_oracle_comparators import _far_camera, _k1_scene
    one = _k1_scene(seed=11, n=400)
    far = _far_camera()
    a = oracle.render_view(one, far, oracle.Options(out_numerator=True))
    ab = oracle.render_alpha(one, far)
    assert (ab["T"] < 1e-4).any()
    np.testing.assert_allclose(a["C"], ab["C"], rtol=0, atol=1e-12)


def test_alpha_skip():
    one = synth.make_scene(200, 1, synth._box(-0.6, 0.6), 0.05, 0.25, 0, seed=13)
    one.cell_v[:] = 1.0
    cam = synth.small_camera(48, 40).as_array()
    base = oracle.render_view(one, cam)
    r = oracle.render_view(one, cam, oracle.Options(alpha_skip=True))
    # with one cell per pixel-hit and K = 1, D is alpha of the first cell plus later cells' terms;
    # restrict to pixels covered by exactly one Gaussian (alpha = D there)
    pv = base["pv"]
    hits = np.zeros((40, 48), dtype=np.int32)
    mu2f, extf = pv["mu2f"], pv["extf"]
    ys, xs = np.mgrid[0:40, 0:48].astype(np.float32) + np.float32(0.5)
    for g in range(one.G):
        if pv["valid"][g]:
            hits += ((np.abs(xs - mu2f[g, 0]) <= extf[g, 0]) & (np.abs(ys - mu2f[g, 1]) <= extf[g, 1])).astype(np.int32)
    single = hits == 1
    assert single.sum() > 50
    D0, D1 = base["D"][single], r["D"][single]
    np.testing.assert_array_equal(D1, np.where(D0 >= 1.0 / 255.0, D0, 0.0))
    assert (D0 < 1.0 / 255.0).any() and (D0 >= 1.0 / 255.0).any()


def test_square_box_radius():
    sc = _scene(seed=7, n_cells=40, K=4)
    cam = synth.sphere_cameras(1, 3.0, 64, 48, seed0=4)[0].as_array()
    mu2f, extf, valid = oracle.gauss_decisions(sc, cam, oracle.Options(aabb_square=True))
    _, tight, _ = oracle.gauss_decisions(sc, cam, oracle.Options())
    proj = oproject.project(torch.tensor(sc.g_mean, dtype=torch.float64), torch.tensor(sc.g_scale, dtype=torch.float64),
                            torch.tensor(sc.g_quat, dtype=torch.float64), torch.zeros(sc.G, dtype=torch.float64),
                            torch.zeros(sc.G, 1, 3, dtype=torch.float64), 0, cam, 0.3)
    cov = proj["cov2"].numpy()
    checked = 0
    for g in np.nonzero(valid)[0]:
        S = np.array([[cov[g, 0], cov[g, 1]], [cov[g, 1], cov[g, 2]]])
        r = math.ceil(3.0 * math.sqrt(np.linalg.eigvalsh(S)[-1]))
        assert extf[g, 0] == extf[g, 1]
        assert abs(extf[g, 0] - r) <= 1.0
        assert extf[g, 0] >= tight[g, 0] and extf[g, 0] >= tight[g, 1]
        checked += 1
    assert checked >= 100


VARIANTS = {
    "w_bg": oracle.Options(bg=(0.3, 0.1, 0.6), w_bg=0.4),
    "numerator": oracle.Options(out_numerator=True),
    "alpha_skip": oracle.Options(alpha_skip=True),
    "term_exclude": oracle.Options(term_exclude=True),
    "aabb_square": oracle.Options(aabb_square=True),
}


@pytest.mark.parametrize("name", sorted(VARIANTS))
def test_variant_adjoint_matches_central_differences(name):
    opt = VARIANTS[name]
    sc = _scene(seed=21)
    cam = synth.small_camera(32, 32).as_array()
    pv = oracle.prepare_view(sc, cam, opt)
    base = oracle.render_view(sc, cam, opt, pv=pv)
    nd = base["ndone"]
    assert base["bad"] == 0
    g = np.random.default_rng(0).standard_normal((3, 32, 32))
    an = oracle.blend_grad_view(sc, pv, g, opt, ndone=nd)

    def loss(proj=None, scene=sc):
        pv2 = dict(pv)
        if proj is not None:
            pv2["proj"] = proj
        return float((oracle.render_view(scene, None, opt, pv=pv2, forced_ndone=nd)["C"] * g).sum())

    rng = np.random.default_rng(1)
    cand = np.nonzero(np.abs(an["opac"]) > 1e-6)[0]
    gs = rng.choice(cand, min(8, len(cand)), replace=False)
    n_checked = 0
    for key, h in (("mu2", 1e-5), ("opac", 1e-6), ("rgb", 1e-6)):
        arr = pv["proj"][key]
        scale = np.abs(an[key]).max()
        for gi in gs:
            for j in range(arr.shape[1] if arr.ndim > 1 else 1):
                idx = (gi, j) if arr.ndim > 1 else (gi,)
                vals = []
                for s in (+1, -1):
                    proj = {k: v.copy() for k, v in pv["proj"].items()}
                    proj[key][idx] += s * h
                    vals.append(loss(proj))
                fd = (vals[0] - vals[1]) / (2 * h)
                assert abs(fd - an[key][idx]) <= 1e-6 * scale + 1e-9, (name, key, idx, fd, an[key][idx])
                n_checked += 1
    cs = np.nonzero(np.abs(an["v"]) > 1e-6)[0][:4]
    for c in cs:
        vals = []
        for s in (+1, -1):
            sc2 = dataclasses.replace(sc, cell_v=sc.cell_v.astype(np.float64).copy())
            sc2.cell_v[c] += s * 1e-6
            vals.append(loss(scene=sc2))
        fd = (vals[0] - vals[1]) / 2e-6
        assert abs(fd - an["v"][c]) <= 1e-6 * np.abs(an["v"]).max() + 1e-9, (name, c, fd, an["v"][c])
    assert n_checked >= 40 and len(cs) >= 2


def _near_plane_scene():
    """Four cells in front of a camera at the origin looking along +z (view
    z = world z): one straddling the near plane (0.2) with its centre in
    front, one wholly behind, one in front, one straddling with its centre
    behind the eye."""
    sc = synth.make_scene(4, 2, synth._box(-0.5, 0.5), 0.15, 0.4, 0, seed=1)
    sc.cell_center[:] = np.array([[0.0, 0.0, 0.25], [0.0, 0.0, -1.0], [0.2, 0.1, 3.0], [0.1, 0.0, -0.1]],
                                 np.float32)
    sc.cell_axes[:] = np.array([[0.3] * 3, [0.3] * 3, [0.3] * 3, [0.5] * 3], np.float32)
    sc.cell_quat[:] = np.array([1.0, 0.0, 0.0, 0.0], np.float32)
    cam = synth.look_at((0.0, 0.0, 0.0), (0.0, 0.0, 1.0), 64, 48).as_array()
    return sc, cam


def test_near_full_footprint():
    sc, cam = _near_plane_scene()
    znear = float(cam[6])
    cz = sc.cell_center[:, 2].astype(np.float64)
    ext = sc.cell_axes[:, 2].astype(np.float64)  # sqrt(S_zz) of an axis-aligned cell
    straddle = (cz - ext <= znear) & (cz + ext > znear)
    assert list(straddle) == [True, False, False, True]
    _, _, Tx, Ty = oracle.grid(cam)
    rect, depth = oracle.cell_rects(sc, cam)
    rect_f, depth_f = oracle.cell_rects(sc, cam, oracle.Options(near_full=True))
    assert (rect[straddle] == -1).all() and (rect[1] == -1).all()       # default: culled
    assert (rect_f[1] == -1).all()                                      # wholly behind: culled either way
    for n in np.nonzero(straddle)[0]:                                   # variant: every tile
        assert list(rect_f[n]) == [0, 0, Tx - 1, Ty - 1]
        assert depth_f[n] == np.float32(max(cz[n], 0.0))
    assert (rect_f[2] == rect[2]).all() and rect[2][0] >= 0 and depth_f[2] == depth[2]
    # every tile's list starts with the straddlers, nearest first (depth 0 before 0.25)
    cells, rng = oracle.tile_lists(rect_f, depth_f, cam, oracle.Options(near_full=True))
    for t in range(Tx * Ty):
        lst = list(cells[rng[t, 0]:rng[t, 1]])
        assert lst[:2] == [3, 0]
        tx, ty = t % Tx, t // Tx
        in2 = rect[2][0] <= tx <= rect[2][2] and rect[2][1] <= ty <= rect[2][3]
        assert lst[2:] == ([2] if in2 else [])
