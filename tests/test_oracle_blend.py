"""Pins of the oracle's hybrid blend (Eq. 12-14, Sec. V-B, Sec. VI-A) against
closed forms, special cases and brute force -- never against itself.

* one Gaussian per cell, v = 1: the numerator is front-to-back alpha blending
  (Eq. 2-3) and the denominator telescopes to 1 - T_final
* a single cell: the image is pure weighted-sum rendering sum a c / sum a
  (Eq. 4 with a constant weight and no background), whatever v is
* permuting the Gaussians inside every cell leaves the image unchanged
  (order independence inside a cell, Sec. V-A)
* cell transmittance never increases along the cell order (Sec. V-B)
* brute force: Eq. 12-14 written as explicit products on tiny scenes
* termination closed form on a stack of half-opaque cells (tests/golden)
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2508_03180_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _alpha(pv, g, x, y, alpha_max=0.99):
    """alpha of Gaussian g at pixel (x, y): FP32 AABB test, FP64 value."""
    if not pv["valid"][g]:
        return 0.0
    px = np.float32(x) + np.float32(0.5)
    py = np.float32(y) + np.float32(0.5)
    if abs(px - pv["mu2f"][g, 0]) > pv["extf"][g, 0] or abs(py - pv["mu2f"][g, 1]) > pv["extf"][g, 1]:
        return 0.0
    pr = pv["proj"]
    dx = float(px) - pr["mu2"][g, 0]
    dy = float(py) - pr["mu2"][g, 1]
    a, b, c = pr["conic"][g]
    G = math.exp(-0.5 * (a * dx * dx + 2 * b * dx * dy + c * dy * dy))
    return min(pr["opac"][g] * G, alpha_max)


def _seq(pv, x, y):
    t = (y // 16) * pv["Tx"] + x // 16
    return pv["cells"][pv["range"][t, 0]:pv["range"][t, 1]]


def test_one_gaussian_per_cell_is_alpha_blending():
    sc = synth.make_scene(150, 1, synth._box(-1, 1), 0.1, 0.4, 0, seed=11)
    cam = synth.small_camera(48, 48).as_array()
    r = oracle.render_view(sc, cam)
    pv = r["pv"]
    rgb = pv["proj"]["rgb"]
    touched = 0
    for y in range(48):
        for x in range(48):
            T, num, n = 1.0, np.zeros(3), 0
            for cell in _seq(pv, x, y):
                if T < 1e-4:
                    break
                a = _alpha(pv, cell, x, y)
                num += T * a * rgb[cell]          # Eq. 2 with T of Eq. 3
                T *= 1.0 - a
                n += 1
            np.testing.assert_allclose(r["N"][:, y, x], num, rtol=1e-12, atol=1e-14)
            assert abs(r["D"][y, x] - (1.0 - T)) <= 1e-12          # telescoping sum
            assert abs(r["T"][y, x] - T) <= 1e-14
            assert r["ndone"][y, x] == n
            touched += n > 3
    assert touched > 300


@pytest.mark.parametrize("v", [1.0, 0.3])
def test_single_cell_is_weighted_sum_rendering(v):
    sc = synth.make_scene(1, 8, lambda rng, n: np.zeros((n, 3)), 0.3, 0.6, 0, seed=4)
    sc.cell_v[:] = v
    cam = synth.small_camera(32, 32).as_array()
    r = oracle.render_view(sc, cam)
    pv = r["pv"]
    rgb = pv["proj"]["rgb"]
    hit = 0
    for y in range(32):
        for x in range(32):
            al = np.array([_alpha(pv, k, x, y) for k in range(8)])
            B = al.sum()
            if B > 1e-10:
                np.testing.assert_allclose(r["C"][:, y, x], (al[:, None] * rgb[:8]).sum(0) / B, rtol=1e-12)
                hit += 1
            else:
                assert np.all(r["C"][:, y, x] == 0.0)
    assert hit > 100


def _permute_within_cells(sc, seed):
    rng = np.random.default_rng(seed)
    perm = np.concatenate([n * sc.K + rng.permutation(sc.K) for n in range(sc.N)])
    out = synth.Scene(sc.K, sc.sh_degree, sc.cell_center, sc.cell_axes, sc.cell_quat, sc.cell_v,
                      sc.g_mean[perm], sc.g_scale[perm], sc.g_quat[perm], sc.g_logit[perm], sc.g_sh[perm])
    return out


def test_order_independence_inside_cells():
    sc = synth.make_scene(400, 8, synth._box(-1, 1), 0.05, 0.25, 3, seed=2)
    sc.cell_v[:] = np.random.default_rng(1).uniform(0.3, 1.0, sc.N).astype(np.float32)
    cam = synth.small_camera(64, 64).as_array()
    a = oracle.render_view(sc, cam)
    b = oracle.render_view(_permute_within_cells(sc, 7), cam)
    assert np.array_equal(a["ndone"], b["ndone"])
    np.testing.assert_allclose(a["C"], b["C"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(a["D"], b["D"], rtol=1e-12, atol=1e-15)
    assert (a["ndone"] > 2).mean() > 0.3


def test_cell_transmittance_is_monotone():
    sc = synth.make_scene(300, 4, synth._box(-1, 1), 0.05, 0.3, 0, seed=3)
    cam = synth.small_camera(40, 40).as_array()
    pv = oracle.prepare_view(sc, cam)
    prev = np.ones((40, 40))
    for n in range(0, 40):
        r = oracle.render_view(sc, cam, pv=pv, forced_ndone=np.full((40, 40), n, np.int32))
        assert np.all(r["T"] <= prev) and np.all(r["T"] >= 0.0)
        prev = r["T"]
    assert prev.min() < 1e-3  # the scene is dense enough to matter


def _direct_image(sc, pv, W, H, eps=1e-4, d_min=1e-10):
    """Eq. 12-14 as written, one pixel at a time, cells ordered by depth."""
    rgb = pv["proj"]["rgb"]
    vis = np.nonzero(pv["rect"][:, 0] >= 0)[0]
    order = vis[np.lexsort((vis, pv["depth"][vis]))]
    img = np.zeros((3, H, W))
    for y in range(H):
        for x in range(W):
            al = {n: [_alpha(pv, n * sc.K + k, x, y) for k in range(sc.K)] for n in order}
            v = {n: float(sc.cell_v[n]) for n in order}
            num, den = np.zeros(3), 0.0
            for j, n in enumerate(order):
                T = 1.0
                for i in order[:j]:                       # Eq. 14
                    for k in range(sc.K):
                        T *= 1.0 - v[i] * al[i][k]
                if T < eps:                               # halted (Sec. V-B)
                    break
                w = v[n] * T                              # Eq. 13
                for k in range(sc.K):                     # Eq. 12
                    num += w * al[n][k] * rgb[n * sc.K + k]
                    den += w * al[n][k]
            img[:, y, x] = num / den if den > d_min else 0.0
    return img


def test_brute_force_tiny_scenes():
    hits = 0
    for seed in range(25):
        rng = np.random.default_rng(100 + seed)
        nc, K = int(rng.integers(1, 5)), int(rng.integers(1, 4))
        sc = synth.make_scene(nc, K, synth._box(-0.3, 0.3), 0.2, 0.5, 0, seed=seed)
        sc.cell_v[:] = rng.uniform(0.2, 1.0, nc).astype(np.float32)
        sc.g_logit[:] = rng.uniform(0.0, 4.0, nc * K).astype(np.float32)
        cam = synth.small_camera(8, 8).as_array()
        r = oracle.render_view(sc, cam)
        ref = _direct_image(sc, r["pv"], 8, 8)
        np.testing.assert_allclose(r["C"], ref, rtol=0, atol=1e-12)
        hits += int((r["D"] > 1e-10).sum())
    assert hits > 200


def _halving_stack(n_cells):
    """n_cells cells on the optical axis of a 9x9 camera, one Gaussian each,
    centred on pixel (4,4), opacity sigmoid(0) = 1/2, large isotropic scale."""
    ys = -1.5 + 0.1 * np.arange(n_cells)
    centre = np.stack([np.zeros(n_cells), ys, np.zeros(n_cells)], 1).astype(np.float32)
    rgb = np.stack([np.arange(n_cells) / n_cells, 1 - np.arange(n_cells) / n_cells,
                    np.full(n_cells, 0.25)], 1)
    sh = ((rgb - 0.5) * 2.0 * math.sqrt(math.pi)).astype(np.float32)[:, None, :]
    rgb = np.maximum(0.5 + sh[:, 0, :].astype(np.float64) / (2.0 * math.sqrt(math.pi)), 0.0)  # stored DC colour, clamped at 0
    q = np.tile(np.array([1, 0, 0, 0], np.float32), (n_cells, 1))
    sc = synth.Scene(1, 0, centre, np.full((n_cells, 3), 0.05, np.float32), q.copy(),
                     np.ones(n_cells, np.float32), centre.copy(), np.full((n_cells, 3), 0.5, np.float32),
                     q.copy(), np.zeros(n_cells, np.float32), sh)
    return sc, rgb


def test_termination_closed_form():
    gold = json.load(open(os.path.join(GOLDEN, "termination_halving.json")))
    sc, rgb = _halving_stack(gold["n_cells_stack"])
    cam = synth.small_camera(9, 9).as_array()
    r = oracle.render_view(sc, cam)
    n = gold["expected_ndone"]
    assert r["ndone"][4, 4] == n
    assert r["T"][4, 4] == gold["expected_T_after"]
    assert abs(r["D"][4, 4] - gold["expected_D"]) <= 1e-15
    w = 2.0 ** -np.arange(n)
    np.testing.assert_allclose(r["C"][:, 4, 4], (w[:, None] * rgb[:n]).sum(0) / w.sum(), rtol=1e-12)
    # a given count is checked against the rule with slack delta = 1e-3
    forced = r["ndone"].copy()
    assert oracle.render_view(sc, cam, forced_ndone=forced)["bad"] == 0
    for wrong in (n - 1, n + 1):
        forced[4, 4] = wrong
        assert oracle.render_view(sc, cam, forced_ndone=forced)["bad"] == 1
