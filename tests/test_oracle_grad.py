"""Pins of the oracle's adjoint against FP64 central finite differences.

Decisions (AABB skip, tile lists, processed-cell counts) are held at the base
point on both sides, so the image is a smooth function of the perturbed
values and central differences converge to the exact derivative.
"""
import numpy as np
import pytest

import oracle
from paper_2508_03180_gb300 import synth


def _loss(sc, pv, g, nd, proj=None):
    pv2 = dict(pv)
    if proj is not None:
        pv2["proj"] = proj
    return float((oracle.render_view(sc, None, pv=pv2, forced_ndone=nd)["C"] * g).sum())


def _scene(seed, n_cells, K, deg):
    sc = synth.make_scene(n_cells, K, synth._box(-0.5, 0.5), 0.15, 0.4, deg, seed=seed)
    rng = np.random.default_rng(seed)
    sc.cell_v[:] = rng.uniform(0.3, 1.0, n_cells).astype(np.float32)
    return sc


def test_blend_adjoint_matches_central_differences():
    sc = _scene(21, 12, 4, 0)
    cam = synth.small_camera(32, 32).as_array()
    pv = oracle.prepare_view(sc, cam)
    base = oracle.render_view(sc, cam, pv=pv)
    nd = base["ndone"]
    g = np.random.default_rng(0).standard_normal((3, 32, 32))
    an = oracle.blend_grad_view(sc, pv, g, ndone=nd)
    # quantities with the pixel-unit scale of each
    checks = [("mu2", 1e-5), ("conic", 1e-6), ("opac", 1e-6), ("rgb", 1e-6)]
    rng = np.random.default_rng(1)
    gs = rng.choice(np.nonzero(np.abs(an["opac"]) > 1e-6)[0], 10, replace=False)
    n_checked = 0
    for key, h in checks:
        arr = pv["proj"][key]
        scale = np.abs(an[key]).max()
        for gi in gs:
            for j in range(arr.shape[1] if arr.ndim > 1 else 1):
                idx = (gi, j) if arr.ndim > 1 else (gi,)
                vals = []
                for s in (+1, -1):
                    proj = {k: v.copy() for k, v in pv["proj"].items()}
                    proj[key][idx] += s * h
                    vals.append(_loss(sc, pv, g, nd, proj))
                fd = (vals[0] - vals[1]) / (2 * h)
                assert abs(fd - an[key][idx]) <= 1e-6 * scale + 1e-9, (key, idx, fd, an[key][idx])
                n_checked += 1
    # the calibration scalar v_n
    cs = np.nonzero(np.abs(an["v"]) > 1e-6)[0][:6]
    for c in cs:
        vals = []
        for s in (+1, -1):
            sc2 = synth.Scene(**{**sc.__dict__})
            sc2.cell_v = sc.cell_v.astype(np.float64).copy()
            sc2.cell_v[c] += s * 1e-6
            vals.append(float((oracle.render_view(sc2, cam, pv=pv, forced_ndone=nd)["C"] * g).sum()))
        fd = (vals[0] - vals[1]) / 2e-6
        assert abs(fd - an["v"][c]) <= 1e-6 * np.abs(an["v"]).max() + 1e-9
    assert n_checked >= 80 and len(cs) >= 3


@pytest.mark.parametrize("deg", [0, 3])
def test_parameter_gradients_match_central_differences(deg):
    """64 Gaussians (16 cells x 4) at 32x32, FP64."""
    sc = _scene(5 + deg, 16, 4, deg)
    cam = synth.small_camera(32, 32).as_array()
    pv = oracle.prepare_view(sc, cam, requires_grad=True)
    base = oracle.render_view(sc, cam, pv=pv)
    nd = base["ndone"]
    g = np.random.default_rng(2).standard_normal((3, 32, 32))
    g2d = oracle.blend_grad_view(sc, pv, g, ndone=nd)
    pg = oracle.param_grads(sc, pv, g2d)
    mask = pv["mask"]
    # float64 copy of the parameters; decisions stay those of pv
    P64 = {k: getattr(sc, k).astype(np.float64) for k in ("g_mean", "g_scale", "g_quat", "g_logit", "g_sh")}

    def loss_with(name, idx, delta):
        p = {k: v.copy() for k, v in P64.items()}
        if name == "log_scale":
            p["g_scale"][idx] *= np.exp(delta)
        else:
            p[{"mean": "g_mean", "quat": "g_quat", "logit": "g_logit", "sh": "g_sh"}[name]][idx] += delta
        sc2 = synth.Scene(sc.K, sc.sh_degree, sc.cell_center, sc.cell_axes, sc.cell_quat, sc.cell_v,
                          p["g_mean"], p["g_scale"], p["g_quat"], p["g_logit"], p["g_sh"])
        proj, _ = oracle.project64(sc2, cam, mask=mask)
        return _loss(sc, pv, g, nd, proj)

    rng = np.random.default_rng(3)
    live = np.nonzero(np.abs(g2d["opac"]) > 1e-6)[0]
    gs = rng.choice(live, min(8, len(live)), replace=False)
    h = 1e-6
    n_checked = 0
    for name, shape in (("mean", 3), ("log_scale", 3), ("quat", 4), ("logit", 1), ("sh", None)):
        an = pg[name]
        scale = np.abs(an).max()
        for gi in gs:
            if name == "sh":
                idxs = [(gi, c, ch) for c in range(an.shape[1]) for ch in range(3)][::5]
            elif name == "logit":
                idxs = [(gi,)]
            else:
                idxs = [(gi, j) for j in range(shape)]
            for idx in idxs:
                fd = (loss_with(name, idx, h) - loss_with(name, idx, -h)) / (2 * h)
                assert abs(fd - an[idx]) <= 1e-6 * scale + 1e-9, (name, idx, fd, an[idx])
                n_checked += 1
    assert n_checked > 60
