"""Pins of the view-dependent calibration v_n (Sec. V-A: v parameterised by
spherical harmonics) in the oracle:

* degree 0 is view-independent and renders exactly like the scalar v_n it
  equals (k_00 Y_00), the reduction to the pinned scalar path;
* direction convention: d points from the eye to the cell centre, so a cell
  at the origin seen from (0, -3, 0) sees d = +y, where the l = 1, m = -1
  function (C1 y, pinned against SciPy elsewhere) is positive;
* the clamp to [0, 1] holds v and zeroes the gradient outside;
* dL/dk_lm of a rendered loss matches FP64 central differences.
"""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from oracle import project as oproject
from paper_2508_03180_gb300 import synth


def _scene(seed=31, n=14, K=4, deg=2):
    sc = synth.make_scene(n, K, synth._box(-0.5, 0.5), 0.15, 0.4, 0, seed=seed)
    return synth.with_view_dependent_v(sc, degree=deg, seed=seed, base=0.6, band_std=0.12)


def test_degree_zero_is_the_scalar_path():
    sc = synth.with_view_dependent_v(_scene(deg=0), degree=0, seed=3, base=0.55)
    y00 = float(oproject.sh_basis(torch.tensor([[0.0, 0.0, 1.0]], dtype=torch.float64), 0)[0, 0])
    scalar = dataclasses.replace(sc, cell_v_sh=None, v_sh_degree=-1,
                                 cell_v=(sc.cell_v_sh[:, 0].astype(np.float64) * y00))
    for cam in (synth.small_camera(32, 32), synth.sphere_cameras(1, 3.0, 40, 24, seed0=2)[0]):
        a = oracle.render_view(sc, cam.as_array())
        b = oracle.render_view(scalar, cam.as_array())
        np.testing.assert_allclose(a["C"], b["C"], rtol=0, atol=1e-12)
        v, info = oracle.cell_v_view(sc, cam.as_array())
        assert np.allclose(v, 0.55, atol=1e-6) and info["mask"].all()


def test_direction_convention():
    sc = _scene(deg=1)
    sc = dataclasses.replace(sc, cell_center=np.zeros_like(sc.cell_center))
    k = np.zeros_like(sc.cell_v_sh)
    k[:, 0] = 0.5 / 0.28209479177387814
    k[:, 1] = 0.3  # Y_1,-1 = C1 y
    sc = dataclasses.replace(sc, cell_v_sh=k)
    c1 = float(oproject.sh_basis(torch.tensor([[0.0, 1.0, 0.0]], dtype=torch.float64), 1)[0, 1])
    v, _ = oracle.cell_v_view(sc, synth.small_camera(32, 32).as_array())  # eye (0,-3,0): d = +y
    np.testing.assert_allclose(v, 0.5 + 0.3 * c1, atol=1e-6)
    v2, _ = oracle.cell_v_view(sc, synth.look_at((0.0, 3.0, 0.0), (0, 0, 0), 32, 32).as_array())
    np.testing.assert_allclose(v2, 0.5 - 0.3 * c1, atol=1e-6)


def test_clamp_holds_and_blocks_the_gradient():
    sc = _scene(deg=1)
    k = sc.cell_v_sh.copy()
    k[:7, 0] = 3.0 / 0.28209479177387814   # raw v ~ 3: clamped to 1
    k[7:, 0] = -3.0 / 0.28209479177387814  # raw v ~ -3: clamped to 0
    sc = dataclasses.replace(sc, cell_v_sh=k)
    cam = synth.small_camera(32, 32).as_array()
    v, info = oracle.cell_v_view(sc, cam)
    assert np.all(v[:7] == 1.0) and np.all(v[7:] == 0.0) and not info["mask"].any()
    pv = oracle.prepare_view(sc, cam, requires_grad=True)
    g = np.random.default_rng(0).standard_normal((3, 32, 32))
    g2d = oracle.blend_grad_view(sc, pv, g)
    assert np.all(oracle.param_grads(sc, pv, g2d)["cell_v_sh"] == 0.0)


def test_sh_v_gradient_matches_central_differences():
    sc = _scene(deg=2)
    cam = synth.small_camera(32, 32).as_array()
    pv = oracle.prepare_view(sc, cam, requires_grad=True)
    base = oracle.render_view(sc, cam, pv=pv)
    nd = base["ndone"]
    g = np.random.default_rng(4).standard_normal((3, 32, 32))
    g2d = oracle.blend_grad_view(sc, pv, g, ndone=nd)
    an = oracle.param_grads(sc, pv, g2d)["cell_v_sh"]
    cells = np.nonzero(np.abs(an).sum(1) > 1e-6)[0][:5]
    assert len(cells) >= 3
    h = 1e-6
    scale = np.abs(an).max()
    for c in cells:
        for lm in range(an.shape[1]):
            vals = []
            for s in (+1, -1):
                k = sc.cell_v_sh.astype(np.float64).copy()
                k[c, lm] += s * h
                sc2 = dataclasses.replace(sc, cell_v_sh=k)
                vals.append(float((oracle.render_view(sc2, cam, pv=pv, forced_ndone=nd)["C"] * g).sum()))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - an[c, lm]) <= 1e-6 * scale + 1e-9, (c, lm, fd, an[c, lm])


def test_cell_centre_gradient_matches_central_differences():
    """dL/dx_n through the direction of a view-dependent v_n (the cells'
    footprints held fixed: the base view's binning) against FP64 central
    differences of the rendered loss in the cell centre."""
    sc = _scene(deg=3, seed=33)
    cam = synth.small_camera(32, 32).as_array()
    pv = oracle.prepare_view(sc, cam, requires_grad=True)
    nd = oracle.render_view(sc, cam, pv=pv)["ndone"]
    g = np.random.default_rng(6).standard_normal((3, 32, 32))
    g2d = oracle.blend_grad_view(sc, pv, g, ndone=nd)
    res = oracle.param_grads(sc, pv, g2d)
    an = res["cell_center"]
    assert np.all(res["cell_axes"] == 0.0) and np.all(res["cell_quat"] == 0.0)
    cells = np.nonzero(np.abs(an).sum(1) > 1e-6 * np.abs(an).max())[0][:5]
    assert len(cells) >= 3
    h = 1e-6
    for c in cells:
        for j in range(3):
            vals = []
            for s in (+1, -1):
                x = sc.cell_center.astype(np.float64).copy()
                x[c, j] += s * h
                sc2 = dataclasses.replace(sc, cell_center=x)
                vals.append(float((oracle.render_view(sc2, cam, pv=pv, forced_ndone=nd)["C"] * g).sum()))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - an[c, j]) <= 1e-6 * np.abs(an).max() + 1e-9, (c, j, fd, an[c, j])
    # a scalar v_n: no path from the centre to the image
    scalar = dataclasses.replace(sc, cell_v_sh=None, v_sh_degree=-1)
    pv2 = oracle.prepare_view(scalar, cam, requires_grad=True)
    g2 = oracle.blend_grad_view(scalar, pv2, g)
    assert np.all(oracle.param_grads(scalar, pv2, g2)["cell_center"] == 0.0)
