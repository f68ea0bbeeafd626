"""View-dependent calibration v_n (SH coefficients per cell, Sec. V-A) on the
GPU against the oracle: v_n per (view, cell), images under the
termination-count protocol, and dL/dv_n with its chain to the SH
coefficients and to the cell centres through the view direction (gradient
tolerance as for the other parameter groups)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2508_03180_gb300 import synth
from tests.gpu_helpers import read_state, view_slices
from tests.test_gpu_grad import _oracle_grads, assert_close_group

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rctx():
    from paper_2508_03180_gb300.renderer import Context
    c = Context()
    yield c
    c.close()


def _scene(deg):
    sc = synth.make_scene(60, 4, synth._box(-0.5, 0.5), 0.15, 0.4, 1, seed=17 + deg)
    return synth.with_view_dependent_v(sc, degree=deg, seed=deg, base=0.6, band_std=0.15)


@pytest.mark.parametrize("deg", [1, 3])
def test_view_dependent_v_render_and_gradients(rctx, deg):
    from paper_2508_03180_gb300 import _lib as L
    sc = _scene(deg)
    cams = synth.sphere_cameras(2, 3.0, 48, 40, seed0=9)
    G, N, C, Cv = sc.G, sc.N, (sc.sh_degree + 1) ** 2, (deg + 1) ** 2
    sid = rctx.upload_scene(sc)
    flat, state, _ = rctx.render(sid, cams, want_state=True)
    dl = torch.randn(flat.numel(), generator=torch.Generator().manual_seed(deg)).cuda()
    gr = dict(g_mean=torch.zeros(G, 3, device="cuda"), g_cell_v=torch.zeros(N, device="cuda"),
              g_cell_v_sh=torch.zeros(N, Cv, device="cuda"), g_cell_center=torch.full((N, 3), 7.0, device="cuda"),
              g_cell_axes=torch.full((N, 3), 7.0, device="cuda"))
    rctx.backward(state, dl, gr)
    torch.cuda.synchronize()
    try:
        gs = read_state(rctx, state, sc, cams)
        vv = rctx.read(state, L.DGS_BUF_CELL_V, np.float32, (len(cams), N))
        imgs = [i.cpu().numpy() for i in rctx.split(flat, cams)]
        for v, cam in enumerate(cams):
            ov, info = oracle.cell_v_view(sc, cam.as_array())
            assert np.abs(vv[v] - ov).max() <= 2e-6
            assert info["mask"].mean() > 0.5  # mostly unclamped: the gradient path is exercised
            gv = view_slices(gs, v)
            r = oracle.render_view(sc, cam.as_array(), forced_ndone=gv["nd"])
            assert r["bad"] == 0
            assert np.abs(imgs[v].reshape(r["C"].shape) - r["C"]).max() <= 1e-4
        ref, _ = _oracle_grads(sc, cams, dl.cpu().numpy(), gs)
        assert_close_group("cell_v", gr["g_cell_v"].cpu(), ref["cell_v"])
        assert_close_group("cell_v_sh", gr["g_cell_v_sh"].cpu(), ref["cell_v_sh"])
        assert_close_group("mean", gr["g_mean"].cpu(), ref["mean"])
        assert_close_group("cell_center", gr["g_cell_center"].cpu(), ref["cell_center"])
        assert torch.all(gr["g_cell_axes"] == 0)  # overwritten: explicit cells reach the image only through v's direction
        assert np.abs(ref["cell_v_sh"]).max() > 0 and np.abs(ref["cell_center"]).max() > 0
    finally:
        rctx.release_state(state)
        rctx.release_scene(sid)


def test_v_sh_gradient_needs_a_view_dependent_scene(rctx):
    from paper_2508_03180_gb300 import _lib as L
    sc = synth.scene_small(n_cells=100)
    sid = rctx.upload_scene(sc)
    flat, state, _ = rctx.render(sid, [synth.small_camera(32, 32)], want_state=True)
    try:
        with pytest.raises(L.DgsError) as ei:
            rctx.backward(state, torch.zeros_like(flat), dict(g_cell_v_sh=torch.zeros(sc.N, 4, device="cuda")))
        assert ei.value.code == L.DGS_ERR_INVALID_ARG
    finally:
        rctx.release_state(state)
        rctx.release_scene(sid)
