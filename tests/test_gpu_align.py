"""Cell alignment on the GPU (Sec. IV-B: Eq. 10 rotation average and the
centre update) against the FP64 oracle, for explicit and neural cells; the
scene renders from the updated cells afterwards (image parity with the
oracle on the GPU's updated FP32 cells); host outputs; a zero weighted sum
keeps the rotation; argument errors."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from paper_2508_03180_gb300 import synth
from tests.gpu_helpers import read_state, view_slices

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rctx():
    from paper_2508_03180_gb300.renderer import Context
    c = Context()
    yield c
    c.close()


def _same_rotation(a, b, atol):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    assert np.abs(a - b).max() <= atol, np.abs(a - b).max()


def test_explicit_align_and_render(rctx):
    sc = synth.make_scene(300, 6, synth._box(-0.6, 0.6), 0.1, 0.3, 1, seed=4)
    ox, oq = oracle.cell_align(sc)
    sid = rctx.upload_scene(sc)
    try:
        x = torch.zeros(sc.N, 3, device="cuda")
        q = torch.zeros(sc.N, 4, device="cuda")
        rctx.cell_align(sid, out_center=x, out_quat=q)
        torch.cuda.synchronize()
        x, q = x.cpu().numpy(), q.cpu().numpy()
        np.testing.assert_allclose(x, ox, rtol=0, atol=2e-6)
        _same_rotation(q, oq, 2e-6)
        # the scene renders from its new cells
        cams = [synth.small_camera(64, 48), synth.sphere_cameras(1, 3.0, 80, 60, seed0=2)[0]]
        flat, state, _ = rctx.render(sid, cams, want_state=True)
        torch.cuda.synchronize()
        try:
            gs = read_state(rctx, state, sc, cams)
            sc2 = dataclasses.replace(sc, cell_center=x.astype(np.float32), cell_quat=q.astype(np.float32))
            for v, (cam, img) in enumerate(zip(cams, rctx.split(flat, cams))):
                gv = view_slices(gs, v)
                r = oracle.render_view(sc2, cam.as_array(), forced_ndone=gv["nd"])
                assert r["bad"] == 0
                assert np.abs(img.cpu().numpy().reshape(r["C"].shape) - r["C"]).max() <= 1e-4
        finally:
            rctx.release_state(state)
    finally:
        rctx.release_scene(sid)


def test_neural_align_host_outputs(rctx):
    sc = synth.neural_scene(n_cells=400, K=5, F=12, H=16, seed=6, box=0.5, axes_lo=0.15, axes_hi=0.4)
    cam = synth.sphere_cameras(1, 3.0, 48, 40, seed0=1)[0]
    ox, oq = oracle.cell_align(sc, cam.as_array())
    sid = rctx.upload_scene(sc)
    try:
        x = np.zeros((sc.N, 3), np.float32)
        q = np.zeros((sc.N, 4), np.float32)
        rctx.cell_align(sid, cam=cam, out_center=x, out_quat=q)
        np.testing.assert_allclose(x, ox, rtol=0, atol=2e-6)
        _same_rotation(q, oq, 2e-5)
        assert np.abs(oq - sc.cell_quat.astype(np.float64)).max() > 0.1  # the rotations did change
    finally:
        rctx.release_scene(sid)


def test_one_of_the_two_and_zero_sum(rctx):
    sc = synth.make_scene(4, 2, synth._box(-0.5, 0.5), 0.1, 0.3, 0, seed=9)
    gq = sc.g_quat.copy()
    gq[1] = -gq[0]                       # cell 0: q and -q with equal opacity: zero sum
    lg = sc.g_logit.copy()
    lg[1] = lg[0]
    sc = dataclasses.replace(sc, g_quat=gq, g_logit=lg)
    ox, oq = oracle.cell_align(sc)
    sid = rctx.upload_scene(sc)
    try:
        x = np.zeros((sc.N, 3), np.float32)
        q = np.zeros((sc.N, 4), np.float32)
        rctx.cell_align(sid, quat=False, center=True, out_center=x, out_quat=q)
        np.testing.assert_array_equal(q, sc.cell_quat)       # rotation untouched
        np.testing.assert_allclose(x, ox, rtol=0, atol=2e-6)
        rctx.cell_align(sid, quat=True, center=False, out_center=x, out_quat=q)
        np.testing.assert_allclose(x, ox, rtol=0, atol=2e-6)  # centre kept from the first call
        np.testing.assert_array_equal(q[0], sc.cell_quat[0])  # zero sum keeps the rotation
        _same_rotation(q[1:], oq[1:], 2e-6)
    finally:
        rctx.release_scene(sid)


def test_argument_errors(rctx):
    from paper_2508_03180_gb300 import _lib as L
    sc = synth.neural_scene(n_cells=20, K=2, F=4, H=4, seed=1)
    sid = rctx.upload_scene(sc)
    try:
        with pytest.raises(L.DgsError) as e1:
            rctx.cell_align(sid, quat=True, center=False)          # neural Eq. 10 needs a view
        with pytest.raises(L.DgsError) as e2:
            L.dgs_cell_align(rctx.ctx, sid, 0, -1, None, None, L.DGS_DEVICE, None)
        with pytest.raises(L.DgsError) as e3:
            L.dgs_cell_align(rctx.ctx, 987654, L.DGS_ALIGN_CENTER, -1, None, None, L.DGS_DEVICE, None)
        assert e1.value.code == e2.value.code == L.DGS_ERR_INVALID_ARG
        assert e3.value.code == L.DGS_ERR_NOT_FOUND
        rctx.cell_align(sid, quat=False, center=True)              # the centre needs no view
    finally:
        rctx.release_scene(sid)
