"""Neural cells on the GPU (the MLP decode before the path) against the
oracle: the decoded Gaussians of every visible (view, cell) against the FP64
decode, then the image against the oracle rendering of the GPU's decoded
FP32 values (so the AABB decisions compare bit for bit), under the
termination-count protocol; the paths not built refuse neural scenes."""
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


@pytest.mark.parametrize("F,H,K", [(32, 32, 6), (16, 24, 10)])
def test_decode_and_render(rctx, F, H, K):
    from paper_2508_03180_gb300 import _lib as L
    sc = synth.neural_scene(n_cells=900, K=K, F=F, H=H, seed=F + K)
    cams = [synth.small_camera(64, 48), synth.sphere_cameras(1, 3.0, 100, 70, seed0=3)[0]]
    sid = rctx.upload_scene(sc)
    flat, state, _ = rctx.render(sid, cams, want_state=True)
    torch.cuda.synchronize()
    try:
        gs = read_state(rctx, state, sc, cams)
        dec = rctx.read(state, L.DGS_BUF_DECODED, np.float32, (len(cams), sc.G, 14))
        imgs = [i.cpu().numpy() for i in rctx.split(flat, cams)]
        for v, cam in enumerate(cams):
            gv = view_slices(gs, v)
            vis = np.repeat(gv["rect"][:, 0] >= 0, sc.K)
            assert vis.sum() > 100
            ref = oracle.decode_view(sc, cam.as_array())
            d = dec[v]
            np.testing.assert_allclose(d[vis, 0:3], ref["mean"].reshape(-1, 3)[vis], rtol=0, atol=2e-6)
            np.testing.assert_allclose(d[vis, 3:6], ref["scale"].reshape(-1, 3)[vis], rtol=2e-5, atol=1e-8)
            np.testing.assert_allclose(d[vis, 6:10], ref["quat"].reshape(-1, 4)[vis], rtol=0, atol=2e-5)
            np.testing.assert_allclose(d[vis, 10], ref["opac"].reshape(-1)[vis], rtol=0, atol=2e-5)
            np.testing.assert_allclose(d[vis, 11:14], ref["rgb"].reshape(-1, 3)[vis], rtol=0, atol=2e-5)
            assert (d[vis, 10] <= 0).any() and (d[vis, 10] > 0).any()  # both drawn and skipped Gaussians
            # the image from the GPU's decoded values (oracle's own values where nothing was decoded)
            take = lambda a, b, n: np.where(vis[:, None], a, b.reshape(-1, n))
            ex = oracle.explicit_scene(sc, take(d[:, 0:3], ref["mean"], 3).astype(np.float32),
                                       take(d[:, 3:6], ref["scale"], 3).astype(np.float32),
                                       take(d[:, 6:10], ref["quat"], 4).astype(np.float32),
                                       np.where(vis, d[:, 10], ref["opac"].reshape(-1)),
                                       take(d[:, 11:14], ref["rgb"], 3))
            r = oracle.render_view(ex, cam.as_array(), forced_ndone=gv["nd"])
            assert r["bad"] == 0
            assert np.abs(imgs[v].reshape(r["C"].shape) - r["C"]).max() <= 1e-4
            assert np.abs(r["C"]).max() > 0.1
    finally:
        rctx.release_state(state)
        rctx.release_scene(sid)


def test_paths_not_built_refuse_neural_scenes(rctx):
    from paper_2508_03180_gb300 import _lib as L
    sc = synth.neural_scene(n_cells=50, K=4, F=8, H=8, seed=1)
    sid = rctx.upload_scene(sc)
    cam = synth.small_camera(32, 32)
    flat, state, _ = rctx.render(sid, [cam], want_state=True)
    try:
        with pytest.raises(L.DgsError) as e1:
            rctx.backward(state, torch.zeros_like(flat), dict(g_mean=torch.zeros(sc.G, 3, device="cuda")))
        with pytest.raises(L.DgsError) as e2:
            rctx.render_compare(sid, [cam], "alpha")
        rctx.serve_start(max_batch=2)
        try:
            with pytest.raises(L.DgsError) as e3:
                rctx.submit(sid, cam, torch.zeros(3 * 32 * 32, device="cuda"))
        finally:
            rctx.serve_stop()
        assert e1.value.code == e2.value.code == e3.value.code == L.DGS_ERR_INVALID_ARG
    finally:
        rctx.release_state(state)
        rctx.release_scene(sid)
