"""Neural cells on the GPU (the MLP decode before the path) against the
oracle: the decoded Gaussians of every visible (view, cell) against the FP64
decode, then the image against the oracle rendering of the GPU's decoded
FP32 values (so the AABB decisions compare bit for bit), under the
termination-count protocol; gradients through the decode against the FP64
oracle; the paths not built refuse neural scenes."""
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


# (32, 32, 10), (32, 32, 6), (16, 24, 10): the tensor-core products (F + 4 <= 40, H <= 32, K <= 10);
# (20, 36, 7), (64, 64, 32): the CUDA-core ones
@pytest.mark.parametrize("F,H,K", [(32, 32, 10), (32, 32, 6), (16, 24, 10), (20, 36, 7), (64, 64, 32)])
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


@pytest.mark.parametrize("F,H,K", [(32, 32, 10), (20, 36, 7)])
def test_neural_scene_out_of_view(rctx, F, H, K):
    """Nothing in view: the decode's device count is 0 while its capacity is
    not (the asynchronous chain), or 0 on the host (stats); both renders give
    the background, and a backward gives zero gradients."""
    from oracle import decode as odec
    sc = synth.neural_scene(n_cells=300, K=K, F=F, H=H, seed=2)
    away = synth.look_at((0.0, -3.0, 0.0), (0.0, -6.0, 0.0), 96, 64)  # looking away from the cells
    sid = rctx.upload_scene(sc)
    try:
        rctx.render(sid, [synth.small_camera(64, 48)])  # the context has rendered: later renders are device-sized
        a, sa, _ = rctx.render(sid, [away], want_state=True)
        b, sb, st = rctx.render(sid, [away], want_state=True, stats=True)
        torch.cuda.synchronize()
        assert st.visible_cells == 0
        assert torch.equal(a, b) and float(a.abs().max()) == 0.0
        P = odec.packed_size(F, H, K)
        g = dict(g_mlp=torch.full((P,), 7.0, device="cuda"), g_feat=torch.full((sc.N, F), 7.0, device="cuda"))
        rctx.backward(sa, torch.ones_like(a), g)
        torch.cuda.synchronize()
        assert float(g["g_mlp"].abs().max()) == 0.0 and float(g["g_feat"].abs().max()) == 0.0
        rctx.release_state(sa)
        rctx.release_state(sb)
    finally:
        rctx.release_scene(sid)


def test_paths_not_built_refuse_neural_scenes(rctx):
    """Explicit-Gaussian gradients of a neural scene and the comparators (which
    project explicit Gaussians) are refused; serving takes neural scenes
    (tests/test_gpu_serving.py)."""
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
        assert e1.value.code == e2.value.code == L.DGS_ERR_INVALID_ARG
    finally:
        rctx.release_state(state)
        rctx.release_scene(sid)


def _neural_oracle_grads(sc, cams, dl_flat, gs, dec):
    """Per-view oracle gradients through the decode, summed over views; the
    AABB decisions and tile lists come from the GPU's decoded FP32 values
    (the oracle's own where nothing was decoded), the per-pixel cell counts
    from the GPU's forward."""
    tot, off = None, 0
    for v, cam in enumerate(cams):
        gv = view_slices(gs, v)
        n = 3 * cam.H * cam.W
        g = dl_flat[off:off + n].astype(np.float64).reshape(3, cam.H, cam.W)
        off += n
        vis = np.repeat(gv["rect"][:, 0] >= 0, sc.K)
        ref = oracle.decode_view(sc, cam.as_array())
        take = lambda a, b, w: np.where(vis[:, None], a, b.reshape(-1, w)).astype(np.float32)
        d = dec[v]
        decided = (take(d[:, 0:3], ref["mean"], 3), take(d[:, 3:6], ref["scale"], 3), take(d[:, 6:10], ref["quat"], 4))
        _, r = oracle.neural_render_and_grad(sc, cam.as_array(), g, decided=decided, ndone=gv["nd"])
        r = {k: r[k] for k in ("mlp", "feat", "offset", "cell_center", "cell_axes", "cell_quat")}
        tot = r if tot is None else {k: tot[k] + r[k] for k in tot}
    return tot


@pytest.mark.parametrize("F,H,K,stretch,location", [(8, 12, 4, 1.0, "device"), (12, 16, 6, 1.6, "host"),
                                                     (32, 32, 10, 1.0, "device"), (20, 36, 7, 1.0, "device"),
                                                     (64, 64, 32, 1.2, "device")])
def test_gradients_through_the_decode(rctx, F, H, K, stretch, location):
    """dL/d(weights, features, offsets) and of the cells' centres, semi-axes
    and quaternions, summed over two views, against the FP64 oracle.  stretch > 1 pushes some offsets outside the unit ball (the
    projection onto it); host outputs go through the staging path.  The
    first three shapes take the weight gradients fused into the adjoint's
    tiles, the last two (a hidden layer wider than 32) the per-sample rows
    and the separate product."""
    from paper_2508_03180_gb300 import _lib as L
    from oracle import decode as odec
    from tests.test_gpu_grad import assert_close_group
    sc = synth.neural_scene(n_cells=160, K=K, F=F, H=H, seed=7 + K, box=0.5, axes_lo=0.15, axes_hi=0.4)
    sc.neural["offset"][:] *= stretch
    cams = synth.sphere_cameras(2, 3.0, 48, 40, seed0=5)
    P = odec.packed_size(F, H, K)
    sid = rctx.upload_scene(sc)
    flat, state, _ = rctx.render(sid, cams, want_state=True)
    dl = torch.randn(flat.numel(), generator=torch.Generator().manual_seed(K)).cuda()
    if location == "device":
        gr = dict(g_mlp=torch.zeros(P, device="cuda"), g_feat=torch.zeros(sc.N, F, device="cuda"),
                  g_offset=torch.zeros(sc.G, 3, device="cuda"), g_cell_center=torch.zeros(sc.N, 3, device="cuda"),
                  g_cell_axes=torch.zeros(sc.N, 3, device="cuda"), g_cell_quat=torch.zeros(sc.N, 4, device="cuda"))
        rctx.backward(state, dl, gr)
    else:
        gr = dict(g_mlp=np.zeros(P, np.float32), g_feat=np.zeros((sc.N, F), np.float32),
                  g_offset=np.zeros((sc.G, 3), np.float32), g_cell_center=np.zeros((sc.N, 3), np.float32),
                  g_cell_axes=np.zeros((sc.N, 3), np.float32), g_cell_quat=np.zeros((sc.N, 4), np.float32))
        rctx.backward(state, dl, gr, location=L.DGS_HOST)
    torch.cuda.synchronize()
    try:
        gs = read_state(rctx, state, sc, cams)
        dec = rctx.read(state, L.DGS_BUF_DECODED, np.float32, (len(cams), sc.G, 14))
        ref = _neural_oracle_grads(sc, cams, dl.cpu().numpy(), gs, dec)
        got = {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v) for k, v in gr.items()}
        for k, name in (("g_mlp", "mlp"), ("g_feat", "feat"), ("g_offset", "offset"),
                        ("g_cell_center", "cell_center"), ("g_cell_axes", "cell_axes"), ("g_cell_quat", "cell_quat")):
            assert np.abs(ref[name]).max() > 0, name
            assert_close_group(name, got[k], ref[name])
        if stretch > 1.0:
            on = np.linalg.norm(sc.neural["offset"].astype(np.float64).reshape(-1, 3), axis=1)
            assert (on > 1.0).any() and (on < 1.0).any()
    finally:
        rctx.release_state(state)
        rctx.release_scene(sid)


def test_second_backward_and_partial_outputs(rctx):
    """A second backward on the same state gives the same gradients; asking
    for the weights alone gives the same weights."""
    sc = synth.neural_scene(n_cells=120, K=3, F=6, H=8, seed=21, box=0.5, axes_lo=0.15, axes_hi=0.4)
    from oracle import decode as odec
    P = odec.packed_size(6, 8, 3)
    cams = [synth.small_camera(40, 32)]
    sid = rctx.upload_scene(sc)
    flat, state, _ = rctx.render(sid, cams, want_state=True)
    dl = torch.randn(flat.numel(), generator=torch.Generator().manual_seed(3)).cuda()
    try:
        a = dict(g_mlp=torch.zeros(P, device="cuda"), g_feat=torch.zeros(sc.N, 6, device="cuda"),
                 g_offset=torch.zeros(sc.G, 3, device="cuda"), g_cell_v=torch.zeros(sc.N, device="cuda"))
        rctx.backward(state, dl, a)
        b = dict(g_mlp=torch.zeros(P, device="cuda"))
        rctx.backward(state, dl, b)
        torch.cuda.synchronize()
        assert a["g_mlp"].abs().max() > 0 and a["g_cell_v"].abs().max() > 0
        assert torch.allclose(a["g_mlp"], b["g_mlp"], rtol=1e-5, atol=1e-6 * float(a["g_mlp"].abs().max()))
    finally:
        rctx.release_state(state)
        rctx.release_scene(sid)
