"""dgs_render without stats is asynchronous on its stream (no host
synchronisation: the pair count and, for neural cells, the decode's sample
count stay on the device and the pair buffers are sized from the context's
pairs-per-tile estimate), gives exactly the image,
binning and gradients of the synchronising render (stats requested), and a
render whose pairs exceed the capacity is reported by the next call, after
which the capacity has grown and the render is exact again."""
import numpy as np
import pytest
import torch

import oracle
from paper_2508_03180_gb300 import _lib as L
from paper_2508_03180_gb300 import synth
from paper_2508_03180_gb300.renderer import Context

pytestmark = pytest.mark.gpu


def _grads(ctx, scene, state, dl):
    G, C = scene.G, (scene.sh_degree + 1) ** 2
    g = dict(g_mean=torch.zeros(G, 3, device="cuda"), g_log_scale=torch.zeros(G, 3, device="cuda"),
             g_quat=torch.zeros(G, 4, device="cuda"), g_logit=torch.zeros(G, device="cuda"),
             g_sh=torch.zeros(G, C, 3, device="cuda"))
    ctx.backward(state, dl, g)
    return g


def test_render_without_stats_returns_before_the_gpu_finishes():
    scene = synth.scene_multiscale(n_cells=40_000, K=10)
    cams = synth.sphere_cameras(8, 15.0, 1920, 1080, seed0=0)
    ctx = Context()
    try:
        sid = ctx.upload_scene(scene)
        ref, ref_state, st = ctx.render(sid, cams, want_state=True, stats=True)  # synchronising, exact sizes
        torch.cuda.synchronize()
        ctx.render(sid, cams)  # warm: the device-sized chain's buffers exist
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        img, state, _ = ctx.render(sid, cams, want_state=True)
        pending = not stream.query()
        torch.cuda.synchronize()
        assert pending, "the render returned only after its kernels had finished"
        assert torch.equal(img, ref)
        for what, dt in ((L.DGS_BUF_TILE_CELLS, np.uint32), (L.DGS_BUF_TILE_RANGES, np.uint32),
                         (L.DGS_BUF_PIX_NDONE, np.int32)):
            assert np.array_equal(ctx.read(state, what, dt), ctx.read(ref_state, what, dt))
        assert len(ctx.read(state, L.DGS_BUF_TILE_CELLS, np.uint32)) == st.sort_length
        dl = torch.randn(img.numel(), generator=torch.Generator().manual_seed(2)).cuda() * 1e-3
        ga, gb = _grads(ctx, scene, state, dl), _grads(ctx, scene, ref_state, dl)
        # the same backward again, three times: the float atomics' order varies from run to run
        again = [_grads(ctx, scene, ref_state, dl) for _ in range(3)]
        torch.cuda.synchronize()
        for k in ga:  # both states hold identical lists and counts: differences are the atomics' order only
            ref = gb[k].double()
            noise = max((g[k].double() - ref).norm() for g in again)
            assert (ga[k].double() - ref).norm() <= 4.0 * noise + 1e-4 * ref.norm(), k
        ctx.release_state(state)
        ctx.release_state(ref_state)
    finally:
        ctx.close()


def test_neural_render_without_stats_is_asynchronous_and_exact():
    """Neural cells: the decode reads the visible-cell count on the device,
    so the render of a neural scene is asynchronous too, and its decoded
    values, image, tile lists and gradients equal the synchronising path's."""
    from oracle import decode as odec
    F, H, K = 32, 32, 10
    scene = synth.neural_scene(n_cells=20_000, K=K, F=F, H=H, seed=4, box=1.0)
    cams = synth.sphere_cameras(8, 3.0, 1920, 1080, seed0=2)
    ctx = Context()
    try:
        sid = ctx.upload_scene(scene)
        ref, ref_state, st = ctx.render(sid, cams, want_state=True, stats=True)
        torch.cuda.synchronize()
        ctx.render(sid, cams)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        img, state, _ = ctx.render(sid, cams, want_state=True)
        pending = not stream.query()
        torch.cuda.synchronize()
        assert pending, "the neural render returned only after its kernels had finished"
        assert torch.equal(img, ref)
        for what, dt in ((L.DGS_BUF_TILE_CELLS, np.uint32), (L.DGS_BUF_PIX_NDONE, np.int32)):
            assert np.array_equal(ctx.read(state, what, dt), ctx.read(ref_state, what, dt))
        V = len(cams)
        vis = np.repeat(ctx.read(ref_state, L.DGS_BUF_CELL_RECT, np.int32, (V, scene.N, 4))[..., 0] >= 0, K, axis=1)
        assert vis.sum() > 1000
        dec = ctx.read(state, L.DGS_BUF_DECODED, np.float32, (V, scene.G, 14))
        dec_ref = ctx.read(ref_state, L.DGS_BUF_DECODED, np.float32, (V, scene.G, 14))
        assert np.array_equal(dec[vis], dec_ref[vis])  # decoded for the visible cells only
        P = odec.packed_size(F, H, K)
        dl = torch.randn(img.numel(), generator=torch.Generator().manual_seed(5)).cuda() * 1e-3

        def grads(s):
            g = dict(g_mlp=torch.zeros(P, device="cuda"), g_feat=torch.zeros(scene.N, F, device="cuda"),
                     g_offset=torch.zeros(scene.G, 3, device="cuda"))
            ctx.backward(s, dl, g)
            return g
        ga, gb = grads(state), grads(ref_state)
        again = [grads(ref_state) for _ in range(3)]
        torch.cuda.synchronize()
        for k in ga:
            ref_k = gb[k].double()
            noise = max((g[k].double() - ref_k).norm() for g in again)
            assert ref_k.abs().max() > 0, k
            assert (ga[k].double() - ref_k).norm() <= 4.0 * noise + 1e-4 * ref_k.norm(), k
        ctx.release_state(state)
        ctx.release_state(ref_state)
    finally:
        ctx.close()


def test_pair_overflow_is_reported_by_the_next_call_and_recovers():
    scene = synth.scene_small(n_cells=2048, sh_degree=1)
    far = synth.sphere_cameras(1, 40.0, 1280, 720, seed0=7)
    near = synth.sphere_cameras(4, 2.2, 1280, 720, seed0=7)
    ppt = lambda cams: sum(oracle.sort_length(scene, c.as_array()) for c in cams) / sum(
        oracle.grid(c.as_array())[2] * oracle.grid(c.as_array())[3] for c in cams)
    L_near = sum(oracle.sort_length(scene, c.as_array()) for c in near)
    T_near = sum(oracle.grid(c.as_array())[2] * oracle.grid(c.as_array())[3] for c in near)
    assert L_near > max(1 << 16, 1.5 * ppt(far) * T_near), "the near views must overflow the far views' capacity"
    ctx = Context()
    try:
        sid = ctx.upload_scene(scene)
        ctx.render(sid, far)  # the context's first render: synchronising, learns the far views' pairs per tile
        torch.cuda.synchronize()
        ctx.render(sid, near)  # device-sized: its pairs overflow the capacity
        torch.cuda.synchronize()
        with pytest.raises(L.DgsError) as ei:
            ctx.render(sid, near)
        assert ei.value.code == L.DGS_ERR_CAPACITY and "render it again" in str(ei.value)
        img, _, _ = ctx.render(sid, near)  # the capacity has grown
        ref, _, st = ctx.render(sid, near, stats=True)
        torch.cuda.synchronize()
        assert st.sort_length == L_near
        assert torch.equal(img, ref)
    finally:
        ctx.close()


def test_backward_of_an_overflowed_state_reports_it():
    """A state whose render overflowed the pair capacity: once its chain has
    completed, dgs_render_backward on it returns DGS_ERR_CAPACITY instead of
    gradients of the incomplete render."""
    scene = synth.scene_small(n_cells=2048, sh_degree=1)
    far = synth.sphere_cameras(1, 40.0, 1280, 720, seed0=7)
    near = synth.sphere_cameras(4, 2.2, 1280, 720, seed0=7)
    ctx = Context()
    try:
        sid = ctx.upload_scene(scene)
        ctx.render(sid, far)
        img, state, _ = ctx.render(sid, near, want_state=True)  # device-sized: overflows
        torch.cuda.synchronize()
        g = dict(g_mean=torch.zeros(scene.G, 3, device="cuda"))
        with pytest.raises(L.DgsError) as ei:
            ctx.backward(state, torch.ones_like(img), g)
        assert ei.value.code == L.DGS_ERR_CAPACITY
        ctx.release_state(state)
        img2, state2, _ = ctx.render(sid, near, want_state=True)  # the capacity has grown
        ctx.backward(state2, torch.ones_like(img2), g)
        torch.cuda.synchronize()
        assert g["g_mean"].abs().max() > 0
        ctx.release_state(state2)
    finally:
        ctx.close()
