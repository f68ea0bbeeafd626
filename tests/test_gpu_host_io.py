"""Host-memory arguments: page-locked host arrays are read and written by the
kernels over the host link, pageable ones are staged through device memory.
Both must give the results of device arrays: the same kernels run, only
where the bytes live differs.  Renders are compared bit for bit; gradients
to within the spread of the blend adjoint's atomic sums, whose order varies
from run to run (each run starts its outputs from a sentinel, so an element
left unwritten fails)."""
import numpy as np
import pytest
import torch

from paper_2508_03180_gb300 import _lib as L
from paper_2508_03180_gb300 import synth

pytestmark = pytest.mark.gpu

GFIELDS = ("g_mean", "g_scale", "g_quat", "g_logit", "g_sh")
OUTS = ("g_mean", "g_scale", "g_log_scale", "g_quat", "g_logit", "g_sh", "g_cell_v")


@pytest.fixture(scope="module")
def rctx():
    from paper_2508_03180_gb300.renderer import Context
    c = Context()
    yield c
    c.close()


def _out_shapes(scene):
    G, N, C = scene.G, scene.N, (scene.sh_degree + 1) ** 2
    return dict(g_mean=(G, 3), g_scale=(G, 3), g_log_scale=(G, 3), g_quat=(G, 4), g_logit=(G,), g_sh=(G, C, 3),
                g_cell_v=(N,))


def _grads_struct(arrays, location):
    g = L.dgs_grads()
    g.location = location
    for f, a in arrays.items():
        setattr(g, f, a.data_ptr() if isinstance(a, torch.Tensor) else a.ctypes.data)
    return g


def _same_grads(got, ref, label):
    for k in OUTS:
        scale = float(np.abs(ref[k]).max())
        np.testing.assert_allclose(got[k], ref[k], rtol=1e-4, atol=1e-4 * scale + 1e-9, err_msg=f"{label} {k}")


def _backward(rctx, state, dl_ptr, dl_loc, arrays, location):
    L.dgs_render_backward(rctx.ctx, state, dl_ptr, dl_loc, _grads_struct(arrays, location),
                          torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if isinstance(v, torch.Tensor) else v).copy() for k, v in arrays.items()}


def test_backward_host_outputs_match_device(rctx):
    scene = synth.scene_small(seed=4, sh_degree=3)
    cams = synth.sphere_cameras(2, 3.0, 200, 150, seed0=7)
    sid = rctx.upload_scene(scene)
    flat, state, _ = rctx.render(sid, cams, want_state=True)
    dl = torch.randn(flat.numel(), generator=torch.Generator().manual_seed(1)).cuda()
    shapes = _out_shapes(scene)
    dev = {k: torch.full(s, 7.0, device="cuda") for k, s in shapes.items()}
    ref = _backward(rctx, state, dl.data_ptr(), L.DGS_DEVICE, dev, L.DGS_DEVICE)
    assert any(np.abs(ref[k]).max() > 0 for k in OUTS)
    # page-locked host outputs (written by the kernels directly), then pageable ones (staged)
    pinned = {k: torch.full(s, 7.0).pin_memory() for k, s in shapes.items()}
    got = _backward(rctx, state, dl.data_ptr(), L.DGS_DEVICE, pinned, L.DGS_HOST)
    _same_grads(got, ref, "pinned")
    pageable = {k: np.full(s, 7.0, np.float32) for k, s in shapes.items()}
    got = _backward(rctx, state, dl.data_ptr(), L.DGS_DEVICE, pageable, L.DGS_HOST)
    _same_grads(got, ref, "pageable")
    # dL/drgb in page-locked host memory (read by the blend adjoint directly) and pageable
    dl_pin = dl.cpu().pin_memory()
    got = _backward(rctx, state, dl_pin.data_ptr(), L.DGS_HOST, dev, L.DGS_DEVICE)
    _same_grads(got, ref, "pinned dL")
    dl_np = dl.cpu().numpy().copy()
    got = _backward(rctx, state, dl_np.ctypes.data, L.DGS_HOST, pinned, L.DGS_HOST)
    _same_grads(got, ref, "pageable dL, pinned outputs")
    # outputs that are views into one page-locked buffer (pointers inside an allocation)
    flat = torch.full((sum(int(np.prod(v)) for v in shapes.values()) + 1,), 7.0).pin_memory()
    views, o = {}, 1  # start one float in, so no output begins at the allocation's base
    for k, shp in shapes.items():
        n = int(np.prod(shp))
        views[k] = flat[o:o + n].view(shp)
        o += n
    got = _backward(rctx, state, dl.data_ptr(), L.DGS_DEVICE, views, L.DGS_HOST)
    _same_grads(got, ref, "views of one pinned buffer")
    assert flat[0].item() == 7.0  # nothing written outside the outputs
    rctx.release_state(state)
    rctx.release_scene(sid)


def _update(rctx, sid, scene, arrays, location):
    d = L.dgs_scene_desc()
    d.num_cells, d.K, d.sh_degree, d.location = scene.N, scene.K, scene.sh_degree, location
    for f, a in arrays.items():
        setattr(d, f, a.data_ptr() if isinstance(a, torch.Tensor) else a.ctypes.data)
    L.dgs_scene_update(rctx.ctx, sid, d, torch.cuda.current_stream().cuda_stream)


def test_scene_update_host_sources_match_device(rctx):
    scene = synth.scene_small(seed=5, sh_degree=3)
    other = synth.scene_small(seed=6, sh_degree=3)  # same sizes, other parameters
    cams = synth.sphere_cameras(2, 3.0, 160, 120, seed0=9)
    sid = rctx.upload_scene(scene)
    src = {f: np.ascontiguousarray(getattr(other, f), dtype=np.float32) for f in GFIELDS}
    _update(rctx, sid, other, {f: torch.from_numpy(a).cuda() for f, a in src.items()}, L.DGS_DEVICE)
    ref = rctx.render(sid, cams)[0].cpu().numpy()
    first = {f: np.ascontiguousarray(getattr(scene, f), dtype=np.float32) for f in GFIELDS}
    for label, arrays in (("pinned", {f: torch.from_numpy(a).pin_memory() for f, a in src.items()}),
                          ("pageable", src)):
        _update(rctx, sid, scene, first, L.DGS_HOST)  # back to the first parameters
        assert not np.array_equal(rctx.render(sid, cams)[0].cpu().numpy(), ref)
        _update(rctx, sid, other, arrays, L.DGS_HOST)
        got, _, _ = rctx.render(sid, cams)
        np.testing.assert_array_equal(got.cpu().numpy(), ref, err_msg=label)
    rctx.release_scene(sid)
