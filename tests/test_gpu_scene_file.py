"""Scene files through the C ABI: dgs_scene_save writes the bytes the host
writer writes for the same scene (the stored planes transposed back to their
row-major layouts), dgs_scene_load of such a file renders bit for bit like
an upload of the scene itself, a save after an in-place update holds the
updated parameters, and files that are missing, truncated or of another
format are refused on the host with NOT_FOUND or INVALID_ARG."""
import numpy as np
import pytest
import torch

from paper_2508_03180_gb300 import _lib as L
from paper_2508_03180_gb300 import scene_file, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rctx():
    from paper_2508_03180_gb300.renderer import Context
    c = Context()
    yield c
    c.close()


def _scenes():
    yield synth.scene_small(seed=3, sh_degree=3, n_cells=1500, K=6)
    yield synth.with_view_dependent_v(synth.scene_small(seed=5, n_cells=1200, K=8), degree=2, seed=9)
    yield synth.neural_scene(n_cells=900, K=5, F=12, H=20, seed=2)


def _render(rctx, sid, cams):
    img, _, _ = rctx.render(sid, cams)
    torch.cuda.synchronize()
    return img.cpu().numpy()


@pytest.mark.parametrize("scene", list(_scenes()), ids=lambda s: s.name)
def test_save_matches_the_host_writer_and_load_renders_the_same(rctx, scene, tmp_path):
    cams = synth.sphere_cameras(2, 3.0, 200, 152, seed0=4)
    sid = rctx.upload_scene(scene)
    want = tmp_path / "host.dgs"
    got = tmp_path / "lib.dgs"
    scene_file.save(scene, want)
    rctx.save_scene(sid, got)
    assert got.read_bytes() == want.read_bytes()
    ref = _render(rctx, sid, cams)
    sid2 = rctx.load_scene(want)
    assert np.array_equal(_render(rctx, sid2, cams), ref)
    again = tmp_path / "again.dgs"
    rctx.save_scene(sid2, again)
    assert again.read_bytes() == want.read_bytes()
    rctx.release_scene(sid)
    rctx.release_scene(sid2)


def test_save_after_update_holds_the_new_parameters(rctx, tmp_path):
    scene = synth.scene_small(seed=8, n_cells=800, K=4)
    sid = rctx.upload_scene(scene)
    rng = np.random.default_rng(1)
    logit = rng.standard_normal(scene.G).astype(np.float32)
    mean = (scene.g_mean + 0.01 * rng.standard_normal(scene.g_mean.shape)).astype(np.float32)
    dev = {f: torch.from_numpy(np.ascontiguousarray(getattr(scene, f))).cuda()
           for f in ("g_scale", "g_quat", "g_sh")}
    rctx.update_scene(sid, scene.N, scene.K, scene.sh_degree, g_logit=torch.from_numpy(logit).cuda(),
                      g_mean=torch.from_numpy(mean).cuda(), **dev)
    torch.cuda.synchronize()
    p = tmp_path / "u.dgs"
    rctx.save_scene(sid, p)
    back = scene_file.load(p)
    assert back.g_logit.tobytes() == logit.tobytes()
    assert back.g_mean.tobytes() == mean.tobytes()
    assert back.g_sh.tobytes() == scene.g_sh.tobytes()
    rctx.release_scene(sid)


def test_bad_files_are_refused(rctx, tmp_path):
    scene = synth.scene_small(seed=0, n_cells=100, K=2)
    p = tmp_path / "s.dgs"
    scene_file.save(scene, p)
    raw = p.read_bytes()
    with pytest.raises(L.DgsError) as e:
        rctx.load_scene(tmp_path / "missing.dgs")
    assert e.value.code == L.DGS_ERR_NOT_FOUND
    for bad in (raw[:-4], raw + b"\0\0\0\0", b"DGS2" + raw[4:], raw[:30]):
        q = tmp_path / "bad.dgs"
        q.write_bytes(bad)
        with pytest.raises(L.DgsError) as e:
            rctx.load_scene(q)
        assert e.value.code == L.DGS_ERR_INVALID_ARG
    with pytest.raises(L.DgsError) as e:
        rctx.save_scene(12345, tmp_path / "x.dgs")
    assert e.value.code == L.DGS_ERR_NOT_FOUND
    # the context still renders after the refusals
    sid = rctx.load_scene(p)
    assert np.isfinite(_render(rctx, sid, [synth.small_camera(64, 48)])).all()
    rctx.release_scene(sid)
