"""Scene files on the host: the byte layout of the header, a bit-exact round
trip of explicit, view-dependent-v and neural scenes, and rejection of files
whose header or length is wrong.  No GPU."""
import struct

import numpy as np
import pytest

import oracle.decode
from paper_2508_03180_gb300 import scene_file, synth

ARRAYS = ("cell_center", "cell_axes", "cell_quat", "cell_v", "g_mean", "g_scale", "g_quat", "g_logit", "g_sh")


def _scenes():
    yield synth.scene_small(seed=3, sh_degree=3, n_cells=300, K=6)
    yield synth.with_view_dependent_v(synth.scene_small(seed=5, n_cells=200, K=4), degree=2, seed=9)
    yield synth.neural_scene(n_cells=150, K=5, F=12, H=20, seed=2)


def _same(a, b):
    assert (a.N, a.K, a.sh_degree, a.v_sh_degree) == (b.N, b.K, b.sh_degree, b.v_sh_degree)
    for f in ARRAYS if a.neural is None else ARRAYS[:4]:
        x, y = getattr(a, f), getattr(b, f)
        assert x.shape == y.shape and x.dtype == y.dtype == np.float32, f
        assert x.tobytes() == y.tobytes(), f
    assert (a.cell_v_sh is None) == (b.cell_v_sh is None)
    if a.cell_v_sh is not None:
        assert a.cell_v_sh.tobytes() == b.cell_v_sh.tobytes()
    assert (a.neural is None) == (b.neural is None)
    if a.neural is not None:
        assert (a.neural["F"], a.neural["H"]) == (b.neural["F"], b.neural["H"])
        for k in ("feat", "offset", "mlp"):
            assert a.neural[k].tobytes() == b.neural[k].tobytes(), k


@pytest.mark.parametrize("scene", list(_scenes()), ids=lambda s: s.name)
def test_round_trip_is_bit_exact(scene, tmp_path):
    p = tmp_path / "s.dgs"
    scene_file.save(scene, p)
    _same(scene, scene_file.load(p))


def test_header_layout(tmp_path):
    s = synth.with_view_dependent_v(synth.scene_small(seed=1, sh_degree=2, n_cells=70, K=3), degree=1)
    p = tmp_path / "s.dgs"
    scene_file.save(s, p)
    raw = p.read_bytes()
    assert raw[:4] == b"DGS1"
    assert struct.unpack_from("<I", raw, 4)[0] == 1
    assert struct.unpack_from("<q", raw, 8)[0] == 70
    assert struct.unpack_from("<5i", raw, 16) == (3, 2, 1, 0, 0)
    assert struct.unpack_from("<I", raw, 36)[0] == 0
    # header, then the arrays in order: the first float is cell 0's centre x,
    # the last ones are the view-dependent v of the last cell
    assert struct.unpack_from("<f", raw, 40)[0] == s.cell_center[0, 0]
    assert np.frombuffer(raw[-16:], "<f4").tolist() == s.cell_v_sh[-1].tolist()
    G = 70 * 3
    assert len(raw) == 40 + 4 * (70 * 11 + G * (11 + 9 * 3) + 70 * 4)


def test_packed_decoder_size_matches_the_oracle():
    for K, F, H in ((5, 12, 20), (10, 32, 32), (1, 1, 1), (16, 64, 64)):
        assert scene_file.mlp_weights(K, F, H) == oracle.decode.packed_size(F, H, K)
    s = synth.neural_scene(n_cells=10, K=7, F=9, H=11)
    assert s.neural["mlp"].size == scene_file.mlp_weights(7, 9, 11)


def test_bad_files_are_rejected(tmp_path):
    s = synth.scene_small(seed=0, n_cells=50, K=2)
    p = tmp_path / "s.dgs"
    scene_file.save(s, p)
    raw = p.read_bytes()
    for bad in (raw[:-4], raw + b"\0\0\0\0", b"DGS2" + raw[4:], raw[:4] + struct.pack("<I", 2) + raw[8:], raw[:20]):
        q = tmp_path / "bad.dgs"
        q.write_bytes(bad)
        with pytest.raises(ValueError):
            scene_file.load(q)
