"""Pins of the oracle's neural-cell decode (the MLP step before the path):

* brute force: every output of a tiny decode recomputed with explicit
  Python loops over the packed weights (checks packing order, transposes
  and reshapes of the vectorised code);
* constant decoders (W1 = W2 = 0): every activation's closed form, with
  distinct biases per decoder so a swapped decoder or channel fails;
* every Gaussian centre lies inside its cell ellipsoid, and the scale ratio
  obeys Eq. 11;
* the view direction enters only through its input columns, the distance
  only through its own;
* gradients of a rendered loss through the decode (autograd of the FP64
  decode and projection) match FP64 central differences.
"""
import math

import numpy as np

import oracle
from oracle import decode as odec
from paper_2508_03180_gb300 import synth


def _tiny(seed=0, K=3, F=5, H=4, N=6):
    return synth.neural_scene(n_cells=N, K=K, F=F, H=H, seed=seed)


def _quat_rot(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_brute_force_loops():
    sc = _tiny()
    K, F, H = sc.K, sc.neural["F"], sc.neural["H"]
    eye = np.array([0.3, -2.5, 0.4])
    d = oracle.decode_view(sc, np.r_[np.zeros(19), eye].astype(np.float32))
    w = sc.neural["mlp"].astype(np.float64)
    sig = lambda t: 1.0 / (1.0 + math.exp(-t))
    for n in range(sc.N):
        x = sc.cell_center[n].astype(np.float64)
        rel = x - eye.astype(np.float32).astype(np.float64)
        dist = math.sqrt(sum(r * r for r in rel))
        z = list(sc.neural["feat"][n].astype(np.float64)) + [dist] + [r / dist for r in rel]
        o, outs = 0, []
        for n_out in (K, 3 * K, 3 * K, 4 * K):
            h = []
            for j in range(H):
                a = w[o + H * (F + 4) + j]
                for i in range(F + 4):
                    a += w[o + j * (F + 4) + i] * z[i]
                h.append(max(a, 0.0))
            o2 = o + H * (F + 4) + H
            vals = []
            for r in range(n_out):
                a = w[o2 + n_out * H + r]
                for j in range(H):
                    a += w[o2 + r * H + j] * h[j]
                vals.append(a)
            outs.append(vals)
            o = o2 + n_out * H + n_out
        S = sc.cell_axes[n].astype(np.float64)
        R = _quat_rot(sc.cell_quat[n].astype(np.float64))
        for k in range(K):
            assert abs(d["opac"][n, k] - math.tanh(outs[0][k])) < 1e-12
            for c in range(3):
                assert abs(d["rgb"][n, k, c] - sig(outs[1][3 * k + c])) < 1e-12
            off = sc.neural["offset"][n * K + k].astype(np.float64)
            off = off / max(1.0, float(np.linalg.norm(off)))
            lim = 1.0 - float(np.linalg.norm(off))
            for c in range(3):
                assert abs(d["scale"][n, k, c] - min(sig(outs[2][3 * k + c]), lim) * S[c]) < 1e-12
            q = np.array(outs[3][4 * k:4 * k + 4])
            assert np.allclose(d["quat"][n, k], q / np.linalg.norm(q), atol=1e-12)
            assert np.allclose(d["mean"][n, k], x + R @ (off * S), atol=1e-12)


def test_constant_decoders_closed_forms():
    sc = _tiny(seed=1)
    K, F, H = sc.K, sc.neural["F"], sc.neural["H"]
    mlp = np.zeros(odec.packed_size(F, H, K), dtype=np.float32)
    o, biases = 0, []
    for i, n_out in enumerate(odec.out_widths(K)):
        o += H * (F + 4) + H + n_out * H
        b = (0.1 * (i + 1) + 0.05 * np.arange(n_out)).astype(np.float32)
        mlp[o:o + n_out] = b
        biases.append(b.astype(np.float64))
        o += n_out
    sc.neural = dict(sc.neural, mlp=mlp)
    d = oracle.decode_view(sc, synth.small_camera(16, 16).as_array())
    off = sc.neural["offset"].astype(np.float64).reshape(sc.N, K, 3)
    off = off / np.maximum(1.0, np.linalg.norm(off, axis=2, keepdims=True))
    lim = 1.0 - np.linalg.norm(off, axis=2, keepdims=True)
    np.testing.assert_allclose(d["opac"], np.tanh(biases[0])[None, :].repeat(sc.N, 0), atol=1e-12)
    np.testing.assert_allclose(d["rgb"], (1 / (1 + np.exp(-biases[1]))).reshape(1, K, 3).repeat(sc.N, 0), atol=1e-12)
    ratio = np.minimum((1 / (1 + np.exp(-biases[2]))).reshape(1, K, 3), lim)
    np.testing.assert_allclose(d["scale"], ratio * sc.cell_axes[:, None, :].astype(np.float64), atol=1e-12)
    q = biases[3].reshape(K, 4)
    np.testing.assert_allclose(d["quat"], (q / np.linalg.norm(q, axis=1, keepdims=True))[None].repeat(sc.N, 0),
                               atol=1e-12)


def test_centres_inside_cells_and_eq11():
    sc = synth.neural_scene(n_cells=200, K=6, F=8, H=8, seed=3)
    sc.neural["offset"][:] *= 1.7  # some offsets outside the unit ball before the projection onto it
    d = oracle.decode_view(sc, synth.small_camera(16, 16).as_array())
    for n in range(sc.N):
        R = _quat_rot(sc.cell_quat[n].astype(np.float64))
        local = (R.T @ (d["mean"][n] - sc.cell_center[n].astype(np.float64)).T).T / sc.cell_axes[n]
        assert np.all(np.linalg.norm(local, axis=1) <= 1.0 + 1e-12)
        ratio = d["scale"][n] / sc.cell_axes[n].astype(np.float64)
        assert np.all(ratio <= (1.0 - np.linalg.norm(local, axis=1))[:, None] + 1e-12)


def test_view_inputs():
    sc = _tiny(seed=2, N=10)
    K, F, H = sc.K, sc.neural["F"], sc.neural["H"]
    sc.cell_center[:] = 0.0
    mlp = sc.neural["mlp"].copy()
    o = 0
    for n_out in odec.out_widths(K):
        W1 = mlp[o:o + H * (F + 4)].reshape(H, F + 4)
        W1[:, F + 1:] = 0.0  # no direction input
        o += H * (F + 4) + H + n_out * H + n_out
    a = oracle.decode_view(dict_scene(sc, mlp), synth.look_at((0, -3, 0), (0, 0, 0), 8, 8).as_array())
    b = oracle.decode_view(dict_scene(sc, mlp), synth.look_at((3, 0, 0), (0, 0, 0), 8, 8).as_array())
    c = oracle.decode_view(dict_scene(sc, mlp), synth.look_at((5, 0, 0), (0, 0, 0), 8, 8).as_array())
    full_a = oracle.decode_view(sc, synth.look_at((0, -3, 0), (0, 0, 0), 8, 8).as_array())
    full_b = oracle.decode_view(sc, synth.look_at((3, 0, 0), (0, 0, 0), 8, 8).as_array())
    for k in ("opac", "rgb", "scale", "quat"):
        np.testing.assert_allclose(a[k], b[k], atol=1e-12)           # same distance, other direction
        assert np.abs(a[k] - c[k]).max() > 1e-6                       # other distance
        assert np.abs(full_a[k] - full_b[k]).max() > 1e-6             # the direction does enter


def dict_scene(sc, mlp):
    import dataclasses
    return dataclasses.replace(sc, neural=dict(sc.neural, mlp=mlp))


def test_neural_gradients_match_central_differences():
    """dL/d(weights, features, offsets) of a rendered loss through the decode,
    against FP64 central differences with the decisions held fixed."""
    import dataclasses
    sc = synth.neural_scene(n_cells=24, K=3, F=6, H=5, seed=11, box=0.5, axes_lo=0.15, axes_hi=0.4)
    cam = synth.small_camera(24, 24).as_array()
    g = np.random.default_rng(5).standard_normal((3, 24, 24))
    img, an = oracle.neural_render_and_grad(sc, cam, g)
    nd = img["ndone"]
    dec = oracle.decode_view(sc, cam)
    decided = tuple(dec[k].reshape(sc.G, -1).astype(np.float32) for k in ("mean", "scale", "quat"))

    def loss(s2):
        im, _ = oracle.neural_render_and_grad(s2, cam, g, decided=decided, ndone=nd)
        return float((im["C"] * g).sum())

    rng = np.random.default_rng(0)
    h = 1e-6
    checked = 0
    for key, arr in (("mlp", sc.neural["mlp"]), ("feat", sc.neural["feat"]), ("offset", sc.neural["offset"])):
        a = an[key].reshape(-1)
        cand = np.nonzero(np.abs(a) > 1e-4 * np.abs(a).max())[0]
        assert len(cand) >= 5, key
        for i in rng.choice(cand, 6, replace=False):
            vals = []
            for s in (+1, -1):
                pert = arr.astype(np.float64).copy().reshape(-1)
                pert[i] += s * h
                s2 = dataclasses.replace(sc, neural=dict(sc.neural, **{key: pert.reshape(arr.shape)}))
                vals.append(loss(s2))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - a[i]) <= 1e-6 * np.abs(a).max() + 1e-9, (key, i, fd, a[i])
            checked += 1
    assert checked == 18


def test_zero_rotation_output_is_the_identity():
    """All weights and the rotation decoder's biases zero: every rotation
    output is exactly zero and decodes to (1, 0, 0, 0); its gradient is zero
    and finite, while the other decoders' gradients stay finite."""
    sc = _tiny(seed=4)
    K, F, H = sc.K, sc.neural["F"], sc.neural["H"]
    mlp = np.zeros(odec.packed_size(F, H, K), dtype=np.float32)
    o = 0
    for i, n_out in enumerate(odec.out_widths(K)):
        o += H * (F + 4) + H + n_out * H
        if i < 3:
            mlp[o:o + n_out] = 0.3
        o += n_out
    import dataclasses
    sc = dataclasses.replace(sc, neural=dict(sc.neural, mlp=mlp))
    eye = synth.small_camera(16, 16).as_array()[19:22]
    d = odec.decode_t(sc.neural, sc.cell_center, sc.cell_axes, sc.cell_quat, K, eye, requires_grad=True)
    np.testing.assert_array_equal(d["quat"].detach().numpy(), np.tile([1.0, 0.0, 0.0, 0.0], (sc.N, K, 1)))
    loss = d["quat"].sum() + d["opac"].sum() + d["scale"].sum()
    g, = __import__("torch").autograd.grad(loss, [d["leaves"]["mlp"]])
    g = g.numpy()
    assert np.isfinite(g).all()
    o_rot = sum(H * (F + 4) + H + n * H + n for n in odec.out_widths(K)[:3])
    assert np.all(g[o_rot:] == 0.0)       # the rotation decoder gets nothing
    assert np.abs(g[:o_rot]).max() > 0.0  # the others do


def test_neural_cell_gradients_match_central_differences():
    """dL/d of the cells' centres, semi-axes and quaternions through the
    decode (decoder inputs delta_n and d_n, the centres x_n + R(Q_n)(O_pos S_n),
    the scales ratio S_n) against FP64 central differences, with the decode's
    decisions and the cells' footprints held fixed."""
    import dataclasses
    sc = synth.neural_scene(n_cells=24, K=3, F=6, H=5, seed=12, box=0.5, axes_lo=0.15, axes_hi=0.4)
    cam = synth.small_camera(24, 24).as_array()
    g = np.random.default_rng(7).standard_normal((3, 24, 24))
    img, an = oracle.neural_render_and_grad(sc, cam, g)
    nd = img["ndone"]
    dec = oracle.decode_view(sc, cam)
    decided = tuple(dec[k].reshape(sc.G, -1).astype(np.float32) for k in ("mean", "scale", "quat"))
    rect0, _ = oracle.cell_rects(sc, cam)

    def loss(s2):
        assert np.array_equal(oracle.cell_rects(s2, cam)[0], rect0), "a footprint moved"
        im, _ = oracle.neural_render_and_grad(s2, cam, g, decided=decided, ndone=nd)
        return float((im["C"] * g).sum())

    rng = np.random.default_rng(1)
    h = 1e-6
    for key in ("cell_center", "cell_axes", "cell_quat"):
        arr = getattr(sc, key)
        a = an[key].reshape(-1)
        cand = np.nonzero(np.abs(a) > 1e-4 * np.abs(a).max())[0]
        assert len(cand) >= 5, key
        for i in rng.choice(cand, 6, replace=False):
            vals = []
            for s in (+1, -1):
                pert = arr.astype(np.float64).copy().reshape(-1)
                pert[i] += s * h
                vals.append(loss(dataclasses.replace(sc, **{key: pert.reshape(arr.shape)})))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - a[i]) <= 1e-6 * np.abs(a).max() + 1e-9, (key, i, fd, a[i])
