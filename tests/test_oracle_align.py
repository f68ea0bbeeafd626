"""Pins of the oracle's cell alignment (Sec. IV-B: Eq. 10 and the centre
update):

* a hand-computed two-Gaussian cell: stored quaternions of different
  lengths, opacities 3/4 and 1/4, so Q = (3, 1, 0, 0) / sqrt(10) exactly
  (fails if the weights, the normalisation of q or of the sum is dropped),
  and the centre is the midpoint;
* identical rotations give that rotation whatever the opacities;
* a zero weighted sum (q and -q with equal opacity) keeps the old Q_n;
* neural cells: offsets in +/- pairs leave the centre where it is; a
  decoder with zero weights and per-Gaussian biases gives the closed form of
  Eq. 10 with tanh opacities, a Gaussian with sigma <= 0 weighted 0;
* brute force: explicit loops over a random explicit and a random neural
  scene.
"""
import dataclasses
import math

import numpy as np

import oracle
from oracle import decode as odec
from paper_2508_03180_gb300 import synth


def _explicit(N=5, K=2, seed=0):
    sc = synth.make_scene(N, K, synth._box(-1.0, 1.0), 0.05, 0.2, 0, seed=seed)
    return sc


def test_two_gaussians_by_hand():
    sc = _explicit(N=1, K=2)
    q = np.array([[2.0, 0.0, 0.0, 0.0], [0.0, 3.0, 0.0, 0.0]], np.float32)
    logit = np.array([math.log(3.0), -math.log(3.0)], np.float32)  # sigma 3/4, 1/4
    mean = np.array([[1.0, 2.0, 3.0], [3.0, -2.0, 5.0]], np.float32)
    sc = dataclasses.replace(sc, g_quat=q, g_logit=logit, g_mean=mean)
    x, Q = oracle.cell_align(sc)
    lo = 1.0 / (1.0 + math.exp(-float(logit[0])))
    np.testing.assert_allclose(Q[0], np.array([3.0, 1.0, 0.0, 0.0]) / math.sqrt(10.0), atol=1e-7)
    assert abs(lo - 0.75) < 1e-7
    np.testing.assert_allclose(x[0], [2.0, 0.0, 4.0], atol=1e-12)


def test_identical_rotations():
    sc = _explicit(N=4, K=3, seed=2)
    r = synth.random_unit_quats(np.random.default_rng(1), 4)
    q = np.repeat(r, 3, axis=0) * np.linspace(0.5, 2.0, 12)[:, None]
    sc = dataclasses.replace(sc, g_quat=q.astype(np.float32))
    _, Q = oracle.cell_align(sc)
    np.testing.assert_allclose(Q, r.astype(np.float32).astype(np.float64) / np.linalg.norm(
        r.astype(np.float32).astype(np.float64), axis=1, keepdims=True), atol=1e-7)


def test_zero_sum_keeps_the_cell_rotation():
    sc = _explicit(N=1, K=2, seed=3)
    q = np.array([[0.5, 0.5, 0.5, 0.5], [-0.5, -0.5, -0.5, -0.5]], np.float32)
    sc = dataclasses.replace(sc, g_quat=q, g_logit=np.zeros(2, np.float32))
    _, Q = oracle.cell_align(sc)
    np.testing.assert_array_equal(Q, sc.cell_quat.astype(np.float64))


def test_neural_symmetric_offsets_keep_the_centre():
    sc = synth.neural_scene(n_cells=6, K=4, F=5, H=4, seed=8)
    off = sc.neural["offset"].reshape(6, 4, 3).copy()
    off[:, 2:] = -off[:, :2]
    sc = dataclasses.replace(sc, neural=dict(sc.neural, offset=off.reshape(-1, 3).astype(np.float32)))
    x, _ = oracle.cell_align(sc, synth.small_camera(16, 16).as_array())
    np.testing.assert_allclose(x, sc.cell_center.astype(np.float64), atol=1e-12)


def test_neural_constant_decoders_closed_form():
    sc = synth.neural_scene(n_cells=3, K=3, F=4, H=4, seed=9)
    F, H, K = 4, 4, 3
    mlp = np.zeros(odec.packed_size(F, H, K), np.float32)
    o = 0
    b_sig = np.array([0.8, -0.3, 0.2], np.float32)       # the second Gaussian is not drawn
    b_q = np.array([1, 0, 0, 0, 0, 2, 0, 0, 0, 0, 0, 5], np.float32)
    for i, n_out in enumerate(odec.out_widths(K)):
        o += H * (F + 4) + H + n_out * H
        if i == 0:
            mlp[o:o + n_out] = b_sig
        if i == 3:
            mlp[o:o + n_out] = b_q
        o += n_out
    sc = dataclasses.replace(sc, neural=dict(sc.neural, mlp=mlp))
    _, Q = oracle.cell_align(sc, synth.small_camera(16, 16).as_array())
    s0, s2 = math.tanh(0.8), math.tanh(0.2)
    want = np.array([s0, 0.0, 0.0, s2]) / math.hypot(s0, s2)
    for n in range(3):
        np.testing.assert_allclose(Q[n], want, atol=1e-6)


def test_brute_force_loops():
    sc = _explicit(N=7, K=3, seed=5)
    x, Q = oracle.cell_align(sc)
    for n in range(sc.N):
        cx, s = [0.0, 0.0, 0.0], [0.0, 0.0, 0.0, 0.0]
        for k in range(sc.K):
            g = n * sc.K + k
            for c in range(3):
                cx[c] += float(sc.g_mean[g, c]) / sc.K
            qq = [float(v) for v in sc.g_quat[g]]
            nq = math.sqrt(sum(v * v for v in qq))
            w = 1.0 / (1.0 + math.exp(-float(sc.g_logit[g])))
            for c in range(4):
                s[c] += w * qq[c] / nq
        ns = math.sqrt(sum(v * v for v in s))
        np.testing.assert_allclose(x[n], cx, atol=1e-12)
        np.testing.assert_allclose(Q[n], [v / ns for v in s], atol=1e-12)
    nsc = synth.neural_scene(n_cells=5, K=3, F=4, H=6, seed=12)
    cam = synth.small_camera(16, 16).as_array()
    x, Q = oracle.cell_align(nsc, cam)
    d = oracle.decode_view(nsc, cam)
    for n in range(nsc.N):
        cx = [sum(d["mean"][n, k, c] for k in range(3)) / 3 for c in range(3)]
        s = [sum(max(d["opac"][n, k], 0.0) * d["quat"][n, k, c] for k in range(3)) for c in range(4)]
        ns = math.sqrt(sum(v * v for v in s))
        np.testing.assert_allclose(x[n], cx, atol=1e-12)
        np.testing.assert_allclose(Q[n], [v / ns for v in s], atol=1e-12)
