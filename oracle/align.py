"""FP64 cell alignment for the oracle -- TEST INFRASTRUCTURE ONLY.  Plain
NumPy / PyTorch CPU float64; shares no code with the CUDA path.

Sec. IV-B keeps each cell aligned with the Gaussians it emits:

* rotation (Eq. 10)  Q_n = norm( sum_k sigma_{n,k} q_{n,k} )
* centre             x_n = (1/K) sum_k mu_{n,k}

Readings:

* q_{n,k} is the Gaussian's unit quaternion (the rotation it denotes), so
  the weights are the opacities alone; quaternions are summed as stored
  (q and -q, the same rotation, are not brought to one hemisphere: the
  equation sums them as they are).
* explicit Gaussians: sigma = sigmoid(logit), q = g_quat / |g_quat|,
  mu = g_mean.  Neural cells: sigma and q decoded for one eye position
  (both depend on the view), a Gaussian with sigma <= 0 (not drawn)
  weighted 0; mu = x_n + R(Q_n)(O_pos * S_n) does not depend on the view.
* a cell whose weighted sum is the zero vector keeps its Q_n.
* both updates read the values from before the call.
"""
from __future__ import annotations

import numpy as np


def _unit(q):
    q = np.asarray(q, dtype=np.float64)
    return q / np.linalg.norm(q, axis=-1, keepdims=True)


def align(scene, eye=None):
    """New (centre (N,3), quaternion (N,4)) of every cell, float64."""
    N, K = scene.N, scene.K
    if getattr(scene, "neural", None) is not None:
        from . import decode as _decode
        e = np.zeros(3) if eye is None else np.asarray(eye, dtype=np.float64)
        d = _decode.decode64(scene.neural, scene.cell_center, scene.cell_axes, scene.cell_quat, K, e)
        mu = d["mean"]                                       # (N,K,3)
        q = d["quat"]                                        # unit already
        sigma = np.maximum(d["opac"], 0.0)                   # (N,K)
    else:
        mu = np.asarray(scene.g_mean, dtype=np.float64).reshape(N, K, 3)
        q = _unit(np.asarray(scene.g_quat, dtype=np.float64).reshape(N, K, 4))
        sigma = 1.0 / (1.0 + np.exp(-np.asarray(scene.g_logit, dtype=np.float64).reshape(N, K)))
    centre = mu.sum(axis=1) / K
    s = (q * sigma[:, :, None]).sum(axis=1)                  # (N,4)
    n = np.linalg.norm(s, axis=1, keepdims=True)
    old = np.asarray(scene.cell_quat, dtype=np.float64)
    quat = np.where(n > 0, s / np.where(n > 0, n, 1.0), old)
    return centre, quat
