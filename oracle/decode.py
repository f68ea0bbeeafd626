"""FP64 decode of neural cells into Gaussians for the oracle -- TEST
INFRASTRUCTURE ONLY.  Plain PyTorch CPU float64 ops; shares no code with the
CUDA path.

The paper decodes the K Gaussians of every visible cell from the cell's
latent feature f_n, viewing distance delta_n and direction d_n with shared
MLPs F_sigma, F_c, F_s, F_q (Sec. III, Eq. 1-7; Sec. IV-A, Eq. 8-11).  It
names their activations but not their shape.  Readings:

* input            z = [f_n, delta_n, d_n], delta_n = |x_n - eye|, d_n = (x_n - eye) / delta_n
* every decoder    h = relu(W1 z + b1), o = W2 h + b2 (one hidden layer of width H)
* opacity          sigma_{n,k} = tanh(o_sigma[k]); a Gaussian with sigma <= 0 is not drawn
* colour           c_{n,k} = sigmoid(o_c[3k .. 3k+2])
* scale            ratio = min(sigmoid(o_s[3k .. 3k+2]), 1 - |O_pos|)   (Eq. 11),
                   s_{n,k} = ratio * S_n                                 (Eq. 8)
* rotation         q_{n,k} = o_q[4k .. 4k+3] / |o_q[4k .. 4k+3]|; an output of exactly zero
                   (no direction to normalise) is the identity rotation (1, 0, 0, 0)
* position         mu_{n,k} = x_n + R(Q_n) (O_pos * S_n), O_pos moved into the unit ball
                   (O / max(1, |O|)): the offset is taken in the cell's frame, so the
                   Gaussian centre lies inside the cell ellipsoid (Sec. IV-A)

Weights are packed decoder after decoder (opacity, colour, scale, rotation
with output widths K, 3K, 3K, 4K): W1 [H][F+4] row-major, b1 [H], W2 [out][H]
row-major, b2 [out].
"""
from __future__ import annotations

import numpy as np
import torch

from .project import quat_to_rotmat

DECODERS = ("opacity", "colour", "scale", "rotation")


def out_widths(K: int):
    return (K, 3 * K, 3 * K, 4 * K)


def unpack(mlp, F: int, H: int, K: int):
    """[(W1, b1, W2, b2)] per decoder, float64 tensors."""
    w = torch.as_tensor(np.asarray(mlp, dtype=np.float64))
    out, o = [], 0
    for n_out in out_widths(K):
        W1 = w[o:o + H * (F + 4)].reshape(H, F + 4); o += H * (F + 4)
        b1 = w[o:o + H]; o += H
        W2 = w[o:o + n_out * H].reshape(n_out, H); o += n_out * H
        b2 = w[o:o + n_out]; o += n_out
        out.append((W1, b1, W2, b2))
    assert o == w.numel(), (o, w.numel())
    return out


def unpack_t(w, F: int, H: int, K: int):
    """unpack() of a float64 tensor (keeps its autograd graph)."""
    out, o = [], 0
    for n_out in out_widths(K):
        W1 = w[o:o + H * (F + 4)].reshape(H, F + 4); o += H * (F + 4)
        b1 = w[o:o + H]; o += H
        W2 = w[o:o + n_out * H].reshape(n_out, H); o += n_out * H
        b2 = w[o:o + n_out]; o += n_out
        out.append((W1, b1, W2, b2))
    assert o == w.numel(), (o, w.numel())
    return out


def packed_size(F: int, H: int, K: int) -> int:
    return sum(H * (F + 4) + H + n * H + n for n in out_widths(K))


def decode64(neural: dict, cell_center, cell_axes, cell_quat, K: int, eye):
    """Gaussians of every cell for one eye position.  Returns float64 numpy
    arrays: mean (N,K,3), scale (N,K,3), quat (N,K,4), opac (N,K), rgb (N,K,3)."""
    out = decode_t(neural, cell_center, cell_axes, cell_quat, K, eye)
    return {k: v.detach().numpy() for k, v in out.items() if k in ("mean", "scale", "quat", "opac", "rgb")}


def decode_t(neural: dict, cell_center, cell_axes, cell_quat, K: int, eye, requires_grad: bool = False):
    """decode64 as torch float64 tensors; with requires_grad the leaves
    (out["leaves"]: mlp, feat, offset, and the cells' cell_center,
    cell_axes, cell_quat) carry gradients."""
    F, H = neural["F"], neural["H"]
    x = torch.tensor(np.asarray(cell_center, dtype=np.float64), requires_grad=requires_grad)
    S = torch.tensor(np.asarray(cell_axes, dtype=np.float64), requires_grad=requires_grad)
    Qc = torch.tensor(np.asarray(cell_quat, dtype=np.float64), requires_grad=requires_grad)
    N = x.shape[0]
    leaves = dict(cell_center=x, cell_axes=S, cell_quat=Qc,
                  mlp=torch.tensor(np.asarray(neural["mlp"], dtype=np.float64), requires_grad=requires_grad),
                  feat=torch.tensor(np.asarray(neural["feat"], dtype=np.float64).reshape(N, F),
                                    requires_grad=requires_grad),
                  offset=torch.tensor(np.asarray(neural["offset"], dtype=np.float64).reshape(N, K, 3),
                                      requires_grad=requires_grad))
    f, off = leaves["feat"], leaves["offset"]
    e = torch.as_tensor(np.asarray(eye, dtype=np.float64))
    rel = x - e[None, :]
    delta = torch.linalg.norm(rel, dim=1, keepdim=True)
    z = torch.cat([f, delta, rel / delta], dim=1)                   # (N, F+4)
    outs = []
    for W1, b1, W2, b2 in unpack_t(leaves["mlp"], F, H, K):
        h = torch.relu(z @ W1.T + b1)
        outs.append(h @ W2.T + b2)
    o_sig, o_col, o_sc, o_q = outs
    opac = torch.tanh(o_sig)                                        # (N, K)
    rgb = torch.sigmoid(o_col).reshape(N, K, 3)
    on = torch.linalg.norm(off, dim=2, keepdim=True)
    off_b = off / torch.clamp_min(on, 1.0)                          # into the unit ball
    ratio = torch.minimum(torch.sigmoid(o_sc).reshape(N, K, 3), 1.0 - torch.linalg.norm(off_b, dim=2, keepdim=True))
    scale = ratio * S[:, None, :]
    q = o_q.reshape(N, K, 4)
    qn = torch.linalg.norm(q, dim=2, keepdim=True)
    ident = torch.tensor([1.0, 0.0, 0.0, 0.0], dtype=torch.float64).expand_as(q)
    quat = torch.where(qn > 0, q / torch.where(qn > 0, qn, torch.ones_like(qn)), ident)
    Rc = quat_to_rotmat(Qc)  # (N,3,3), Q_n normalised
    local = off_b * S[:, None, :]
    mean = x[:, None, :] + torch.einsum("nij,nkj->nki", Rc, local)
    return dict(mean=mean, scale=scale, quat=quat, opac=opac, rgb=rgb, leaves=leaves)
