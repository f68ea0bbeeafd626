"""FP64 per-Gaussian projection for the oracle -- TEST INFRASTRUCTURE ONLY.

Plain PyTorch CPU float64 ops; torch.autograd supplies the chain rule from
screen-space quantities back to the Gaussian parameters, so the adjoint of
this stage is exact by construction.  Shares no code with the CUDA path.

What is computed (the paper only names "the projected 2D gaussian kernel"
G'(x') of Eq. 2; the readings below are the 3DGS conventions it builds on):

* view-space mean  t = R mu + t_cam;  screen mean mu2 = (fx t_x/t_z + cx, fy t_y/t_z + cy)
* 3D covariance    Sigma = R(q) diag(s)^2 R(q)^T,  q normalised, [w,x,y,z]
* EWA screen cov.  Sigma' = J R Sigma R^T J^T + dilation I, J the Jacobian of
  the pinhole map at t with t_x/t_z, t_y/t_z clamped to +-1.3 tan(half FOV)
* conic            (a, b, c) = inverse of Sigma', so q(d) = a dx^2 + 2 b dx dy + c dy^2
* opacity          sigma = sigmoid(logit)  (alpha in [0,1], Sec. V-A)
* colour           c = max(0, 0.5 + sum_lm k_lm Y_lm(dir)), dir = (mu - eye)/|mu - eye|,
                   real spherical harmonics of degree <= 3.
"""
from __future__ import annotations

import math

import torch

# Real spherical harmonics without the Condon-Shortley phase, index l^2+l+m.
# Each constant is the normalisation of Y_lm written from its definition.
_C0 = 0.5 / math.sqrt(math.pi)
_C1 = math.sqrt(3.0 / (4.0 * math.pi))
_C2a = 0.5 * math.sqrt(15.0 / math.pi)
_C2b = 0.25 * math.sqrt(5.0 / math.pi)
_C2c = 0.25 * math.sqrt(15.0 / math.pi)
_C3a = 0.25 * math.sqrt(35.0 / (2.0 * math.pi))
_C3b = 0.5 * math.sqrt(105.0 / math.pi)
_C3c = 0.25 * math.sqrt(21.0 / (2.0 * math.pi))
_C3d = 0.25 * math.sqrt(7.0 / math.pi)
_C3e = 0.25 * math.sqrt(105.0 / math.pi)


def sh_basis(d: torch.Tensor, degree: int) -> torch.Tensor:
    """Y_lm(d) for unit vectors d (G,3): returns (G, (degree+1)^2)."""
    x, y, z = d[:, 0], d[:, 1], d[:, 2]
    out = [torch.full_like(x, _C0)]
    if degree >= 1:
        out += [_C1 * y, _C1 * z, _C1 * x]
    if degree >= 2:
        out += [_C2a * x * y, _C2a * y * z, _C2b * (3.0 * z * z - 1.0),
                _C2a * x * z, _C2c * (x * x - y * y)]
    if degree >= 3:
        out += [_C3a * y * (3.0 * x * x - y * y), _C3b * x * y * z,
                _C3c * y * (5.0 * z * z - 1.0), _C3d * z * (5.0 * z * z - 3.0),
                _C3c * x * (5.0 * z * z - 1.0), _C3e * z * (x * x - y * y),
                _C3a * x * (x * x - 3.0 * y * y)]
    return torch.stack(out, dim=1)


def quat_to_rotmat(q: torch.Tensor) -> torch.Tensor:
    """(G,4) [w,x,y,z] -> (G,3,3) rotation of the normalised quaternion."""
    q = q / torch.linalg.norm(q, dim=1, keepdim=True)
    w, x, y, z = q.unbind(1)
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], 1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], 1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], 1),
    ], 1)


def camera_tensors(cam):
    """Unpack the float32[22] camera array into float64 pieces."""
    c = torch.as_tensor(cam, dtype=torch.float64)
    return dict(W=float(c[0]), H=float(c[1]), fx=float(c[2]), fy=float(c[3]), cx=float(c[4]),
                cy=float(c[5]), znear=float(c[6]), R=c[7:16].reshape(3, 3), t=c[16:19], eye=c[19:22])


def project_direct(mean, scale, quat, opac, rgb, cam, dilation: float = 0.3):
    """As project(), with opacity and colour given directly (decoded neural
    Gaussians): the same geometry, opac and rgb passed through."""
    out = project(mean, scale, quat, torch.zeros_like(opac), torch.zeros(mean.shape[0], 1, 3, dtype=mean.dtype), 0,
                  cam, dilation)
    out["opac"] = opac
    out["rgb"] = rgb
    return out


def project(mean, scale, quat, logit, sh, sh_degree: int, cam, dilation: float = 0.3):
    """Screen-space quantities of Gaussians (all float64 tensors; gradients
    flow to every input).  Returns dict(mu2 (G,2), conic (G,3), opac (G,),
    rgb (G,3), depth (G,))."""
    cv = camera_tensors(cam)
    R, tc = cv["R"], cv["t"]
    fx, fy = cv["fx"], cv["fy"]
    tv = mean @ R.T + tc
    tx, ty, tz = tv.unbind(1)
    x = tx / tz
    y = ty / tz
    mu2 = torch.stack([fx * x + cv["cx"], fy * y + cv["cy"]], 1)
    limx = 1.3 * (0.5 * cv["W"] / fx)
    limy = 1.3 * (0.5 * cv["H"] / fy)
    xc = torch.clamp(x, -limx, limx)
    yc = torch.clamp(y, -limy, limy)
    zero = torch.zeros_like(tz)
    J = torch.stack([
        torch.stack([fx / tz, zero, -fx * xc / tz], 1),
        torch.stack([zero, fy / tz, -fy * yc / tz], 1),
    ], 1)                                              # (G,2,3)
    Rg = quat_to_rotmat(quat)
    M = Rg * scale[:, None, :]                          # R diag(s)
    Sigma = M @ M.transpose(1, 2)
    T = J @ R                                           # (G,2,3)
    S2 = T @ Sigma @ T.transpose(1, 2)
    sxx = S2[:, 0, 0] + dilation
    syy = S2[:, 1, 1] + dilation
    sxy = S2[:, 0, 1]
    det = sxx * syy - sxy * sxy
    conic = torch.stack([syy / det, -sxy / det, sxx / det], 1)
    opac = torch.sigmoid(logit)
    d = mean - cv["eye"]
    d = d / torch.linalg.norm(d, dim=1, keepdim=True)
    Y = sh_basis(d, sh_degree)                          # (G,C)
    rgb = torch.clamp_min(0.5 + torch.einsum("gc,gck->gk", Y, sh), 0.0)
    return dict(mu2=mu2, conic=conic, opac=opac, rgb=rgb, depth=tz,
                cov2=torch.stack([sxx, sxy, syy], 1))
