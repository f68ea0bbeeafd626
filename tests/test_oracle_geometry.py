"""Pins of the oracle's geometry against things other than itself.

* real spherical harmonics vs SciPy's complex Y_l^m and quadrature orthonormality
* quaternion rotation matrix vs the Hamilton sandwich product q v q*
* EWA screen covariance vs a finite-difference Jacobian of the pinhole map
* projected mean vs the camera ray through it
* FP32 AABB inputs vs the FP64 projection
* cell footprint vs a dense silhouette scan of the ellipsoid (Sec. IV-B)
* tile lists vs a per-tile brute-force scan (Sec. IV-B)
"""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import project as P
from paper_2508_03180_gb300 import synth


def _real_sh_scipy(l, m, theta, phi):
    from scipy.special import sph_harm_y
    if m == 0:
        return np.real(sph_harm_y(l, 0, theta, phi))
    Y = sph_harm_y(l, abs(m), theta, phi)
    if m > 0:
        return math.sqrt(2.0) * (-1) ** m * np.real(Y)
    return math.sqrt(2.0) * (-1) ** m * np.imag(Y)


def test_sh_basis_matches_scipy():
    rng = np.random.default_rng(3)
    d = rng.standard_normal((500, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    Y = P.sh_basis(torch.tensor(d), 3).numpy()
    for l in range(4):
        for m in range(-l, l + 1):
            ref = _real_sh_scipy(l, m, theta, phi)
            np.testing.assert_allclose(Y[:, l * l + l + m], ref, atol=1e-12, err_msg=f"l={l} m={m}")


def test_sh_basis_orthonormal_quadrature():
    # Gauss-Legendre in cos(theta) x uniform phi is exact for these products
    xg, wg = np.polynomial.legendre.leggauss(24)
    nphi = 48
    phi = (np.arange(nphi) + 0.5) * 2 * math.pi / nphi
    ct = np.repeat(xg, nphi)
    w = np.repeat(wg, nphi) * (2 * math.pi / nphi)
    ph = np.tile(phi, len(xg))
    st = np.sqrt(1 - ct * ct)
    d = np.stack([st * np.cos(ph), st * np.sin(ph), ct], 1)
    Y = P.sh_basis(torch.tensor(d), 3).numpy()
    gram = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-12)


def test_dc_colour_reading():
    """Degree-0 colour 0.5 + k00 Y00 returns the drawn base colour u."""
    sc = synth.scene_small(n_cells=64)
    Y00 = P.sh_basis(torch.tensor([[0.0, 0.0, 1.0]]), 0).numpy()[0, 0]
    u = 0.5 + sc.g_sh[:, 0, :].astype(np.float64) * Y00
    assert u.min() >= -1e-6 and u.max() <= 1 + 1e-6
    assert u.min() < 0.05 and u.max() > 0.95  # spans the drawn range [0,1]


def _sandwich(q, v):
    """Rotate v by unit quaternion q with Hamilton products q (0,v) q*."""
    def mul(a, b):
        w1, x1, y1, z1 = a
        w2, x2, y2, z2 = b
        return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                         w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                         w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                         w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])
    q = q / np.linalg.norm(q)
    qc = q * np.array([1, -1, -1, -1])
    return mul(mul(q, np.concatenate([[0.0], v])), qc)[1:]


def test_rotation_matches_sandwich_product():
    rng = np.random.default_rng(5)
    q = rng.standard_normal((50, 4)) * rng.uniform(0.2, 3.0, (50, 1))  # unnormalised on purpose
    R = P.quat_to_rotmat(torch.tensor(q)).numpy()
    for i in range(50):
        for e in np.eye(3):
            np.testing.assert_allclose(R[i] @ e, _sandwich(q[i], e), atol=1e-13)


def _pinhole(cam, tv):
    c = P.camera_tensors(cam)
    return np.array([c["fx"] * tv[0] / tv[2] + c["cx"], c["fy"] * tv[1] / tv[2] + c["cy"]])


def test_ewa_covariance_matches_fd_jacobian():
    sc = synth.scene_small(n_cells=200, K=4)
    cam = synth.small_camera().as_array()
    proj, _ = oracle.project64(sc, cam)
    c = P.camera_tensors(cam)
    R = c["R"].numpy()
    t = c["t"].numpy()
    h = 1e-6
    for g in range(0, sc.G, 37):
        mean = sc.g_mean[g].astype(np.float64)
        tv = R @ mean + t
        J = np.zeros((2, 3))
        for j in range(3):
            e = np.zeros(3); e[j] = h
            J[:, j] = (_pinhole(cam, tv + e) - _pinhole(cam, tv - e)) / (2 * h)
        Rq = np.stack([_sandwich(sc.g_quat[g].astype(np.float64), e) for e in np.eye(3)], 1)
        s = sc.g_scale[g].astype(np.float64)
        Sigma = Rq @ np.diag(s * s) @ Rq.T
        S2 = J @ R @ Sigma @ R.T @ J.T
        sxx, sxy, syy = proj["cov2"][g]
        np.testing.assert_allclose([sxx - 0.3, sxy, syy - 0.3], [S2[0, 0], S2[0, 1], S2[1, 1]],
                                   rtol=1e-6, atol=1e-9 * abs(S2).max())
        # the conic is the inverse of the screen covariance
        a, b, cc = proj["conic"][g]
        np.testing.assert_allclose(np.array([[a, b], [b, cc]]) @ np.array([[sxx, sxy], [sxy, syy]]),
                                   np.eye(2), atol=1e-10)


def test_projected_mean_lies_on_camera_ray():
    sc = synth.scene_small(n_cells=100, K=4)
    cam = synth.small_camera().as_array()
    proj, _ = oracle.project64(sc, cam)
    c = P.camera_tensors(cam)
    R, eye = c["R"].numpy(), c["eye"].numpy()
    mu2 = proj["mu2"]
    ray = np.stack([(mu2[:, 0] - c["cx"]) / c["fx"], (mu2[:, 1] - c["cy"]) / c["fy"], np.ones(sc.G)], 1) @ R
    to = sc.g_mean.astype(np.float64) - eye
    cos = (ray * to).sum(1) / np.linalg.norm(ray, axis=1) / np.linalg.norm(to, axis=1)
    assert np.all(cos > 1 - 1e-11)


def test_fp32_decision_inputs_match_fp64_projection():
    sc = synth.scene_multiscale(n_cells=3000, K=4)
    cam = synth.sphere_cameras(1, 15.0, 480, 270)[0].as_array()
    mu2f, extf, valid = oracle.gauss_decisions(sc, cam)
    proj, _ = oracle.project64(sc, cam)
    v = valid.astype(bool)
    assert np.array_equal(v, proj["depth"] > 0.2)
    np.testing.assert_allclose(mu2f[v], proj["mu2"][v], atol=1e-3, rtol=1e-5)
    ext64 = 3.0 * np.sqrt(proj["cov2"][:, [0, 2]])
    np.testing.assert_allclose(extf[v], ext64[v], rtol=1e-4)


def _fibonacci_sphere(n):
    i = np.arange(n) + 0.5
    z = 1 - 2 * i / n
    r = np.sqrt(1 - z * z)
    phi = i * math.pi * (3 - math.sqrt(5))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], 1)


@pytest.mark.parametrize("kind", ["small", "multiscale"])
def test_cell_footprint_matches_silhouette_scan(kind):
    if kind == "small":
        sc = synth.scene_small(n_cells=60)
        cam = synth.small_camera().as_array()
    else:
        sc = synth.scene_multiscale(n_cells=60, K=1)
        cam = synth.sphere_cameras(1, 15.0, 480, 270, seed0=2)[0].as_array()
    rect, depth, bounds = oracle.cell_rects(sc, cam, with_bounds=True)
    c = P.camera_tensors(cam)
    R, t = c["R"].numpy(), c["t"].numpy()
    U = _fibonacci_sphere(200_000)
    checked = 0
    for n in range(sc.N):
        Rq = np.stack([_sandwich(sc.cell_quat[n].astype(np.float64), e) for e in np.eye(3)], 1)
        pts = sc.cell_center[n].astype(np.float64) + (U * sc.cell_axes[n].astype(np.float64)) @ Rq.T
        tv = pts @ R.T + t
        centre_z = (R @ sc.cell_center[n].astype(np.float64) + t)[2]
        assert abs(depth[n] - centre_z) <= 1e-5 * abs(centre_z) + 1e-6
        if np.isnan(bounds[n, 0]):
            assert tv[:, 2].min() <= 0.2 + 1e-4 * abs(centre_z)
            continue
        assert tv[:, 2].min() > 0.2
        u = c["fx"] * tv[:, 0] / tv[:, 2] + c["cx"]
        v = c["fy"] * tv[:, 1] / tv[:, 2] + c["cy"]
        ext = max(u.max() - u.min(), v.max() - v.min(), 1.0)
        tol = 2e-3 + 1e-4 * ext + 2e-6 * np.abs(bounds[n]).max()
        for got, ref in zip(bounds[n], [u.min(), u.max(), v.min(), v.max()]):
            assert abs(got - ref) <= tol, (n, got, ref, tol)
        checked += 1
    assert checked > 10


def test_tile_lists_match_per_tile_scan():
    sc = synth.make_scene(300, 2, synth._box(-1, 1), 0.05, 0.4, 0, seed=9)
    cam = synth.small_camera(96, 80).as_array()
    rect, depth = oracle.cell_rects(sc, cam)
    cells, rng = oracle.tile_lists(rect, depth, cam)
    W, H, Tx, Ty = oracle.grid(cam)
    total = 0
    for ty in range(Ty):
        for tx in range(Tx):
            cov = np.nonzero((rect[:, 0] >= 0) & (rect[:, 0] <= tx) & (rect[:, 2] >= tx)
                             & (rect[:, 1] <= ty) & (rect[:, 3] >= ty))[0]
            order = cov[np.lexsort((cov, depth[cov]))]
            tid = ty * Tx + tx
            got = cells[rng[tid, 0]:rng[tid, 1]]
            assert np.array_equal(got, order), (tx, ty)
            total += len(order)
    assert total == len(cells) and total > 500
    # rectangles lie inside the grid and are consistent with the pixel box
    vis = rect[:, 0] >= 0
    assert (rect[vis, 0] <= rect[vis, 2]).all() and (rect[vis, 2] < Tx).all()
    assert (rect[vis, 1] <= rect[vis, 3]).all() and (rect[vis, 3] < Ty).all()


def _axis_camera(W, H):
    """Camera at the origin looking along +z with R = I (view space = world
    space), vertical FOV 60 deg."""
    cam = synth.look_at((0.0, 0.0, 0.0), (0.0, 0.0, 1.0), W, H, 60.0, up=(0.0, -1.0, 0.0))
    assert np.allclose(cam.R, np.eye(3)) and np.allclose(cam.t, 0.0)
    return cam.as_array()


@pytest.mark.parametrize("W,H", [(320, 240), (180, 300)])
def test_ewa_jacobian_clamp_outside_the_view(W, H):
    """Eq. 2's projected kernel with the EWA reading: the Jacobian of the
    pinhole map is taken at the point of the same depth whose view direction
    is clamped per axis to 1.3 x the tangent of that axis' half field of view.
    The limits come from the camera's construction (vertical FOV 60 deg,
    square pixels, so tan(half FOV_x) = tan(30 deg) W / H), the Jacobian from
    central differences of the pinhole map at the clamped point, and the
    covariance from the Hamilton sandwich rotation: none of it from the
    oracle.  Directions inside, between the two axes' limits, and beyond
    them, on both sides; the screen mean itself stays unclamped."""
    cam = _axis_camera(W, H)
    ty = math.tan(math.radians(30.0))
    lim = np.array([1.3 * ty * W / H, 1.3 * ty])
    lo, hi = lim.min(), lim.max()
    # ratios t_x/t_z and t_y/t_z relative to each axis' own limit, plus ones
    # that lie between the smaller and the larger limit (they tell the axes apart)
    rel = np.array([-3.0, -1.2, -0.97, 0.0, 0.4, 0.96, 1.04, 2.5])
    between = 0.5 * (lo + hi)
    rng = np.random.default_rng(11)
    pts = []
    for rx in list(rel * lim[0]) + [between, -between]:
        for ry in list(rel * lim[1]) + [between, -between]:
            z = rng.uniform(1.0, 6.0)
            pts.append([rx * z, ry * z, z])
    tv = np.array(pts)
    G = len(tv)
    scale = np.exp(rng.normal(np.log(0.2), 0.5, (G, 3)))
    quat = rng.standard_normal((G, 4))
    out = P.project(torch.tensor(tv), torch.tensor(scale), torch.tensor(quat), torch.zeros(G),
                    torch.zeros(G, 1, 3, dtype=torch.float64), 0, cam)
    cov2 = out["cov2"].numpy()
    mu2 = out["mu2"].numpy()
    c = P.camera_tensors(cam)
    h = 1e-6
    clamped = 0
    for g in range(G):
        t = tv[g]
        r = np.clip(t[:2] / t[2], -lim, lim)
        clamped += int(np.any(np.abs(t[:2] / t[2]) > lim))
        tc = np.array([r[0] * t[2], r[1] * t[2], t[2]])
        J = np.zeros((2, 3))
        for j in range(3):
            e = np.zeros(3); e[j] = h * max(1.0, abs(tc[j]))
            J[:, j] = (_pinhole(cam, tc + e) - _pinhole(cam, tc - e)) / (2 * e[j])
        Rq = np.stack([_sandwich(quat[g], e) for e in np.eye(3)], 1)
        Sigma = Rq @ np.diag(scale[g] ** 2) @ Rq.T
        S2 = J @ Sigma @ J.T
        ref = [S2[0, 0] + 0.3, S2[0, 1], S2[1, 1] + 0.3]
        np.testing.assert_allclose(cov2[g], ref, rtol=1e-6, atol=1e-8 * abs(S2).max(), err_msg=str(t))
        np.testing.assert_allclose(mu2[g], _pinhole(cam, t), rtol=1e-12)
    assert clamped > G // 2 and clamped < G


def test_colour_clamp_at_zero():
    """Reading 8: c = max(0, 0.5 + sum_lm k_lm Y_lm(d)).  The raw sum is
    evaluated with SciPy's spherical harmonics at d = (mu - eye)/|mu - eye|;
    a channel whose raw value is negative is exactly 0 with zero gradient to
    its coefficients and to the mean, and a positive one equals the raw value
    with gradient Y_lm(d) to k_lm."""
    rng = np.random.default_rng(4)
    G = 400
    cam = synth.small_camera(64, 64).as_array()
    mean = rng.uniform(-1.0, 1.0, (G, 3))
    sh = rng.normal(0.0, 0.3, (G, 16, 3))
    sh[:, 0, :] = rng.uniform(-2.0, 1.0, (G, 3))  # DC pushes many channels below zero
    sh[:3, 0, :] = -5.0                               # three Gaussians negative in every channel
    eye = cam[19:22].astype(np.float64)
    d = mean - eye
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    Y = np.stack([_real_sh_scipy(l, m, theta, phi) for l in range(4) for m in range(-l, l + 1)], 1)
    raw = 0.5 + np.einsum("gc,gck->gk", Y, sh)
    neg = raw < 0.0
    assert 0.2 < neg.mean() < 0.8 and np.abs(raw).min() > 1e-9
    mt = torch.tensor(mean, requires_grad=True)
    st = torch.tensor(sh, requires_grad=True)
    out = P.project(mt, torch.full((G, 3), 0.05, dtype=torch.float64), torch.tensor([[1.0, 0, 0, 0]] * G),
                    torch.zeros(G, dtype=torch.float64), st, 3, cam)
    rgb = out["rgb"]
    assert torch.all(rgb.detach()[torch.tensor(neg)] == 0.0)
    np.testing.assert_allclose(rgb.detach().numpy()[~neg], raw[~neg], atol=1e-12)
    for k in range(3):
        gm, gs = torch.autograd.grad(rgb[:, k].sum(), (mt, st), retain_graph=True)
        gs = gs.numpy()[:, :, k]
        assert np.all(gs[neg[:, k]] == 0.0)
        np.testing.assert_allclose(gs[~neg[:, k]], Y[~neg[:, k]], atol=1e-12)
        assert np.all(gm.numpy()[neg[:, k]] == 0.0)
    assert np.all(neg[:3])
