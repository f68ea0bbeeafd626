"""CPU oracle of the Duplex-GS hybrid renderer -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import this package.  It shares no code with the CUDA path and never calls
it; the product path must not import it.

Pieces:
  dgs_oracle.c  FP32-exact decisions (cell footprint, tile lists, AABB inputs)
                and the FP64 hybrid blend (Eq. 12-14) with its adjoint; the
                comparators: per-Gaussian alpha-blending (Eq. 2-3) and
                weighted-sum rendering (Eq. 4-6).
  project.py    FP64 projection of Gaussians (EWA, opacity, SH colour) in
                plain PyTorch CPU ops; autograd gives its chain rule.
  decode.py     FP64 decode of neural cells into Gaussians (the MLP step
                before the path).

Parity protocol helpers live here too: `render(..., forced_ndone=...)`
renders with a given per-pixel processed-cell count and reports how many of
those counts are not valid outcomes of the stopping rule within a relative
transmittance slack `delta`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np
import torch

from . import project as _project

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dgs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libdgs_oracle.so")


def build(force: bool = False) -> str:
    """Compile the C part with gcc (no contraction, no fast-math)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
            "-o", _SO + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32 = ctypes.c_int64, ctypes.c_int
        L.or_cell_rects.argtypes = [i64, P, P, P, P, i32, i32, P, P, P]
        L.or_cell_rects.restype = None
        L.or_tile_lists.argtypes = [i64, P, P, i32, i32, P, i64, P]
        L.or_tile_lists.restype = i64
        L.or_gauss_decisions.argtypes = [i64, P, P, P, P, ctypes.c_float, ctypes.c_float, ctypes.c_int, P, P, P]
        L.or_gauss_decisions.restype = None
        L.or_blend.argtypes = [i32, i32, i32, i32, P, P, P, P, P, P, P, P, P, P, P, P, i32, i32,
                               P, P, P, P, P]
        L.or_blend.restype = i64
        L.or_blend_grad.argtypes = [i32, i32, i32, i32, P, P, P, P, P, P, P, P, P, P, P, P, P, i32, i32,
                                    P, P, P, P, P]
        L.or_blend_grad.restype = None
        L.or_gauss_rects.argtypes = [i64, P, P, P, P, P, i32, P, P]
        L.or_gauss_rects.restype = None
        L.or_alpha_blend.argtypes = [i32, i32, i32, P, P, P, P, P, P, P, P, P, P, P, i32, i32, P, P, P]
        L.or_alpha_blend.restype = i64
        L.or_wsr.argtypes = [i32, i32, i32, P, P, P, P, P, P, P, P, P, P, ctypes.c_double, P, i32, i32, P]
        L.or_wsr.restype = None
        L.or_num_threads.argtypes = []
        L.or_num_threads.restype = i32
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


@dataclass
class Options:
    """Renderer settings shared by the oracle and the CUDA path (same defaults).

    eps: termination threshold on cell transmittance (the 3DGS value 1e-4,
    Sec. VII-D); alpha_max: alpha clamp (3DGS 0.99); d_min: a pixel whose
    weight sum D is not above this keeps the background; dilation: EWA
    low-pass 0.3 px^2; ksigma: AABB half extent in standard deviations;
    delta: relative slack on T when checking a given termination count.
    Variants of the hybrid renderer (off by default; the same meaning as the
    renderer's config flags): w_bg, a background weight in the normalisation
    (Eq. 4's term: C = (N + w_bg bg) / (D + w_bg)); alpha_skip, alpha < 1/255
    contributes nothing; term_exclude, a cell that would take T below eps is
    not blended; aabb_square, the AABB is the square of radius
    ceil(ksigma sqrt(lambda_max(Sigma'))); out_numerator, the output is the
    numerator N of Eq. 12; near_full, a cell reaching the near plane without
    lying wholly behind it covers every tile (sort depth max(c_z, 0)) instead
    of being culled.
    """
    eps: float = 1e-4
    alpha_max: float = 0.99
    d_min: float = 1e-10
    bg: tuple = (0.0, 0.0, 0.0)
    dilation: float = 0.3
    ksigma: float = 3.0
    tile: int = 16
    delta: float = 1e-3
    w_bg: float = 0.0
    alpha_skip: bool = False
    term_exclude: bool = False
    aabb_square: bool = False
    out_numerator: bool = False
    near_full: bool = False

    def flags(self) -> int:
        return (1 if self.alpha_skip else 0) | (2 if self.term_exclude else 0) | \
            (4 if self.aabb_square else 0) | (8 if self.out_numerator else 0) | (16 if self.near_full else 0)

    def blend_opts(self) -> np.ndarray:
        return np.array([self.eps, self.alpha_max, self.d_min, *self.bg, self.delta, self.w_bg, float(self.flags())],
                        dtype=np.float64)


def num_threads() -> int:
    return int(lib().or_num_threads())


def cell_rects(scene, cam, opt: Options = Options(), with_bounds=False):
    """Per cell: tile rectangle (tx0, ty0, tx1, ty1; tx0 = -1 culled) and
    view depth; with_bounds adds the FP32 pixel box (lo_x, hi_x, lo_y, hi_y)."""
    N = scene.N
    rect = np.empty((N, 4), dtype=np.int32)
    depth = np.empty(N, dtype=np.float32)
    bounds = np.empty((N, 4), dtype=np.float32) if with_bounds else None
    lib().or_cell_rects(N, _p(_c(scene.cell_center, np.float32)), _p(_c(scene.cell_axes, np.float32)),
                        _p(_c(scene.cell_quat, np.float32)), _p(_c(cam, np.float32)), opt.tile, opt.flags(),
                        _p(rect), _p(depth), _p(bounds))
    if with_bounds:
        return rect, depth, bounds
    return rect, depth


def grid(cam, tile=16):
    W, H = int(cam[0]), int(cam[1])
    return W, H, (W + tile - 1) // tile, (H + tile - 1) // tile


def tile_lists(rect, depth, cam, opt: Options = Options()):
    """(cells (L,), range (Tx*Ty, 2) int64) ordered by (tile, depth, cell)."""
    _, _, Tx, Ty = grid(cam, opt.tile)
    rect = _c(rect, np.int32)
    depth = _c(depth, np.float32)
    vis = rect[:, 0] >= 0
    L = int(((rect[vis, 2] - rect[vis, 0] + 1).astype(np.int64) * (rect[vis, 3] - rect[vis, 1] + 1)).sum())
    cells = np.empty(max(L, 1), dtype=np.int32)
    rng = np.empty((Tx * Ty, 2), dtype=np.int64)
    got = lib().or_tile_lists(rect.shape[0], _p(rect), _p(depth), Tx, Ty, _p(cells), L, _p(rng))
    assert got == L, (got, L)
    return cells[:L], rng


def gauss_decisions(scene, cam, opt: Options = Options()):
    G = scene.G
    mu2 = np.empty((G, 2), dtype=np.float32)
    ext = np.empty((G, 2), dtype=np.float32)
    valid = np.empty(G, dtype=np.uint8)
    lib().or_gauss_decisions(G, _p(_c(scene.g_mean, np.float32)), _p(_c(scene.g_scale, np.float32)),
                             _p(_c(scene.g_quat, np.float32)), _p(_c(cam, np.float32)),
                             opt.dilation, opt.ksigma, 1 if opt.aabb_square else 0, _p(mu2), _p(ext), _p(valid))
    return mu2, ext, valid


def _params64(scene, idx, requires_grad=False):
    t = lambda a: torch.tensor(np.asarray(a)[idx], dtype=torch.float64, requires_grad=requires_grad)
    return dict(mean=t(scene.g_mean), scale=t(scene.g_scale), quat=t(scene.g_quat),
                logit=t(scene.g_logit), sh=t(scene.g_sh))


def project64(scene, cam, opt: Options = Options(), mask=None, requires_grad=False):
    """FP64 projected values for the Gaussians in `mask` (bool (G,)); rows
    outside the mask are zero.  Returns (numpy dict, torch graph or None)."""
    G = scene.G
    idx = np.nonzero(mask)[0] if mask is not None else np.arange(G)
    prm = _params64(scene, idx, requires_grad)
    out = _project.project(prm["mean"], prm["scale"], prm["quat"], prm["logit"], prm["sh"],
                           scene.sh_degree, cam, opt.dilation)
    full = {}
    for k in ("mu2", "conic", "opac", "rgb", "depth", "cov2"):
        v = out[k].detach().numpy()
        arr = np.zeros((G,) + v.shape[1:], dtype=np.float64)
        arr[idx] = v
        full[k] = arr
    graph = dict(idx=idx, params=prm, out=out) if requires_grad else None
    return full, graph


def cell_v_view(scene, cam):
    """v_n of every cell as rendered from camera `cam` (FP64), and for a
    view-dependent v (Sec. V-A: v parameterised by spherical harmonics) the
    basis values and the unclamped mask: v_n = clamp(sum_lm k_lm Y_lm(d), 0, 1)
    with d the unit vector from the eye to the cell centre."""
    vsh = getattr(scene, "cell_v_sh", None)
    if vsh is None:
        return np.asarray(scene.cell_v, dtype=np.float64), None
    eye = np.asarray(cam, dtype=np.float64)[19:22]
    d = np.asarray(scene.cell_center, dtype=np.float64) - eye[None, :]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = _project.sh_basis(torch.from_numpy(d), scene.v_sh_degree).numpy()
    raw = (np.asarray(vsh, dtype=np.float64) * Y).sum(1)
    return np.clip(raw, 0.0, 1.0), dict(Y=Y, mask=(raw > 0.0) & (raw < 1.0))


def cell_v_center_grad(scene, cam, g_v):
    """dL/dx_n (N,3) of the cell centres through the direction d of a
    view-dependent v_n, given dL/dv_n (N,) of one view (torch autograd
    through the SH basis at d = (x_n - eye)/|x_n - eye|; zero where the clamp
    holds v_n); zeros for a scalar v_n."""
    vsh = getattr(scene, "cell_v_sh", None)
    N = scene.N
    if vsh is None or N == 0:
        return np.zeros((N, 3))
    eye = torch.as_tensor(np.asarray(cam, dtype=np.float64)[19:22])
    x = torch.tensor(np.asarray(scene.cell_center, dtype=np.float64), requires_grad=True)
    d = x - eye[None, :]
    d = d / torch.linalg.norm(d, dim=1, keepdim=True)
    raw = (torch.as_tensor(np.asarray(vsh, dtype=np.float64)) * _project.sh_basis(d, scene.v_sh_degree)).sum(1)
    free = ((raw > 0.0) & (raw < 1.0)).detach().to(torch.float64)
    (gx,) = torch.autograd.grad((raw * free * torch.as_tensor(np.asarray(g_v, dtype=np.float64))).sum(), x)
    return gx.numpy()


def prepare_view(scene, cam, opt: Options = Options(), tile_rows=None, requires_grad=False):
    """All per-view inputs of the blend: tile lists, FP32 decisions, FP64
    projected values (only for valid Gaussians of cells that reach the
    rendered tile rows)."""
    rect, depth = cell_rects(scene, cam, opt)
    cells, rng = tile_lists(rect, depth, cam, opt)
    mu2f, extf, valid = gauss_decisions(scene, cam, opt)
    W, H, Tx, Ty = grid(cam, opt.tile)
    ty0, ty1 = (0, Ty) if tile_rows is None else tile_rows
    used_cells = np.zeros(scene.N, dtype=bool)
    win = rng[ty0 * Tx: ty1 * Tx]
    ne = win[:, 1] > win[:, 0]
    if ne.any():
        used_cells[cells[win[ne, 0].min(): win[ne, 1].max()]] = True
    mask = np.repeat(used_cells, scene.K) & (valid != 0)
    proj, graph = project64(scene, cam, opt, mask, requires_grad)
    return dict(rect=rect, depth=depth, cells=cells, range=rng, mu2f=mu2f, extf=extf, valid=valid,
                proj=proj, graph=graph, W=W, H=H, Tx=Tx, Ty=Ty, rows=(ty0, ty1), mask=mask,
                cam=np.asarray(cam, dtype=np.float32))


def _blend_args(scene, pv, opt):
    pr = pv["proj"]
    pv["_v"] = _c(cell_v_view(scene, pv["cam"])[0], np.float64)  # kept alive during the call
    return (pv["W"], pv["H"], opt.tile, scene.K, _p(pv["range"]), _p(pv["cells"]),
            _p(_c(pr["mu2"], np.float64)), _p(_c(pr["conic"], np.float64)), _p(_c(pr["opac"], np.float64)),
            _p(_c(pr["rgb"], np.float64)), _p(pv["mu2f"]), _p(pv["extf"]), _p(pv["valid"]),
            _p(pv["_v"]), _p(opt.blend_opts()))


def render_view(scene, cam, opt: Options = Options(), forced_ndone=None, tile_rows=None, pv=None):
    """FP64 image of one view.  Returns dict(C (3,H,W), N, D, T, ndone,
    bad (count of invalid forced counts), pv)."""
    if pv is None:
        pv = prepare_view(scene, cam, opt, tile_rows)
    W, H = pv["W"], pv["H"]
    ty0, ty1 = pv["rows"]
    C = np.zeros((3, H, W)); N = np.zeros((3, H, W)); D = np.zeros((H, W)); T = np.ones((H, W))
    nd = np.zeros((H, W), dtype=np.int32)
    pr = pv["proj"]
    keep = [pr["mu2"], pr["conic"], pr["opac"], pr["rgb"]]  # noqa: F841 (alive during the call)
    fn = None if forced_ndone is None else _c(forced_ndone, np.int32)
    bad = lib().or_blend(*_blend_args(scene, pv, opt), _p(fn), ty0, ty1, _p(C), _p(N), _p(D), _p(T), _p(nd))
    return dict(C=C, N=N, D=D, T=T, ndone=nd, bad=int(bad), pv=pv)


def blend_grad_view(scene, pv, dL_dC, opt: Options = Options(), ndone=None):
    """FP64 adjoint of the blend for one view: per-Gaussian dL/d(mu2, conic,
    opac, rgb) and per-cell dL/dv."""
    G, N = scene.G, scene.N
    g_mu2 = np.zeros((G, 2)); g_conic = np.zeros((G, 3)); g_opac = np.zeros(G); g_rgb = np.zeros((G, 3))
    g_v = np.zeros(N)
    ty0, ty1 = pv["rows"]
    dl = _c(dL_dC, np.float64)
    nd = None if ndone is None else _c(ndone, np.int32)
    lib().or_blend_grad(*_blend_args(scene, pv, opt), _p(nd), _p(dl), ty0, ty1,
                        _p(g_mu2), _p(g_conic), _p(g_opac), _p(g_rgb), _p(g_v))
    return dict(mu2=g_mu2, conic=g_conic, opac=g_opac, rgb=g_rgb, v=g_v)


def param_grads(scene, pv, g2d):
    """Chain screen-space gradients back to the Gaussian parameters through
    the FP64 projection (torch autograd).  Returns numpy float64 arrays:
    mean (G,3), scale (G,3), log_scale (G,3), quat (G,4), logit (G,), sh."""
    graph = pv["graph"]
    assert graph is not None, "prepare_view(..., requires_grad=True) needed"
    idx, prm, out = graph["idx"], graph["params"], graph["out"]
    outs = [out["mu2"], out["conic"], out["opac"], out["rgb"]]
    gos = [torch.tensor(g2d[k][idx], dtype=torch.float64) for k in ("mu2", "conic", "opac", "rgb")]
    ins = [prm["mean"], prm["scale"], prm["quat"], prm["logit"], prm["sh"]]
    grads = torch.autograd.grad(outs, ins, gos, allow_unused=True)
    G = scene.G
    res = {}
    for name, gr, ref in zip(("mean", "scale", "quat", "logit", "sh"), grads, ins):
        arr = np.zeros((G,) + tuple(ref.shape[1:]), dtype=np.float64)
        if gr is not None:
            arr[idx] = gr.numpy()
        res[name] = arr
    res["log_scale"] = res["scale"] * np.asarray(scene.g_scale, dtype=np.float64)
    res["cell_v"] = g2d["v"]
    _, info = cell_v_view(scene, pv["cam"])
    if info is not None:  # through the clamp and the SH basis
        res["cell_v_sh"] = (g2d["v"] * info["mask"])[:, None] * info["Y"]
    # the cells' own parameters: with the footprints held fixed, explicit
    # Gaussians see them only through a view-dependent v_n's direction
    res["cell_center"] = cell_v_center_grad(scene, pv["cam"], g2d["v"])
    res["cell_axes"] = np.zeros((scene.N, 3))
    res["cell_quat"] = np.zeros((scene.N, 4))
    return res


def render_and_grad(scene, cam, dL_dC, opt: Options = Options(), ndone=None, tile_rows=None):
    pv = prepare_view(scene, cam, opt, tile_rows, requires_grad=True)
    img = render_view(scene, cam, opt, pv=pv, forced_ndone=ndone)
    g2d = blend_grad_view(scene, pv, dL_dC, opt, ndone=ndone)
    return img, g2d, param_grads(scene, pv, g2d)


def sort_length(scene, cam, opt: Options = Options()) -> int:
    rect, _ = cell_rects(scene, cam, opt)
    vis = rect[:, 0] >= 0
    return int(((rect[vis, 2] - rect[vis, 0] + 1).astype(np.int64) * (rect[vis, 3] - rect[vis, 1] + 1)).sum())


# --------------------------------------------------------------------------
# Comparators (per-Gaussian alpha-blending, weighted-sum rendering)


def gauss_rects(scene, cam, opt: Options = Options()):
    """Per Gaussian: tile rectangle of its FP32 AABB box (tx0 = -1 culled) and
    FP32 view depth of its mean."""
    mu2f, extf, valid = gauss_decisions(scene, cam, opt)
    G = scene.G
    rect = np.empty((G, 4), dtype=np.int32)
    depth = np.empty(G, dtype=np.float32)
    lib().or_gauss_rects(G, _p(_c(scene.g_mean, np.float32)), _p(mu2f), _p(extf), _p(valid),
                         _p(_c(cam, np.float32)), opt.tile, _p(rect), _p(depth))
    return rect, depth, (mu2f, extf, valid)


def lc_wsr_weights(scene, depth64, tau: float):
    """Eq. 5-6: w_i = max(0, 1 - d_i / tau) v_i with v_i the calibration
    scalar of Gaussian i's cell; tau = inf gives w_i = v_i (plain WSR)."""
    v = np.repeat(np.asarray(scene.cell_v, dtype=np.float64), scene.K)
    if not np.isfinite(tau):
        return v
    return np.maximum(0.0, 1.0 - np.asarray(depth64, dtype=np.float64) / tau) * v


def _prepare_gauss_view(scene, cam, opt, tile_rows, ordered):
    rect, depth, (mu2f, extf, valid) = gauss_rects(scene, cam, opt)
    vis = rect[:, 0] >= 0
    L = int(((rect[vis, 2] - rect[vis, 0] + 1).astype(np.int64) * (rect[vis, 3] - rect[vis, 1] + 1)).sum())
    if not ordered:  # weighted sums do not need a depth order: list in index order
        depth = np.zeros_like(depth)
    W, H, Tx, Ty = grid(cam, opt.tile)
    ty0, ty1 = (0, Ty) if tile_rows is None else tile_rows
    if tile_rows is not None:  # lists of the rendered rows only (the same lists for those tiles)
        rect = rect.copy()
        rect[(rect[:, 3] < ty0) | (rect[:, 1] >= ty1)] = -1
    lst, rng = tile_lists(rect, depth, cam, opt)
    used = np.zeros(scene.G, dtype=bool)
    win = rng[ty0 * Tx: ty1 * Tx]
    for b, e in win:
        used[lst[b:e]] = True
    proj, _ = project64(scene, cam, opt, used & (valid != 0))
    return dict(rect=rect, list=lst, range=rng, mu2f=mu2f, extf=extf, valid=valid, proj=proj,
                W=W, H=H, Tx=Tx, Ty=Ty, rows=(ty0, ty1), L=L)


def render_alpha(scene, cam, opt: Options = Options(), forced_ndone=None, tile_rows=None):
    """Per-Gaussian depth-sorted alpha-blending (Eq. 2-3) of one view.
    Returns dict(C (3,H,W), T, ndone, bad, L (tile-Gaussian pairs))."""
    pv = _prepare_gauss_view(scene, cam, opt, tile_rows, ordered=True)
    W, H = pv["W"], pv["H"]
    ty0, ty1 = pv["rows"]
    pr = pv["proj"]
    mu2, conic, opac, rgb = (_c(pr[k], np.float64) for k in ("mu2", "conic", "opac", "rgb"))
    C = np.zeros((3, H, W)); T = np.ones((H, W)); nd = np.zeros((H, W), dtype=np.int32)
    fn = None if forced_ndone is None else _c(forced_ndone, np.int32)
    bad = lib().or_alpha_blend(W, H, opt.tile, _p(pv["range"]), _p(pv["list"]), _p(mu2), _p(conic), _p(opac),
                               _p(rgb), _p(pv["mu2f"]), _p(pv["extf"]), _p(pv["valid"]), _p(opt.blend_opts()),
                               _p(fn), ty0, ty1, _p(C), _p(T), _p(nd))
    return dict(C=C, T=T, ndone=nd, bad=int(bad), L=pv["L"])


def render_wsr(scene, cam, tau: float = float("inf"), w_bg: float = 0.0, opt: Options = Options(),
               tile_rows=None):
    """Weighted-sum rendering (Eq. 4) with the LC-WSR weight (Eq. 5-6) of one
    view.  Returns dict(C (3,H,W), L (tile-Gaussian pairs))."""
    pv = _prepare_gauss_view(scene, cam, opt, tile_rows, ordered=False)
    W, H = pv["W"], pv["H"]
    ty0, ty1 = pv["rows"]
    pr = pv["proj"]
    mu2, conic, opac, rgb = (_c(pr[k], np.float64) for k in ("mu2", "conic", "opac", "rgb"))
    w = _c(lc_wsr_weights(scene, pr["depth"], tau), np.float64)
    C = np.zeros((3, H, W))
    lib().or_wsr(W, H, opt.tile, _p(pv["range"]), _p(pv["list"]), _p(mu2), _p(conic), _p(opac), _p(rgb),
                 _p(pv["mu2f"]), _p(pv["extf"]), _p(pv["valid"]), _p(w), float(w_bg), _p(opt.blend_opts()),
                 ty0, ty1, _p(C))
    return dict(C=C, L=pv["L"])


# --------------------------------------------------------------------------
# Neural cells


def decode_view(scene, cam):
    """FP64 Gaussians of every cell of a neural scene as seen from `cam`."""
    from . import decode as _decode
    return _decode.decode64(scene.neural, scene.cell_center, scene.cell_axes, scene.cell_quat, scene.K,
                            np.asarray(cam, dtype=np.float64)[19:22])


def explicit_scene(scene, mean, scale, quat, opac, rgb):
    """An explicit-Gaussian scene with the given per-Gaussian values ((G,...)
    arrays): colour as SH degree 0 with 0.5 + k_00 Y_00 = rgb, opacity as the
    logit of sigma (sigma <= 0: opacity 0, never contributing)."""
    import dataclasses
    y00 = 0.5 / np.sqrt(np.pi)
    G = scene.G
    op = np.asarray(opac, dtype=np.float64).reshape(G)
    with np.errstate(divide="ignore"):
        logit = np.where(op > 0, np.log(np.clip(op, 1e-300, None)) - np.log1p(-np.clip(op, None, 1 - 1e-16)), -np.inf)
    sh = ((np.asarray(rgb, dtype=np.float64).reshape(G, 1, 3) - 0.5) / y00)
    return dataclasses.replace(scene, neural=None, g_mean=np.asarray(mean).reshape(G, 3),
                               g_scale=np.asarray(scale).reshape(G, 3), g_quat=np.asarray(quat).reshape(G, 4),
                               g_logit=logit, g_sh=sh, sh_degree=0)


def neural_render_and_grad(scene, cam, dL_dC, decided=None, opt: Options = Options(), ndone=None, tile_rows=None):
    """FP64 image and gradients of sum(dL_dC * C) for a neural scene in one
    view: dL/d(packed weights), dL/d(features) (N,F), dL/d(offsets) (G,3),
    dL/d of the cells' centres (N,3), semi-axes (N,3) and quaternions (N,4)
    through the decode (and a view-dependent v_n's direction), and dL/d(decoded
    mean, scale, quat, opacity, rgb) per Gaussian.
    decided: (mean, scale, quat) float32 arrays (G,...) whose FP32 AABB
    decisions and tile lists to use (the renderer's own decoded values);
    default: the FP64 decode rounded to FP32."""
    from . import decode as _decode
    d = _decode.decode_t(scene.neural, scene.cell_center, scene.cell_axes, scene.cell_quat, scene.K,
                         np.asarray(cam, dtype=np.float64)[19:22], requires_grad=True)
    G = scene.G
    flat = {k: d[k].reshape(G, -1) for k in ("mean", "scale", "quat", "opac", "rgb")}
    if decided is None:
        decided = tuple(flat[k].detach().numpy().astype(np.float32) for k in ("mean", "scale", "quat"))
    ex = explicit_scene(scene, decided[0], decided[1], decided[2], flat["opac"].detach().numpy().reshape(G),
                        flat["rgb"].detach().numpy())
    pv = prepare_view(ex, cam, opt, tile_rows)
    # sigma <= 0 is not drawn: zero opacity, no gradient
    proj = _project.project_direct(flat["mean"], flat["scale"], flat["quat"], torch.clamp_min(flat["opac"].reshape(G), 0.0),
                                   flat["rgb"], cam, opt.dilation)
    pv["proj"] = {k: v.detach().numpy() for k, v in proj.items()}
    img = render_view(ex, cam, opt, pv=pv, forced_ndone=ndone)
    g2d = blend_grad_view(ex, pv, dL_dC, opt, ndone=ndone)
    outs = [proj["mu2"], proj["conic"], proj["opac"], proj["rgb"]]
    gos = [torch.tensor(g2d[k], dtype=torch.float64) for k in ("mu2", "conic", "opac", "rgb")]
    dec_vals = [flat[k] for k in ("mean", "scale", "quat", "opac", "rgb")]
    leaves = d["leaves"]
    names = ("mlp", "feat", "offset", "cell_center", "cell_axes", "cell_quat")
    grads = torch.autograd.grad(outs, [leaves[k] for k in names] + dec_vals, gos, allow_unused=True,
                                retain_graph=False)
    z = lambda t, ref: np.zeros(tuple(ref.shape)) if t is None else t.numpy()
    res = {k: z(g_, leaves[k]) for k, g_ in zip(names, grads)}
    res["offset"] = res["offset"].reshape(G, 3)
    res["cell_center"] = res["cell_center"] + cell_v_center_grad(scene, cam, g2d["v"])
    for name, g_, ref in zip(("mean", "scale", "quat", "opac", "rgb"), grads[len(names):], dec_vals):
        res["dec_" + name] = z(g_, ref).reshape(G, -1)
    return img, res


# --------------------------------------------------------------------------
# Cell alignment (Sec. IV-B, Eq. 10 and the centre update)


def cell_align(scene, cam=None):
    """New (centre (N,3), quaternion (N,4)) of every cell in FP64; neural
    scenes decode sigma and q for the eye of `cam`."""
    from . import align as _align
    eye = None if cam is None else np.asarray(cam, dtype=np.float64)[19:22]
    return _align.align(scene, eye)
