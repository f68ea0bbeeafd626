"""Scene files: a synth.Scene on disk, in the format dgs_scene_save writes.

Little-endian.  A 40-byte header -- magic b"DGS1", uint32 version (1), int64
number of cells N, int32 K, sh_degree, v_sh_degree (-1 when v_n is a scalar),
feat_dim and hidden (both 0 for explicit Gaussians), uint32 reserved (0) --
then float32 arrays, row-major, in this order:

    cell_center (N,3)  cell_axes (N,3)  cell_quat (N,4)  cell_v (N,)
    explicit:  g_mean (G,3)  g_scale (G,3)  g_quat (G,4)  g_logit (G,)  g_sh (G,C,3)
    neural:    feat (N,F)  offset (G,3)  mlp (P,)
    cell_v_sh (N,Cv)   only when v_sh_degree >= 0

with G = N*K, C = (sh_degree+1)^2, Cv = (v_sh_degree+1)^2 and P the packed
decoder weight count.  This module only reads and writes bytes: it is the
same format as the C entry points, usable without a GPU.
"""
from __future__ import annotations

import struct

import numpy as np

from .synth import Scene

MAGIC = b"DGS1"
VERSION = 1
_HEADER = struct.Struct("<4sIqiiiiiI")
assert _HEADER.size == 40


def mlp_weights(K: int, F: int, H: int) -> int:
    """Packed decoder weight count: four one-hidden-layer decoders (opacity K,
    colour 3K, scale 3K, rotation 4K outputs) on the input [feature,
    distance, direction], each W1 (H, F+4), b1 (H), W2 (out, H), b2 (out)."""
    return sum(H * (F + 4) + H + o * H + o for o in (K, 3 * K, 3 * K, 4 * K))


def _arrays(scene: Scene) -> list[np.ndarray]:
    out = [scene.cell_center, scene.cell_axes, scene.cell_quat, scene.cell_v]
    if scene.neural is not None:
        out += [scene.neural["feat"], scene.neural["offset"], scene.neural["mlp"]]
    else:
        out += [scene.g_mean, scene.g_scale, scene.g_quat, scene.g_logit, scene.g_sh]
    if scene.cell_v_sh is not None:
        out.append(scene.cell_v_sh)
    return [np.ascontiguousarray(a, dtype="<f4") for a in out]


def save(scene: Scene, path) -> None:
    """Write `scene` to `path`."""
    F, H = (scene.neural["F"], scene.neural["H"]) if scene.neural is not None else (0, 0)
    vdeg = scene.v_sh_degree if scene.cell_v_sh is not None else -1
    with open(path, "wb") as f:
        f.write(_HEADER.pack(MAGIC, VERSION, scene.N, scene.K, scene.sh_degree, vdeg, F, H, 0))
        for a in _arrays(scene):
            f.write(a.tobytes())


def load(path, name: str = "") -> Scene:
    """Read a scene file.  A neural scene gets zero placeholders for the
    explicit Gaussian arrays (the renderer decodes those per view)."""
    with open(path, "rb") as f:
        raw = f.read()
    if len(raw) < _HEADER.size:
        raise ValueError(f"{path}: shorter than a scene file header")
    magic, version, N, K, deg, vdeg, F, H, _ = _HEADER.unpack_from(raw)
    if magic != MAGIC or version != VERSION:
        raise ValueError(f"{path}: not a version-{VERSION} scene file")
    G, Cc = N * K, (deg + 1) ** 2
    shapes = [(N, 3), (N, 3), (N, 4), (N,)]
    if F > 0:
        shapes += [(N, F), (G, 3), (mlp_weights(K, F, H),)]
    else:
        shapes += [(G, 3), (G, 3), (G, 4), (G,), (G, Cc, 3)]
    if vdeg >= 0:
        shapes.append((N, (vdeg + 1) ** 2))
    need = _HEADER.size + 4 * sum(int(np.prod(s)) for s in shapes)
    if len(raw) != need:
        raise ValueError(f"{path}: {len(raw)} bytes, the header describes {need}")
    arrs, o = [], _HEADER.size
    for s in shapes:
        n = int(np.prod(s))
        arrs.append(np.frombuffer(raw, dtype="<f4", count=n, offset=o).reshape(s).astype(np.float32))
        o += 4 * n
    cells, rest = arrs[:4], arrs[4:]
    v_sh = rest.pop() if vdeg >= 0 else None
    if F > 0:
        feat, offset, mlp = rest
        z = lambda *s: np.zeros(s, np.float32)
        gauss = [z(G, 3), z(G, 3), z(G, 4), z(G), z(G, 1, 3)]
        neural = dict(F=F, H=H, feat=feat, offset=offset, mlp=mlp)
    else:
        gauss, neural = rest, None
    return Scene(K, deg, *cells, *gauss, name=name, cell_v_sh=v_sh, v_sh_degree=vdeg, neural=neural)
