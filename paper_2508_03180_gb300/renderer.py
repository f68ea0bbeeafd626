"""Python-side marshalling over the C ABI: torch tensors in, torch tensors out.

Nothing here computes any part of the renderer; every call forwards pointers
and sizes to libdgs.so (see _lib.py for the one-to-one ABI wrappers).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L


def _camera_struct(cam) -> L.dgs_camera:
    """From a synth.Camera or its float32[22] array."""
    a = cam.as_array() if hasattr(cam, "as_array") else np.asarray(cam, dtype=np.float32)
    c = L.dgs_camera()
    c.W, c.H = int(a[0]), int(a[1])
    c.fx, c.fy, c.cx, c.cy, c.znear = (float(x) for x in a[2:7])
    c.R[:] = [float(x) for x in a[7:16]]
    c.t[:] = [float(x) for x in a[16:19]]
    c.eye[:] = [float(x) for x in a[19:22]]
    return c


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


class Context:
    """One dgs_ctx on one CUDA device."""

    def __init__(self, device: int = 0, **cfg):
        self.lib = L.load()
        c = L.dgs_config_default()
        c.device = device
        for k, v in cfg.items():
            if k == "bg":
                c.bg[:] = list(v)
            else:
                setattr(c, k, v)
        self.ctx = L.dgs_create(c)
        self.device = torch.device("cuda", device)
        self._keep = {}
        self._next_slot = 0

    def close(self):
        if self.ctx is not None:
            L.dgs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ scenes
    def _desc(self, arrays: dict, N: int, K: int, deg: int, location: int, v_sh_degree: int = -1) -> L.dgs_scene_desc:
        d = L.dgs_scene_desc()
        d.num_cells, d.K, d.sh_degree, d.location = N, K, deg, location
        d.v_sh_degree = v_sh_degree
        for f in ("cell_center", "cell_axes", "cell_quat", "cell_v", "g_mean", "g_scale", "g_quat", "g_logit", "g_sh",
                  "cell_v_sh"):
            a = arrays.get(f)
            if a is None:
                setattr(d, f, None)
                continue
            setattr(d, f, a.data_ptr() if isinstance(a, torch.Tensor) else a.ctypes.data)
        return d

    def upload_scene(self, scene) -> int:
        """Upload a synth.Scene (host numpy arrays) or a dict of CUDA tensors
        with the same field names plus N, K, sh_degree."""
        if isinstance(scene, dict):
            arrays = {k: v.contiguous() for k, v in scene.items() if isinstance(v, torch.Tensor)}
            d = self._desc(arrays, scene["N"], scene["K"], scene["sh_degree"], L.DGS_DEVICE,
                           scene.get("v_sh_degree", -1))
        else:
            arrays = {f: np.ascontiguousarray(getattr(scene, f), dtype=np.float32)
                      for f in ("cell_center", "cell_axes", "cell_quat", "cell_v", "g_mean", "g_scale", "g_quat",
                                "g_logit", "g_sh")}
            vdeg = getattr(scene, "v_sh_degree", -1)
            if getattr(scene, "cell_v_sh", None) is not None:
                arrays["cell_v_sh"] = np.ascontiguousarray(scene.cell_v_sh, dtype=np.float32)
            d = self._desc(arrays, scene.N, scene.K, scene.sh_degree, L.DGS_HOST, vdeg)
            if getattr(scene, "neural", None) is not None:
                nr = scene.neural
                keep = {k: np.ascontiguousarray(nr[k], dtype=np.float32) for k in ("feat", "offset", "mlp")}
                nd = L.dgs_neural_desc()
                nd.feat_dim, nd.hidden = nr["F"], nr["H"]
                nd.cell_feat, nd.g_offset, nd.mlp = (keep[k].ctypes.data for k in ("feat", "offset", "mlp"))
                d.neural = C.pointer(nd)
                arrays["_neural"] = (nd, keep)  # alive during the call
        return L.dgs_scene_upload(self.ctx, d)

    def update_scene(self, scene_id: int, N: int, K: int, deg: int, **tensors):
        """Overwrite Gaussian parameters (CUDA tensors, ABI layout) in place."""
        arrays = {k: v.contiguous() for k, v in tensors.items()}
        d = self._desc(arrays, N, K, deg, L.DGS_DEVICE)
        L.dgs_scene_update(self.ctx, scene_id, d, _stream())
        self._keep["update"] = arrays  # alive until the stream has consumed them

    def release_scene(self, scene_id: int):
        L.dgs_scene_release(self.ctx, scene_id)

    def save_scene(self, scene_id: int, path) -> None:
        """Write the scene's current parameters to a scene file."""
        L.dgs_scene_save(self.ctx, scene_id, path)

    def load_scene(self, path) -> int:
        """Upload the scene stored in a scene file; returns its id."""
        return L.dgs_scene_load(self.ctx, path)

    # ------------------------------------------------------------ cameras
    def set_camera(self, slot: int, cam):
        L.dgs_camera_set(self.ctx, slot, _camera_struct(cam))

    def set_cameras(self, cams) -> list[int]:
        slots = list(range(len(cams)))
        for s, c in zip(slots, cams):
            self.set_camera(s, c)
        return slots

    # ------------------------------------------------------------ render
    @staticmethod
    def image_sizes(cams):
        out = []
        for c in cams:
            a = c.as_array() if hasattr(c, "as_array") else np.asarray(c)
            out.append((int(a[1]), int(a[0])))
        return out

    def render(self, scene_id: int, cams, want_state: bool = False, out: torch.Tensor | None = None,
               stats: bool = False, slots=None):
        """Render views; returns (flat image tensor, state or None, stats or None).

        The flat tensor holds view v as [3][H_v][W_v] back to back."""
        if slots is None:
            slots = self.set_cameras(cams)
        sizes = self.image_sizes(cams)
        n = sum(3 * h * w for h, w in sizes)
        if out is None:
            out = torch.empty(n, dtype=torch.float32, device=self.device)
        st = L.dgs_stats() if stats else None
        state = L.dgs_render(self.ctx, scene_id, slots, _ptr(out), L.DGS_DEVICE, want_state, _stream(), st)
        return out, state, st

    def render_compare(self, scene_id: int, cams, mode: str = "alpha", tau: float = float("inf"),
                       w_bg: float = 0.0, want_ndone: bool = False, stats: bool = False):
        """Comparator renderers: mode "alpha" (per-Gaussian depth-sorted
        alpha-blending) or "wsr" (weighted-sum rendering with the LC-WSR
        weight; tau = inf for plain WSR).  Returns (flat image, ndone or None,
        stats or None)."""
        slots = self.set_cameras(cams)
        sizes = self.image_sizes(cams)
        out = torch.empty(sum(3 * h * w for h, w in sizes), dtype=torch.float32, device=self.device)
        nd = torch.empty(sum(h * w for h, w in sizes), dtype=torch.int32, device=self.device) if want_ndone else None
        cfg = L.dgs_compare_config()
        cfg.mode = {"alpha": L.DGS_COMPARE_ALPHA, "wsr": L.DGS_COMPARE_WSR}[mode]
        cfg.tau = tau if np.isfinite(tau) else 0.0
        cfg.w_bg = w_bg
        st = L.dgs_stats() if stats else None
        L.dgs_render_compare(self.ctx, scene_id, slots, cfg, _ptr(out), _ptr(nd) if nd is not None else 0,
                             _stream(), st)
        return out, nd, st

    def render_host(self, scene_id: int, cams, out: np.ndarray):
        slots = self.set_cameras(cams)
        L.dgs_render(self.ctx, scene_id, slots, out.ctypes.data, L.DGS_HOST, False, _stream(), None)
        return out

    @staticmethod
    def split(flat: torch.Tensor, cams):
        outs, o = [], 0
        for h, w in Context.image_sizes(cams):
            outs.append(flat[o:o + 3 * h * w].view(3, h, w))
            o += 3 * h * w
        return outs

    def backward(self, state, dL: torch.Tensor, grads: dict, location: int = L.DGS_DEVICE):
        """grads: dict of preallocated tensors/arrays keyed g_mean, g_scale,
        g_log_scale, g_quat, g_logit, g_sh, g_cell_v, g_cell_v_sh, g_cell_center,
        g_cell_axes, g_cell_quat (any subset; neural scenes: g_mlp, g_feat,
        g_offset and the cell gradients)."""
        g = L.dgs_grads()
        g.location = location
        for f in ("g_mean", "g_scale", "g_log_scale", "g_quat", "g_logit", "g_sh", "g_cell_v", "g_cell_v_sh",
                  "g_mlp", "g_feat", "g_offset", "g_cell_center", "g_cell_axes", "g_cell_quat"):
            a = grads.get(f)
            setattr(g, f, None if a is None else (a.data_ptr() if isinstance(a, torch.Tensor) else a.ctypes.data))
        dl_ptr = dL.data_ptr() if isinstance(dL, torch.Tensor) else dL.ctypes.data
        dl_loc = L.DGS_DEVICE if isinstance(dL, torch.Tensor) and dL.is_cuda else L.DGS_HOST
        L.dgs_render_backward(self.ctx, state, dl_ptr, dl_loc, g, _stream())

    def release_state(self, state):
        L.dgs_state_release(self.ctx, state)

    def read(self, state, what: int, dtype, shape=None) -> np.ndarray:
        need = L.dgs_state_read(self.ctx, state, what, None, 0)
        buf = np.empty(need // np.dtype(dtype).itemsize, dtype=dtype)
        if need:
            L.dgs_state_read(self.ctx, state, what, buf.ctypes.data, need)
        return buf if shape is None else buf.reshape(shape)

    def loss_l1(self, rgb: torch.Tensor, target: torch.Tensor, dL: torch.Tensor, loss: torch.Tensor):
        L.dgs_loss_l1(self.ctx, _ptr(rgb), _ptr(target), rgb.numel(), _ptr(dL), _ptr(loss), _stream())

    def sort_pairs(self, keys: torch.Tensor, vals: torch.Tensor, bits: int):
        L.dgs_sort_pairs(self.ctx, _ptr(keys), _ptr(vals), keys.numel(), bits, _stream())

    # ------------------------------------------------------------ diagnostics
    def counts(self, state) -> dict:
        c = L.dgs_state_counts(self.ctx, state)
        return dict(pairs_blended=c.pairs_blended, inbox_rendered=c.inbox_rendered, inbox_all=c.inbox_all,
                    cells_blended=c.cells_blended)

    def profile_enable(self, on: bool = True):
        L.dgs_profile_enable(self.ctx, on)

    def profile_read(self) -> dict:
        p = L.dgs_profile_read(self.ctx)
        return {name: (p.ms[i], p.launches[i]) for i, name in enumerate(L.STAGES)}

    def cell_align(self, scene_id: int, quat: bool = True, center: bool = True, cam=None,
                   out_center=None, out_quat=None):
        """Cell alignment (Sec. IV-B) in place: Q_n by Eq. 10 and/or x_n as the
        mean of the Gaussians' centres.  Neural scenes need `cam` for Eq. 10.
        out_center [N][3] / out_quat [N][4]: optional tensors (device) or
        arrays (host) that receive the new values."""
        what = (L.DGS_ALIGN_QUAT if quat else 0) | (L.DGS_ALIGN_CENTER if center else 0)
        slot = self.set_cameras([cam])[0] if cam is not None else -1
        outs = [a for a in (out_center, out_quat) if a is not None]
        host = bool(outs) and not isinstance(outs[0], torch.Tensor)
        ptr = lambda a: None if a is None else (a.ctypes.data if host else a.data_ptr())
        L.dgs_cell_align(self.ctx, scene_id, what, slot, ptr(out_center), ptr(out_quat),
                         L.DGS_HOST if host else L.DGS_DEVICE, _stream())

    def probe_alu(self) -> dict:
        r = L.dgs_probe_alu(self.ctx)
        return {"fp32_tflops": r.fp32_tflops, "ex2_per_s": r.ex2_per_s, "ms_fma": r.ms_fma, "ms_ex2": r.ms_ex2,
                "sm_count": r.sm_count}

    # ------------------------------------------------------------ serving
    def serve_start(self, max_batch: int = 8, queue_cap: int = 1024, graphs: bool = True):
        """graphs=False runs each batch as a plain launch chain instead of a
        replay of a captured graph."""
        L.dgs_serve_start(self.ctx, max_batch, queue_cap, 0 if graphs else L.DGS_SERVE_NO_GRAPHS)

    def serve_stats(self) -> dict:
        r = L.dgs_serve_read_stats(self.ctx)
        return {"batches": r.batches, "graphs_captured": r.graphs_captured,
                "overflow_retries": r.overflow_retries, "pairs_per_tile": r.pairs_per_tile}

    def serve_stop(self):
        L.dgs_serve_stop(self.ctx)

    def submit(self, scene_id: int, cam, out: torch.Tensor) -> int:
        r = L.dgs_request()
        r.scene_id = scene_id
        r.out_location = L.DGS_DEVICE if out.is_cuda else L.DGS_HOST
        r.camera = _camera_struct(cam)
        r.out_rgb = out.data_ptr()
        return L.dgs_submit(self.ctx, r)

    def poll(self, ticket: int, timeout_us: int = -1):
        return L.dgs_poll(self.ctx, ticket, timeout_us)

    def cancel(self, ticket: int):
        L.dgs_cancel(self.ctx, ticket)
