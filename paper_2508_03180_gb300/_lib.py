"""ctypes binding of the C ABI in include/dgs.h (argument marshalling only).

Every function below has the name of the C entry point it calls.  The
library is the in-tree libdgs.so built by paper_2508_03180_gb300.build;
importing a function that needs it fails loudly when it cannot be loaded --
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

DGS_OK = 0
DGS_ERR_INVALID_ARG = -1
DGS_ERR_OOM = -2
DGS_ERR_NOT_FOUND = -3
DGS_ERR_CUDA = -4
DGS_ERR_TIMEOUT = -5
DGS_ERR_BUSY = -6
DGS_ERR_CAPACITY = -7
DGS_ERR_GUARD = -8
DGS_ERR_WORKER = -9
DGS_ERR_CANCELLED = -10
DGS_FAULT_ALLOC = 1
DGS_FAULT_SORT_WAIT = 2
DGS_FAULT_SERVE_WORKER = 3
DGS_FAULT_GUARD = 4
DGS_FAULT_TC_WAIT = 5
DGS_HOST = 0
DGS_DEVICE = 1

DGS_BUF_CELL_RECT = 1
DGS_BUF_CELL_DEPTH = 2
DGS_BUF_TILE_CELLS = 3
DGS_BUF_TILE_RANGES = 4
DGS_BUF_GAUSS_REC = 5
DGS_BUF_PIX_D = 6
DGS_BUF_PIX_NDONE = 7
DGS_BUF_GRAD2D = 8
DGS_BUF_CELL_V = 9
DGS_BUF_DECODED = 10

_P = C.c_void_p
_FP = C.POINTER(C.c_float)


class dgs_config(C.Structure):
    _fields_ = [("eps", C.c_float), ("alpha_max", C.c_float), ("d_min", C.c_float), ("bg", C.c_float * 3),
                ("dilation", C.c_float), ("ksigma", C.c_float), ("device", C.c_int32), ("flags", C.c_int32),
                ("hbm_budget_bytes", C.c_int64), ("w_bg", C.c_float), ("reserved", C.c_int32)]


DGS_FLAG_ALPHA_SKIP = 1
DGS_FLAG_TERM_EXCLUDE = 2
DGS_FLAG_AABB_SQUARE = 4
DGS_FLAG_NUMERATOR = 8
DGS_FLAG_NEAR_FULL = 16


class dgs_neural_desc(C.Structure):
    _fields_ = [("feat_dim", C.c_int32), ("hidden", C.c_int32), ("cell_feat", _P), ("g_offset", _P), ("mlp", _P)]


class dgs_scene_desc(C.Structure):
    _fields_ = [("num_cells", C.c_int64), ("K", C.c_int32), ("sh_degree", C.c_int32), ("location", C.c_int32),
                ("reserved", C.c_int32), ("cell_center", _P), ("cell_axes", _P), ("cell_quat", _P), ("cell_v", _P),
                ("g_mean", _P), ("g_scale", _P), ("g_quat", _P), ("g_logit", _P), ("g_sh", _P),
                ("cell_v_sh", _P), ("v_sh_degree", C.c_int32), ("reserved2", C.c_int32),
                ("neural", C.POINTER(dgs_neural_desc))]


class dgs_camera(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float),
                ("cy", C.c_float), ("znear", C.c_float), ("R", C.c_float * 9), ("t", C.c_float * 3),
                ("eye", C.c_float * 3)]


class dgs_stats(C.Structure):
    _fields_ = [("sort_length", C.c_int64), ("visible_cells", C.c_int64), ("num_tiles", C.c_int64),
                ("ms_total", C.c_float), ("timing", C.c_int32), ("reserved", C.c_int32)]


class dgs_grads(C.Structure):
    _fields_ = [("location", C.c_int32), ("reserved", C.c_int32), ("g_mean", _P), ("g_scale", _P), ("g_log_scale", _P),
                ("g_quat", _P), ("g_logit", _P), ("g_sh", _P), ("g_cell_v", _P), ("g_cell_v_sh", _P),
                ("g_mlp", _P), ("g_feat", _P), ("g_offset", _P), ("g_cell_center", _P), ("g_cell_axes", _P),
                ("g_cell_quat", _P)]


class dgs_counts(C.Structure):
    _fields_ = [("pairs_blended", C.c_int64), ("inbox_rendered", C.c_int64), ("inbox_all", C.c_int64),
                ("cells_blended", C.c_int64)]


class dgs_profile(C.Structure):
    _fields_ = [("ms", C.c_double * 16), ("launches", C.c_int64 * 16)]


STAGES = ["cell_project", "depth_sort", "count_scan", "emit", "tile_sort", "tile_ranges", "project_fwd",
          "blend_fwd", "blend_bwd", "project_bwd", "decode", "decode_bwd"]


class dgs_request(C.Structure):
    _fields_ = [("scene_id", C.c_uint32), ("out_location", C.c_int32), ("camera", dgs_camera), ("out_rgb", _P)]


class dgs_serve_stats(C.Structure):
    _fields_ = [("batches", C.c_int64), ("graphs_captured", C.c_int64), ("overflow_retries", C.c_int64),
                ("pairs_per_tile", C.c_double)]


class dgs_alu_peaks(C.Structure):
    _fields_ = [("fp32_tflops", C.c_double), ("ex2_per_s", C.c_double), ("ms_fma", C.c_float),
                ("ms_ex2", C.c_float), ("sm_count", C.c_int32), ("reserved", C.c_int32)]


DGS_SERVE_NO_GRAPHS = 1
DGS_COMPARE_ALPHA = 1
DGS_COMPARE_WSR = 2
DGS_ALIGN_QUAT = 1
DGS_ALIGN_CENTER = 2


class dgs_compare_config(C.Structure):
    _fields_ = [("mode", C.c_int32), ("tau", C.c_float), ("w_bg", C.c_float), ("reserved", C.c_int32)]


class dgs_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("batch_size", C.c_int32), ("t_submit_ms", C.c_double),
                ("t_start_ms", C.c_double), ("t_done_ms", C.c_double)]


_SIGS = {
    "dgs_config_default": (None, [C.POINTER(dgs_config)]),
    "dgs_create": (C.c_int32, [C.POINTER(dgs_config), C.POINTER(_P)]),
    "dgs_destroy": (None, [_P]),
    "dgs_last_error": (C.c_char_p, [_P]),
    "dgs_scene_upload": (C.c_int32, [_P, C.POINTER(dgs_scene_desc), C.POINTER(C.c_uint32)]),
    "dgs_scene_update": (C.c_int32, [_P, C.c_uint32, C.POINTER(dgs_scene_desc), _P]),
    "dgs_scene_release": (C.c_int32, [_P, C.c_uint32]),
    "dgs_scene_save": (C.c_int32, [_P, C.c_uint32, C.c_char_p]),
    "dgs_scene_load": (C.c_int32, [_P, C.c_char_p, C.POINTER(C.c_uint32)]),
    "dgs_camera_set": (C.c_int32, [_P, C.c_uint32, C.POINTER(dgs_camera)]),
    "dgs_render": (C.c_int32, [_P, C.c_uint32, C.c_int32, C.POINTER(C.c_uint32), _P, C.c_int32, C.POINTER(_P), _P,
                               C.POINTER(dgs_stats)]),
    "dgs_render_backward": (C.c_int32, [_P, _P, _P, C.c_int32, C.POINTER(dgs_grads), _P]),
    "dgs_state_release": (C.c_int32, [_P, _P]),
    "dgs_loss_l1": (C.c_int32, [_P, _P, _P, C.c_int64, _P, _P, _P]),
    "dgs_state_read": (C.c_int32, [_P, _P, C.c_int32, _P, C.c_int64, C.POINTER(C.c_int64)]),
    "dgs_sort_pairs": (C.c_int32, [_P, _P, _P, C.c_int64, C.c_int32, _P]),
    "dgs_sort_pairs_noalloc": (C.c_int32, [_P, _P, C.c_int64, C.c_int32, _P]),
    "dgs_state_counts": (C.c_int32, [_P, _P, C.POINTER(dgs_counts)]),
    "dgs_profile_enable": (C.c_int32, [_P, C.c_int32]),
    "dgs_profile_read": (C.c_int32, [_P, C.POINTER(dgs_profile)]),
    "dgs_render_compare": (C.c_int32, [_P, C.c_uint32, C.c_int32, C.POINTER(C.c_uint32),
                                       C.POINTER(dgs_compare_config), _P, _P, _P, C.POINTER(dgs_stats)]),
    "dgs_probe_alu": (C.c_int32, [_P, C.POINTER(dgs_alu_peaks)]),
    "dgs_cell_align": (C.c_int32, [_P, C.c_uint32, C.c_int32, C.c_int32, _P, _P, C.c_int32, _P]),
    "dgs_serve_start": (C.c_int32, [_P, C.c_int32, C.c_int32, C.c_int32]),
    "dgs_serve_read_stats": (C.c_int32, [_P, C.POINTER(dgs_serve_stats)]),
    "dgs_serve_stop": (C.c_int32, [_P]),
    "dgs_submit": (C.c_int32, [_P, C.POINTER(dgs_request), C.POINTER(C.c_uint64)]),
    "dgs_poll": (C.c_int32, [_P, C.c_uint64, C.c_int64, C.POINTER(dgs_result)]),
    "dgs_cancel": (C.c_int32, [_P, C.c_uint64]),
    "dgs_debug_guards": (C.c_int32, [C.c_int32]),
    "dgs_debug_check_guards": (C.c_int32, [C.POINTER(C.c_int64)]),
    "dgs_debug_inject_fault": (C.c_int32, [_P, C.c_int32, C.c_int32]),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libdgs.so (building it first if sources changed)."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_needed else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libdgs.so not found at {path}; run paper_2508_03180_gb300.build.build()")
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return sorted(_SIGS)


class DgsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"dgs error {code}: {msg}")
        self.code = code


def check(code, ctx=None):
    if code != DGS_OK:
        msg = load().dgs_last_error(ctx)
        raise DgsError(code, msg.decode() if msg else "")
    return code


# thin wrappers with the C names ------------------------------------------------------------


def dgs_config_default() -> dgs_config:
    c = dgs_config()
    load().dgs_config_default(C.byref(c))
    return c


def dgs_create(cfg: dgs_config | None = None):
    ctx = _P()
    check(load().dgs_create(C.byref(cfg) if cfg is not None else None, C.byref(ctx)))
    return ctx


def dgs_destroy(ctx):
    load().dgs_destroy(ctx)


def dgs_last_error(ctx=None) -> str:
    m = load().dgs_last_error(ctx)
    return m.decode() if m else ""


def dgs_scene_upload(ctx, desc: dgs_scene_desc) -> int:
    sid = C.c_uint32()
    check(load().dgs_scene_upload(ctx, C.byref(desc), C.byref(sid)), ctx)
    return sid.value


def dgs_scene_update(ctx, scene_id: int, desc: dgs_scene_desc, stream: int = 0):
    check(load().dgs_scene_update(ctx, scene_id, C.byref(desc), _P(stream)), ctx)


def dgs_scene_release(ctx, scene_id: int):
    check(load().dgs_scene_release(ctx, scene_id), ctx)


def dgs_scene_save(ctx, scene_id: int, path) -> None:
    check(load().dgs_scene_save(ctx, scene_id, os.fsencode(path)), ctx)


def dgs_scene_load(ctx, path) -> int:
    sid = C.c_uint32()
    check(load().dgs_scene_load(ctx, os.fsencode(path), C.byref(sid)), ctx)
    return sid.value


def dgs_camera_set(ctx, slot: int, cam: dgs_camera):
    check(load().dgs_camera_set(ctx, slot, C.byref(cam)), ctx)


def dgs_render(ctx, scene_id: int, cam_slots, out_ptr: int, out_location: int, want_state: bool, stream: int = 0,
               stats: dgs_stats | None = None):
    slots = (C.c_uint32 * len(cam_slots))(*cam_slots)
    state = _P()
    check(load().dgs_render(ctx, scene_id, len(cam_slots), slots, _P(out_ptr), out_location,
                            C.byref(state) if want_state else None, _P(stream),
                            C.byref(stats) if stats is not None else None), ctx)
    return state if want_state else None


def dgs_render_compare(ctx, scene_id: int, cam_slots, cfg: dgs_compare_config, out_ptr: int, ndone_ptr,
                       stream: int = 0, stats: dgs_stats | None = None):
    slots = (C.c_uint32 * len(cam_slots))(*cam_slots)
    check(load().dgs_render_compare(ctx, scene_id, len(cam_slots), slots, C.byref(cfg), _P(out_ptr),
                                    _P(ndone_ptr) if ndone_ptr else None, _P(stream),
                                    C.byref(stats) if stats is not None else None), ctx)


def dgs_render_backward(ctx, state, dl_ptr: int, location: int, grads: dgs_grads, stream: int = 0):
    check(load().dgs_render_backward(ctx, state, _P(dl_ptr), location, C.byref(grads), _P(stream)), ctx)


def dgs_state_release(ctx, state):
    check(load().dgs_state_release(ctx, state), ctx)


def dgs_loss_l1(ctx, rgb_ptr: int, target_ptr: int, n: int, dl_ptr: int, loss_ptr: int, stream: int = 0):
    check(load().dgs_loss_l1(ctx, _P(rgb_ptr), _P(target_ptr), n, _P(dl_ptr), _P(loss_ptr), _P(stream)), ctx)


def dgs_state_read(ctx, state, what: int, dst_ptr: int | None, nbytes: int) -> int:
    need = C.c_int64()
    check(load().dgs_state_read(ctx, state, what, _P(dst_ptr) if dst_ptr else None, nbytes, C.byref(need)), ctx)
    return need.value


def dgs_sort_pairs(ctx, keys_ptr: int, vals_ptr: int, n: int, bits: int, stream: int = 0):
    check(load().dgs_sort_pairs(ctx, _P(keys_ptr), _P(vals_ptr), n, bits, _P(stream)), ctx)


def dgs_sort_pairs_noalloc(keys_ptr: int, vals_ptr: int, n: int, bits: int, stream: int = 0):
    """Sort without allocating (fixed scratch, n <= 1,048,576)."""
    check(load().dgs_sort_pairs_noalloc(_P(keys_ptr), _P(vals_ptr), n, bits, _P(stream)))


def dgs_state_counts(ctx, state) -> dgs_counts:
    c = dgs_counts()
    check(load().dgs_state_counts(ctx, state, C.byref(c)), ctx)
    return c


def dgs_profile_enable(ctx, on: bool):
    check(load().dgs_profile_enable(ctx, 1 if on else 0), ctx)


def dgs_profile_read(ctx) -> dgs_profile:
    p = dgs_profile()
    check(load().dgs_profile_read(ctx, C.byref(p)), ctx)
    return p


def dgs_cell_align(ctx, scene_id: int, what: int, cam_slot: int, center_ptr, quat_ptr, location: int, stream):
    check(load().dgs_cell_align(ctx, scene_id, what, cam_slot, _P(center_ptr) if center_ptr else None,
                                _P(quat_ptr) if quat_ptr else None, location, stream), ctx)


def dgs_probe_alu(ctx) -> dgs_alu_peaks:
    r = dgs_alu_peaks()
    check(load().dgs_probe_alu(ctx, C.byref(r)), ctx)
    return r


def dgs_serve_start(ctx, max_batch: int, queue_cap: int, flags: int = 0):
    check(load().dgs_serve_start(ctx, max_batch, queue_cap, flags), ctx)


def dgs_serve_read_stats(ctx) -> dgs_serve_stats:
    r = dgs_serve_stats()
    check(load().dgs_serve_read_stats(ctx, C.byref(r)), ctx)
    return r


def dgs_serve_stop(ctx):
    check(load().dgs_serve_stop(ctx), ctx)


def dgs_submit(ctx, req: dgs_request) -> int:
    t = C.c_uint64()
    check(load().dgs_submit(ctx, C.byref(req), C.byref(t)), ctx)
    return t.value


def dgs_cancel(ctx, ticket: int):
    check(load().dgs_cancel(ctx, ticket), ctx)


def dgs_poll(ctx, ticket: int, timeout_us: int):
    """Returns a dgs_result, or None on DGS_ERR_TIMEOUT."""
    r = dgs_result()
    code = load().dgs_poll(ctx, ticket, timeout_us, C.byref(r))
    if code == DGS_ERR_TIMEOUT:
        return None
    check(code, ctx)
    return r


def dgs_debug_guards(on: bool):
    check(load().dgs_debug_guards(1 if on else 0))


def dgs_debug_check_guards() -> int:
    n = C.c_int64()
    check(load().dgs_debug_check_guards(C.byref(n)))
    return n.value


def dgs_debug_inject_fault(ctx, kind: int, count: int):
    check(load().dgs_debug_inject_fault(ctx, kind, count), ctx)
