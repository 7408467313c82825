"""ctypes binding of liblinprim.so (include/linprim.h).  Argument marshalling
only: every step of rendering and differentiation runs in the library's CUDA
kernels.  Loading fails loudly when the library has not been built."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblinprim.so")

LP_OK, LP_ERR_INVALID, LP_ERR_CAPACITY, LP_ERR_CUDA, LP_ERR_TIMEOUT, LP_ERR_UNSUPPORTED, \
    LP_ERR_STATE = range(7)
LP_TETRAHEDRON, LP_OCTAHEDRON = 4, 6
LP_MAX_CAMERAS = 32

# Every symbol include/linprim.h declares.
EXPORTS = ("lp_create", "lp_destroy", "lp_set_tuning", "lp_get_tuning", "lp_set_filter_2d", "lp_get_filter_2d",
           "lp_reserve",
           "lp_render_forward", "lp_render_backward", "lp_sync_status", "lp_get_stats",
           "lp_debug_keys", "lp_debug_counts", "lp_debug_pixel_state", "lp_count_pairs",
           "lp_last_error", "lp_status_string", "lp_set_timing", "lp_stage_times",
           "lp_render_forward_noalloc", "lp_params_forward", "lp_params_backward",
           "lp_l1_loss_grad", "lp_adam_step", "lp_render_depth", "lp_set_exact", "lp_get_exact",
           "lp_set_densify_stats", "lp_population_scratch", "lp_population_decide", "lp_population_apply",
           "lp_set_debug_guard", "lp_check_guards", "lp_debug_sort_stall", "lp_debug_scan")
LP_ADAM_MAX_GROUPS = 8
STAGES = ("preprocess", "scan_emit", "sort", "ranges", "blend_fwd", "blend_bwd", "chain")


class lp_camera(C.Structure):
    _fields_ = [("viewmat", C.c_float * 16), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int), ("height", C.c_int)]


class lp_prims(C.Structure):
    _fields_ = [("kind", C.c_int), ("n", C.c_int), ("sh_degree", C.c_int),
                ("centre", C.c_void_p), ("verts", C.c_void_p), ("opacity", C.c_void_p),
                ("sh", C.c_void_p)]


class lp_tuning(C.Structure):
    _fields_ = [("tile", C.c_int), ("batch", C.c_int), ("blocks_per_sm", C.c_int),
                ("sort_mode", C.c_int), ("pixels_per_thread", C.c_int), ("chain_split", C.c_int),
                ("radix_bits", C.c_int), ("tile_order", C.c_int), ("onesweep", C.c_int)]


class lp_stats(C.Structure):
    _fields_ = [("records", C.c_longlong), ("entries", C.c_longlong), ("tiles", C.c_longlong),
                ("pixels", C.c_longlong), ("sort_passes", C.c_int), ("key_bits", C.c_int),
                ("launches_fwd", C.c_int), ("launches_bwd", C.c_int)]


class lp_adam_group(C.Structure):
    _fields_ = [("offset", C.c_longlong), ("count", C.c_longlong), ("lr", C.c_float),
                ("lr_final", C.c_float), ("decay_steps", C.c_int), ("period", C.c_int),
                ("head", C.c_int), ("lr_tail", C.c_float)]


LP_POP_PRUNE, LP_POP_KEEP, LP_POP_CLONE, LP_POP_SPLIT = range(4)


class lp_population_rules(C.Structure):
    _fields_ = [("scene_extent", C.c_float), ("min_opacity", C.c_float), ("max_scene_frac", C.c_float),
                ("max_pixels", C.c_uint), ("grad_threshold", C.c_float), ("clone_scene_frac", C.c_float)]


class lp_param_arrays(C.Structure):
    _fields_ = [("centre", C.c_void_p), ("quat", C.c_void_p), ("dist", C.c_void_p), ("logit", C.c_void_p),
                ("sh", C.c_void_p)]


class LinPrimError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(msg)
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load the library once; raise if it is missing (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    L = C.CDLL(path)
    vp, ll, i = C.c_void_p, C.c_longlong, C.c_int
    L.lp_create.argtypes = [C.POINTER(vp), i]
    L.lp_destroy.argtypes = [vp]
    L.lp_destroy.restype = None
    L.lp_set_tuning.argtypes = [vp, C.POINTER(lp_tuning)]
    L.lp_get_tuning.argtypes = [vp, C.POINTER(lp_tuning)]
    L.lp_set_filter_2d.argtypes = [vp, C.c_float]
    L.lp_get_filter_2d.argtypes = [vp, C.POINTER(C.c_float)]
    L.lp_reserve.argtypes = [vp, ll, ll, ll, ll]
    L.lp_render_forward.argtypes = [vp, C.POINTER(lp_prims), C.POINTER(lp_camera), i,
                                    C.POINTER(C.c_float), vp, vp]
    L.lp_render_backward.argtypes = [vp, vp, vp, vp, vp, vp, i, vp]
    L.lp_sync_status.argtypes = [vp, vp]
    L.lp_get_stats.argtypes = [vp, C.POINTER(lp_stats)]
    L.lp_debug_keys.argtypes = [vp, vp, vp, ll, C.POINTER(ll)]
    L.lp_debug_counts.argtypes = [vp, vp, ll]
    L.lp_debug_pixel_state.argtypes = [vp, vp, vp, ll]
    L.lp_count_pairs.argtypes = [vp, C.POINTER(ll)]
    L.lp_set_debug_guard.argtypes = [vp, i]
    L.lp_debug_sort_stall.argtypes = [vp, i]
    L.lp_debug_scan.argtypes = [vp, vp, ll, vp, C.POINTER(C.c_uint), vp]
    L.lp_check_guards.argtypes = [vp, C.POINTER(ll), C.POINTER(ll)]
    L.lp_render_depth.argtypes = [vp, vp, vp]
    L.lp_set_exact.argtypes = [vp, i]
    L.lp_get_exact.argtypes = [vp, C.POINTER(i)]
    L.lp_last_error.argtypes = [vp]
    L.lp_last_error.restype = C.c_char_p
    L.lp_status_string.argtypes = [i]
    L.lp_status_string.restype = C.c_char_p
    L.lp_set_timing.argtypes = [vp, i]
    L.lp_stage_times.argtypes = [vp, C.POINTER(C.c_float)]
    L.lp_render_forward_noalloc.argtypes = [C.POINTER(lp_prims), C.POINTER(lp_camera),
                                            C.POINTER(C.c_float), vp, vp]
    L.lp_params_forward.argtypes = [i, i, vp, vp, vp, vp, vp, vp, vp]
    L.lp_params_backward.argtypes = [i, i, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.lp_l1_loss_grad.argtypes = [vp, vp, ll, vp, vp, vp]
    L.lp_adam_step.argtypes = [vp, vp, vp, vp, C.POINTER(lp_adam_group), i, C.c_float, C.c_float,
                               C.c_float, vp, vp]
    L.lp_set_densify_stats.argtypes = [vp, vp, vp, vp, ll]
    L.lp_population_scratch.argtypes = [ll]
    L.lp_population_scratch.restype = ll
    L.lp_population_decide.argtypes = [i, i, vp, vp, vp, vp, vp, C.POINTER(lp_population_rules), vp, vp, vp,
                                       vp, vp]
    L.lp_population_apply.argtypes = [i, i, i, vp, vp, vp, C.POINTER(lp_param_arrays),
                                      C.POINTER(lp_param_arrays), i, vp]
    for name in EXPORTS:
        getattr(L, name)
    _lib = L
    return L


def check(ctx, status: int, what: str):
    if status != LP_OK:
        L = load()
        msg = L.lp_last_error(ctx).decode() if ctx else ""
        raise LinPrimError(status, f"{what}: {L.lp_status_string(status).decode()} {msg}".strip())


def camera_struct(cameras):
    arr = (lp_camera * max(1, len(cameras)))()
    for k, c in enumerate(cameras):
        vm = [float(x) for x in __import__("numpy").asarray(c.viewmat, "float32").reshape(16)]
        arr[k].viewmat[:] = vm
        arr[k].fx, arr[k].fy, arr[k].cx, arr[k].cy = (float(c.fx), float(c.fy), float(c.cx),
                                                       float(c.cy))
        arr[k].width, arr[k].height = int(c.width), int(c.height)
    return arr
