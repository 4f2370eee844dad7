"""ctypes binding of libgsr.so (include/gsr.h): argument marshalling only.

Every compute step runs in the library's CUDA kernels; this module converts
Python/torch objects into the C structs and raises on any non-OK status.  It
fails loudly when the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional

_PKG = os.path.dirname(os.path.abspath(__file__))
# GSR_LIBRARY selects another build of the library, e.g. libgsr_checked.so
LIB_PATH = os.environ.get("GSR_LIBRARY") or os.path.join(_PKG, "_build", "libgsr.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "gsr.h")

MAX_VIEWS = 64
ABI_VERSION = 7   # GSR_ABI_VERSION these structs follow
STATUS = {0: "GSR_OK", -1: "GSR_EINVAL", -2: "GSR_ECAPACITY", -3: "GSR_ECUDA", -4: "GSR_ETIMEOUT",
          -5: "GSR_ENOTREADY", -6: "GSR_EINTERNAL"}
OK, EINVAL, ECAPACITY, ECUDA, ETIMEOUT, ENOTREADY, EINTERNAL = 0, -1, -2, -3, -4, -5, -6
TEST_STALL_SORT = 1
BIN_TILE, BIN_RADIX = 0, 1
STAGE_EVENTS = 10
# stage k lasts from event STAGE_SPANS[k][0] to STAGE_SPANS[k][1]
STAGES = ("preprocess", "scan_duplicate", "sort", "ranges", "blend_fwd", "clear", "blend_bwd", "preprocess_bwd")
STAGE_SPANS = ((0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (6, 7), (7, 8), (8, 9))

_p = ctypes.c_void_p


class Config(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int), ("spin_limit", ctypes.c_uint32), ("flags", ctypes.c_int),
                ("binning", ctypes.c_int), ("batch", ctypes.c_int), ("fwd_rows", ctypes.c_int)]


class Gaussians(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("sh_degree", ctypes.c_int), ("means", _p), ("log_scales", _p),
                ("quats", _p), ("opacity_logits", _p), ("sh", _p)]


class View(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("T_cw", _p), ("color", _p), ("depth", _p),
                ("alpha", _p), ("median_depth", _p)]


class ViewGrad(ctypes.Structure):
    _fields_ = [("d_color", _p), ("d_depth", _p), ("d_alpha", _p), ("d_median_depth", _p), ("d_pose", _p)]


class Grads(ctypes.Structure):
    _fields_ = [("means", _p), ("log_scales", _p), ("quats", _p), ("opacity_logits", _p), ("sh", _p),
                ("accumulate", ctypes.c_int), ("densify_grad", _p), ("densify_count", _p), ("densify_radius", _p)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("keys", ctypes.c_uint32), ("key_capacity", ctypes.c_uint32),
                ("tiles", ctypes.c_uint32), ("pairs_contributing", ctypes.c_uint64), ("pairs_visible", ctypes.c_uint32),
                ("pairs_backward", ctypes.c_uint32)]


class L1View(ctypes.Structure):
    _fields_ = [("target_color", _p), ("target_depth", _p), ("d_color", _p), ("d_depth", _p)]


class SurfelOut(ctypes.Structure):
    _fields_ = [("normal", _p), ("distortion", _p)]


class SurfelGrad(ctypes.Structure):
    _fields_ = [("d_normal", _p), ("d_distortion", _p)]


class AdcParams(ctypes.Structure):
    _fields_ = [("grad_threshold", ctypes.c_float), ("split_scale", ctypes.c_float), ("min_opacity", ctypes.c_float),
                ("max_screen_radius", ctypes.c_float), ("max_world_scale", ctypes.c_float)]


class GaussiansOut(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("means", _p), ("log_scales", _p), ("quats", _p), ("opacity_logits", _p),
                ("sh", _p)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int), ("binning", ctypes.c_int), ("batch", ctypes.c_int), ("fwd_rows", ctypes.c_int),
                ("ms", ctypes.c_float), ("status", ctypes.c_int32)]


ABI_STRUCTS = [Config, Gaussians, View, ViewGrad, Grads, Info, L1View, SurfelOut, SurfelGrad, AdcParams,
               GaussiansOut, TuneEntry]

_lib: Optional[ctypes.CDLL] = None


class GsrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def declared_functions() -> list:
    """Names of the functions include/gsr.h declares."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(gsr_[a-z_0-9]+)\s*\(", text, re.M)))


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libgsr.so is not built ({path}); run `python -m paper_2411_17660_b300.build`")
    lib = ctypes.CDLL(path)
    c_int, c_size = ctypes.c_int, ctypes.c_size_t
    sig = {
        "gsr_create": (c_int, [ctypes.POINTER(Config), ctypes.POINTER(_p)]),
        "gsr_destroy": (c_int, [_p]),
        "gsr_workspace_size": (c_int, [_p, c_int, ctypes.POINTER(View), c_int, c_size, ctypes.POINTER(c_size)]),
        "gsr_render": (c_int, [_p, ctypes.POINTER(Gaussians), ctypes.POINTER(View), c_int, _p, c_size, _p]),
        "gsr_render_l1": (c_int, [_p, ctypes.POINTER(Gaussians), ctypes.POINTER(View), c_int,
                                  ctypes.POINTER(L1View), ctypes.c_float, ctypes.c_float, _p, _p, c_size, _p]),
        "gsr_render_backward": (c_int, [_p, ctypes.POINTER(Gaussians), ctypes.POINTER(View),
                                         ctypes.POINTER(ViewGrad), c_int, ctypes.POINTER(Grads), _p, c_size, _p]),
        "gsr_read_info": (c_int, [_p, _p, c_size, ctypes.POINTER(Info), _p]),
        "gsr_get_status": (c_int, [_p, _p, c_size, _p]),
        "gsr_autotune": (c_int, [_p, ctypes.POINTER(Gaussians), ctypes.POINTER(View), c_int, ctypes.POINTER(Grads),
                                 _p, c_size, c_int, ctypes.POINTER(TuneEntry), c_int, ctypes.POINTER(c_int), _p]),
        "gsr_l1_loss": (c_int, [_p, ctypes.POINTER(View), ctypes.POINTER(L1View), c_int, ctypes.c_float,
                                ctypes.c_float, _p, _p]),
        "gsr_set_stage_events": (c_int, [_p, ctypes.POINTER(_p)]),
        "gsr_rgbd_loss": (c_int, [_p, ctypes.POINTER(View), ctypes.POINTER(L1View), c_int, ctypes.c_float,
                                  ctypes.c_float, _p, _p]),
        "gsr_render_noalloc": (c_int, [_p, ctypes.POINTER(Gaussians), ctypes.POINTER(View), c_int, _p, _p]),
        "gsr_render_surfels": (c_int, [_p, ctypes.POINTER(Gaussians), ctypes.POINTER(View),
                                       ctypes.POINTER(SurfelOut), c_int, _p, c_size, _p]),
        "gsr_render_surfels_backward": (c_int, [_p, ctypes.POINTER(Gaussians), ctypes.POINTER(View),
                                                ctypes.POINTER(ViewGrad), ctypes.POINTER(SurfelGrad), c_int,
                                                ctypes.POINTER(Grads), _p, c_size, _p]),
        "gsr_density_workspace_size": (c_int, [_p, c_int, ctypes.POINTER(c_size)]),
        "gsr_densify_adc": (c_int, [_p, ctypes.POINTER(Gaussians), _p, _p, _p, _p, ctypes.POINTER(AdcParams),
                                    ctypes.POINTER(GaussiansOut), _p, _p, c_size, _p]),
        "gsr_mcmc_relocate": (c_int, [_p, ctypes.POINTER(Gaussians), _p, ctypes.c_float,
                                      ctypes.POINTER(GaussiansOut), _p, _p, c_size, _p]),
        "gsr_mcmc_noise": (c_int, [_p, ctypes.POINTER(Gaussians), _p, ctypes.c_float, _p, _p]),
        "gsr_last_error": (ctypes.c_char_p, [_p]),
        "gsr_status_string": (ctypes.c_char_p, [c_int]),
        "gsr_abi_version": (c_int, []),
        "gsr_abi_sizeof": (c_size, [c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if lib.gsr_abi_version() != ABI_VERSION:
        raise RuntimeError(f"{path} has ABI version {lib.gsr_abi_version()}, this binding expects {ABI_VERSION}; "
                           "rebuild with `python -m paper_2411_17660_b300.build`")
    _lib = lib
    return lib


class Context:
    """Owns one gsr_ctx (host memory only)."""

    def __init__(self, tile: int = 16, spin_limit: int = 0, flags: int = 0, binning: int = BIN_TILE,
                 batch: int = 32, fwd_rows: int = 0):
        self.lib = load()
        cfg = Config(tile, spin_limit, flags, binning, batch, fwd_rows)
        h = _p()
        st = self.lib.gsr_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != OK:
            raise GsrError(st, f"gsr_create(tile={tile}, binning={binning}, batch={batch}, fwd_rows={fwd_rows})")
        self.h = h
        self.tile = tile

    def __del__(self):
        lib, h = getattr(self, "lib", None), getattr(self, "h", None)
        if lib is not None and h:
            lib.gsr_destroy(h)
            self.h = None

    def check(self, st: int, what: str):
        if st != OK:
            raise GsrError(st, f"{what}: {self.lib.gsr_last_error(self.h).decode()}")

    def workspace_size(self, N: int, views, key_capacity: int = 0) -> int:
        arr = (View * len(views))(*views)
        out = ctypes.c_size_t()
        self.check(self.lib.gsr_workspace_size(self.h, N, arr, len(views), key_capacity, ctypes.byref(out)),
                   "gsr_workspace_size")
        return out.value

    def render(self, g: Gaussians, views, ws_ptr: int, ws_bytes: int, stream: int) -> int:
        arr = (View * len(views))(*views)
        return self.lib.gsr_render(self.h, ctypes.byref(g), arr, len(views), ws_ptr, ws_bytes, stream)

    def render_l1(self, g: Gaussians, views, targets, color_weight: float, depth_weight: float, loss_ptr: int,
                  ws_ptr: int, ws_bytes: int, stream: int) -> int:
        arr = (View * len(views))(*views)
        tarr = (L1View * len(targets))(*targets)
        return self.lib.gsr_render_l1(self.h, ctypes.byref(g), arr, len(views), tarr, color_weight, depth_weight,
                                      loss_ptr, ws_ptr, ws_bytes, stream)

    def render_backward(self, g: Gaussians, views, vgrads, out: Grads, ws_ptr: int, ws_bytes: int,
                        stream: int) -> int:
        arr = (View * len(views))(*views)
        garr = (ViewGrad * len(vgrads))(*vgrads)
        return self.lib.gsr_render_backward(self.h, ctypes.byref(g), arr, garr, len(views), ctypes.byref(out),
                                            ws_ptr, ws_bytes, stream)

    def render_surfels(self, g: Gaussians, views, extra, ws_ptr: int, ws_bytes: int, stream: int) -> int:
        arr = (View * len(views))(*views)
        ex = None if extra is None else (SurfelOut * len(extra))(*extra)
        return self.lib.gsr_render_surfels(self.h, ctypes.byref(g), arr, ex, len(views), ws_ptr, ws_bytes, stream)

    def render_surfels_backward(self, g: Gaussians, views, vgrads, extra, out: Grads, ws_ptr: int, ws_bytes: int,
                                stream: int) -> int:
        arr = (View * len(views))(*views)
        garr = (ViewGrad * len(vgrads))(*vgrads)
        ex = None if extra is None else (SurfelGrad * len(extra))(*extra)
        return self.lib.gsr_render_surfels_backward(self.h, ctypes.byref(g), arr, garr, ex, len(views),
                                                    ctypes.byref(out), ws_ptr, ws_bytes, stream)

    def render_noalloc(self, g: Gaussians, views, status_ptr: int, stream: int) -> int:
        """Forward render into the library's static scratch (no allocation);
        status_ptr: device int32 receiving the device-side status, or 0."""
        arr = (View * len(views))(*views)
        return self.lib.gsr_render_noalloc(self.h, ctypes.byref(g), arr, len(views), status_ptr or None, stream)

    def get_status(self, ws_ptr: int, ws_bytes: int, stream: int) -> int:
        """gsr_get_status: the workspace's device status (after the stream)."""
        return self.lib.gsr_get_status(self.h, ws_ptr, ws_bytes, stream)

    def autotune(self, g: Gaussians, views, grads: Grads, ws_ptr: int, ws_bytes: int, reps: int, stream: int):
        """gsr_autotune; returns (status, [TuneEntry])."""
        arr = (View * len(views))(*views)
        entries = (TuneEntry * 32)()
        n = ctypes.c_int(0)
        st = self.lib.gsr_autotune(self.h, ctypes.byref(g), arr, len(views), ctypes.byref(grads), ws_ptr, ws_bytes,
                                   reps, entries, 32, ctypes.byref(n), stream)
        return st, list(entries[:n.value])

    def read_info(self, ws_ptr: int, ws_bytes: int, stream: int) -> Info:
        info = Info()
        self.check(self.lib.gsr_read_info(self.h, ws_ptr, ws_bytes, ctypes.byref(info), stream), "gsr_read_info")
        return info

    def set_stage_events(self, handles):
        """handles: GSR_STAGE_EVENTS raw cudaEvent_t values, or None to stop."""
        if handles is None:
            self.check(self.lib.gsr_set_stage_events(self.h, None), "gsr_set_stage_events")
            return
        arr = (_p * STAGE_EVENTS)(*handles)
        self.check(self.lib.gsr_set_stage_events(self.h, arr), "gsr_set_stage_events")

    def rgbd_loss(self, views, targets, lambda1: float, lambda2: float, loss_ptr: int, stream: int):
        arr = (View * len(views))(*views)
        tarr = (L1View * len(targets))(*targets)
        self.check(self.lib.gsr_rgbd_loss(self.h, arr, tarr, len(views), lambda1, lambda2, loss_ptr, stream),
                   "gsr_rgbd_loss")

    def density_workspace_size(self, N: int) -> int:
        b = ctypes.c_size_t()
        self.check(self.lib.gsr_density_workspace_size(self.h, N, ctypes.byref(b)), "gsr_density_workspace_size")
        return b.value

    def densify_adc(self, g: Gaussians, grad: int, count: int, radius: int, normals: int, params: AdcParams,
                    out: GaussiansOut, out_count: int, ws_ptr: int, ws_bytes: int, stream: int) -> int:
        return self.lib.gsr_densify_adc(self.h, ctypes.byref(g), grad, count, radius, normals, ctypes.byref(params),
                                        ctypes.byref(out), out_count, ws_ptr, ws_bytes, stream)

    def mcmc_relocate(self, g: Gaussians, draws: int, min_opacity: float, out: GaussiansOut, relocated: int,
                      ws_ptr: int, ws_bytes: int, stream: int) -> int:
        return self.lib.gsr_mcmc_relocate(self.h, ctypes.byref(g), draws, min_opacity, ctypes.byref(out), relocated,
                                          ws_ptr, ws_bytes, stream)

    def mcmc_noise(self, g: Gaussians, eta: int, scale: float, means_out: int, stream: int) -> int:
        return self.lib.gsr_mcmc_noise(self.h, ctypes.byref(g), eta, scale, means_out, stream)

    def l1_loss(self, views, targets, color_weight: float, depth_weight: float, loss_ptr: int, stream: int):
        arr = (View * len(views))(*views)
        tarr = (L1View * len(targets))(*targets)
        self.check(self.lib.gsr_l1_loss(self.h, arr, tarr, len(views), color_weight, depth_weight, loss_ptr,
                                        stream), "gsr_l1_loss")
