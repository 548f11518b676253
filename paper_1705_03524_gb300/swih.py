"""Thin ctypes binding of libswih (C ABI in include/swih.h).

Argument marshalling only: every function here forwards to the C entry point
of the same name, which enqueues CUDA kernels; nothing is computed in Python.
Pointers may be given as integers or as objects with ``data_ptr()`` (torch
tensors); streams as integers, ``None`` (the legacy default stream) or objects
with a ``cuda_stream`` attribute (``torch.cuda.Stream``).

Importing this module loads the shared library and fails loudly if it has not
been built (``paper_1705_03524_gb300.build.build()``): there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

from . import build as _build

SWIH_OK = 0
SWIH_ERR_INVALID_ARG = 1
SWIH_ERR_UNSUPPORTED = 2
SWIH_ERR_OOM = 3
SWIH_ERR_BUDGET = 4
SWIH_ERR_CUDA = 5
SWIH_ERR_TIMEOUT = 6
SWIH_ERR_CANCELLED = 7

SWIH_PIXEL_U8 = 0
SWIH_PIXEL_U16 = 1

SWIH_KERNEL_PLAIN = 0
SWIH_KERNEL_MANHATTAN = 1
SWIH_KERNEL_EUCLIDEAN = 2
SWIH_KERNEL_GAUSSIAN = 3
SWIH_KERNEL_WEDDING = 4
SWIH_KERNEL_EXPONENTIAL = 5

SWIH_PREC_AUTO = 0
SWIH_PREC_RING32 = 1
SWIH_PREC_RING64 = 2
SWIH_PREC_RING128 = 3

KERNELS = {"plain": SWIH_KERNEL_PLAIN, "manhattan": SWIH_KERNEL_MANHATTAN,
           "euclidean": SWIH_KERNEL_EUCLIDEAN, "gaussian": SWIH_KERNEL_GAUSSIAN,
           "wedding": SWIH_KERNEL_WEDDING, "exponential": SWIH_KERNEL_EXPONENTIAL}


def kernel_bit(k: int) -> int:
    return 1 << k


class SwihError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"swih status {status}: {message}")
        self.status = status


class swih_plan_desc(ctypes.Structure):
    _fields_ = [
        ("height", ctypes.c_int32),
        ("width", ctypes.c_int32),
        ("pitch_bytes", ctypes.c_int64),
        ("pixel_type", ctypes.c_int32),
        ("bitdepth", ctypes.c_int32),
        ("bins", ctypes.c_int32),
        ("kernel_mask", ctypes.c_uint32),
        ("gauss_degree", ctypes.c_int32),
        ("gauss_sigma_frac", ctypes.c_double),
        ("max_win_w", ctypes.c_int32),
        ("max_win_h", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("band_rows", ctypes.c_int32),
        ("hbm_budget_bytes", ctypes.c_uint64),
        ("wedding_rings", ctypes.c_int32),
        ("exp_lambda", ctypes.c_double),
    ]


class swih_plan_info(ctypes.Structure):
    _fields_ = [
        ("height", ctypes.c_int32),
        ("width", ctypes.c_int32),
        ("bins", ctypes.c_int32),
        ("elem_bytes", ctypes.c_int32),
        ("n_terms", ctypes.c_int32),
        ("term_p", ctypes.c_int32 * 96),
        ("term_q", ctypes.c_int32 * 96),
        ("d_bins", ctypes.c_void_p),
        ("bins_pitch", ctypes.c_int64),
        ("d_ih", ctypes.c_void_p),
        ("ih_pitch", ctypes.c_int64),
        ("plane_elems", ctypes.c_int64),
        ("band_rows", ctypes.c_int32),
        ("n_bands", ctypes.c_int32),
        ("workspace_bytes", ctypes.c_uint64),
        ("d_exp", ctypes.c_void_p),
        ("exp_frac_bits", ctypes.c_int32),
        ("d_row_map", ctypes.c_void_p),
        ("n_channels", ctypes.c_int32),
    ]


SWIH_MAX_SCALES = 8
SWIH_MAX_CHANNELS = 8


class swih_channel_desc(ctypes.Structure):
    _fields_ = [
        ("pitch_bytes", ctypes.c_int64),
        ("pixel_type", ctypes.c_int32),
        ("bitdepth", ctypes.c_int32),
        ("bins", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class swih_batch_desc(ctypes.Structure):
    _fields_ = [
        ("height", ctypes.c_int32),
        ("width", ctypes.c_int32),
        ("pitch_bytes", ctypes.c_int64),
        ("pixel_type", ctypes.c_int32),
        ("bitdepth", ctypes.c_int32),
        ("bins", ctypes.c_int32),
        ("kernel_mask", ctypes.c_uint32),
        ("gauss_degree", ctypes.c_int32),
        ("gauss_sigma_frac", ctypes.c_double),
        ("precision", ctypes.c_int32),
        ("band_rows", ctypes.c_int32),
        ("hbm_budget_bytes", ctypes.c_uint64),
    ]


class swih_roi_desc(ctypes.Structure):
    _fields_ = [
        ("x0", ctypes.c_int32),
        ("y0", ctypes.c_int32),
        ("width", ctypes.c_int32),
        ("height", ctypes.c_int32),
        ("kernel", ctypes.c_int32),
        ("n_windows", ctypes.c_int32),
        ("win_w", ctypes.c_int32 * SWIH_MAX_SCALES),
        ("win_h", ctypes.c_int32 * SWIH_MAX_SCALES),
        ("d_target", ctypes.c_void_p),
        ("d_map", ctypes.c_void_p * SWIH_MAX_SCALES),
        ("bins", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


SWIH_MAX_TARGETS = 8


class swih_server_desc(ctypes.Structure):
    _fields_ = [
        ("hbm_budget_bytes", ctypes.c_uint64),
        ("max_inflight", ctypes.c_int32),
        ("max_batch_queries", ctypes.c_int32),
        ("merge_regions", ctypes.c_int32),
        ("gauss_degree", ctypes.c_int32),
        ("gauss_sigma_frac", ctypes.c_double),
        ("staging_bytes", ctypes.c_uint64),
        ("keep_ih", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class swih_frame_desc(ctypes.Structure):
    _fields_ = [
        ("d_pixels", ctypes.c_void_p),
        ("height", ctypes.c_int32),
        ("width", ctypes.c_int32),
        ("pitch_bytes", ctypes.c_int64),
        ("pixel_type", ctypes.c_int32),
        ("bitdepth", ctypes.c_int32),
    ]


class swih_query(ctypes.Structure):
    _fields_ = [
        ("frame", ctypes.c_int32),
        ("x0", ctypes.c_int32),
        ("y0", ctypes.c_int32),
        ("width", ctypes.c_int32),
        ("height", ctypes.c_int32),
        ("bins", ctypes.c_int32),
        ("kernel", ctypes.c_int32),
        ("n_targets", ctypes.c_int32),
        ("n_scales", ctypes.c_int32),
        ("win_w", ctypes.c_int32 * SWIH_MAX_SCALES),
        ("win_h", ctypes.c_int32 * SWIH_MAX_SCALES),
        ("d_targets", ctypes.c_void_p),
        ("d_out", ctypes.c_void_p),
        ("user_tag", ctypes.c_uint64),
    ]


class swih_completion(ctypes.Structure):
    _fields_ = [
        ("id", ctypes.c_uint64),
        ("user_tag", ctypes.c_uint64),
        ("status", ctypes.c_int32),
        ("batch_queries", ctypes.c_int32),
        ("submit_ns", ctypes.c_uint64),
        ("start_ns", ctypes.c_uint64),
        ("done_ns", ctypes.c_uint64),
        ("ih_reused", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class swih_server_stats(ctypes.Structure):
    _fields_ = [
        ("queries", ctypes.c_uint64),
        ("ih_reused", ctypes.c_uint64),
        ("regions_built", ctypes.c_uint64),
        ("evictions", ctypes.c_uint64),
        ("resident_bytes", ctypes.c_uint64),
    ]


class swih_frame_job(ctypes.Structure):
    _fields_ = [
        ("kernel", ctypes.c_int32),
        ("win_w", ctypes.c_int32),
        ("win_h", ctypes.c_int32),
        ("d_target", ctypes.c_void_p),
        ("d_map", ctypes.c_void_p),
    ]


def _load() -> ctypes.CDLL:
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built ({path}); run paper_1705_03524_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, I, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_int
    lib.swih_plan_workspace_bytes.argtypes = [ctypes.POINTER(swih_plan_desc), ctypes.POINTER(ctypes.c_uint64)]
    lib.swih_plan_workspace_bytes.restype = S
    lib.swih_plan.argtypes = [ctypes.POINTER(swih_plan_desc), ctypes.POINTER(P)]
    lib.swih_plan.restype = S
    lib.swih_build_ih.argtypes = [P, P, P]
    lib.swih_build_ih.restype = S
    lib.swih_local_hist.argtypes = [P, I, I, I, I, I, I, I, P, P]
    lib.swih_local_hist.restype = S
    lib.swih_likelihood.argtypes = [P, I, I, I, P, P, P]
    lib.swih_likelihood.restype = S
    lib.swih_likelihood_scales.argtypes = [P, I, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(P),
                                           ctypes.POINTER(P), P]
    lib.swih_likelihood_scales.restype = S
    lib.swih_sync_status.argtypes = [P, P]
    lib.swih_sync_status.restype = S
    lib.swih_destroy.argtypes = [P]
    lib.swih_destroy.restype = S
    lib.swih_last_error.argtypes = [P]
    lib.swih_last_error.restype = ctypes.c_char_p
    lib.swih_build_ih_noalloc.argtypes = [ctypes.POINTER(swih_plan_desc), P, P, ctypes.c_uint64, P,
                                          ctypes.POINTER(swih_plan_info), P]
    lib.swih_build_ih_noalloc.restype = S
    lib.swih_plan_channels.argtypes = [ctypes.POINTER(swih_plan_desc), I, ctypes.POINTER(swih_channel_desc),
                                       ctypes.POINTER(P)]
    lib.swih_plan_channels.restype = S
    lib.swih_build_ih_channels.argtypes = [P, ctypes.POINTER(P), P]
    lib.swih_build_ih_channels.restype = S
    lib.swih_likelihood_channels.argtypes = [P, I, I, I, P, P, P]
    lib.swih_likelihood_channels.restype = S
    lib.swih_set_gather_config.argtypes = [P, I, I, I, I]
    lib.swih_set_gather_config.restype = S
    lib.swih_debug_inject.argtypes = [P, I]
    lib.swih_debug_inject.restype = S
    lib.swih_plan_get_info.argtypes = [P, ctypes.POINTER(swih_plan_info)]
    lib.swih_plan_get_info.restype = S
    lib.swih_launch_count.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
    lib.swih_plan_load_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_uint64), I]
    lib.swih_plan_load_bytes.restype = S
    lib.swih_launch_count.restype = S
    BD, RD = ctypes.POINTER(swih_batch_desc), ctypes.POINTER(swih_roi_desc)
    lib.swih_batch_workspace_bytes.argtypes = [BD, RD, I, ctypes.POINTER(ctypes.c_uint64)]
    lib.swih_batch_workspace_bytes.restype = S
    lib.swih_batch_plan.argtypes = [BD, RD, I, P, ctypes.POINTER(P)]
    lib.swih_batch_plan.restype = S
    for name in ("swih_batch_run", "swih_batch_autotune", "swih_batch_sync_status"):
        getattr(lib, name).argtypes = [P, P]
        getattr(lib, name).restype = S
    lib.swih_batch_destroy.argtypes = [P]
    lib.swih_batch_destroy.restype = S
    SD, FD, QD = (ctypes.POINTER(swih_server_desc), ctypes.POINTER(swih_frame_desc),
                  ctypes.POINTER(swih_query))
    U64P = ctypes.POINTER(ctypes.c_uint64)
    lib.swih_server_create.argtypes = [SD, ctypes.POINTER(P)]
    lib.swih_server_add_frame.argtypes = [P, FD, ctypes.POINTER(ctypes.c_int32)]
    lib.swih_query_out_elems.argtypes = [QD, U64P]
    lib.swih_server_query_bytes.argtypes = [P, QD, U64P]
    lib.swih_server_submit.argtypes = [P, QD, U64P]
    lib.swih_server_poll.argtypes = [P, ctypes.POINTER(swih_completion), ctypes.c_int32,
                                     ctypes.POINTER(ctypes.c_int32), ctypes.c_int32]
    lib.swih_server_drain.argtypes = [P]
    lib.swih_server_cancel.argtypes = [P, ctypes.c_uint64]
    lib.swih_server_frame_changed.argtypes = [P, ctypes.c_int32]
    lib.swih_server_get_stats.argtypes = [P, ctypes.POINTER(swih_server_stats)]
    lib.swih_server_destroy.argtypes = [P]
    lib.swih_stream_plan.argtypes = [ctypes.POINTER(swih_plan_desc), ctypes.POINTER(swih_frame_job), I, P,
                                     ctypes.c_int32, ctypes.POINTER(P)]
    lib.swih_stream_run.argtypes = [P, P]
    lib.swih_stream_sync_status.argtypes = [P, P]
    lib.swih_stream_get_info.argtypes = [P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_uint64)]
    lib.swih_stream_set_host_maps.argtypes = [P, ctypes.POINTER(ctypes.c_void_p)]
    lib.swih_stream_destroy.argtypes = [P]
    lib.swih_stream_run_timed.argtypes = [P, P, ctypes.POINTER(ctypes.c_float)]
    lib.swih_stream_load_bytes.argtypes = [P, U64P, I]
    for name in ("swih_stream_plan", "swih_stream_run", "swih_stream_sync_status", "swih_stream_get_info",
                 "swih_stream_destroy", "swih_stream_run_timed", "swih_stream_load_bytes",
                 "swih_stream_set_host_maps"):
        getattr(lib, name).restype = S
    for name in ("swih_server_create", "swih_server_add_frame", "swih_query_out_elems",
                 "swih_server_query_bytes", "swih_server_submit", "swih_server_poll",
                 "swih_server_drain", "swih_server_destroy", "swih_server_cancel", "swih_server_frame_changed",
                 "swih_server_get_stats"):
        getattr(lib, name).restype = S
    return lib


LIB = _load()
LIB_PATH = _build.LIB


def header_functions() -> list:
    """Names of the functions declared in include/swih.h."""
    hdr = os.path.join(_build.ROOT, "include", "swih.h")
    text = open(hdr).read()
    return sorted(set(re.findall(r"^\s*(?:swih_status|const char \*)\s*(swih_\w+)\s*\(", text, re.M)))


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(s) -> int | None:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


def _check(status: int, plan=None):
    if status != SWIH_OK:
        msg = LIB.swih_last_error(plan).decode(errors="replace")
        raise SwihError(status, msg)


def make_desc(height, width, *, pitch_bytes=None, pixel_type=SWIH_PIXEL_U8, bitdepth=None,
              bins=16, kernels=("manhattan",), gauss_degree=2, gauss_sigma_frac=0.25,
              max_win=(3, 3), precision=SWIH_PREC_AUTO, band_rows=0, hbm_budget_bytes=0,
              wedding_rings=0, exp_lambda=0.0):
    pb = 1 if pixel_type == SWIH_PIXEL_U8 else 2
    mask = 0
    for k in kernels:
        mask |= kernel_bit(KERNELS[k] if isinstance(k, str) else int(k))
    d = swih_plan_desc()
    d.height, d.width = int(height), int(width)
    d.pitch_bytes = int(pitch_bytes if pitch_bytes is not None else width * pb)
    d.pixel_type = int(pixel_type)
    d.bitdepth = int(bitdepth if bitdepth is not None else 8 * pb)
    d.bins = int(bins)
    d.kernel_mask = mask
    d.gauss_degree = int(gauss_degree)
    d.gauss_sigma_frac = float(gauss_sigma_frac)
    d.max_win_w, d.max_win_h = int(max_win[0]), int(max_win[1])
    d.precision = int(precision)
    d.band_rows = int(band_rows)
    d.hbm_budget_bytes = int(hbm_budget_bytes)
    d.wedding_rings = int(wedding_rings)
    d.exp_lambda = float(exp_lambda)
    return d


def swih_plan_workspace_bytes(desc: swih_plan_desc) -> int:
    out = ctypes.c_uint64(0)
    _check(LIB.swih_plan_workspace_bytes(ctypes.byref(desc), ctypes.byref(out)))
    return int(out.value)


def swih_plan(desc: swih_plan_desc) -> int:
    h = ctypes.c_void_p()
    _check(LIB.swih_plan(ctypes.byref(desc), ctypes.byref(h)))
    return int(h.value)


def swih_build_ih(plan: int, image, stream=None) -> None:
    _check(LIB.swih_build_ih(plan, _ptr(image), _stream(stream)), plan)


def swih_local_hist(plan: int, kernel: int, win_w: int, win_h: int, cx0: int, cy0: int,
                    ncx: int, ncy: int, hist, stream=None) -> None:
    _check(LIB.swih_local_hist(plan, int(kernel), win_w, win_h, cx0, cy0, ncx, ncy, _ptr(hist),
                               _stream(stream)), plan)


def swih_likelihood(plan: int, kernel: int, win_w: int, win_h: int, target, out_map,
                    stream=None) -> None:
    _check(LIB.swih_likelihood(plan, int(kernel), win_w, win_h, _ptr(target), _ptr(out_map),
                               _stream(stream)), plan)


def swih_likelihood_scales(plan: int, kernel: int, windows, targets, maps, stream=None) -> None:
    """windows: [(w, h), ...]; targets, maps: device tensors or pointers, one per window."""
    n = len(windows)
    ww = (ctypes.c_int * n)(*[int(w) for w, _ in windows])
    wh = (ctypes.c_int * n)(*[int(h) for _, h in windows])
    tg = (ctypes.c_void_p * n)(*[_ptr(t) for t in targets])
    mp = (ctypes.c_void_p * n)(*[_ptr(m) for m in maps])
    _check(LIB.swih_likelihood_scales(plan, int(kernel), n, ww, wh, tg, mp, _stream(stream)), plan)


def swih_sync_status(plan: int, stream=None) -> None:
    _check(LIB.swih_sync_status(plan, _stream(stream)), plan)


def swih_destroy(plan: int) -> None:
    _check(LIB.swih_destroy(plan))


def swih_last_error(plan=None) -> str:
    return LIB.swih_last_error(plan).decode(errors="replace")


def swih_build_ih_noalloc(desc: swih_plan_desc, image, d_ih, ih_bytes: int, d_status=None,
                          stream=None) -> swih_plan_info:
    """Allocation-free build into caller memory; d_ih=None only queries the layout
    (layout.workspace_bytes = bytes d_ih must hold)."""
    info = swih_plan_info()
    _check(LIB.swih_build_ih_noalloc(ctypes.byref(desc), _ptr(image), _ptr(d_ih), int(ih_bytes),
                                     _ptr(d_status), ctypes.byref(info), _stream(stream)))
    return info


def swih_set_gather_config(plan: int, kernel: int, tile_cols: int = 0, stages: int = 0,
                           bins_per_step: int = 0) -> None:
    _check(LIB.swih_set_gather_config(plan, int(kernel), int(tile_cols), int(stages),
                                      int(bins_per_step)), plan)


SWIH_INJECT_STALL_SCAN_TILE = 1
SWIH_INJECT_DIRECT_GATHER = 2


def swih_debug_inject(plan: int, what: int) -> None:
    _check(LIB.swih_debug_inject(plan, int(what)), plan)


def swih_plan_load_bytes(plan: int, reset: bool = False) -> int:
    out = ctypes.c_uint64(0)
    _check(LIB.swih_plan_load_bytes(plan, ctypes.byref(out), 1 if reset else 0), plan)
    return int(out.value)


def swih_launch_count() -> int:
    out = ctypes.c_uint64(0)
    _check(LIB.swih_launch_count(ctypes.byref(out)))
    return int(out.value)


def swih_plan_get_info(plan: int) -> swih_plan_info:
    info = swih_plan_info()
    _check(LIB.swih_plan_get_info(plan, ctypes.byref(info)), plan)
    return info


class Plan:
    """Owning wrapper: ``with Plan(desc) as p: p.build_ih(img); p.likelihood(...)``."""

    def __init__(self, desc: swih_plan_desc):
        self.desc = desc
        self.handle = swih_plan(desc)

    def build_ih(self, image, stream=None):
        swih_build_ih(self.handle, image, stream)

    def local_hist(self, kernel, win_w, win_h, cx0, cy0, ncx, ncy, hist, stream=None):
        k = KERNELS[kernel] if isinstance(kernel, str) else kernel
        swih_local_hist(self.handle, k, win_w, win_h, cx0, cy0, ncx, ncy, hist, stream)

    def likelihood(self, kernel, win_w, win_h, target, out_map, stream=None):
        k = KERNELS[kernel] if isinstance(kernel, str) else kernel
        swih_likelihood(self.handle, k, win_w, win_h, target, out_map, stream)

    def likelihood_scales(self, kernel, windows, targets, maps, stream=None):
        k = KERNELS[kernel] if isinstance(kernel, str) else kernel
        swih_likelihood_scales(self.handle, k, windows, targets, maps, stream)

    def sync_status(self, stream=None):
        swih_sync_status(self.handle, stream)

    def info(self) -> swih_plan_info:
        return swih_plan_get_info(self.handle)

    def load_bytes(self, reset=False) -> int:
        return swih_plan_load_bytes(self.handle, reset)

    def close(self):
        if self.handle:
            swih_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_channel(width, *, pixel_type=SWIH_PIXEL_U8, bitdepth=None, bins=16, pitch_bytes=None) -> swih_channel_desc:
    """One feature channel of a channel plan (image row stride defaults to width pixels)."""
    pb = 1 if pixel_type == SWIH_PIXEL_U8 else 2
    c = swih_channel_desc()
    c.pitch_bytes = int(pitch_bytes if pitch_bytes is not None else width * pb)
    c.pixel_type = int(pixel_type)
    c.bitdepth = int(bitdepth if bitdepth is not None else 8 * pb)
    c.bins = int(bins)
    c.reserved = 0
    return c


class ChannelPlan(Plan):
    """Owning wrapper of a feature-channel plan (swih_plan_channels): one bin
    plane per channel, every channel's map from one gather launch."""

    def __init__(self, desc: swih_plan_desc, channels):
        self.desc = desc
        self.channels = list(channels)
        arr = (swih_channel_desc * len(self.channels))(*self.channels)
        h = ctypes.c_void_p()
        _check(LIB.swih_plan_channels(ctypes.byref(desc), len(self.channels), arr, ctypes.byref(h)))
        self.handle = int(h.value)
        self.bins = sum(c.bins for c in self.channels)

    def build_ih(self, images, stream=None):
        ptrs = (ctypes.c_void_p * len(images))(*[_ptr(im) for im in images])
        _check(LIB.swih_build_ih_channels(self.handle, ptrs, _stream(stream)), self.handle)

    def likelihood_channels(self, kernel, win_w, win_h, target, out_maps, stream=None):
        """target: [B] (the channels' targets side by side); out_maps: [C][H-h+1][W-w+1]."""
        k = KERNELS[kernel] if isinstance(kernel, str) else kernel
        _check(LIB.swih_likelihood_channels(self.handle, k, int(win_w), int(win_h), _ptr(target), _ptr(out_maps),
                                            _stream(stream)), self.handle)


# ---------------------------------------------------------------- batches

def make_batch_desc(height, width, *, pitch_bytes=None, pixel_type=SWIH_PIXEL_U8, bitdepth=None,
                    bins=16, kernels=("manhattan",), gauss_degree=2, gauss_sigma_frac=0.25,
                    precision=SWIH_PREC_AUTO, band_rows=0, hbm_budget_bytes=0) -> swih_batch_desc:
    pb = 1 if pixel_type == SWIH_PIXEL_U8 else 2
    mask = 0
    for k in kernels:
        mask |= kernel_bit(KERNELS[k] if isinstance(k, str) else int(k))
    d = swih_batch_desc()
    d.height, d.width = int(height), int(width)
    d.pitch_bytes = int(pitch_bytes if pitch_bytes is not None else width * pb)
    d.pixel_type = int(pixel_type)
    d.bitdepth = int(bitdepth if bitdepth is not None else 8 * pb)
    d.bins = int(bins)
    d.kernel_mask = mask
    d.gauss_degree = int(gauss_degree)
    d.gauss_sigma_frac = float(gauss_sigma_frac)
    d.precision = int(precision)
    d.band_rows = int(band_rows)
    d.hbm_budget_bytes = int(hbm_budget_bytes)
    return d


def make_roi(x0, y0, width, height, kernel, windows, target, maps, bins=0) -> swih_roi_desc:
    """windows: [(w, h), ...] (at most SWIH_MAX_SCALES); maps: one device buffer per window;
    bins: this ROI's bin count (0: the batch's)."""
    if len(windows) != len(maps) or not 1 <= len(windows) <= SWIH_MAX_SCALES:
        raise ValueError("need 1..SWIH_MAX_SCALES windows, one map each")
    r = swih_roi_desc()
    r.x0, r.y0, r.width, r.height = int(x0), int(y0), int(width), int(height)
    r.kernel = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    r.n_windows = len(windows)
    for k, (w, h) in enumerate(windows):
        r.win_w[k], r.win_h[k] = int(w), int(h)
        r.d_map[k] = _ptr(maps[k])
    r.d_target = _ptr(target)
    r.bins = int(bins)
    r.reserved = 0
    return r


def _roi_array(rois):
    arr = (swih_roi_desc * len(rois))()
    for i, r in enumerate(rois):
        arr[i] = r
    return arr


def swih_batch_workspace_bytes(desc: swih_batch_desc, rois) -> int:
    out = ctypes.c_uint64(0)
    arr = _roi_array(rois)
    _check(LIB.swih_batch_workspace_bytes(ctypes.byref(desc), arr, len(rois), ctypes.byref(out)))
    return int(out.value)


def swih_batch_plan(desc: swih_batch_desc, rois, frame) -> int:
    h = ctypes.c_void_p()
    arr = _roi_array(rois)
    _check(LIB.swih_batch_plan(ctypes.byref(desc), arr, len(rois), _ptr(frame), ctypes.byref(h)))
    return int(h.value)


def swih_batch_run(batch: int, stream=None) -> None:
    _check(LIB.swih_batch_run(batch, _stream(stream)))


def swih_batch_autotune(batch: int, stream=None) -> None:
    _check(LIB.swih_batch_autotune(batch, _stream(stream)))


def swih_batch_sync_status(batch: int, stream=None) -> None:
    _check(LIB.swih_batch_sync_status(batch, _stream(stream)))


def swih_batch_destroy(batch: int) -> None:
    _check(LIB.swih_batch_destroy(batch))


class Batch:
    """Owning wrapper of a batch; keeps the frame, targets and maps it was given alive."""

    def __init__(self, desc: swih_batch_desc, rois, frame, keep=()):
        self.desc = desc
        self.rois = list(rois)
        self._keep = (frame, tuple(keep))
        self.handle = swih_batch_plan(desc, self.rois, frame)

    def run(self, stream=None):
        swih_batch_run(self.handle, stream)

    def autotune(self, stream=None):
        swih_batch_autotune(self.handle, stream)

    def sync_status(self, stream=None):
        swih_batch_sync_status(self.handle, stream)

    def close(self):
        if self.handle:
            swih_batch_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- serving

def make_query(frame, x0, y0, width, height, bins, kernel, windows, targets, out, n_targets=1,
               user_tag=0) -> swih_query:
    """windows: [(w, h), ...]; targets: device [n_targets][bins]; out: device buffer of
    swih_query_out_elems(q) floats (maps target-major, then scale, packed)."""
    if not 1 <= len(windows) <= SWIH_MAX_SCALES:
        raise ValueError("need 1..SWIH_MAX_SCALES windows")
    q = swih_query()
    q.frame, q.x0, q.y0, q.width, q.height = int(frame), int(x0), int(y0), int(width), int(height)
    q.bins = int(bins)
    q.kernel = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    q.n_targets = int(n_targets)
    q.n_scales = len(windows)
    for k, (w, h) in enumerate(windows):
        q.win_w[k], q.win_h[k] = int(w), int(h)
    q.d_targets = _ptr(targets)
    q.d_out = _ptr(out)
    q.user_tag = int(user_tag)
    return q


def swih_query_out_elems(q: swih_query) -> int:
    out = ctypes.c_uint64(0)
    _check(LIB.swih_query_out_elems(ctypes.byref(q), ctypes.byref(out)))
    return int(out.value)


def query_map_shapes(q: swih_query):
    """[(offset, (rows, cols))] of every map in d_out, target-major then scale."""
    shapes = []
    off = 0
    for _t in range(q.n_targets):
        for k in range(q.n_scales):
            r, c = q.height - q.win_h[k] + 1, q.width - q.win_w[k] + 1
            shapes.append((off, (r, c)))
            off += r * c
    return shapes


class Server:
    """Owning wrapper of swih_server_*; frames are device buffers kept alive here."""

    def __init__(self, hbm_budget_bytes, max_inflight=4, max_batch_queries=16, merge_regions=True,
                 gauss_degree=0, gauss_sigma_frac=0.0, staging_bytes=0, keep_ih=False):
        d = swih_server_desc()
        d.keep_ih = 1 if keep_ih else 0
        d.reserved = 0
        d.hbm_budget_bytes = int(hbm_budget_bytes)
        d.max_inflight = int(max_inflight)
        d.max_batch_queries = int(max_batch_queries)
        d.merge_regions = 1 if merge_regions else 0
        d.gauss_degree = int(gauss_degree)
        d.gauss_sigma_frac = float(gauss_sigma_frac)
        d.staging_bytes = int(staging_bytes)
        h = ctypes.c_void_p()
        _check(LIB.swih_server_create(ctypes.byref(d), ctypes.byref(h)))
        self.handle = int(h.value)
        self._frames = []

    def add_frame(self, pixels, height, width, pitch_bytes=None, pixel_type=SWIH_PIXEL_U8,
                  bitdepth=None) -> int:
        pb = 1 if pixel_type == SWIH_PIXEL_U8 else 2
        f = swih_frame_desc()
        f.d_pixels = _ptr(pixels)
        f.height, f.width = int(height), int(width)
        f.pitch_bytes = int(pitch_bytes if pitch_bytes is not None else width * pb)
        f.pixel_type = int(pixel_type)
        f.bitdepth = int(bitdepth if bitdepth is not None else 8 * pb)
        fid = ctypes.c_int32(0)
        _check(LIB.swih_server_add_frame(self.handle, ctypes.byref(f), ctypes.byref(fid)))
        self._frames.append(pixels)
        return int(fid.value)

    def query_bytes(self, q: swih_query) -> int:
        out = ctypes.c_uint64(0)
        _check(LIB.swih_server_query_bytes(self.handle, ctypes.byref(q), ctypes.byref(out)))
        return int(out.value)

    def submit(self, q: swih_query) -> int:
        qid = ctypes.c_uint64(0)
        _check(LIB.swih_server_submit(self.handle, ctypes.byref(q), ctypes.byref(qid)))
        return int(qid.value)

    def poll(self, max_n=256, wait_us=0):
        buf = (swih_completion * max_n)()
        n = ctypes.c_int32(0)
        _check(LIB.swih_server_poll(self.handle, buf, int(max_n), ctypes.byref(n), int(wait_us)))
        return [buf[i] for i in range(n.value)]

    def drain(self):
        _check(LIB.swih_server_drain(self.handle))

    def cancel(self, qid: int):
        _check(LIB.swih_server_cancel(self.handle, int(qid)))

    def frame_changed(self, frame_id: int):
        _check(LIB.swih_server_frame_changed(self.handle, int(frame_id)))

    def stats(self) -> dict:
        st = swih_server_stats()
        _check(LIB.swih_server_get_stats(self.handle, ctypes.byref(st)))
        return {name: int(getattr(st, name)) for name, _ in swih_server_stats._fields_}

    def close(self):
        if self.handle:
            _check(LIB.swih_server_destroy(self.handle))
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- streamed frames

def make_frame_job(kernel, win_w, win_h, target, out_map) -> swih_frame_job:
    j = swih_frame_job()
    j.kernel = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    j.win_w, j.win_h = int(win_w), int(win_h)
    j.d_target = _ptr(target)
    j.d_map = _ptr(out_map)
    return j


class Stream:
    """Owning wrapper of swih_stream_*: likelihood maps of a large frame, band by band."""

    def __init__(self, desc: swih_plan_desc, jobs, image, band_height=0, keep=()):
        arr = (swih_frame_job * len(jobs))()
        for i, j in enumerate(jobs):
            arr[i] = j
        h = ctypes.c_void_p()
        _check(LIB.swih_stream_plan(ctypes.byref(desc), arr, len(jobs), _ptr(image), int(band_height),
                                    ctypes.byref(h)))
        self.handle = int(h.value)
        self._keep = (image, tuple(keep))
        self._host = ()

    def run(self, stream=None):
        _check(LIB.swih_stream_run(self.handle, _stream(stream)))

    def sync_status(self, stream=None):
        _check(LIB.swih_stream_sync_status(self.handle, _stream(stream)))

    def set_host_maps(self, h_maps):
        """Host copies of the maps made during each pass, band by band (one
        page-locked host tensor or pointer per job, or None; h_maps None: off)."""
        if h_maps is None:
            _check(LIB.swih_stream_set_host_maps(self.handle, None))
            self._host = ()
            return
        arr = (ctypes.c_void_p * len(h_maps))(*[_ptr(m) for m in h_maps])
        _check(LIB.swih_stream_set_host_maps(self.handle, arr))
        self._host = tuple(h_maps)  # kept alive while passes copy into them

    def run_timed(self, stream=None):
        """One pass launched stage by stage with CUDA events; returns
        {"scan": ms, kernel name: ms of its gathers} summed over the bands."""
        ms = (ctypes.c_float * 7)()
        _check(LIB.swih_stream_run_timed(self.handle, _stream(stream), ms))
        out = {"scan": float(ms[0])}
        for name, k in KERNELS.items():
            if 0 <= k <= 5 and ms[1 + k] > 0:
                out[name] = float(ms[1 + k])
        return out

    def load_bytes(self, reset=False):
        """Integral-histogram bytes the tiled gathers requested, per kernel name."""
        b = (ctypes.c_uint64 * 5)()
        _check(LIB.swih_stream_load_bytes(self.handle, b, int(bool(reset))))
        return {name: int(b[k]) for name, k in KERNELS.items() if 0 <= k < 5}

    def info(self):
        bh, nb, wb = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_uint64(0)
        _check(LIB.swih_stream_get_info(self.handle, ctypes.byref(bh), ctypes.byref(nb), ctypes.byref(wb)))
        return dict(band_height=bh.value, n_bands=nb.value, workspace_bytes=wb.value)

    def close(self):
        if self.handle:
            _check(LIB.swih_stream_destroy(self.handle))
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
