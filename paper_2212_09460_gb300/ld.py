"""Thin Python binding of libld.so (include/ld.h), argument marshalling only.

Every step of the path runs in the library's CUDA kernels; this module only
converts torch tensors into device pointers and the current CUDA stream, and
turns non-zero ``ld_status`` codes into exceptions.  The C functions are
exposed under their own names (``ld_sobel_binarize`` ...), taking raw
integer pointers; :class:`Context` wraps them for torch tensors.  There is
no fallback: if libld.so is missing, importing the library raises.
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass

from . import build as _build

LD_OK, LD_ERR_INVALID, LD_ERR_CUDA, LD_ERR_NOMEM, LD_ERR_CAPACITY, LD_ERR_TIMEOUT = range(6)
LD_BORDER_ZERO, LD_BORDER_CLEAR = 0, 1
HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ld.h")


class LdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"ld status {status}: {msg}")
        self.status = status


class ld_params(ctypes.Structure):
    _fields_ = [("n_theta", ctypes.c_int32), ("threshold", ctypes.c_int32), ("border", ctypes.c_int32),
                ("top_k", ctypes.c_int32), ("nms_theta", ctypes.c_int32), ("nms_rho", ctypes.c_int32),
                ("min_votes", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("edge_capacity", ctypes.c_int64)]


class ld_peak(ctypes.Structure):
    _fields_ = [("theta_idx", ctypes.c_int32), ("rho_idx", ctypes.c_int32), ("votes", ctypes.c_int32)]


class ld_lines_params(ctypes.Structure):
    _fields_ = [("fill_gap", ctypes.c_int32), ("min_length", ctypes.c_int32), ("max_segments", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class ld_segment(ctypes.Structure):
    _fields_ = [("x1", ctypes.c_int32), ("y1", ctypes.c_int32), ("x2", ctypes.c_int32), ("y2", ctypes.c_int32),
                ("theta_idx", ctypes.c_int32), ("rho_idx", ctypes.c_int32)]


class ld_canny_params(ctypes.Structure):
    _fields_ = [("t_low", ctypes.c_int32), ("t_high", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("reserved1", ctypes.c_int32)]


class ld_frame(ctypes.Structure):
    _fields_ = [("img", ctypes.c_void_p), ("w", ctypes.c_int32), ("h", ctypes.c_int32),
                ("pitch", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ld_synth_stripe(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("c", ctypes.c_int64), ("tx", ctypes.c_int64),
                ("ty", ctypes.c_int64), ("t0", ctypes.c_int64), ("dash", ctypes.c_int32), ("gap", ctypes.c_int32),
                ("value", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ld_synth_frame(ctypes.Structure):
    _fields_ = [("img", ctypes.c_void_p), ("w", ctypes.c_int32), ("h", ctypes.c_int32),
                ("pitch", ctypes.c_int32), ("n_stripes", ctypes.c_int32), ("base", ctypes.c_uint64 * 3),
                ("k_top", ctypes.c_int64), ("k_road", ctypes.c_int64), ("salt_thr", ctypes.c_uint64),
                ("stripes", ld_synth_stripe * 4)]


class ld_proposal_net(ctypes.Structure):
    _fields_ = [("w", ctypes.c_void_p * 4), ("b", ctypes.c_void_p * 4), ("wh", ctypes.c_void_p),
                ("bh", ctypes.c_void_p)]


class ld_proposal_params(ctypes.Structure):
    _fields_ = [("p_band", ctypes.c_float), ("p_fallback", ctypes.c_float), ("margin", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


_lib = None
_P = ctypes.c_void_p
_SIGS = {
    "ld_params_default": [ctypes.POINTER(ld_params)],
    "ld_ctx_create": [ctypes.POINTER(_P), ctypes.c_int],
    "ld_ctx_destroy": [_P],
    "ld_ctx_reserve": [_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ld_params)],
    "ld_query_sizes": [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ld_params),
                       ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t),
                       ctypes.POINTER(ctypes.c_int32)],
    "ld_sobel_binarize": [_P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ld_params),
                          _P, _P, _P, _P],
    "ld_hough_vote": [_P, _P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ld_params), _P, _P],
    "ld_hough_peaks": [_P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ld_params), _P, _P, _P],
    "ld_detect_batch": [_P, ctypes.POINTER(ld_frame), ctypes.c_int32, ctypes.POINTER(ld_params), _P, _P, _P,
                        _P],
    "ld_detect_batch_host": [_P, ctypes.POINTER(ld_frame), ctypes.c_int32, ctypes.POINTER(ld_params), _P, _P,
                             _P, _P],
    "ld_ctx_set_wait_limit": [_P, ctypes.c_int64],
    "ld_lines_params_default": [ctypes.POINTER(ld_lines_params)],
    "ld_sobel_hough_fused": [_P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ld_params),
                             _P, _P],
    "ld_detect_fused_batch": [_P, ctypes.POINTER(ld_frame), ctypes.c_int32, ctypes.POINTER(ld_params), _P, _P, _P,
                              _P],
    "ld_canny_params_default": [ctypes.POINTER(ld_canny_params)],
    "ld_canny": [_P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ld_params),
                 ctypes.POINTER(ld_canny_params), _P, _P, _P, _P],
    "ld_detect_canny_batch": [_P, ctypes.POINTER(ld_frame), ctypes.c_int32, ctypes.POINTER(ld_params),
                              ctypes.POINTER(ld_canny_params), _P, _P, _P, _P],
    "ld_hough_lines": [_P, _P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ld_params), _P, _P,
                       ctypes.POINTER(ld_lines_params), _P, _P, _P, _P],
    "ld_detect_lines_batch": [_P, ctypes.POINTER(ld_frame), ctypes.c_int32, ctypes.POINTER(ld_params),
                              ctypes.POINTER(ld_lines_params), _P, _P, _P, _P, _P, _P, _P],
    "ld_hough_peaks_static": [_P, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ld_params), _P, _P, _P],
    "ld_autotune": [_P, ctypes.POINTER(ld_frame), ctypes.c_int32, ctypes.POINTER(ld_params), ctypes.c_int32, _P],
    "ld_ctx_plan": [_P, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ld_params), ctypes.POINTER(ctypes.c_int32),
                    ctypes.POINTER(ctypes.c_int32)],
    "ld_synth_frames": [_P, ctypes.c_int32, _P],
    "ld_probe_smem_red": [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, _P],
    "ld_proposal_targets": [_P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                            ctypes.c_int32, ctypes.c_float, _P, _P],
    "ld_detect_batch_proposal": [_P, ctypes.POINTER(ld_frame), ctypes.c_int32, ctypes.POINTER(ld_params),
                                 ctypes.POINTER(ld_proposal_net), ctypes.POINTER(ld_proposal_params), _P, _P, _P, _P,
                                 _P, _P],
    "ld_edge_pool_batch": [_P, ctypes.POINTER(ld_frame), ctypes.c_int32, ctypes.POINTER(ld_params), _P, _P],
    "ld_conv3x3_forward": [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                           ctypes.c_int32, _P, _P, _P, _P],
    "ld_conv3x3_backward": [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                            ctypes.c_int32, _P, _P, _P, _P, _P, _P, _P],
    "ld_pool_head_forward": [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P, _P],
    "ld_pool_head_backward": [_P, _P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P],
    "ld_bce_loss": [_P, _P, ctypes.c_int32, ctypes.c_int32, _P, _P, _P],
    "ld_adam_step": [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                     ctypes.c_float, ctypes.c_int32, _P, _P],
    "ld_conv_faults": [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)],
    "ld_proposal_logits": [_P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ld_proposal_net),
                           _P, _P],
    "ld_ctx_enable_timing": [_P, ctypes.c_int],
    "ld_ctx_stage_ms": [_P, ctypes.POINTER(ctypes.c_float * 3)],
}


def library_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Load libld.so (built by ``build.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libld.so not built ({path}); run paper_2212_09460_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.ld_last_error.argtypes = []
    lib.ld_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def header_functions() -> list[str]:
    """Names of the functions include/ld.h declares."""
    with open(HEADER) as f:
        text = f.read()
    return re.findall(r"^LD_API\s+[\w\s\*]*?\b(ld_\w+)\s*\(", text, flags=re.M)


def _check(status: int) -> None:
    if status != LD_OK:
        raise LdError(status, load().ld_last_error().decode())


def params(n_theta=180, threshold=128, border=LD_BORDER_ZERO, top_k=4, nms_theta=5, nms_rho=5,
           min_votes=1, edge_capacity=0) -> ld_params:
    p = ld_params()
    _check(load().ld_params_default(ctypes.byref(p)))
    p.n_theta, p.threshold, p.border, p.top_k = n_theta, threshold, border, top_k
    p.nms_theta, p.nms_rho, p.min_votes, p.edge_capacity = nms_theta, nms_rho, min_votes, edge_capacity
    return p


# ------------------------------------------------------------------ raw C names

def ld_params_default() -> ld_params:
    p = ld_params()
    _check(load().ld_params_default(ctypes.byref(p)))
    return p


def ld_ctx_create(device: int = 0) -> int:
    h = _P()
    _check(load().ld_ctx_create(ctypes.byref(h), device))
    return h.value


def ld_ctx_destroy(ctx: int) -> None:
    _check(load().ld_ctx_destroy(ctx))


def ld_ctx_reserve(ctx: int, max_pixels: int, max_frames: int, max_acc_cells: int, p: ld_params) -> None:
    _check(load().ld_ctx_reserve(ctx, max_pixels, max_frames, max_acc_cells, ctypes.byref(p)))


def ld_query_sizes(w: int, h: int, p: ld_params | None = None):
    a, e, d = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_int32()
    _check(load().ld_query_sizes(w, h, ctypes.byref(p) if p is not None else None,
                                 ctypes.byref(a), ctypes.byref(e), ctypes.byref(d)))
    return a.value, e.value, d.value


def ld_sobel_binarize(ctx, d_img, w, h, pitch, p, d_bin, d_edges, d_edge_count, stream) -> None:
    _check(load().ld_sobel_binarize(ctx, d_img, w, h, pitch, ctypes.byref(p), d_bin, d_edges, d_edge_count,
                                    stream))


def ld_hough_vote(ctx, d_edges, d_edge_count, w, h, p, d_acc, stream) -> None:
    _check(load().ld_hough_vote(ctx, d_edges, d_edge_count, w, h, ctypes.byref(p), d_acc, stream))


def ld_hough_peaks(ctx, d_acc, n_theta, n_rho, p, d_peaks, d_n_peaks, stream) -> None:
    _check(load().ld_hough_peaks(ctx, d_acc, n_theta, n_rho, ctypes.byref(p), d_peaks, d_n_peaks, stream))


def ld_detect_batch(ctx, frames, p, d_peaks, d_n_peaks, d_status, stream) -> None:
    """frames: sequence of (device_ptr, w, h, pitch), or a ctypes ld_frame array."""
    arr = frames if isinstance(frames, ctypes.Array) else _frames_array(frames)
    _check(load().ld_detect_batch(ctx, arr, len(arr), ctypes.byref(p), d_peaks, d_n_peaks, d_status, stream))


def ld_detect_batch_host(ctx, frames, p, h_peaks, h_n_peaks, h_status, stream) -> None:
    """frames: sequence of (host_ptr, w, h, pitch), or a ctypes ld_frame array;
    outputs are host pointers, valid once the stream's work has completed."""
    arr = frames if isinstance(frames, ctypes.Array) else _frames_array(frames)
    _check(load().ld_detect_batch_host(ctx, arr, len(arr), ctypes.byref(p), h_peaks, h_n_peaks, h_status, stream))


def ld_sobel_hough_fused(ctx, d_img, w, h, pitch, p, d_acc, stream) -> None:
    _check(load().ld_sobel_hough_fused(ctx, d_img, w, h, pitch, None if p is None else ctypes.byref(p), d_acc,
                                       stream))


def ld_detect_fused_batch(ctx, frames, p, d_peaks, d_n_peaks, d_status, stream) -> None:
    arr = frames if isinstance(frames, ctypes.Array) else _frames_array(frames)
    _check(load().ld_detect_fused_batch(ctx, arr, len(arr), ctypes.byref(p), d_peaks, d_n_peaks, d_status, stream))


def ld_canny_params_default() -> ld_canny_params:
    q = ld_canny_params()
    _check(load().ld_canny_params_default(ctypes.byref(q)))
    return q


def canny_params(t_low=100, t_high=200) -> ld_canny_params:
    q = ld_canny_params_default()
    q.t_low, q.t_high = t_low, t_high
    return q


def ld_canny(ctx, d_img, w, h, pitch, p, cp, d_bin, d_edges, d_count, stream) -> None:
    _check(load().ld_canny(ctx, d_img, w, h, pitch, None if p is None else ctypes.byref(p),
                           None if cp is None else ctypes.byref(cp), d_bin, d_edges, d_count, stream))


def ld_detect_canny_batch(ctx, frames, p, cp, d_peaks, d_n_peaks, d_status, stream) -> None:
    arr = frames if isinstance(frames, ctypes.Array) else _frames_array(frames)
    _check(load().ld_detect_canny_batch(ctx, arr, len(arr), ctypes.byref(p), ctypes.byref(cp), d_peaks, d_n_peaks,
                                        d_status, stream))


def ld_lines_params_default() -> ld_lines_params:
    q = ld_lines_params()
    _check(load().ld_lines_params_default(ctypes.byref(q)))
    return q


def lines_params(fill_gap=20, min_length=40, max_segments=16) -> ld_lines_params:
    q = ld_lines_params()
    _check(load().ld_lines_params_default(ctypes.byref(q)))
    q.fill_gap, q.min_length, q.max_segments = fill_gap, min_length, max_segments
    return q


def ld_hough_lines(ctx, d_edges, d_count, w, h, p, d_peaks, d_n_peaks, lp, d_segs, d_nsegs, d_support,
                   stream) -> None:
    _check(load().ld_hough_lines(ctx, d_edges, d_count, w, h, None if p is None else ctypes.byref(p), d_peaks,
                                 d_n_peaks, None if lp is None else ctypes.byref(lp), d_segs, d_nsegs, d_support,
                                 stream))


def ld_detect_lines_batch(ctx, frames, p, lp, d_peaks, d_n_peaks, d_status, d_segs, d_nsegs, d_support,
                          stream) -> None:
    arr = frames if isinstance(frames, ctypes.Array) else _frames_array(frames)
    _check(load().ld_detect_lines_batch(ctx, arr, len(arr), ctypes.byref(p), ctypes.byref(lp), d_peaks, d_n_peaks,
                                        d_status, d_segs, d_nsegs, d_support, stream))


def ld_hough_peaks_static(d_acc, n_theta, n_rho, p, d_peaks, d_n_peaks, stream) -> None:
    """ld_hough_peaks without a context and without any device allocation (p None: the defaults)."""
    _check(load().ld_hough_peaks_static(d_acc, n_theta, n_rho, None if p is None else ctypes.byref(p), d_peaks,
                                        d_n_peaks, stream))


def _frames_array(frames):
    arr = (ld_frame * len(frames))()
    for i, (ptr, w, h, pitch) in enumerate(frames):
        arr[i].img, arr[i].w, arr[i].h, arr[i].pitch, arr[i].reserved = ptr, w, h, pitch, 0
    return arr


def ld_autotune(ctx, frames, p, iters, stream) -> None:
    """frames: sequence of (device_ptr, w, h, pitch)."""
    _check(load().ld_autotune(ctx, _frames_array(frames), len(frames), ctypes.byref(p), iters, stream))


def ld_ctx_plan(ctx, w, h, p) -> tuple[int, int]:
    pairs, rows = ctypes.c_int32(), ctypes.c_int32()
    _check(load().ld_ctx_plan(ctx, w, h, ctypes.byref(p), ctypes.byref(pairs), ctypes.byref(rows)))
    return pairs.value, rows.value


def ld_ctx_set_wait_limit(ctx: int, polls: int) -> None:
    """Voting kernels' edge-chunk waits give up after `polls` polls (0: at once, < 0: the default)."""
    _check(load().ld_ctx_set_wait_limit(ctx, polls))


def ld_ctx_enable_timing(ctx: int, enable: bool) -> None:
    _check(load().ld_ctx_enable_timing(ctx, 1 if enable else 0))


def ld_ctx_stage_ms(ctx: int) -> tuple[float, float, int]:
    """(Steps 1-2 ms, Steps 3-4 ms, calls): summed over the calls timed since the last read."""
    ms = (ctypes.c_float * 3)()
    _check(load().ld_ctx_stage_ms(ctx, ctypes.byref(ms)))
    return ms[0], ms[1], int(ms[2])


def ld_synth_frames(d_descs, n, stream) -> None:
    _check(load().ld_synth_frames(d_descs, n, stream))


def ld_probe_smem_red(n_ctas, iters, pattern, d_sink, stream) -> None:
    _check(load().ld_probe_smem_red(n_ctas, iters, pattern, d_sink, stream))


def synth_descriptors(specs, bufs):
    """ld_synth_frame array (host bytes) for (seed, w, h, style) specs and their
    uint8 [h][pitch] device buffers."""
    from . import synth
    arr = (ld_synth_frame * len(specs))()
    for i, ((seed, w, h, style), buf) in enumerate(zip(specs, bufs)):
        fp = synth.frame_params(seed, w, h, style)
        d = arr[i]
        d.img, d.w, d.h, d.pitch = buf.data_ptr(), w, h, buf.stride(0)
        d.n_stripes = len(fp["stripes"])
        for k in range(3):
            d.base[k] = fp["base"][k]
        d.k_top, d.k_road, d.salt_thr = fp["k_top"], fp["k_road"], fp["salt_thr"]
        for k, st in enumerate(fp["stripes"]):
            s = d.stripes[k]
            s.nx, s.ny, s.c, s.tx, s.ty, s.t0 = st.nx, st.ny, st.c, st.tx, st.ty, st.t0
            s.dash, s.gap, s.value, s.reserved = st.dash, st.gap, st.value, 0
    return arr


def synth_frames_device(specs, device, stream=None):
    """Generate frames on the device: list of uint8 [h][pitch] tensors (pitch = w
    rounded up to 16), byte-identical to synth.road_frame for each spec."""
    torch = _torch()
    bufs = [torch.empty((h, (w + 15) // 16 * 16), dtype=torch.uint8, device=device) for _, w, h, _ in specs]
    arr = synth_descriptors(specs, bufs)
    raw = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8).to(device)
    ld_synth_frames(raw.data_ptr(), len(specs), _stream_handle(stream))
    return bufs, raw   # keep `raw` (the descriptors) alive until the kernel has run


def ld_edge_pool_batch(ctx, frames, p, d_pool, stream) -> None:
    arr = frames if isinstance(frames, ctypes.Array) else _frames_array(frames)
    _check(load().ld_edge_pool_batch(ctx, arr, len(arr), ctypes.byref(p), d_pool, stream))


def ld_proposal_targets(d_peaks, d_n_peaks, n, top_k, w, h, n_theta, always_k, rel_votes, d_targets,
                        stream) -> None:
    _check(load().ld_proposal_targets(d_peaks, d_n_peaks, n, top_k, w, h, n_theta, always_k, rel_votes, d_targets,
                                      stream))


def proposal_params(p_band=0.2, p_fallback=0.5, margin=2) -> ld_proposal_params:
    q = ld_proposal_params()
    q.p_band, q.p_fallback, q.margin, q.reserved = p_band, p_fallback, margin, 0
    return q


def ld_detect_batch_proposal(ctx, frames, p, net, q, d_peaks, d_n_peaks, d_status, d_fallback, d_active,
                             stream) -> None:
    arr = frames if isinstance(frames, ctypes.Array) else _frames_array(frames)
    _check(load().ld_detect_batch_proposal(ctx, arr, len(arr), ctypes.byref(p), ctypes.byref(net), ctypes.byref(q),
                                           d_peaks, d_n_peaks, d_status, d_fallback, d_active, stream))


def ld_conv3x3_forward(d_x, n, h, w, cin, cout, stride, d_w, d_b, d_y, stream) -> None:
    _check(load().ld_conv3x3_forward(d_x, n, h, w, cin, cout, stride, d_w, d_b, d_y, stream))


def ld_proposal_logits(ctx, d_pool, n, ph, pw, net, d_logits, stream) -> None:
    _check(load().ld_proposal_logits(ctx, d_pool, n, ph, pw, ctypes.byref(net), d_logits, stream))


def ld_conv_faults(device: int = 0) -> int:
    """Tensor-core convolution faults recorded on `device` since the last call (read and cleared)."""
    v = ctypes.c_int32(0)
    _check(load().ld_conv_faults(device, ctypes.byref(v)))
    return v.value


def ld_conv3x3_backward(d_x, n, h, w, cin, cout, stride, d_w, d_y, d_dy, d_dx, d_dw, d_db, stream) -> None:
    _check(load().ld_conv3x3_backward(d_x, n, h, w, cin, cout, stride, d_w, d_y, d_dy, d_dx, d_dw, d_db, stream))


def ld_pool_head_forward(d_y4, n, h4, w4, d_wh, d_bh, d_feat, d_logits, stream) -> None:
    _check(load().ld_pool_head_forward(d_y4, n, h4, w4, d_wh, d_bh, d_feat, d_logits, stream))


def ld_pool_head_backward(d_feat, d_dlogits, d_wh, n, h4, w4, d_dwh, d_dbh, d_dy4, stream) -> None:
    _check(load().ld_pool_head_backward(d_feat, d_dlogits, d_wh, n, h4, w4, d_dwh, d_dbh, d_dy4, stream))


def ld_bce_loss(d_logits, d_target, n, k, d_loss, d_dlogits, stream) -> None:
    _check(load().ld_bce_loss(d_logits, d_target, n, k, d_loss, d_dlogits, stream))


def ld_adam_step(d_param, d_grad, d_m, d_v, count, lr, beta1, beta2, eps, step, d_param_bf16, stream) -> None:
    _check(load().ld_adam_step(d_param, d_grad, d_m, d_v, count, lr, beta1, beta2, eps, step, d_param_bf16,
                               stream))


def ld_last_error() -> str:
    return load().ld_last_error().decode()


# ------------------------------------------------------------------ torch wrappers

def _torch():
    import torch
    return torch


def _stream_handle(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


@dataclass
class PreparedBatch:
    array: "ctypes.Array"   # ld_frame descriptors
    device: "object"


@dataclass
class SobelOut:
    edges: "object"        # torch.uint32/int32 [capacity]
    count: "object"        # torch.int32 [1]
    binary: "object|None"  # torch.uint8 [h][pitch] or None


class Context:
    """An ld_ctx on one CUDA device, with torch-tensor wrappers of the calls."""

    def __init__(self, device: int = 0):
        self.device = device
        self.handle = ld_ctx_create(device)

    def close(self) -> None:
        if self.handle:
            ld_ctx_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @staticmethod
    def _img(img):
        torch = _torch()
        if img.dtype != torch.uint8 or img.dim() != 2 or not img.is_cuda or img.stride(1) != 1:
            raise ValueError("image must be a 2-D uint8 CUDA tensor with unit column stride")
        return img.data_ptr(), img.shape[1], img.shape[0], img.stride(0)

    def set_wait_limit(self, polls: int) -> None:
        ld_ctx_set_wait_limit(self.handle, polls)

    def reserve(self, max_pixels: int, max_frames: int, max_acc_cells: int, p: ld_params) -> None:
        ld_ctx_reserve(self.handle, max_pixels, max_frames, max_acc_cells, p)

    def sobel_binarize(self, img, p: ld_params, want_binary: bool = False, edges=None, count=None,
                       width: int | None = None, stream=None) -> SobelOut:
        """Steps 1-2 on a [h][pitch] uint8 tensor (``width`` = w if the tensor is padded)."""
        torch = _torch()
        ptr, pw, h, pitch = self._img(img)
        w = pw if width is None else width
        cap = p.edge_capacity if p.edge_capacity > 0 else w * h
        if edges is None:
            edges = torch.empty(cap, dtype=torch.int32, device=img.device)
        if count is None:
            count = torch.empty(1, dtype=torch.int32, device=img.device)
        binary = torch.empty((h, pitch), dtype=torch.uint8, device=img.device) if want_binary else None
        ld_sobel_binarize(self.handle, ptr, w, h, pitch, p, binary.data_ptr() if binary is not None else None,
                          edges.data_ptr(), count.data_ptr(), _stream_handle(stream))
        return SobelOut(edges, count, binary)

    def hough_vote(self, edges, count, w: int, h: int, p: ld_params, acc=None, stream=None):
        """Step 3: returns the int32 [n_theta][2D+1] accumulator."""
        torch = _torch()
        n_acc, _, D = ld_query_sizes(w, h, p)
        if acc is None:
            acc = torch.empty((p.n_theta, 2 * D + 1), dtype=torch.int32, device=edges.device)
        ld_hough_vote(self.handle, edges.data_ptr(), count.data_ptr(), w, h, p, acc.data_ptr(),
                      _stream_handle(stream))
        return acc

    def hough_peaks(self, acc, p: ld_params, stream=None):
        """Step 4: returns (peaks int32 [top_k][3], n_peaks int32 [1]) on the device."""
        torch = _torch()
        n_theta, n_rho = acc.shape
        peaks = torch.zeros((p.top_k, 3), dtype=torch.int32, device=acc.device)
        n = torch.zeros(1, dtype=torch.int32, device=acc.device)
        ld_hough_peaks(self.handle, acc.data_ptr(), n_theta, n_rho, p, peaks.data_ptr(), n.data_ptr(),
                       _stream_handle(stream))
        return peaks, n

    def _descs(self, frames, widths=None):
        descs = []
        for i, f in enumerate(frames):
            ptr, pw, h, pitch = self._img(f)
            descs.append((ptr, pw if widths is None else widths[i], h, pitch))
        return descs

    def autotune(self, frames, p: ld_params, iters: int = 3, widths=None, stream=None) -> None:
        """Tune tile sizes on representative frames (synchronises the stream)."""
        ld_autotune(self.handle, self._descs(frames, widths), p, iters, _stream_handle(stream))

    def plan(self, w: int, h: int, p: ld_params) -> tuple[int, int]:
        """(theta pairs per voting tile, Sobel rows per warp) used for w x h
        frames; pairs < 0: the interleaved-column voting kernel, -pairs per tile."""
        return ld_ctx_plan(self.handle, w, h, p)

    def prepare(self, frames, widths=None) -> "PreparedBatch":
        """Build the frame descriptors once, for repeated detect_batch calls on the same tensors."""
        return PreparedBatch(_frames_array(self._descs(frames, widths)), frames[0].device)

    def detect_batch_proposal(self, frames, p: ld_params, net, q: ld_proposal_params | None = None, widths=None,
                              out=None, stream=None):
        """Steps 1-4 with the learned proposal (net: a ProposalNet); returns
        (peaks [n][top_k][3], n_peaks [n], status [n], fallback [n], active_pairs [n])."""
        torch = _torch()
        if isinstance(frames, PreparedBatch):
            descs, dev = frames.array, frames.device
        else:
            descs, dev = self._descs(frames, widths), frames[0].device
        n = len(descs)
        if out is None:
            out = (torch.zeros((n, p.top_k, 3), dtype=torch.int32, device=dev),) + tuple(
                torch.zeros(n, dtype=torch.int32, device=dev) for _ in range(4))
        pk, npk, st, fb, act = out
        ld_detect_batch_proposal(self.handle, descs, p, net.c_struct(), q or proposal_params(), pk.data_ptr(),
                                 npk.data_ptr(), st.data_ptr(), fb.data_ptr(), act.data_ptr(), _stream_handle(stream))
        return out

    def proposal_logits(self, pool, net, out=None, stream=None):
        """The proposal network's inference (fused first layer) on uint8 edge
        counts [n][ph][pw] on the device: logits float32 [n][44]."""
        torch = _torch()
        n, ph, pw = pool.shape
        if out is None:
            out = torch.empty((n, 44), dtype=torch.float32, device=pool.device)
        ld_proposal_logits(self.handle, pool.data_ptr(), n, ph, pw, net.c_struct(), out.data_ptr(),
                           _stream_handle(stream))
        return out

    def edge_pool(self, frames, p: ld_params, widths=None, out=None, stream=None):
        """Edge pixels per 8x8 block (0..64) of equal-size frames: uint8 [n][ceil(h/8)][ceil(w/8)]."""
        torch = _torch()
        descs = self._descs(frames, widths)
        w, h = descs[0][1], descs[0][2]
        if out is None:
            out = torch.empty((len(descs), (h + 7) // 8, (w + 7) // 8), dtype=torch.uint8, device=frames[0].device)
        ld_edge_pool_batch(self.handle, descs, p, out.data_ptr(), _stream_handle(stream))
        return out

    def sobel_hough_fused(self, img, p: ld_params, width: int | None = None, acc=None, stream=None):
        """Steps 1-3 without an edge list: the int32 [n_theta][2D+1] accumulator."""
        torch = _torch()
        ptr, pw, h, pitch = self._img(img)
        w = pw if width is None else width
        _, _, D = ld_query_sizes(w, h, p)
        if acc is None:
            acc = torch.empty((p.n_theta, 2 * D + 1), dtype=torch.int32, device=img.device)
        ld_sobel_hough_fused(self.handle, ptr, w, h, pitch, p, acc.data_ptr(), _stream_handle(stream))
        return acc

    def detect_fused_batch(self, frames, p: ld_params, widths=None, out=None, stream=None):
        """Steps 1-4 with Steps 1-3 fused; returns (peaks, n_peaks, status) as detect_batch."""
        torch = _torch()
        if isinstance(frames, PreparedBatch):
            descs, dev = frames.array, frames.device
        else:
            descs, dev = self._descs(frames, widths), frames[0].device
        n = len(descs)
        if out is None:
            out = (torch.zeros((n, p.top_k, 3), dtype=torch.int32, device=dev),
                   torch.zeros(n, dtype=torch.int32, device=dev), torch.zeros(n, dtype=torch.int32, device=dev))
        peaks, npk, st = out
        ld_detect_fused_batch(self.handle, descs, p, peaks.data_ptr(), npk.data_ptr(), st.data_ptr(),
                              _stream_handle(stream))
        return peaks, npk, st

    def canny(self, img, p: ld_params, cp: ld_canny_params, want_binary: bool = False, width: int | None = None,
              stream=None) -> SobelOut:
        """Canny edges of a [h][pitch] uint8 tensor (``width`` = w if padded)."""
        torch = _torch()
        ptr, pw, h, pitch = self._img(img)
        w = pw if width is None else width
        cap = p.edge_capacity if p.edge_capacity > 0 else w * h
        edges = torch.empty(max(cap, 4), dtype=torch.int32, device=img.device)
        count = torch.empty(1, dtype=torch.int32, device=img.device)
        binary = torch.empty_like(img) if want_binary else None
        ld_canny(self.handle, ptr, w, h, pitch, p, cp, binary.data_ptr() if binary is not None else None,
                 edges.data_ptr(), count.data_ptr(), _stream_handle(stream))
        return SobelOut(edges, count, binary)

    def detect_canny_batch(self, frames, p: ld_params, cp: ld_canny_params, widths=None, stream=None):
        """Steps 1-4 with Canny edges; returns (peaks [n][top_k][3], n_peaks [n], status [n])."""
        torch = _torch()
        if isinstance(frames, PreparedBatch):
            descs, dev = frames.array, frames.device
        else:
            descs, dev = self._descs(frames, widths), frames[0].device
        n = len(descs)
        peaks = torch.zeros((n, p.top_k, 3), dtype=torch.int32, device=dev)
        npk = torch.zeros(n, dtype=torch.int32, device=dev)
        st = torch.zeros(n, dtype=torch.int32, device=dev)
        ld_detect_canny_batch(self.handle, descs, p, cp, peaks.data_ptr(), npk.data_ptr(), st.data_ptr(),
                              _stream_handle(stream))
        return peaks, npk, st

    def hough_lines(self, edges, count, w: int, h: int, p: ld_params, peaks, n_peaks, lp: ld_lines_params,
                    stream=None):
        """Hough lines of one frame from device tensors (edge list, count [1],
        peaks [top_k][3], n_peaks [1]); returns (segments [top_k][max_segments][6],
        n_segments [top_k], support [top_k])."""
        torch = _torch()
        dev = edges.device
        segs = torch.zeros((p.top_k, lp.max_segments, 6), dtype=torch.int32, device=dev)
        nseg = torch.zeros(p.top_k, dtype=torch.int32, device=dev)
        sup = torch.zeros(p.top_k, dtype=torch.int32, device=dev)
        ld_hough_lines(self.handle, edges.data_ptr(), count.data_ptr(), w, h, p, peaks.data_ptr(), n_peaks.data_ptr(),
                       lp, segs.data_ptr(), nseg.data_ptr(), sup.data_ptr(), _stream_handle(stream))
        return segs, nseg, sup

    def detect_lines_batch(self, frames, p: ld_params, lp: ld_lines_params, widths=None, stream=None):
        """Steps 1-4 and the Hough lines; returns (peaks, n_peaks, status,
        segments [n][top_k][max_segments][6], n_segments [n][top_k], support [n][top_k])."""
        torch = _torch()
        if isinstance(frames, PreparedBatch):
            descs, dev = frames.array, frames.device
        else:
            descs, dev = self._descs(frames, widths), frames[0].device
        n = len(descs)
        peaks = torch.zeros((n, p.top_k, 3), dtype=torch.int32, device=dev)
        npk = torch.zeros(n, dtype=torch.int32, device=dev)
        st = torch.zeros(n, dtype=torch.int32, device=dev)
        segs = torch.zeros((n, p.top_k, lp.max_segments, 6), dtype=torch.int32, device=dev)
        nseg = torch.zeros((n, p.top_k), dtype=torch.int32, device=dev)
        sup = torch.zeros((n, p.top_k), dtype=torch.int32, device=dev)
        ld_detect_lines_batch(self.handle, descs, p, lp, peaks.data_ptr(), npk.data_ptr(), st.data_ptr(),
                              segs.data_ptr(), nseg.data_ptr(), sup.data_ptr(), _stream_handle(stream))
        return peaks, npk, st, segs, nseg, sup

    @staticmethod
    def _host_descs(frames, widths=None):
        torch = _torch()
        if isinstance(frames, torch.Tensor) and frames.dim() == 3:
            frames = list(frames.unbind(0))
        descs = []
        for i, f in enumerate(frames):
            if f.dtype != torch.uint8 or f.dim() != 2 or f.is_cuda or f.stride(1) != 1:
                raise ValueError("host frames must be 2-D uint8 CPU tensors with unit column stride")
            descs.append((f.data_ptr(), f.shape[1] if widths is None else widths[i], f.shape[0], f.stride(0)))
        return descs

    def detect_batch_host(self, frames, p: ld_params, widths=None, out=None, stream=None, sync: bool = True):
        """Steps 1-4 on frames in host memory (a list of uint8 CPU tensors, or
        one [n][h][pitch] tensor; pinned memory lets the upload overlap):
        returns host (peaks [n][top_k][3], n_peaks [n], status [n]).  With
        sync=False the outputs are valid only after the stream is synchronised,
        and the frames must stay unchanged until then."""
        torch = _torch()
        descs = frames if isinstance(frames, ctypes.Array) else _frames_array(self._host_descs(frames, widths))
        n = len(descs)
        if out is None:
            out = (torch.zeros((n, p.top_k, 3), dtype=torch.int32).pin_memory(),
                   torch.zeros(n, dtype=torch.int32).pin_memory(), torch.zeros(n, dtype=torch.int32).pin_memory())
        peaks, npk, st = out
        ld_detect_batch_host(self.handle, descs, p, peaks.data_ptr(), npk.data_ptr(), st.data_ptr(),
                             _stream_handle(stream))
        if sync:
            (stream if stream is not None else torch.cuda.current_stream(torch.device("cuda", self.device))).synchronize()
        return peaks, npk, st

    def prepare_host(self, frames, widths=None):
        """Frame descriptors of host frames, built once for repeated detect_batch_host calls."""
        return _frames_array(self._host_descs(frames, widths))

    def detect_batch(self, frames, p: ld_params, widths=None, out=None, stream=None):
        """Steps 1-4 on a list of uint8 CUDA tensors (or a PreparedBatch);
        returns (peaks [n][top_k][3], n_peaks [n], status [n])."""
        torch = _torch()
        if isinstance(frames, PreparedBatch):
            descs, dev = frames.array, frames.device
        else:
            descs, dev = self._descs(frames, widths), frames[0].device
        n = len(descs)
        if out is None:
            out = (torch.zeros((n, p.top_k, 3), dtype=torch.int32, device=dev),
                   torch.zeros(n, dtype=torch.int32, device=dev),
                   torch.zeros(n, dtype=torch.int32, device=dev))
        peaks, npk, st = out
        ld_detect_batch(self.handle, descs, p, peaks.data_ptr(), npk.data_ptr(), st.data_ptr(),
                        _stream_handle(stream))
        return peaks, npk, st
