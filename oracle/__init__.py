"""CPU oracle for the lane-detection hot path (arXiv 2212.09460).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg load this package; the product path (the CUDA library and its
Python binding) never does.  The arithmetic lives in ``ld_oracle.c``, plain
loops following Sec. 2-4 of the paper (Eq. 1, Sec. 2.2, Eq. 3, Eqs. 4-5,
Hough peaks); this module only compiles it with gcc and marshals numpy
arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ld_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libld_oracle.so")
_lock = threading.Lock()
_lib = None

BORDER_ZERO = 0
BORDER_CLEAR = 1


def build(force: bool = False) -> str:
    """Compile ld_oracle.c into a shared object with gcc (-O2, no -march)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC",
                           "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64 = ctypes.c_int, ctypes.c_int64
        lib.ldo_rho_max.argtypes = [i32, i32]
        lib.ldo_rho_max.restype = i32
        lib.ldo_sobel_mag.argtypes = [P, i32, i32, i32, i32, i32, P]
        lib.ldo_sobel_mag.restype = None
        lib.ldo_binarize.argtypes = [P, i32, i32, i32, P]
        lib.ldo_binarize.restype = None
        lib.ldo_edge_list.argtypes = [P, i32, i32, P, i64]
        lib.ldo_edge_list.restype = i64
        lib.ldo_trig_q16.argtypes = [i32, P, P]
        lib.ldo_trig_q16.restype = None
        lib.ldo_hough.argtypes = [P, i64, i32, i32, i32, P]
        lib.ldo_hough.restype = i64
        lib.ldo_peaks.argtypes = [P, i32, i32, i32, i32, i32, i32, P]
        lib.ldo_peaks.restype = i32
        lib.ldo_detect.argtypes = [P, i32, i32, i32, i32, i32, i32, i32, i32,
                                   i32, i32, P, P, P, P, P]
        lib.ldo_detect.restype = i32
        lib.ldo_hough_lines.argtypes = [P, i64, i32, i32, i32, P, i32, i32, i32, i32, P, P, P]
        lib.ldo_hough_lines.restype = None
        lib.ldo_canny.argtypes = [P, i32, i32, i32, i32, i32, P, P]
        lib.ldo_canny.restype = None
        lib.ldo_canny_blur.argtypes = [P, i32, i32, i32, P]
        lib.ldo_canny_blur.restype = None
        _lib = lib
        return lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _img(img: np.ndarray):
    img = np.asarray(img)
    if img.dtype != np.uint8 or img.ndim != 2:
        raise ValueError("image must be a 2-D uint8 array")
    if img.strides[1] != 1:
        img = np.ascontiguousarray(img)
    h, w = img.shape
    pitch = img.strides[0]
    return img, w, h, pitch


def rho_max(w: int, h: int) -> int:
    """D = ceil(sqrt(w^2 + h^2)), the rho range bound."""
    return _load().ldo_rho_max(int(w), int(h))


def sobel_mag(img: np.ndarray, border: int = BORDER_ZERO, variant: int = 0) -> np.ndarray:
    """Eq. 1 with zero padding, saturated to 255 (uint8 [h][w])."""
    img, w, h, pitch = _img(img)
    out = np.empty((h, w), np.uint8)
    _load().ldo_sobel_mag(_ptr(img), w, h, pitch, int(border), int(variant), _ptr(out))
    return out


def binarize(mag: np.ndarray, threshold: int = 128) -> np.ndarray:
    """Sec. 2.2: 255 where mag >= threshold, else 0."""
    mag = np.ascontiguousarray(mag, dtype=np.uint8)
    h, w = mag.shape
    out = np.empty((h, w), np.uint8)
    _load().ldo_binarize(_ptr(mag), w, h, int(threshold), _ptr(out))
    return out


def edge_list(binimg: np.ndarray) -> np.ndarray:
    """Row-major packed (y << 16) | x coordinates of the 255 pixels."""
    binimg = np.ascontiguousarray(binimg, dtype=np.uint8)
    h, w = binimg.shape
    cap = int(np.count_nonzero(binimg == 255))
    out = np.empty(max(cap, 1), np.uint32)
    n = _load().ldo_edge_list(_ptr(binimg), w, h, _ptr(out), cap)
    assert n == cap
    return out[:n].copy()


def trig_q16(n_theta: int):
    """Q16 (cos, sin) table, Sec. 3.3 Eqs. 4-5; two int32 arrays."""
    c = np.empty(n_theta, np.int32)
    s = np.empty(n_theta, np.int32)
    _load().ldo_trig_q16(int(n_theta), _ptr(c), _ptr(s))
    return c, s


def hough(edges: np.ndarray, w: int, h: int, n_theta: int, return_dropped: bool = False):
    """Eq. 3 voting into int32 acc[n_theta][2D+1] (theta-major)."""
    edges = np.ascontiguousarray(edges, dtype=np.uint32)
    D = rho_max(w, h)
    acc = np.empty((n_theta, 2 * D + 1), np.int32)
    dropped = _load().ldo_hough(_ptr(edges) if edges.size else None, edges.size,
                                int(w), int(h), int(n_theta), _ptr(acc))
    return (acc, dropped) if return_dropped else acc


def peaks(acc: np.ndarray, top_k: int, nms_theta: int = 5, nms_rho: int = 5,
          min_votes: int = 1) -> np.ndarray:
    """Greedy NMS top-k; int32 [n][3] rows of (theta_idx, rho_idx, votes)."""
    acc = np.ascontiguousarray(acc, dtype=np.int32)
    n_theta, n_rho = acc.shape
    out = np.zeros((max(top_k, 1), 3), np.int32)
    n = _load().ldo_peaks(_ptr(acc), n_theta, n_rho, int(top_k), int(nms_theta),
                          int(nms_rho), int(min_votes), _ptr(out))
    return out[:n].copy()


def detect(img: np.ndarray, n_theta: int, top_k: int, threshold: int = 128,
           border: int = BORDER_ZERO, nms_theta: int = 5, nms_rho: int = 5,
           min_votes: int = 1) -> np.ndarray:
    """Steps 1-4 for one frame in one C call; returns the peaks like peaks()."""
    img, w, h, pitch = _img(img)
    D = rho_max(w, h)
    mag = np.empty(w * h, np.uint8)
    binimg = np.empty(w * h, np.uint8)
    edges = np.empty(w * h, np.uint32)
    acc = np.empty(n_theta * (2 * D + 1), np.int32)
    out = np.zeros((max(top_k, 1), 3), np.int32)
    n = _load().ldo_detect(_ptr(img), w, h, pitch, int(border), int(threshold),
                           int(n_theta), int(top_k), int(nms_theta), int(nms_rho),
                           int(min_votes), _ptr(mag), _ptr(binimg), _ptr(edges),
                           _ptr(acc), _ptr(out))
    return out[:n].copy()


def hough_lines(edges: np.ndarray, w: int, h: int, n_theta: int, peaks: np.ndarray,
                fill_gap: int = 20, min_length: int = 40, max_segments: int = 16):
    """Segments behind each peak (the paper's Step 4 "Hough lines" without the
    drawing): returns (segments, counts, support) with segments int32
    [n_peaks][max_segments][6] rows (x1, y1, x2, y2, theta_idx, rho_idx) (rows
    past counts[p] are zero), counts [n_peaks] kept segments per peak, support
    [n_peaks] supporting pixels per peak."""
    edges = np.ascontiguousarray(edges, dtype=np.uint32)
    peaks = np.ascontiguousarray(np.asarray(peaks, dtype=np.int32).reshape(-1, 3))
    n_p = peaks.shape[0]
    segs = np.zeros((max(n_p, 1), max(max_segments, 1), 6), np.int32)
    counts = np.zeros(max(n_p, 1), np.int32)
    support = np.zeros(max(n_p, 1), np.int32)
    _load().ldo_hough_lines(_ptr(edges) if edges.size else None, edges.size, int(w), int(h),
                            int(n_theta), _ptr(peaks) if n_p else None, n_p, int(fill_gap),
                            int(min_length), int(max_segments), _ptr(segs), _ptr(counts),
                            _ptr(support))
    return segs[:n_p], counts[:n_p], support[:n_p]


def canny(img: np.ndarray, t_low: int = 100, t_high: int = 200, return_mag: bool = False):
    """Canny edges in place of Steps 1-2 (the paper's future work): 0/255 map
    [h][w] (and the magnitude |gx| + |gy| of the blurred image, int32 [h][w])."""
    img, w, h, pitch = _img(img)
    out = np.empty((h, w), np.uint8)
    mag = np.empty((h, w), np.int32) if return_mag else None
    _load().ldo_canny(_ptr(img), w, h, pitch, int(t_low), int(t_high), _ptr(out),
                      _ptr(mag) if return_mag else None)
    return (out, mag) if return_mag else out


def canny_blur(img: np.ndarray) -> np.ndarray:
    """The Canny Gaussian stage alone: (sum of 5x5 binomial x pixels + 128) >> 8."""
    img, w, h, pitch = _img(img)
    out = np.empty((h, w), np.uint8)
    _load().ldo_canny_blur(_ptr(img), w, h, pitch, _ptr(out))
    return out
