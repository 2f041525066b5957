"""Seeded synthetic road frames (uint8 grayscale) -- input generator only.

This module holds no step of the detection method (no Sobel, no
binarization, no voting, no peak picking); it only draws pixels.  Both the
CUDA path and the CPU oracle consume its frames, so the two always see the
same input.

The paper's only workload is a 512x512 gray road image that is not
available, so these frames stand in for it.  Every pixel is a pure function
of (seed, x, y): random numbers come from SplitMix64 (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014) used as a
counter-based generator, and all per-pixel arithmetic is integer, so a
device-side generator can reproduce a frame bit for bit.

Frame recipe (all quantities per frame, drawn from the frame's seed):
  * background: vertical gradient 40 (top row) .. 120 (bottom row);
  * 2 solid stripes (``style='solid'``) or 2-4 dashed stripes
    (``style='dashed'``, dash and gap lengths U[30, 60] px) of 6 px width and
    intensity U[200, 255]; stripe directions alternate between U[25, 65] and
    U[115, 155] degrees from the x-axis, each through a point in the lower half;
  * additive noise, approximately Gaussian (Irwin-Hall sum of eight 16-bit
    uniforms) with std ``sigma`` above the horizon (y < h/2) and
    ``sigma_road`` below it (road texture), rounded, clamped to [0, 255];
  * salt: each pixel set to 255 with probability ``salt``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
# std of a sum of eight independent uniforms on {0..65535}
_IH8_STD = math.sqrt(8.0 * (65536.0 ** 2 - 1.0) / 12.0)
_IH8_MEAN = 8 * 65535 // 2  # 262140


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied to a uint64 array."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


_U64 = (1 << 64) - 1


def _mix64_int(z: int) -> int:
    """_mix64 on one Python integer (the per-frame scalars; no numpy overhead)."""
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _U64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _U64
    return z ^ (z >> 31)


def _stream_base_int(seed: int, stream: int) -> int:
    return _mix64_int(((int(seed) * 8 + int(stream)) + 0x9E3779B97F4A7C15) & _U64)


def _stream_base(seed: int, stream: int) -> np.uint64:
    return np.uint64(_stream_base_int(seed, stream))


def _draws(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """The idx-th SplitMix64 outputs of the stream (seed, stream)."""
    base = _stream_base(seed, stream)
    with np.errstate(over="ignore"):
        return _mix64(base + (idx.astype(np.uint64) + np.uint64(1)) * _GAMMA)


class _Scalars:
    """Sequential uniform draws for the per-frame parameters (stream 0)."""

    def __init__(self, seed: int):
        self.base = _stream_base_int(seed, 0)
        self.i = 0

    def u(self) -> float:
        v = _mix64_int((self.base + (self.i + 1) * 0x9E3779B97F4A7C15) & _U64)
        self.i += 1
        return float(v >> 11) / float(1 << 53)

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi]."""
        return lo + min(int(self.u() * (hi - lo + 1)), hi - lo)


@dataclass(frozen=True)
class FrameStyle:
    style: str = "solid"        # 'solid' (two stripes) or 'dashed' (2-4 stripes)
    sigma: float = 8.0          # noise std above the horizon
    sigma_road: float = 8.0     # noise std below the horizon (road texture)
    salt: float = 0.0           # probability of a 255 salt pixel


# Workload presets.  ``LATENCY_640x480`` is the single-frame latency frame
# (solid stripes, sigma 8, no salt).  ``THROUGHPUT_1080P`` is the dashed-lane
# frame with 0.5% salt; its road texture sigma_road was tuned once so that the
# binarized edge density of every frame lies in [5%, 10%].
LATENCY_640x480 = FrameStyle("solid", 8.0, 8.0, 0.0)
THROUGHPUT_1080P = FrameStyle("dashed", 8.0, 12.0, 0.005)


@dataclass(frozen=True)
class Stripe:
    nx: int      # Q16 unit normal
    ny: int
    c: int       # Q16 offset: inside if |x*nx + y*ny - c| < 3*65536
    tx: int      # Q16 unit tangent
    ty: int
    t0: int      # Q16 phase along the stripe
    dash: int    # dash length in px (0: solid)
    gap: int
    value: int   # stripe intensity


def frame_stripes(seed: int, w: int, h: int, style: FrameStyle):
    """Per-frame stripe descriptors (integer Q16 geometry)."""
    r = _Scalars(seed)
    n_lines = 2 if style.style == "solid" else 2 + min(int(r.u() * 3), 2)
    out = []
    for j in range(n_lines):
        lo, hi = (25.0, 65.0) if j % 2 == 0 else (115.0, 155.0)
        phi = math.radians(lo + (hi - lo) * r.u())
        px = (0.2 + 0.6 * r.u()) * (w - 1)
        py = (0.5 + 0.5 * r.u()) * (h - 1)
        value = r.randint(200, 255)
        if style.style == "dashed":
            dash, gap = r.randint(30, 60), r.randint(30, 60)
            phase = r.randint(0, dash + gap - 1)
        else:
            dash, gap, phase = 0, 0, 0
        dx, dy = math.cos(phi), math.sin(phi)
        nx, ny = -dy, dx
        q = 65536.0
        out.append(Stripe(nx=int(round(nx * q)), ny=int(round(ny * q)),
                          c=int(round((px * nx + py * ny) * q)),
                          tx=int(round(dx * q)), ty=int(round(dy * q)),
                          t0=int(round((px * dx + py * dy) * q)) - phase * 65536,
                          dash=dash, gap=gap, value=value))
    return out


def _stripe_mask(st: Stripe, w: int, h: int):
    """Rows, columns of the pixels inside a stripe (and inside a dash).

    The test is the exact integer predicate |x*nx + y*ny - c| < 3*65536 (and
    the dash phase); it is only evaluated on a window of columns around the
    centre line of each row, wide enough to hold every pixel that passes.
    """
    ys = np.arange(h, dtype=np.int64)
    half = 3 * 65536 // max(abs(st.nx), 1) + 3
    xc = np.floor((st.c - ys * st.ny) / st.nx).astype(np.int64)
    xs = xc[:, None] + np.arange(-half, half + 1, dtype=np.int64)[None, :]
    yy = np.broadcast_to(ys[:, None], xs.shape)
    ok = (xs >= 0) & (xs < w) & (np.abs(xs * st.nx + yy * st.ny - st.c) < 3 * 65536)
    if st.dash:
        t = np.floor_divide(xs * st.tx + yy * st.ty - st.t0, 65536)
        ok &= np.mod(t, st.dash + st.gap) < st.dash
    return yy[ok], xs[ok]


_M16x2 = np.uint64(0x0000FFFF0000FFFF)


def road_frame(seed: int, w: int, h: int, style: FrameStyle = LATENCY_640x480) -> np.ndarray:
    """One uint8 [h][w] frame, a pure function of (seed, w, h, style)."""
    ys = np.arange(h, dtype=np.int32)[:, None]
    v = np.empty((h, w), np.int32)
    v[:] = 40 + (80 * ys) // max(h - 1, 1)
    for st in frame_stripes(seed, w, h, style):
        ry, rx = _stripe_mask(st, w, h)
        v[ry, rx] = st.value
    idx = np.arange(w * h, dtype=np.uint64).reshape(h, w)
    a = _draws(seed, 1, idx)
    b = _draws(seed, 2, idx)
    # sum of the eight 16-bit fields of a and b (two 32-bit partial sums)
    t = (a & _M16x2) + ((a >> np.uint64(16)) & _M16x2) + (b & _M16x2) + ((b >> np.uint64(16)) & _M16x2)
    s8 = ((t & np.uint64(0xFFFFFFFF)) + (t >> np.uint64(32))).astype(np.int64)
    n = s8 - _IH8_MEAN
    k_top = int(round(style.sigma / _IH8_STD * 2.0 ** 32))
    k_road = int(round(style.sigma_road / _IH8_STD * 2.0 ** 32))
    kk = np.where(ys >= h // 2, k_road, k_top).astype(np.int64)
    noise = ((n * kk + (1 << 31)) >> 32).astype(np.int32)
    v += noise
    np.clip(v, 0, 255, out=v)
    if style.salt > 0:
        c = _draws(seed, 3, idx)
        thr = np.uint64(int(style.salt * 2.0 ** 32))
        v[(c & np.uint64(0xFFFFFFFF)) < thr] = 255
    return v.astype(np.uint8)


def frame_params(seed: int, w: int, h: int, style: FrameStyle = LATENCY_640x480) -> dict:
    """The integer parameters road_frame draws for a frame, for a device-side
    generator that reproduces it: stream bases, Q32 noise scales, salt
    threshold and stripe geometry."""
    return {
        "base": [_stream_base_int(seed, s) for s in (1, 2, 3)],
        "k_top": int(round(style.sigma / _IH8_STD * 2.0 ** 32)),
        "k_road": int(round(style.sigma_road / _IH8_STD * 2.0 ** 32)),
        "salt_thr": int(style.salt * 2.0 ** 32) if style.salt > 0 else 0,
        "stripes": frame_stripes(seed, w, h, style),
    }


def pitched(frame: np.ndarray, pitch: int | None = None, fill: int | None = None,
            seed: int = 0) -> np.ndarray:
    """Copy a [h][w] frame into a [h][pitch] buffer (pitch a multiple of 16).

    The columns beyond w are filled with ``fill`` or, when None, with seeded
    garbage, so that tests can check that nothing reads them.
    """
    h, w = frame.shape
    if pitch is None:
        pitch = (w + 15) // 16 * 16
    buf = np.empty((h, pitch), np.uint8)
    if fill is None:
        idx = np.arange(h * pitch, dtype=np.uint64).reshape(h, pitch)
        buf[:] = (_draws(seed, 7, idx) & np.uint64(0xFF)).astype(np.uint8)
    else:
        buf[:] = fill
    buf[:, :w] = frame
    return buf


def random_image(seed: int, w: int, h: int, density: float | None = None) -> np.ndarray:
    """Uniform random uint8 image; with ``density`` a 0/255 pattern instead."""
    idx = np.arange(w * h, dtype=np.uint64).reshape(h, w)
    z = _draws(seed, 5, idx)
    if density is None:
        return (z & np.uint64(0xFF)).astype(np.uint8)
    thr = np.uint64(int(density * 2.0 ** 32))
    return np.where((z & np.uint64(0xFFFFFFFF)) < thr, 255, 0).astype(np.uint8)
