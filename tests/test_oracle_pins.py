"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these re-types the oracle's own formulas: each checks it against a
library routine, a closed form derived by hand, an invariant, the exact
fp64 value of Eq. 3 within the Q16 error bound, or an independent brute
force.  A plausible slip in the oracle (a dropped Sobel term, a sign, a
transposed coordinate, a wrong mirror in Eqs. 4-5, an off-by-one in the
rho offset, a wrong tie-break) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy import ndimage

from paper_2212_09460_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _sobel_scipy(img):
    """|Gx| + |Gy| via scipy.ndimage.sobel with zero padding (mode='constant')."""
    a = img.astype(np.int64)
    gx = ndimage.sobel(a, axis=1, mode="constant", cval=0)
    gy = ndimage.sobel(a, axis=0, mode="constant", cval=0)
    return np.minimum(np.abs(gx) + np.abs(gy), 255).astype(np.uint8)


# ---------------------------------------------------------------- Step 1: Eq. 1

@pytest.mark.parametrize("w,h,seed", [(3, 3, 1), (5, 4, 2), (17, 9, 3), (64, 48, 4), (131, 37, 5)])
def test_sobel_matches_library_routine(ora, w, h, seed):
    img = synth.random_image(seed, w, h)
    np.testing.assert_array_equal(ora.sobel_mag(img), _sobel_scipy(img))


def test_sobel_ignores_pitch_padding(ora):
    img = synth.random_image(9, 37, 11)
    buf = synth.pitched(img, 48, seed=3)
    np.testing.assert_array_equal(ora.sobel_mag(buf[:, :37]), ora.sobel_mag(img))


def test_sobel_convention_invariance(ora):
    # Fig. 2 (the coefficient figure) is lost; |Gx|+|Gy| is the same for all
    # eight sign / transpose conventions of the kernel pair.
    img = synth.random_image(11, 23, 19)
    ref = ora.sobel_mag(img, variant=0)
    for v in range(1, 8):
        np.testing.assert_array_equal(ora.sobel_mag(img, variant=v), ref)


@pytest.mark.parametrize("c", [1, 20, 31, 32, 42, 60, 200])
def test_sobel_constant_image_closed_form(ora, c):
    # Zero padding (Sec. 3.1): interior 0, edge pixels 4c, corners 6c, capped at 255.
    w, h = 9, 7
    m = ora.sobel_mag(np.full((h, w), c, np.uint8)).astype(int)
    exp = np.zeros((h, w), int)
    exp[0, :] = exp[-1, :] = exp[:, 0] = exp[:, -1] = 4 * c
    for y, x in ((0, 0), (0, w - 1), (h - 1, 0), (h - 1, w - 1)):
        exp[y, x] = 6 * c
    np.testing.assert_array_equal(m, np.minimum(exp, 255))
    # binarized frame: edges exactly when 4c >= 128 (c >= 32), Sec. 2.2 with T = 128
    b = ora.binarize(m.astype(np.uint8), 128)
    assert (b[0, 1:-1] == 255).all() == (c >= 32)
    assert (b[1:-1, 1:-1] == 0).all()


def test_sobel_border_clear(ora):
    img = np.full((6, 8), 90, np.uint8)
    m = ora.sobel_mag(img, border=ora.BORDER_CLEAR)
    assert (m == 0).all()


@pytest.mark.parametrize("v", [1, 63, 64, 100, 255])
def test_sobel_impulse_closed_form(ora, v):
    # A single pixel v at (x0, y0): its 8 neighbours get |G| = 2v (saturated), the
    # centre and everything else 0.
    w, h, x0, y0 = 11, 9, 4, 5
    img = np.zeros((h, w), np.uint8)
    img[y0, x0] = v
    m = ora.sobel_mag(img).astype(int)
    exp = np.zeros((h, w), int)
    exp[y0 - 1:y0 + 2, x0 - 1:x0 + 2] = min(2 * v, 255)
    exp[y0, x0] = 0
    np.testing.assert_array_equal(m, exp)


def test_sobel_ramps_threshold_and_saturation(ora):
    # I = 16x: interior Gx = 4*16*2 = 128 -> exactly at T -> 255 (test is >=).
    # I = 15x: interior 120 -> 0.  I = 32x: interior 256 -> saturates to 255.
    x = np.arange(8)
    for slope, mag, b in ((16, 128, 255), (15, 120, 0), (32, 255, 255)):
        img = np.tile((slope * x).astype(np.uint8), (6, 1))
        m = ora.sobel_mag(img)
        assert (m[1:-1, 1:-1] == mag).all()
        assert (ora.binarize(m, 128)[1:-1, 1:-1] == b).all()


# ---------------------------------------------------------------- Step 2: Sec. 2.2

def test_binarize_values_and_boundary(ora):
    mag = np.arange(256, dtype=np.uint8).reshape(16, 16)
    for t in (1, 127, 128, 200, 255):
        b = ora.binarize(mag, t)
        assert set(np.unique(b)) <= {0, 255}
        np.testing.assert_array_equal(b == 255, mag >= t)


def test_edge_list_row_major(ora):
    b = synth.random_image(21, 29, 13, density=0.3)
    e = ora.edge_list(b)
    ys, xs = np.nonzero(b == 255)          # numpy's row-major order
    np.testing.assert_array_equal(e >> 16, ys)
    np.testing.assert_array_equal(e & 0xFFFF, xs)


# ---------------------------------------------------------------- Step 3: Eqs. 3-5

@pytest.mark.parametrize("n", [2, 4, 8, 90, 180, 360, 720])
def test_trig_table_closed_forms_and_symmetry(ora, n):
    c, s = ora.trig_q16(n)
    assert c[0] == 65536 and s[0] == 0
    assert c[n // 2] == 0 and s[n // 2] == 65536
    if n % 4 == 0:
        assert c[n // 4] == s[n // 4] == 46341 and c[3 * n // 4] == -46341
    for k in range(1, n):                              # Eqs. 4-5
        assert s[n - k] == s[k] and c[n - k] == -c[k]
    t = np.arange(n) * math.pi / n
    assert np.abs(c - 65536 * np.cos(t)).max() <= 0.5
    assert np.abs(s - 65536 * np.sin(t)).max() <= 0.5


@pytest.mark.parametrize("n", [180, 360])
def test_trig_table_no_rounding_ties(n):
    # No table entry lies near a .5 tie, so fp64 rounding on any libm gives the
    # same table (margin checked independently of the oracle).
    m = 1.0
    for k in range(n // 2 + 1):
        for v in (math.cos(k * math.pi / n) * 65536, math.sin(k * math.pi / n) * 65536):
            m = min(m, abs(v - math.floor(v) - 0.5))
    assert m > 1e-3


def test_rho_max(ora):
    for w, h in ((3, 4), (640, 480), (1920, 1080), (3840, 2160), (512, 512), (7, 7)):
        D = ora.rho_max(w, h)
        assert D * D >= w * w + h * h and (D - 1) ** 2 < w * w + h * h
    assert ora.rho_max(3, 4) == 5 and ora.rho_max(640, 480) == 800


def _line_pixels(kind, a, n):
    t = np.arange(n)
    if kind == "vline":
        return np.full(n, a), t
    if kind == "hline":
        return t, np.full(n, a)
    if kind == "diag":
        return t, t
    if kind == "anti":
        return t, a - t
    raise ValueError(kind)


def _golden_lines():
    rows = []
    with open(os.path.join(GOLDEN, "hough_lines.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, *vals = line.split()
            rows.append((k, *map(int, vals)))
    return rows


@pytest.mark.parametrize("row", _golden_lines())
def test_hough_golden_lines(ora, row):
    kind, w, h, n_theta, a, n, ti, rho, votes = row
    xs, ys = _line_pixels(kind, a, n)
    edges = ((ys.astype(np.uint32) << 16) | xs.astype(np.uint32))
    acc, dropped = ora.hough(edges, w, h, n_theta, return_dropped=True)
    D = ora.rho_max(w, h)
    assert dropped == 0
    assert acc.shape == (n_theta, 2 * D + 1)
    assert acc[ti, rho + D] == votes
    assert acc[ti].sum() == votes          # every vote of that theta in one cell


def test_hough_single_pixel_matches_fp64_eq3(ora):
    # For every pixel of a small image and every theta, the Q16 rho equals
    # round-half-up of the exact x cos + y sin (Eq. 3) unless the exact value is
    # within the Q16 error bound of a .5 tie; it never differs by more than 1.
    w, h, n_theta = 41, 29, 180
    D = ora.rho_max(w, h)
    t = np.arange(n_theta) * math.pi / n_theta
    checked = 0
    for y in range(0, h, 2):
        for x in range(0, w, 3):
            e = np.array([(y << 16) | x], np.uint32)
            acc = ora.hough(e, w, h, n_theta)
            assert (acc.sum(axis=1) == 1).all()
            rho = acc.argmax(axis=1) - D
            exact = x * np.cos(t) + y * np.sin(t)
            ref = np.floor(exact + 0.5)
            bound = (x + y) * 0.5 / 65536 + 1e-9
            frac = exact + 0.5 - np.floor(exact + 0.5)
            safe = (frac > bound) & (frac < 1 - bound)
            assert (np.abs(rho - ref) <= 1).all()
            np.testing.assert_array_equal(rho[safe], ref[safe])
            checked += safe.sum()
    assert checked > 0.99 * n_theta * len(range(0, h, 2)) * len(range(0, w, 3))


@pytest.mark.parametrize("w,h,n_theta,dens", [(37, 23, 180, 0.2), (64, 64, 360, 0.05), (13, 200, 8, 0.5)])
def test_hough_column_sums_and_bruteforce(ora, w, h, n_theta, dens):
    # Invariant: every theta column sums to the number of edge pixels.  Brute force:
    # an independent dictionary count with exact fp64 rho away from ties.
    b = synth.random_image(w * h + n_theta, w, h, density=dens)
    e = ora.edge_list(b)
    acc, dropped = ora.hough(e, w, h, n_theta, return_dropped=True)
    assert dropped == 0
    assert (acc.sum(axis=1) == len(e)).all()
    D = ora.rho_max(w, h)
    xs, ys = (e & 0xFFFF).astype(float), (e >> 16).astype(float)
    for k in range(0, n_theta, max(1, n_theta // 12)):
        th = k * math.pi / n_theta
        exact = xs * math.cos(th) + ys * math.sin(th) + 0.5
        fl = np.floor(exact)
        bound = (xs + ys) * 0.5 / 65536 + 1e-9
        safe = ((exact - fl) > bound) & ((exact - fl) < 1 - bound)
        counts = {}
        for r in fl[safe].astype(int):
            counts[r] = counts.get(r, 0) + 1
        n_unsafe = int((~safe).sum())
        for r, cnt in counts.items():
            assert cnt <= acc[k, r + D] <= cnt + n_unsafe


def test_hough_extreme_corner_int64(ora):
    # The largest accepted image (w + h <= 32767): the corner pixel's rho agrees
    # with exact arithmetic and stays inside [-D, D].
    w, h = 32764, 3
    e = np.array([((h - 1) << 16) | (w - 1), 0, (h - 1) << 16, w - 1], np.uint32)
    acc, dropped = ora.hough(e, w, h, 360, return_dropped=True)
    assert dropped == 0 and (acc.sum(axis=1) == 4).all()
    D = ora.rho_max(w, h)
    assert acc[0, (w - 1) + D] == 2      # theta = 0: rho = x for (w-1, 0) and (w-1, h-1)


# ---------------------------------------------------------------- Step 4: peaks

def _golden_peaks():
    with open(os.path.join(GOLDEN, "peaks_small.txt")) as f:
        lines = [ln for ln in f if not ln.startswith("#") and ln.strip()]
    nt, nr = map(int, lines[0].split()[1:])
    acc = np.array([list(map(int, lines[1 + i].split())) for i in range(nt)], np.int32)
    k = int(lines[1 + nt].split()[1])
    exp = np.array([list(map(int, ln.split())) for ln in lines[2 + nt:]], np.int32)
    return acc, k, exp


def test_peaks_golden(ora):
    acc, k, exp = _golden_peaks()
    np.testing.assert_array_equal(ora.peaks(acc, k, 5, 5, 1), exp)


def test_peaks_k1_is_argmax(ora):
    rng = np.random.default_rng(5)
    for _ in range(20):
        acc = rng.integers(0, 6, size=(13, 31)).astype(np.int32)
        p = ora.peaks(acc, 1)
        i = int(np.argmax(acc))          # first max in row-major = theta asc, rho asc
        assert tuple(p[0]) == (i // 31, i % 31, acc.flat[i])


def _greedy_bruteforce(acc, k, nt, nr, minv):
    """Independent greedy: sort every cell once, then walk with a suppressed set."""
    T, R = acc.shape
    cells = sorted(((-int(acc[t, r]), t, r) for t in range(T) for r in range(R)))
    sup, out = set(), []
    while len(out) < k:
        pick = next(((t, r) for v, t, r in cells
                     if (t, r) not in sup and -v >= minv), None)
        if pick is None:
            break
        t, r = pick
        out.append((t, r, int(acc[t, r])))
        for dt in range(-(nt // 2), nt // 2 + 1):
            for dr in range(-(nr // 2), nr // 2 + 1):
                sup.add((t + dt, r + dr))
    return np.array(out, np.int32).reshape(-1, 3)


@pytest.mark.parametrize("seed", range(6))
def test_peaks_bruteforce_with_ties(ora, seed):
    rng = np.random.default_rng(seed)
    T, R = int(rng.integers(3, 15)), int(rng.integers(3, 40))
    acc = rng.integers(0, 4, size=(T, R)).astype(np.int32)   # many ties and plateaus
    for k, nt, nr, mv in ((4, 5, 5, 1), (16, 3, 7, 2), (8, 1, 1, 1), (3, 5, 5, 4)):
        np.testing.assert_array_equal(ora.peaks(acc, k, nt, nr, mv),
                                      _greedy_bruteforce(acc, k, nt, nr, mv))


# ---------------------------------------------------------------- whole path

def test_detect_finds_generated_stripes(ora):
    # Sanity, not parity: with the frame border cleared, the top peaks of a
    # two-stripe frame lie near the stripe edges the generator drew.
    w, h = 640, 480
    img = synth.road_frame(0, w, h, synth.LATENCY_640x480)
    p = ora.detect(img, 180, 4, border=ora.BORDER_CLEAR)
    D = ora.rho_max(w, h)
    st = synth.frame_stripes(0, w, h, synth.LATENCY_640x480)
    for row in p[:2]:
        th = math.radians(row[0])
        rho = row[1] - D
        ok = False
        for s in st:
            nx, ny, c = s.nx / 65536, s.ny / 65536, s.c / 65536
            phi_n = math.atan2(ny, nx) % math.pi      # normal direction of the stripe
            sign = 1 if math.atan2(ny, nx) >= 0 else -1
            for off in (-3, 3):
                r_line = sign * (c + off)
                dth = min(abs(th - phi_n), math.pi - abs(th - phi_n))
                if dth <= math.radians(1.5) and abs(rho - r_line) <= 5:
                    ok = True
        assert ok, (row, st)


def test_detect_composes_steps(ora):
    img = synth.road_frame(3, 96, 64, synth.THROUGHPUT_1080P)
    m = ora.sobel_mag(img)
    e = ora.edge_list(ora.binarize(m, 128))
    acc = ora.hough(e, 96, 64, 360)
    np.testing.assert_array_equal(ora.detect(img, 360, 4), ora.peaks(acc, 4))
