"""Pins of the oracle's Canny stage (oracle.canny), the edge detector the paper
proposes in place of Sobel (Sec. 7).  Pinned against what mathematics and
independent routines fix:

  * the 5x5 binomial blur: its impulse response is the kernel itself, a
    constant interior stays constant, and it equals scipy.ndimage.convolve
    with the same kernel (rounded);
  * the magnitude equals |Sobel_x * G| + |Sobel_y * G| from scipy on the blur;
  * a vertical step edge gives a one-pixel ridge, at the column derived by hand;
  * non-maximum suppression, the thresholds and the hysteresis equal an
    independent numpy restatement whose connectivity comes from
    scipy.ndimage.label (8-connected components that hold a strong pixel).
"""
import numpy as np
import pytest

scipy_ndimage = pytest.importorskip("scipy.ndimage")

from paper_2212_09460_gb300 import synth

B5 = np.array([1, 4, 6, 4, 1])
K5 = np.outer(B5, B5)


def test_blur_impulse_response(ora):
    img = np.zeros((16, 17), np.uint8)
    img[7, 8] = 255
    g = ora.canny_blur(img)
    ref = np.zeros_like(g)
    for j in range(-2, 3):
        for i in range(-2, 3):
            ref[7 + j, 8 + i] = (K5[j + 2, i + 2] * 255 + 128) >> 8
    np.testing.assert_array_equal(g, ref)


def test_blur_constant_interior_and_library(ora):
    img = np.full((20, 24), 173, np.uint8)
    g = ora.canny_blur(img)
    assert (g[2:-2, 2:-2] == 173).all()
    rng = np.random.default_rng(1)
    img = rng.integers(0, 256, (37, 29)).astype(np.uint8)
    conv = scipy_ndimage.convolve(img.astype(np.int64), K5, mode="constant", cval=0)
    np.testing.assert_array_equal(ora.canny_blur(img), ((conv + 128) >> 8).astype(np.uint8))


def _sobel_mag(g):
    kx = np.array([[-1, 0, 1], [-2, 0, 2], [-1, 0, 1]])
    gx = scipy_ndimage.correlate(g.astype(np.int64), kx, mode="constant", cval=0)
    gy = scipy_ndimage.correlate(g.astype(np.int64), kx.T, mode="constant", cval=0)
    return gx, gy


def test_magnitude_matches_library(ora):
    img = synth.road_frame(3, 120, 90, synth.THROUGHPUT_1080P)
    _, mag = ora.canny(img, 100, 200, return_mag=True)
    gx, gy = _sobel_mag(ora.canny_blur(img))
    np.testing.assert_array_equal(mag, np.abs(gx) + np.abs(gy))


def test_step_edge_one_pixel_ridge(ora):
    # columns < 20 are 50, >= 20 are 200.  Interior rows: the 1-D blur gives
    # 50, 59, 97, 153, 191, 200 at x = 17..22 (round(sum b_i I / 16)), so
    # M = 4 |G(x+1) - G(x-1)| = 36, 188, 376, 376, 188, 36 at x = 17..22; the
    # pair 376, 376 keeps x = 19 (M > M(x-1) and M >= M(x+1)), x = 20 fails
    # M > M(x-1).  With t_high 300 it is strong.
    img = np.full((40, 48), 50, np.uint8)
    img[:, 20:] = 200
    b, mag = ora.canny(img, 100, 300, return_mag=True)
    np.testing.assert_array_equal(mag[10, 16:24], [0, 36, 188, 376, 376, 188, 36, 0])
    for y in range(4, 36):
        assert list(np.nonzero(b[y, 12:28])[0] + 12) == [19], y


def _restated(img, t_low, t_high, ora):
    # independent restatement of steps 3-5 on the oracle's own blur
    g = ora.canny_blur(img)
    gx, gy = _sobel_mag(g)
    ax, ay = np.abs(gx), np.abs(gy)
    m = ax + ay
    sec = np.where(ay * 65536 <= 27146 * ax, 0, np.where(ay * 65536 >= 158218 * ax, 2, np.where(gx * gy > 0, 1, 3)))
    h, w = m.shape
    mp = np.zeros((h + 2, w + 2), np.int64)
    mp[1:-1, 1:-1] = m
    d1 = {0: (0, -1), 1: (-1, -1), 2: (-1, 0), 3: (-1, 1)}   # (dy, dx) of n1
    keep = np.zeros_like(m, bool)
    for s, (dy, dx) in d1.items():
        n1 = mp[1 + dy:1 + dy + h, 1 + dx:1 + dx + w]
        n2 = mp[1 - dy:1 - dy + h, 1 - dx:1 - dx + w]
        keep |= (sec == s) & (m > 0) & (m > n1) & (m >= n2)
    strong = keep & (m >= t_high)
    cand = keep & (m >= t_low)
    lab, _ = scipy_ndimage.label(cand, structure=np.ones((3, 3), int))
    on = np.unique(lab[strong])
    return np.where(np.isin(lab, on[on > 0]), 255, 0).astype(np.uint8)


@pytest.mark.parametrize("case", [(0, 640, 480, 100, 200), (1001, 400, 300, 60, 150), (7, 97, 61, 20, 40)])
def test_canny_matches_restatement(ora, case):
    seed, w, h, tl, th = case
    img = synth.road_frame(seed, w, h, synth.THROUGHPUT_1080P if seed else synth.LATENCY_640x480)
    np.testing.assert_array_equal(ora.canny(img, tl, th), _restated(img, tl, th, ora))


def test_canny_random_images_match_restatement(ora):
    rng = np.random.default_rng(5)
    for _ in range(5):
        h, w = (int(v) for v in rng.integers(5, 40, 2))
        img = (rng.integers(0, 256, (h, w)) * (rng.random((h, w)) < 0.5)).astype(np.uint8)
        np.testing.assert_array_equal(ora.canny(img, 80, 240), _restated(img, 80, 240, ora))
