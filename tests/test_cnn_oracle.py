"""Pins of the proposal-network CPU oracle (oracle/cnn.py).

The network is not from the paper; it is pinned against mathematics:
finite-difference gradients, closed-form responses of the conv and pooling
layers, the BCE value at zero logits, and brute-force pooling/labels."""
import math

import numpy as np
import pytest

import oracle.cnn as cnn


def _small_x(seed, h=21, w=26):
    rng = np.random.default_rng(seed)
    return (rng.random((2, h, w)) < 0.2).astype(np.float64)


def test_shapes_on_full_input():
    p = cnn.init_params(1)
    x = np.zeros((1, cnn.IN_H, cnn.IN_W))
    x[0, 60, 100] = 1
    logits, acts = cnn.forward(p, x, keep=True)
    assert [a.shape for a in acts[:4]] == [(1, 16, 135, 240), (1, 32, 68, 120), (1, 32, 34, 60), (1, 32, 17, 30)]
    assert acts[4].shape == (1, 1024) and logits.shape == (1, 44)


def test_conv1_impulse_response_closed_form():
    # one input pixel at (y0, x0): conv1 (correlation, pad 1) puts w[co, ky, kx]
    # at output (y0 + 1 - ky, x0 + 1 - kx); zero bias, positive weights survive ReLU
    p = cnn.init_params(2)
    p["w0"] = np.abs(p["w0"])
    x = np.zeros((1, 9, 11))
    y0, x0 = 4, 5
    x[0, y0, x0] = 1.0
    _, acts = cnn.forward(p, x, keep=True)
    a = acts[0][0]
    for co in range(16):
        for ky in range(3):
            for kx in range(3):
                assert a[co, y0 + 1 - ky, x0 + 1 - kx] == pytest.approx(p["w0"][co, ky, kx, 0], abs=1e-12)
    assert np.count_nonzero(a) == 16 * 9


def test_pool_bins_hand_derived():
    assert cnn.pool_bins(17, 4) == [(0, 5), (4, 9), (8, 13), (12, 17)]
    assert cnn.pool_bins(30, 8) == [(0, 4), (3, 8), (7, 12), (11, 15), (15, 19), (18, 23), (22, 27), (26, 30)]


def test_pool_and_head_on_constant_activation():
    # conv4 output constant c in every channel -> every pooled feature is c, so
    # logits = c * rowsum(wh) + bh
    p = cnn.init_params(3)
    for i in range(4):
        p[f"w{i}"] = np.zeros_like(p[f"w{i}"])
    p["b3"] = np.full(32, 0.75)
    logits, acts = cnn.forward(p, np.zeros((1, 17 * 8, 30 * 8)), keep=True)
    np.testing.assert_allclose(acts[4][0], 0.75, rtol=0, atol=1e-12)
    np.testing.assert_allclose(logits[0], 0.75 * p["wh"].sum(axis=1) + p["bh"], rtol=1e-12)


def test_bce_at_zero_logits_is_log2():
    p = cnn.init_params(4)
    p["wh"] = np.zeros_like(p["wh"])
    t = np.random.default_rng(0).integers(0, 2, size=(2, 44)).astype(float)
    loss, _ = cnn.loss_and_grads(p, _small_x(0), t)
    assert loss == pytest.approx(math.log(2.0), abs=1e-12)


@pytest.mark.parametrize("name", ["w0", "b0", "w1", "b1", "w2", "w3", "b3", "wh", "bh"])
def test_gradients_match_finite_differences(name):
    p = cnn.init_params(5)
    for i in range(4):
        p[f"b{i}"] = np.full_like(p[f"b{i}"], 0.05)   # keep most ReLUs active
    x = _small_x(1)
    t = (np.random.default_rng(2).random((2, 44)) < 0.3).astype(float)
    _, g = cnn.loss_and_grads(p, x, t)
    rng = np.random.default_rng(hash(name) % 1000)
    flat = p[name].reshape(-1)
    for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
        eps = 1e-6
        old = flat[idx]
        flat[idx] = old + eps
        lp, _ = cnn.loss_and_grads(p, x, t)
        flat[idx] = old - eps
        lm, _ = cnn.loss_and_grads(p, x, t)
        flat[idx] = old
        fd = (lp - lm) / (2 * eps)
        assert g[name].reshape(-1)[idx] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_count_pool8_bruteforce():
    rng = np.random.default_rng(6)
    b = np.where(rng.random((37, 29)) < 0.2, 255, 0).astype(np.uint8)
    p = cnn.count_pool8(b)
    assert p.shape == (5, 4)
    for i in range(5):
        for j in range(4):
            assert p[i, j] == int((b[8 * i:8 * i + 8, 8 * j:8 * j + 8] == 255).sum())


def test_band_targets():
    peaks = np.array([[0, 10, 5], [9, 3, 4], [10, 3, 4], [359, 0, 1]])
    t = cnn.theta_band_targets(peaks, 360)
    assert list(np.nonzero(t)[0]) == [0, 1, 35]
    # a vertical line x = 100 (theta 0, rho 100) crosses every row
    D = int(np.ceil(np.hypot(1920, 1080)))
    r = cnn.row_band_targets(np.array([[0, 100 + D, 1]]), 1920, 1080, 360)
    assert r.sum() == 8
    # a horizontal line y = 500 (theta 90 deg, rho 500) only in band 500*8//1080 = 3
    r = cnn.row_band_targets(np.array([[180, 500 + D, 1]]), 1920, 1080, 360)
    assert list(np.nonzero(r)[0]) == [3]


def _golden_row_bands():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "row_bands.txt")
    rows = []
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if line:
            w, h, th, rho, bands = line.split()
            rows.append((int(w), int(h), int(th), int(rho), [int(b) for b in bands.split(",")]))
    return rows


@pytest.mark.parametrize("case", _golden_row_bands(), ids=lambda c: f"theta{c[2]}_rho{c[3]}")
def test_row_band_targets_oblique_lines(case):
    # hand-derived bands of oblique lines (tests/golden/row_bands.txt): a sign
    # or index slip in the cos != 0 branch changes the band set
    w, h, th, rho, bands = case
    D = int(np.ceil(np.hypot(w, h)))
    t = cnn.row_band_targets(np.array([[th, rho + D, 1]]), w, h, 360)
    assert list(np.nonzero(t)[0]) == bands


def _conv_bruteforce(x, w, b, stride):
    # y[n,i,j,co] = relu(b[co] + sum w[co,ky,kx,ci] x[n, i*s+ky-1, j*s+kx-1, ci]), zero outside
    n, h, wd, ci = x.shape
    co = w.shape[0]
    oh, ow = (h - 1) // stride + 1, (wd - 1) // stride + 1
    y = np.zeros((n, oh, ow, co))
    for a in range(n):
        for i in range(oh):
            for j in range(ow):
                for o in range(co):
                    acc = b[o]
                    for ky in range(3):
                        for kx in range(3):
                            yy, xx = i * stride + ky - 1, j * stride + kx - 1
                            if 0 <= yy < h and 0 <= xx < wd:
                                for c in range(ci):
                                    acc += w[o, ky, kx, c] * x[a, yy, xx, c]
                    y[a, i, j, o] = max(acc, 0.0)
    return y


@pytest.mark.parametrize("cin,cout,stride,h,w", [(1, 4, 1, 5, 6), (3, 2, 2, 7, 5), (2, 3, 2, 6, 8), (4, 2, 1, 4, 3)])
def test_conv3x3_relu_bruteforce(cin, cout, stride, h, w):
    # the single-layer definition against plain loops (tap order, padding,
    # stride, weight layout [Cout][3][3][Cin], bias, ReLU)
    rng = np.random.default_rng(cin * 31 + stride)
    x = rng.standard_normal((2, h, w, cin))
    wt = rng.standard_normal((cout, 3, 3, cin))
    b = rng.standard_normal(cout) * 0.3
    np.testing.assert_allclose(cnn.conv3x3_relu(x, wt, b, stride), _conv_bruteforce(x, wt, b, stride),
                               rtol=1e-12, atol=1e-12)
