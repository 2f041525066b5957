"""Pins of the oracle's Hough-line segments (oracle.hough_lines), the paper's
Step 4 "Hough lines" (Sec. 1, Sec. 5, Fig. 12) without the drawing.

  * hand-derived segments of horizontal, vertical and diagonal dashed lines
    (tests/golden/hough_segments.txt);
  * the supporting pixels of a peak are exactly its votes (same Q16 rounding as
    Eq. 3), on real frames;
  * an independent brute-force restatement on random images and peaks;
  * every segment end is a supporting pixel of its peak.
"""
import math
import os

import numpy as np
import pytest

from paper_2212_09460_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hough_segments.txt")


def _golden():
    cases = []
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if line:
            f = line.split()
            segs = [tuple(int(v) for v in s.split(",")) for s in f[10].split(";")]
            cases.append(dict(name=f[0], kind=f[1], w=int(f[2]), h=int(f[3]), n_theta=int(f[4]), theta=int(f[5]),
                              rho=int(f[6]), gap=int(f[7]), minlen=int(f[8]), support=int(f[9]), segs=segs))
    return cases


def _golden_image(kind, w, h):
    img = np.zeros((h, w), np.uint8)
    if kind == "h":
        for x in list(range(2, 21)) + list(range(31, 51)) + [62, 63]:
            img[10, x] = 255
    elif kind == "v":
        for y in list(range(0, 10)) + list(range(15, 41)):
            img[y, 7] = 255
    else:
        for t in list(range(0, 16)) + list(range(20, 31)):
            img[t, t] = 255
        img[10, 3] = 255
        img[2, 25] = 255
    return img


@pytest.mark.parametrize("case", _golden(), ids=lambda c: c["name"])
def test_golden_segments(ora, case):
    img = _golden_image(case["kind"], case["w"], case["h"])
    D = ora.rho_max(case["w"], case["h"])
    peak = np.array([[case["theta"], case["rho"] + D, 0]])
    segs, counts, support = ora.hough_lines(ora.edge_list(img), case["w"], case["h"], case["n_theta"], peak,
                                            fill_gap=case["gap"], min_length=case["minlen"], max_segments=8)
    assert support[0] == case["support"]
    assert counts[0] == len(case["segs"])
    got = [tuple(int(v) for v in segs[0, i, :4]) for i in range(counts[0])]
    assert got == case["segs"]
    assert (segs[0, : counts[0], 4] == case["theta"]).all() and (segs[0, : counts[0], 5] == case["rho"] + D).all()


def test_support_equals_votes_on_frames(ora):
    for seed, (w, h), nt in ((0, (640, 480), 180), (1003, (1920, 1080), 360)):
        style = synth.LATENCY_640x480 if seed == 0 else synth.THROUGHPUT_1080P
        img = synth.road_frame(seed, w, h, style)
        e = ora.edge_list(ora.binarize(ora.sobel_mag(img)))
        acc = ora.hough(e, w, h, nt)
        pk = ora.peaks(acc, 6)
        rng = np.random.default_rng(seed)
        extra = np.stack([rng.integers(0, nt, 10), rng.integers(0, acc.shape[1], 10), np.zeros(10, int)], 1)
        allp = np.concatenate([pk, extra]).astype(np.int32)
        _, _, support = ora.hough_lines(e, w, h, nt, allp)
        np.testing.assert_array_equal(support, acc[allp[:, 0], allp[:, 1]])


def _brute(edges, w, h, n_theta, peaks, gap, minlen, max_segments):
    # independent restatement: fp64 angle only to pick the table entry's sign
    # pattern is not used; the Q16 table is rebuilt from its definition here
    half = n_theta // 2
    c = np.zeros(n_theta, np.int64)
    s = np.zeros(n_theta, np.int64)
    for k in range(half + 1):
        c[k] = int(round(math.cos(k * math.pi / n_theta) * 65536.0))
        s[k] = int(round(math.sin(k * math.pi / n_theta) * 65536.0))
    for k in range(half + 1, n_theta):
        c[k], s[k] = -c[n_theta - k], s[n_theta - k]
    D = math.isqrt(w * w + h * h - 1) + 1
    xs = (edges & 0xFFFF).astype(np.int64)
    ys = (edges >> 16).astype(np.int64)
    out = []
    for k, r, _ in peaks:
        rho = (xs * c[k] + ys * s[k] + 32768) // 65536      # floor division
        sel = rho == r - D
        pts = list(zip(xs[sel].tolist(), ys[sel].tolist()))
        if abs(c[k]) <= abs(s[k]):
            pts.sort()
        else:
            pts.sort(key=lambda p: (p[1], p[0]))
        segs, start = [], 0
        for i in range(1, len(pts) + 1):
            if i == len(pts) or (pts[i][0] - pts[i - 1][0]) ** 2 + (pts[i][1] - pts[i - 1][1]) ** 2 > gap * gap:
                a, b = pts[start], pts[i - 1]
                if (b[0] - a[0]) ** 2 + (b[1] - a[1]) ** 2 >= minlen * minlen:
                    segs.append((a[0], a[1], b[0], b[1]))
                start = i
        out.append((segs, int(sel.sum())))
    return out


@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_random_images(ora, seed):
    rng = np.random.default_rng(seed)
    w, h = int(rng.integers(8, 60)), int(rng.integers(8, 60))
    img = np.where(rng.random((h, w)) < 0.25, 255, 0).astype(np.uint8)
    for _ in range(3):   # a few straight runs so that segments exist
        y0 = int(rng.integers(0, h))
        img[y0, :] = 255 * (rng.random(w) < 0.8)
    e = ora.edge_list(img)
    nt = int(rng.choice([8, 36, 180]))
    acc = ora.hough(e, w, h, nt)
    pk = np.concatenate([ora.peaks(acc, 4, 3, 3),
                         np.stack([rng.integers(0, nt, 4), rng.integers(0, acc.shape[1], 4), np.zeros(4, int)], 1)])
    gap, minlen = int(rng.integers(1, 6)), int(rng.integers(0, 8))
    segs, counts, support = ora.hough_lines(e, w, h, nt, pk, fill_gap=gap, min_length=minlen, max_segments=64)
    for p, (ref_segs, ref_support) in enumerate(_brute(e, w, h, nt, pk, gap, minlen, 64)):
        assert support[p] == ref_support
        assert counts[p] == len(ref_segs)
        assert [tuple(int(v) for v in segs[p, i, :4]) for i in range(counts[p])] == ref_segs


def test_segment_ends_support_their_peak(ora):
    img = synth.road_frame(5, 640, 480, synth.LATENCY_640x480)
    e = ora.edge_list(ora.binarize(ora.sobel_mag(img, border=1)))
    acc = ora.hough(e, 640, 480, 180)
    pk = ora.peaks(acc, 4)
    segs, counts, _ = ora.hough_lines(e, 640, 480, 180, pk, fill_gap=20, min_length=40)
    c, s = ora.trig_q16(180)
    D = ora.rho_max(640, 480)
    ok = set(int(v) for v in e)
    assert counts.sum() > 0
    for p in range(len(pk)):
        k, r = pk[p, 0], pk[p, 1]
        for i in range(min(counts[p], 16)):
            for x, y in ((segs[p, i, 0], segs[p, i, 1]), (segs[p, i, 2], segs[p, i, 3])):
                assert (int(y) << 16) | int(x) in ok
                assert (int(x) * int(c[k]) + int(y) * int(s[k]) + 32768) // 65536 == r - D
