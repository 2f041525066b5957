"""Canny on the GPU (ld_canny, ld_detect_canny_batch) against the oracle
(oracle.canny): the 0/255 map byte for byte, the edge set exactly (the list's
order is unspecified), and the Hough peaks of the Canny edges."""
import numpy as np
import pytest
import torch

from paper_2212_09460_gb300 import synth

pytestmark = pytest.mark.gpu


def _gpu_canny(ctx, ld, raw, tl, th, border=0, cap=0, seed=0):
    h, w = raw.shape
    img = torch.from_numpy(synth.pitched(raw, seed=seed)).cuda()
    p = ld.params(border=border, edge_capacity=cap)
    out = ctx.canny(img, p, ld.canny_params(tl, th), want_binary=True, width=w)
    torch.cuda.synchronize()
    n = int(out.count.item())
    edges = out.edges.cpu().numpy().view(np.uint32)[: min(n, cap if cap else w * h)]
    return out.binary.cpu().numpy()[:, :w], n, edges


def _ref(ora, raw, tl, th, border):
    b = ora.canny(raw, tl, th)
    if border:
        b[0, :] = 0
        b[-1, :] = 0
        b[:, 0] = 0
        b[:, -1] = 0
    return b


CASES = [
    (0, 640, 480, 100, 200, 0), (1, 640, 480, 40, 80, 1), (1000, 1920, 1080, 100, 200, 0),
    (7, 333, 201, 60, 150, 0), (9, 37, 29, 20, 40, 0), (11, 3, 3, 1, 1, 0), (13, 1280, 720, 150, 300, 1),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[1]}x{c[2]}_{c[3]}_{c[4]}_b{c[5]}")
def test_canny_matches_oracle(ctx, ldlib, ora, case):
    seed, w, h, tl, th, border = case
    style = synth.LATENCY_640x480 if w == 640 else synth.THROUGHPUT_1080P
    raw = synth.road_frame(seed, w, h, style)
    ref = _ref(ora, raw, tl, th, border)
    got, n, edges = _gpu_canny(ctx, ldlib, raw, tl, th, border, seed=seed)
    np.testing.assert_array_equal(got, ref)
    ref_edges = np.sort(ora.edge_list(ref))
    assert n == len(ref_edges)
    np.testing.assert_array_equal(np.sort(edges), ref_edges)


def test_canny_long_weak_chains(ctx, ldlib, ora):
    # a long winding ridge of weak edges touched by one strong point at its far
    # end: hysteresis must follow it across the whole frame (many tiles), and
    # an identical ridge without a strong point must vanish
    h, w = 300, 500
    img = np.full((h, w), 60, np.uint8)
    for x in range(10, 490):
        y = int(150 + 100 * np.sin(x / 37.0))
        img[y:y + 6, x] = 110        # weak contrast
        img[(y + 60) % h:(y + 60) % h + 6, x] = 110
    img[140:170, 480:492] = 250       # a strong blob touching the first ridge's end
    for tl, th in ((60, 400), (100, 300)):
        ref = ora.canny(img, tl, th)
        got, n, edges = _gpu_canny(ctx, ldlib, img, tl, th)
        np.testing.assert_array_equal(got, ref)
        assert n == int((ref == 255).sum())


def test_canny_capacity_overflow(ctx, ldlib, ora):
    raw = synth.road_frame(2, 640, 480, synth.LATENCY_640x480)
    ref = ora.canny(raw, 40, 80)
    total = int((ref == 255).sum())
    got, n, edges = _gpu_canny(ctx, ldlib, raw, 40, 80, cap=100)
    assert n == total and len(edges) == 100
    assert set(edges.tolist()) <= set(ora.edge_list(ref).tolist())


def test_detect_canny_batch_matches_oracle(ctx, ldlib, ora):
    sizes = [(640, 480), (1920, 1080), (97, 61), (1280, 720)]
    raw = [synth.road_frame(2200 + i, w, h, synth.THROUGHPUT_1080P) for i, (w, h) in enumerate(sizes)]
    p = ldlib.params(n_theta=360, top_k=4)
    cp = ldlib.canny_params(100, 200)
    dev = [torch.from_numpy(synth.pitched(r, seed=i)).cuda() for i, r in enumerate(raw)]
    pk, npk, st = ctx.detect_canny_batch(dev, p, cp, widths=[w for w, h in sizes])
    torch.cuda.synchronize()
    pk, npk, st = pk.cpu().numpy(), npk.cpu().numpy(), st.cpu().numpy()
    assert (st == 0).all()
    for i, (r, (w, h)) in enumerate(zip(raw, sizes)):
        e = ora.edge_list(ora.canny(r, 100, 200))
        ref = ora.peaks(ora.hough(e, w, h, 360), 4)
        assert npk[i] == len(ref)
        np.testing.assert_array_equal(pk[i, : npk[i]], ref)
