"""Steps 1-3 without an edge list (ld_sobel_hough_fused, ld_detect_fused_batch)
against the oracle: the accumulator cell for cell, and the peaks."""
import numpy as np
import pytest
import torch

from paper_2212_09460_gb300 import synth

pytestmark = pytest.mark.gpu

CASES = [
    (0, 640, 480, 180, 128, 0), (1000, 1920, 1080, 360, 128, 0), (7, 333, 201, 90, 128, 1),
    (3, 37, 29, 2, 60, 0), (5, 3, 3, 8, 1, 0), (9, 1280, 720, 1024, 200, 1), (11, 1000, 33, 360, 100, 0),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[1]}x{c[2]}_t{c[3]}_T{c[4]}_b{c[5]}")
def test_fused_accumulator_matches_oracle(ctx, ldlib, ora, case):
    seed, w, h, nt, thr, border = case
    style = synth.LATENCY_640x480 if w == 640 else synth.THROUGHPUT_1080P
    raw = synth.road_frame(seed, w, h, style)
    p = ldlib.params(n_theta=nt, threshold=thr, border=border)
    acc = ctx.sobel_hough_fused(torch.from_numpy(synth.pitched(raw, seed=seed)).cuda(), p, width=w)
    torch.cuda.synchronize()
    ref = ora.hough(ora.edge_list(ora.binarize(ora.sobel_mag(raw, border=border), thr)), w, h, nt)
    np.testing.assert_array_equal(acc.cpu().numpy(), ref)


def test_fused_detect_batch_matches_oracle(ctx, ldlib, ora):
    sizes = [(640, 480), (1920, 1080), (97, 61), (1280, 720), (3840, 2160), (200, 900)]
    raw = [synth.road_frame(2300 + i, w, h, synth.THROUGHPUT_1080P) for i, (w, h) in enumerate(sizes)]
    for kw in (dict(n_theta=360, top_k=4), dict(n_theta=180, top_k=16, border=1, nms_theta=3, nms_rho=9)):
        p = ldlib.params(**kw)
        dev = [torch.from_numpy(synth.pitched(r, seed=i)).cuda() for i, r in enumerate(raw)]
        pk, npk, st = ctx.detect_fused_batch(dev, p, widths=[w for w, h in sizes])
        torch.cuda.synchronize()
        pk, npk, st = pk.cpu().numpy(), npk.cpu().numpy(), st.cpu().numpy()
        assert (st == 0).all()
        for i, r in enumerate(raw):
            ref = ora.detect(r, kw["n_theta"], kw["top_k"], border=kw.get("border", 0),
                             nms_theta=kw.get("nms_theta", 5), nms_rho=kw.get("nms_rho", 5))
            assert npk[i] == len(ref)
            np.testing.assert_array_equal(pk[i, : npk[i]], ref)


def test_fused_rejects_too_many_thetas(ctx, ldlib):
    img = torch.zeros((32, 32), dtype=torch.uint8, device="cuda")
    with pytest.raises(ldlib.LdError) as ei:
        ctx.sobel_hough_fused(img, ldlib.params(n_theta=2048))
    assert ei.value.status == ldlib.LD_ERR_INVALID
