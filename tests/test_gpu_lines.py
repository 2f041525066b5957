"""Hough lines on the GPU (ld_hough_lines, ld_detect_lines_batch) against the
oracle (oracle.hough_lines), bit for bit: segments, per-peak segment counts
and supporting-pixel counts, which must also equal the peaks' votes."""
import numpy as np
import pytest
import torch

from paper_2212_09460_gb300 import synth

pytestmark = pytest.mark.gpu


def _dev_u32(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()


def _gpu_lines(ctx, ld, edges, w, h, nt, peaks, top_k, lp):
    e = _dev_u32(edges if edges.size else np.zeros(4, np.uint32))
    cnt = torch.tensor([edges.size], dtype=torch.int32, device="cuda")
    pk = torch.zeros((top_k, 3), dtype=torch.int32, device="cuda")
    pk[: len(peaks)] = torch.from_numpy(np.asarray(peaks, np.int32).reshape(-1, 3)).cuda()
    npk = torch.tensor([len(peaks)], dtype=torch.int32, device="cuda")
    p = ld.params(n_theta=nt, top_k=top_k)
    segs, nseg, sup = ctx.hough_lines(e, cnt, w, h, p, pk, npk, lp)
    torch.cuda.synchronize()
    return segs.cpu().numpy(), nseg.cpu().numpy(), sup.cpu().numpy()


def _compare(ora_out, gpu_out, n_peaks, max_segments):
    osegs, ocnt, osup = ora_out
    gsegs, gcnt, gsup = gpu_out
    np.testing.assert_array_equal(gsup[:n_peaks], osup)
    np.testing.assert_array_equal(gcnt[:n_peaks], ocnt)
    assert (gcnt[n_peaks:] == 0).all()
    for j in range(n_peaks):
        m = min(int(ocnt[j]), max_segments)
        np.testing.assert_array_equal(gsegs[j, :m], osegs[j, :m], err_msg=f"peak {j}")


CASES = [
    ("latency", 0, 640, 480, 180, 6, dict(fill_gap=20, min_length=40, max_segments=16)),
    ("latency_tight", 1, 640, 480, 180, 4, dict(fill_gap=0, min_length=0, max_segments=64)),
    ("hd", 1002, 1920, 1080, 360, 4, dict(fill_gap=20, min_length=40, max_segments=16)),
    ("hd_trunc", 1003, 1920, 1080, 360, 8, dict(fill_gap=3, min_length=2, max_segments=3)),
    ("ragged", 7, 333, 201, 90, 5, dict(fill_gap=10, min_length=5, max_segments=32)),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_hough_lines_matches_oracle(ctx, ldlib, ora, case):
    _, seed, w, h, nt, top_k, lk = case
    style = synth.LATENCY_640x480 if w == 640 else synth.THROUGHPUT_1080P
    img = synth.road_frame(seed, w, h, style)
    e = ora.edge_list(ora.binarize(ora.sobel_mag(img)))
    acc = ora.hough(e, w, h, nt)
    peaks = ora.peaks(acc, top_k)
    lp = ldlib.lines_params(**lk)
    ref = ora.hough_lines(e, w, h, nt, peaks, **lk)
    got = _gpu_lines(ctx, ldlib, e, w, h, nt, peaks, top_k, lp)
    _compare(ref, got, len(peaks), lk["max_segments"])
    np.testing.assert_array_equal(got[2][: len(peaks)], peaks[:, 2])   # support = votes


def test_hough_lines_edge_cases(ctx, ldlib, ora):
    w, h, nt = 64, 48, 180
    img = np.zeros((h, w), np.uint8)
    img[10, 2:60] = 255
    img[5:40, 30] = 255
    e = ora.edge_list(img)
    D = ora.rho_max(w, h)
    lp = ldlib.lines_params(fill_gap=2, min_length=3, max_segments=4)
    # fewer peaks than slots, a cell with no support, and the two lines
    peaks = np.array([[90, 10 + D, 58], [0, 30 + D, 35], [45, 3, 0]], np.int32)
    ref = ora.hough_lines(e, w, h, nt, peaks, fill_gap=2, min_length=3, max_segments=4)
    got = _gpu_lines(ctx, ldlib, e, w, h, nt, peaks, 6, lp)
    _compare(ref, got, 3, 4)
    # an empty edge list
    got = _gpu_lines(ctx, ldlib, np.zeros(0, np.uint32), w, h, nt, peaks, 6, lp)
    assert (got[1] == 0).all() and (got[2] == 0).all()


def test_hough_lines_rejects_large_frames(ctx, ldlib):
    lp = ldlib.lines_params()
    p = ldlib.params(n_theta=180, top_k=2)
    z = torch.zeros(16, dtype=torch.int32, device="cuda")
    pk = torch.zeros((2, 3), dtype=torch.int32, device="cuda")
    with pytest.raises(ldlib.LdError) as ei:
        ldlib.ld_hough_lines(ctx.handle, z.data_ptr(), z.data_ptr(), 8200, 100, p, pk.data_ptr(), z.data_ptr(), lp,
                             z.data_ptr(), z.data_ptr(), None, torch.cuda.current_stream().cuda_stream)
    assert ei.value.status == ldlib.LD_ERR_INVALID


def test_detect_lines_batch(ctx, ldlib, ora):
    sizes = [(640, 480), (1920, 1080), (1280, 720), (97, 61), (1920, 1080)]
    raw = [synth.road_frame(2100 + i, w, h, synth.THROUGHPUT_1080P) for i, (w, h) in enumerate(sizes)]
    p = ldlib.params(n_theta=360, top_k=4, border=1)
    lp = ldlib.lines_params(fill_gap=15, min_length=30, max_segments=8)
    dev = [torch.from_numpy(synth.pitched(r, seed=i)).cuda() for i, r in enumerate(raw)]
    pk, npk, st, segs, nseg, sup = ctx.detect_lines_batch(dev, p, lp, widths=[w for w, h in sizes])
    torch.cuda.synchronize()
    pk, npk, st = pk.cpu().numpy(), npk.cpu().numpy(), st.cpu().numpy()
    segs, nseg, sup = segs.cpu().numpy(), nseg.cpu().numpy(), sup.cpu().numpy()
    assert (st == 0).all()
    for i, (r, (w, h)) in enumerate(zip(raw, sizes)):
        e = ora.edge_list(ora.binarize(ora.sobel_mag(r, border=1)))
        peaks = ora.detect(r, 360, 4, border=1)
        np.testing.assert_array_equal(pk[i, : npk[i]], peaks)
        ref = ora.hough_lines(e, w, h, 360, peaks, fill_gap=15, min_length=30, max_segments=8)
        _compare(ref, (segs[i], nseg[i], sup[i]), len(peaks), 8)


def test_detect_lines_headline_batch_support_equals_votes(ctx, ldlib, ora):
    # the 64-frame 1080p workload: support = votes for every peak of every
    # frame, and two frames' segments against the oracle
    seeds = list(range(1000, 1064))
    raw = [synth.road_frame(s, 1920, 1080, synth.THROUGHPUT_1080P) for s in seeds]
    p = ldlib.params(n_theta=360, top_k=4)
    lp = ldlib.lines_params()
    pk, npk, st, segs, nseg, sup = ctx.detect_lines_batch([torch.from_numpy(r).cuda() for r in raw], p, lp)
    torch.cuda.synchronize()
    pk, st, sup, segs, nseg = pk.cpu().numpy(), st.cpu().numpy(), sup.cpu().numpy(), segs.cpu().numpy(), \
        nseg.cpu().numpy()
    assert (st == 0).all()
    np.testing.assert_array_equal(sup, pk[:, :, 2])
    for i in (0, 63):
        e = ora.edge_list(ora.binarize(ora.sobel_mag(raw[i])))
        ref = ora.hough_lines(e, 1920, 1080, 360, pk[i], max_segments=16)
        _compare(ref, (segs[i], nseg[i], sup[i]), 4, 16)
