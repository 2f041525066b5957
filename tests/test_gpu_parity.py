"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer work, so every comparison is bit-exact: the 0/255 map byte for byte,
the edge list as a set (its order is unspecified), the accumulator cell for
cell, the peaks entry for entry.  Sizes span several Sobel warp strips (480
output pixels wide, runs of 8-row groups) with ragged right and bottom
edges, and several theta tiles with ragged tails.
"""
import numpy as np
import pytest
import torch

from paper_2212_09460_gb300 import synth

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _sorted_edges(e):
    return np.sort(np.asarray(e, dtype=np.uint32))


def _gpu_sobel(ctx, ld, img, w, threshold=128, border=0, cap=0):
    p = ld.params(threshold=threshold, border=border, edge_capacity=cap)
    out = ctx.sobel_binarize(_dev(img), p, want_binary=True, width=w)
    torch.cuda.synchronize()
    n = int(out.count.item())
    e = out.edges.cpu().numpy().view(np.uint32)[:min(n, out.edges.numel())]
    return out.binary.cpu().numpy()[:, :w], e, n


SOBEL_CASES = [
    (3, 3, 1), (17, 5, 2), (640, 480, 3), (513, 67, 4), (1000, 129, 5), (1920, 1080, 6), (31, 300, 7),
    (1024, 17, 8), (480, 9, 9), (481, 33, 10), (961, 40, 11), (959, 8, 12),
]


@pytest.mark.parametrize("w,h,seed", SOBEL_CASES)
@pytest.mark.parametrize("border", [0, 1])
def test_sobel_binarize_parity(ctx, ldlib, ora, w, h, seed, border):
    img = synth.road_frame(seed, w, h, synth.THROUGHPUT_1080P) if w * h > 5000 else synth.random_image(seed, w, h)
    buf = synth.pitched(img, seed=seed)            # garbage in the padding columns
    b, e, n = _gpu_sobel(ctx, ldlib, buf, w, border=border)
    ref_b = ora.binarize(ora.sobel_mag(img, border=border), 128)
    np.testing.assert_array_equal(b, ref_b)
    ref_e = ora.edge_list(ref_b)
    assert n == len(ref_e)
    np.testing.assert_array_equal(_sorted_edges(e), ref_e)   # oracle list is row-major = sorted


@pytest.mark.parametrize("thr", [1, 64, 128, 200, 255])
def test_sobel_thresholds(ctx, ldlib, ora, thr):
    img = synth.random_image(11, 300, 77)
    b, e, n = _gpu_sobel(ctx, ldlib, synth.pitched(img), 300, threshold=thr)
    ref_b = ora.binarize(ora.sobel_mag(img), thr)
    np.testing.assert_array_equal(b, ref_b)
    assert n == int((ref_b == 255).sum())


def test_sobel_capacity_overflow(ctx, ldlib, ora):
    img = synth.random_image(12, 200, 100)
    ref = ora.edge_list(ora.binarize(ora.sobel_mag(img), 128))
    cap = len(ref) // 3
    b, e, n = _gpu_sobel(ctx, ldlib, synth.pitched(img), 200, cap=cap)
    assert n == len(ref) and len(e) == cap
    assert np.isin(e, ref).all() and len(np.unique(e)) == cap


def test_sobel_blank_and_full_images(ctx, ldlib, ora):
    for v in (0, 31, 32, 255):
        img = np.full((50, 70), v, np.uint8)
        b, e, n = _gpu_sobel(ctx, ldlib, synth.pitched(img, fill=7), 70)
        ref_b = ora.binarize(ora.sobel_mag(img), 128)
        np.testing.assert_array_equal(b, ref_b)
        assert n == int((ref_b == 255).sum())


def _gpu_hough(ctx, ld, edges, w, h, n_theta):
    p = ld.params(n_theta=n_theta)
    e = torch.from_numpy(np.ascontiguousarray(edges, dtype=np.uint32).view(np.int32)).cuda() \
        if len(edges) else torch.zeros(4, dtype=torch.int32, device="cuda")
    cnt = torch.tensor([len(edges)], dtype=torch.int32, device="cuda")
    acc = ctx.hough_vote(e, cnt, w, h, p)
    torch.cuda.synchronize()
    return acc.cpu().numpy()


HOUGH_CASES = [
    (640, 480, 180, 0.03), (97, 61, 360, 0.2), (1920, 1080, 360, 0.075), (3, 3, 2, 1.0), (33, 20, 8, 0.5),
    (800, 3, 180, 0.6), (5, 700, 360, 0.6), (3840, 2160, 360, 0.002), (512, 512, 180, 0.9), (257, 129, 4096, 0.01),
]


@pytest.mark.parametrize("w,h,n_theta,dens", HOUGH_CASES)
def test_hough_vote_parity(ctx, ldlib, ora, w, h, n_theta, dens):
    b = synth.random_image(w + h + n_theta, w, h, density=dens)
    edges = ora.edge_list(b)
    rng = np.random.default_rng(w * h)
    perm = rng.permutation(len(edges))           # any order gives the same counts
    acc = _gpu_hough(ctx, ldlib, edges[perm], w, h, n_theta)
    ref = ora.hough(edges, w, h, n_theta)
    np.testing.assert_array_equal(acc, ref)


def test_hough_empty_edge_list(ctx, ldlib, ora):
    acc = _gpu_hough(ctx, ldlib, np.zeros(0, np.uint32), 64, 48, 180)
    assert acc.shape == (180, 2 * ora.rho_max(64, 48) + 1) and (acc == 0).all()


@pytest.mark.parametrize("w,h,n_theta", [(700, 300, 360), (24000, 3, 180)])
def test_hough_full_image_16bit_counts(ctx, ldlib, ora, w, h, n_theta):
    # every pixel an edge: the fullest cells hold max(w, h) votes or more
    # (24000 at theta = 90 deg for the 24000 x 3 image), close to the 16-bit
    # bound the packed counters rely on
    edges = ora.edge_list(np.full((h, w), 255, np.uint8))
    acc = _gpu_hough(ctx, ldlib, edges, w, h, n_theta)
    ref = ora.hough(edges, w, h, n_theta)
    assert ref.max() >= max(w, h)
    np.testing.assert_array_equal(acc, ref)


def test_hough_skips_out_of_image_entries(ctx, ldlib, ora):
    w, h = 50, 40
    good = ora.edge_list(synth.random_image(3, w, h, density=0.3))
    bad = np.array([(h << 16) | 3, (5 << 16) | w, 0xFFFFFFFF], np.uint32)
    acc = _gpu_hough(ctx, ldlib, np.concatenate([good, bad]), w, h, 180)
    np.testing.assert_array_equal(acc, ora.hough(good, w, h, 180))


def _gpu_peaks(ctx, ld, acc, k, nt=5, nr=5, mv=1):
    p = ld.params(top_k=k, nms_theta=nt, nms_rho=nr, min_votes=mv)
    pk, n = ctx.hough_peaks(_dev(acc.astype(np.int32)), p)
    torch.cuda.synchronize()
    return pk.cpu().numpy()[: int(n.item())]


@pytest.mark.parametrize("seed", range(8))
def test_peaks_parity_random_with_ties(ctx, ldlib, ora, seed):
    rng = np.random.default_rng(seed)
    T, R = int(rng.integers(2, 400)), int(rng.integers(3, 3000))
    acc = rng.integers(0, 5, size=(T, R)).astype(np.int32)       # many ties and plateaus
    for k, nt, nr, mv in ((4, 5, 5, 1), (16, 3, 7, 2), (1, 1, 1, 1), (8, 5, 5, 4), (2, 9, 3, 0)):
        np.testing.assert_array_equal(_gpu_peaks(ctx, ldlib, acc, k, nt, nr, mv),
                                      ora.peaks(acc, k, nt, nr, mv))


def test_peaks_parity_signed_and_large(ctx, ldlib, ora):
    rng = np.random.default_rng(99)
    acc = rng.integers(-2**31, 2**31 - 1, size=(37, 1001), dtype=np.int64).astype(np.int32)
    acc[5, 7] = 2**31 - 1
    acc[30, 900] = 2**31 - 1
    for mv in (-2**31, 0, 1):
        np.testing.assert_array_equal(_gpu_peaks(ctx, ldlib, acc, 16, 5, 5, mv), ora.peaks(acc, 16, 5, 5, mv))


def test_peaks_plateau_across_chunks(ctx, ldlib, ora):
    # one flat plateau larger than a select chunk: ties decided by (theta, rho)
    acc = np.zeros((40, 3000), np.int32)
    acc[3:30, 100:2900] = 7
    np.testing.assert_array_equal(_gpu_peaks(ctx, ldlib, acc, 16), ora.peaks(acc, 16))


def test_peaks_none_above_min_votes(ctx, ldlib, ora):
    acc = np.zeros((10, 20), np.int32)
    assert len(_gpu_peaks(ctx, ldlib, acc, 4)) == 0
    assert len(ora.peaks(acc, 4)) == 0


def test_peaks_on_real_accumulator(ctx, ldlib, ora):
    img = synth.road_frame(5, 640, 480, synth.LATENCY_640x480)
    acc = ora.hough(ora.edge_list(ora.binarize(ora.sobel_mag(img))), 640, 480, 180)
    for k in (1, 2, 4, 16):
        np.testing.assert_array_equal(_gpu_peaks(ctx, ldlib, acc, k), ora.peaks(acc, k))
