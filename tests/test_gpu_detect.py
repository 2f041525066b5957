"""End-to-end parity of ld_detect_batch (Steps 1-4, fused candidate path)
with the oracle: single frames, mixed-resolution batches, and sampled frames
of the 64 x 1920x1080 batch in the launch configuration the benchmark times."""
import numpy as np
import pytest
import torch

from paper_2212_09460_gb300 import synth

pytestmark = pytest.mark.gpu


def _detect(ctx, ld, frames, widths, **kw):
    p = ld.params(**kw)
    dev = [torch.from_numpy(np.ascontiguousarray(f)).cuda() for f in frames]
    pk, n, st = ctx.detect_batch(dev, p, widths=widths)
    torch.cuda.synchronize()
    return pk.cpu().numpy(), n.cpu().numpy(), st.cpu().numpy()


def _check(ora, frames_raw, pk, n, st, **kw):
    for i, img in enumerate(frames_raw):
        ref = ora.detect(img, kw.get("n_theta", 180), kw.get("top_k", 4), threshold=kw.get("threshold", 128),
                         border=kw.get("border", 0), nms_theta=kw.get("nms_theta", 5),
                         nms_rho=kw.get("nms_rho", 5), min_votes=kw.get("min_votes", 1))
        assert st[i] == 0
        assert n[i] == len(ref), (i, n[i], ref)
        np.testing.assert_array_equal(pk[i, : n[i]], ref, err_msg=f"frame {i}")


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_detect_latency_frame(ctx, ldlib, ora, seed):
    img = synth.road_frame(seed, 640, 480, synth.LATENCY_640x480)
    kw = dict(n_theta=180, top_k=2)
    pk, n, st = _detect(ctx, ldlib, [img], [640], **kw)
    _check(ora, [img], pk, n, st, **kw)


def test_detect_mixed_batch(ctx, ldlib, ora):
    sizes = [(640, 480), (97, 61), (1280, 720), (3, 3), (513, 300), (200, 900), (1920, 1080), (33, 17)]
    raw = [synth.road_frame(100 + i, w, h, synth.THROUGHPUT_1080P) for i, (w, h) in enumerate(sizes)]
    frames = [synth.pitched(r, seed=i) for i, r in enumerate(raw)]
    for kw in (dict(n_theta=360, top_k=4), dict(n_theta=180, top_k=16, border=1, nms_theta=3, nms_rho=9)):
        pk, n, st = _detect(ctx, ldlib, frames, [w for w, h in sizes], **kw)
        _check(ora, raw, pk, n, st, **kw)


def test_detect_blank_frames(ctx, ldlib, ora):
    raw = [np.zeros((40, 64), np.uint8), np.full((40, 64), 200, np.uint8)]
    kw = dict(n_theta=180, top_k=4)
    pk, n, st = _detect(ctx, ldlib, raw, [64, 64], **kw)
    _check(ora, raw, pk, n, st, **kw)
    assert n[0] == 0


def test_detect_more_frames_than_one_launch(ctx, ldlib, ora):
    # 130 frames: more descriptors than one launch carries
    raw = [synth.road_frame(300 + i, 48 + (i % 5) * 16, 32 + (i % 3), synth.THROUGHPUT_1080P) for i in range(130)]
    kw = dict(n_theta=90, top_k=3)
    pk, n, st = _detect(ctx, ldlib, raw, [r.shape[1] for r in raw], **kw)
    _check(ora, raw, pk, n, st, **kw)


def test_detect_full_size_batch_sampled(ctx, ldlib, ora):
    # the benchmark's workload: 64 seeded 1920x1080 dashed-lane frames, 360 theta,
    # top-4, in one call; the oracle checks a sample of the frames
    seeds = list(range(1000, 1064))
    raw = {s: synth.road_frame(s, 1920, 1080, synth.THROUGHPUT_1080P) for s in seeds}
    kw = dict(n_theta=360, top_k=4)
    pk, n, st = _detect(ctx, ldlib, [raw[s] for s in seeds], [1920] * 64, **kw)
    assert (st == 0).all() and (n == 4).all()
    for i in (0, 21, 42, 63):
        ref = ora.detect(raw[seeds[i]], 360, 4)
        np.testing.assert_array_equal(pk[i], ref, err_msg=f"frame {i}")


MIXED_SIZES = [(640, 480), (1280, 720), (1920, 1080), (3840, 2160)]


def test_detect_mixed_resolution_batch_sampled(ctx, ldlib, ora):
    # the batching workload's four resolutions, two frames each, in one call
    # (one persistent voting launch over all of them), 360 theta, top-4
    sizes = [s for s in MIXED_SIZES for _ in range(2)]
    raw = [synth.road_frame(2000 + i, w, h, synth.THROUGHPUT_1080P) for i, (w, h) in enumerate(sizes)]
    kw = dict(n_theta=360, top_k=4)
    pk, n, st = _detect(ctx, ldlib, raw, [w for w, h in sizes], **kw)
    for i in (0, 3, 4, 7):
        ref = ora.detect(raw[i], 360, 4)
        assert st[i] == 0 and n[i] == len(ref)
        np.testing.assert_array_equal(pk[i, : n[i]], ref, err_msg=f"frame {i} {sizes[i]}")


def test_autotune_keeps_results_and_sets_plans(ldlib, ora):
    # a fresh context: tuning changes tile sizes, never results
    c = ldlib.Context(0)
    try:
        sizes = [(640, 480), (640, 480), (1280, 720)]
        raw = [synth.road_frame(3000 + i, w, h, synth.THROUGHPUT_1080P) for i, (w, h) in enumerate(sizes)]
        p = ldlib.params(n_theta=360, top_k=4)
        dev = [torch.from_numpy(r).cuda() for r in raw]
        before = [c.plan(w, h, p) for w, h in sizes]
        c.autotune(dev, p, iters=2)
        after = [c.plan(w, h, p) for w, h in sizes]
        for pairs, rows in after:
            assert 1 <= abs(pairs) <= 30 and rows in (1, 2, 4)
        pk, n, st = c.detect_batch(dev, p)
        torch.cuda.synchronize()
        pk, n, st = pk.cpu().numpy(), n.cpu().numpy(), st.cpu().numpy()
        for i, r in enumerate(raw):
            ref = ora.detect(r, 360, 4)
            assert st[i] == 0 and n[i] == len(ref)
            np.testing.assert_array_equal(pk[i, : n[i]], ref)
        assert len(before) == len(after)
    finally:
        c.close()


# Both voting kernels against the oracle.  The interleaved-column kernel votes
# when min_votes >= 1 and the frame fits (plan pairs < 0); min_votes <= 0
# takes the packed-pair kernel.  Cases: one full 16-pair tile (32 theta), a
# cut of M > 1024 candidates per tile (the radix select instead of the
# survivor sort), a checkerboard frame whose accumulator is full of equal
# counts (the ordered emission of ties), 1440p (the largest common size that
# fits the interleaved accumulator), and min_votes 0 and 2.
KERNEL_CASES = [
    dict(n_theta=32, top_k=16, min_votes=3),
    dict(n_theta=180, top_k=16, nms_theta=63, nms_rho=3),
    dict(n_theta=360, top_k=8, nms_theta=1, nms_rho=1, min_votes=0),
    dict(n_theta=360, top_k=16, nms_theta=1, nms_rho=1, min_votes=2),
]


def _checker(w, h, cell):
    yy, xx = np.mgrid[0:h, 0:w]
    return ((((xx // cell) + (yy // cell)) & 1) * 255).astype(np.uint8)


@pytest.mark.parametrize("kw", KERNEL_CASES)
def test_detect_voting_kernels(ctx, ldlib, ora, kw):
    sizes = [(640, 480), (2560, 1440), (37, 23)]
    raw = [synth.road_frame(5000 + i, w, h, synth.THROUGHPUT_1080P) for i, (w, h) in enumerate(sizes)]
    raw.append(_checker(1280, 720, 7))
    sizes.append((1280, 720))
    p = ldlib.params(**kw)
    for w, h in sizes:
        pairs, _ = ctx.plan(w, h, p)
        assert (pairs < 0) == (kw.get("min_votes", 1) >= 1), (w, h, pairs)
    frames = [synth.pitched(r, seed=i) for i, r in enumerate(raw)]
    pk, n, st = _detect(ctx, ldlib, frames, [w for w, h in sizes], **kw)
    _check(ora, raw, pk, n, st, **kw)


def test_benchmark_config_uses_interleaved_kernel(ctx, ldlib):
    p = ldlib.params(n_theta=360, top_k=4)
    pairs, rows = ctx.plan(1920, 1080, p)
    assert pairs == -15 and rows in (1, 2, 4)
    pairs4k, _ = ctx.plan(3840, 2160, p)
    assert pairs4k == -8   # 4K windows take 8-slot interleaved tiles (16 x 4407 rows do not fit)


# Split tiles: when a launch's last wave would be at most half full, the tiles
# of its last frames are voted in edge-range pieces that meet in a partial
# accumulator.  13 x 1080p at 360 theta: 156 tiles on 152 SMs, the last frame
# split 8 ways; 60 x 640x480 at 90 theta: 180 tiles, the last 10 frames split
# 5 ways (pieces of a frame with only a few edge chunks get none).  Small
# batches of large frames split every tile to fill the GPU: 1 x 1080p (12
# tiles, 8 pieces each), 3 x 720p (36 tiles, 4 each).  Every frame against
# the oracle.
@pytest.mark.parametrize("n,w,h,n_theta", [(13, 1920, 1080, 360), (60, 640, 480, 90), (1, 1920, 1080, 360),
                                           (3, 1280, 720, 360)])
def test_detect_split_tiles(ctx, ldlib, ora, n, w, h, n_theta):
    raw = [synth.road_frame(6000 + i, w, h, synth.THROUGHPUT_1080P) for i in range(n)]
    kw = dict(n_theta=n_theta, top_k=4)
    pk, cnt, st = _detect(ctx, ldlib, raw, [w] * n, **kw)
    _check(ora, raw, pk, cnt, st, **kw)


def test_shared_memory_reduction_probe(ldlib):
    # the measurement probe of the voting ceiling: every reduction lands (sums exact)
    sink = torch.zeros(8, dtype=torch.int32, device="cuda")
    for pattern in (0, 1):
        ldlib.ld_probe_smem_red(8, 64, pattern, sink.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert (sink.cpu().numpy() == 1024 * 64).all()
    with pytest.raises(ldlib.LdError):
        ldlib.ld_probe_smem_red(8, 12, 0, sink.data_ptr(), 0)   # iters not a multiple of 8


def test_detect_split_tiles_mixed_sizes(ctx, ldlib, ora):
    # 12 x 1080p + 1 x 720p at 360 theta: 156 tiles; the 720p frame is last in
    # queue order (fewest pixels), so its tiles are the ones split, and its
    # partial accumulators are smaller than the launch's stride (sized for
    # 1080p rows).  Every frame against the oracle.
    sizes = [(1920, 1080)] * 12 + [(1280, 720)]
    raw = [synth.road_frame(6500 + i, w, h, synth.THROUGHPUT_1080P) for i, (w, h) in enumerate(sizes)]
    kw = dict(n_theta=360, top_k=4)
    pk, cnt, st = _detect(ctx, ldlib, raw, [w for w, h in sizes], **kw)
    _check(ora, raw, pk, cnt, st, **kw)


@pytest.mark.parametrize("n_theta,top_k,nms_theta,nms_rho", [(4096, 16, 7, 3), (1000, 8, 5, 5)])
def test_detect_many_theta_bins(ctx, ldlib, ora, n_theta, top_k, nms_theta, nms_rho):
    # the interleaved-column kernel with many tiles a frame (4096 theta: 128
    # tiles of 16 pairs; 1000 theta: 500 pairs in tiles of 16 and 15)
    sizes = [(97, 61), (640, 480)]
    raw = [synth.road_frame(6800 + i, w, h, synth.THROUGHPUT_1080P) for i, (w, h) in enumerate(sizes)]
    kw = dict(n_theta=n_theta, top_k=top_k, nms_theta=nms_theta, nms_rho=nms_rho)
    p = ldlib.params(**kw)
    for w, h in sizes:
        assert ctx.plan(w, h, p)[0] < 0
    frames = [synth.pitched(r, seed=i) for i, r in enumerate(raw)]
    pk, cnt, st = _detect(ctx, ldlib, frames, [w for w, h in sizes], **kw)
    _check(ora, raw, pk, cnt, st, **kw)


def test_detect_two_voting_launches(ctx, ldlib, ora):
    # 14 x 1080p + 5 x 4K at 360 theta: the 1080p frames' 168 interleaved tiles
    # and the 4K frames' 180 packed-pair tiles each fill the GPU, so the group
    # votes in two launches (one per kernel).  Every frame against the oracle.
    sizes = [(1920, 1080)] * 14 + [(3840, 2160)] * 5
    raw = [synth.road_frame(6900 + i, w, h, synth.THROUGHPUT_1080P) for i, (w, h) in enumerate(sizes)]
    kw = dict(n_theta=360, top_k=4)
    pk, cnt, st = _detect(ctx, ldlib, raw, [w for w, h in sizes], **kw)
    _check(ora, raw, pk, cnt, st, **kw)


def test_detect_noise_frames_nearly_all_edges(ctx, ldlib, ora):
    # uniform noise: ~93% of the pixels are edges (edge lists near w*h, cells
    # with ~2000 votes, hundreds of streamed chunks per tile); a lone 1080p
    # frame (tiles split over the GPU) and a 640x480 one in one call
    rng = np.random.default_rng(77)
    raw = [rng.integers(0, 256, size=(1080, 1920), dtype=np.uint8),
           rng.integers(0, 256, size=(480, 640), dtype=np.uint8)]
    for frames in ([raw[0]], raw):
        kw = dict(n_theta=360, top_k=4)
        pk, cnt, st = _detect(ctx, ldlib, frames, [f.shape[1] for f in frames], **kw)
        _check(ora, frames, pk, cnt, st, **kw)


def _dots(w, h, pts):
    img = np.zeros((h, w), np.uint8)
    for x, y in pts:
        img[y, x] = 255
    return img


def _tile_totals(acc, n_theta, width, min_votes):
    """Cells >= min_votes in each tile of `width` theta pairs (pairs split
    evenly over the tiles; pair j holds theta j and n - j, pair 0 holds 0 and
    n/2), the counts a tile's top-M selection sees."""
    n_pairs = n_theta // 2
    n_tiles = -(-n_pairs // width)
    base, extra = divmod(n_pairs, n_tiles)
    per_theta = (acc >= min_votes).sum(axis=1)
    out = []
    for t in range(n_tiles):
        j0 = t * base + min(t, extra)
        js = range(j0, j0 + base + (1 if t < extra else 0))
        out.append(int(sum(per_theta[j] + per_theta[n_theta // 2 if j == 0 else n_theta - j] for j in js)))
    return out


@pytest.mark.parametrize("min_votes", [1, 2])
def test_detect_tiles_near_candidate_count(ctx, ldlib, ora, min_votes):
    # A few isolated bright pixels (a ring of 8 edge pixels each) leave 45 to
    # 300 voted cells per tile.  Sweeping top_k and the suppression window moves
    # M = nms_theta * nms_rho * (top_k - 1) + 1 across those counts, so tiles
    # hold fewer cells >= min_votes than M, exactly M, and more: the tile
    # selection's threshold path and its general path both run, and both
    # must give the oracle's peaks.
    raw = [_dots(48, 40, [(20, 18)]), _dots(64, 33, [(10, 10), (40, 20), (43, 23)])]
    n_theta = 32
    totals = set()
    for r in raw:
        acc = ora.hough(ora.edge_list(ora.binarize(ora.sobel_mag(r), 128)), r.shape[1], r.shape[0], n_theta)
        for width in (8, 16):
            totals.update(_tile_totals(acc, n_theta, width, min_votes))
    swept = set()
    for nms_theta in (1, 3):
        for nms_rho in (1, 3, 5, 7):
            for top_k in range(1, 17):
                kw = dict(n_theta=n_theta, top_k=top_k, nms_theta=nms_theta, nms_rho=nms_rho, min_votes=min_votes)
                swept.add(nms_theta * nms_rho * (top_k - 1) + 1)
                pk, n, st = _detect(ctx, ldlib, raw, [r.shape[1] for r in raw], **kw)
                _check(ora, raw, pk, n, st, **kw)
    assert totals & swept, (sorted(totals), sorted(swept))
