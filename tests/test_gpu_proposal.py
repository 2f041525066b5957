"""The proposal path (ld_detect_batch_proposal) is exact where it votes.

With forced band probabilities (head weights 0, biases +-20), the kept theta
pairs are known; the peaks must equal the oracle's greedy over the full
accumulator with every other theta row removed.  With the fallback forced,
the path must equal the plain ld_detect_batch.  With the trained network,
frames of one batch keep different bands (and some fall back), so the device
plan gives them different tile counts; every frame whose band decision the
oracle's own network forward fixes must still equal the masked oracle.  Also:
the training targets kernel against the oracle's definition."""
import os

import numpy as np
import pytest
import torch

import oracle.cnn as cnn
from paper_2212_09460_gb300 import synth

pytestmark = pytest.mark.gpu

W, H, NT = 1920, 1080, 360
WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(__file__)), "paper_2212_09460_gb300", "weights",
                       "proposal_1080p.npz")


def _frames(seeds):
    raw = [synth.road_frame(s, W, H, synth.THROUGHPUT_1080P) for s in seeds]
    return raw, [torch.from_numpy(r).cuda() for r in raw]


def _forced_net(bands):
    from paper_2212_09460_gb300.proposal import ProposalNet, init_numpy
    p = init_numpy(0)
    p["wh"][:] = 0.0
    p["bh"][:] = -20.0
    p["bh"][list(bands)] = 20.0
    return ProposalNet(p, 0)


def _voted_rows(bands, margin, n_theta=NT):
    bpb = n_theta // 36
    on = np.zeros(n_theta, bool)
    for b in bands:
        on[max(0, b * bpb - margin): min(n_theta, (b + 1) * bpb + margin)] = True
    pairs = [j for j in range(n_theta // 2) if (on[0] or on[n_theta // 2]) if j == 0] + \
            [j for j in range(1, n_theta // 2) if on[j] or on[n_theta - j]]
    rows = np.zeros(n_theta, bool)
    for j in pairs:
        rows[j] = True
        rows[n_theta // 2 if j == 0 else n_theta - j] = True
    return rows, len(pairs)


# min_votes 1: the interleaved-column kernel votes the kept pairs; min_votes 0:
# the packed-pair kernel (the frames have far more than top_k voted cells, so
# the peaks are the same either way)
@pytest.mark.parametrize("bands,margin,mv", [([27, 10], 2, 1), ([0, 18, 35], 0, 1), ([5], 4, 1), ([27, 10], 2, 0),
                                             ([0, 18, 35], 0, 0)])
def test_restricted_vote_matches_masked_oracle(ctx, ldlib, ora, bands, margin, mv):
    raw, dev = _frames([4000, 4001, 4002])
    p = ldlib.params(n_theta=NT, top_k=4, border=1, min_votes=mv)
    net = _forced_net(bands)
    q = ldlib.proposal_params(0.5, 0.9, margin)
    pk, npk, st, fb, act = (t.cpu().numpy() for t in ctx.detect_batch_proposal(dev, p, net, q))
    rows, n_pairs = _voted_rows(bands, margin)
    for i, r in enumerate(raw):
        e = ora.edge_list(ora.binarize(ora.sobel_mag(r, border=1), 128))
        acc = ora.hough(e, W, H, NT)
        acc[~rows] = 0
        ref = ora.peaks(acc, 4, min_votes=mv)
        assert st[i] == 0 and fb[i] == 0 and act[i] == n_pairs
        assert npk[i] == len(ref)
        np.testing.assert_array_equal(pk[i, : npk[i]], ref)


def test_fallback_equals_plain_path(ctx, ldlib, ora):
    raw, dev = _frames([4100, 4101])
    p = ldlib.params(n_theta=NT, top_k=4, border=1)
    net = _forced_net([])                      # every band at sigmoid(-20): falls back
    pk, npk, st, fb, act = (t.cpu().numpy() for t in ctx.detect_batch_proposal(dev, p, net))
    plain = ctx.detect_batch(dev, p)
    torch.cuda.synchronize()
    ppk, pn, pst = (t.cpu().numpy() for t in plain)
    assert (fb == 1).all() and (act == NT // 2).all() and (st == 0).all()
    np.testing.assert_array_equal(npk, pn)
    np.testing.assert_array_equal(pk, ppk)
    ref = ora.detect(raw[0], NT, 4, border=1)
    np.testing.assert_array_equal(pk[0, : npk[0]], ref)


def _oracle_rows(ora, params, raw, p_band, p_fallback, margin, tol=0.25):
    """The oracle's band decision for one frame (its float64 network on the
    same bf16-rounded weights): (rows, n_pairs, fell_back), or None when a band
    logit lies within tol of a threshold's logit, where the GPU's bf16
    network could decide the other way."""
    x = cnn.count_pool8(ora.binarize(ora.sobel_mag(raw, border=1), 128))
    z = cnn.forward(params, x[None].astype(np.float64) / 64.0)[0, :36]
    lb, lf = np.log(p_band / (1 - p_band)), np.log(p_fallback / (1 - p_fallback))
    if np.min(np.abs(z - lb)) < tol or abs(z.max() - lf) < tol:
        return None
    if z.max() < lf or z.max() < lb:
        return np.ones(NT, bool), NT // 2, 1
    rows, n_pairs = _voted_rows(np.nonzero(z >= lb)[0], margin)
    return rows, n_pairs, 0


@pytest.mark.parametrize("n,p_fallback", [(64, 0.5), (64, 0.99), (5, 0.99), (128, 0.9)])
def test_planned_units_exact_with_trained_network(ctx, ldlib, ora, n, p_fallback):
    from paper_2212_09460_gb300.proposal import ProposalNet
    z = np.load(WEIGHTS)
    params = {k: z[k].astype(np.float64) for k in z.files if not k.startswith("adam_") and k != "step"}
    for i in range(4):
        params[f"w{i}"] = torch.tensor(params[f"w{i}"], dtype=torch.float32).to(torch.bfloat16).double().numpy()
    net = ProposalNet.load(WEIGHTS, 0)
    seeds = 4300 + 1000 * n + np.arange(n)
    raw = [synth.road_frame(int(s), W, H, synth.THROUGHPUT_1080P) for s in seeds]
    dev = [torch.from_numpy(r).cuda() for r in raw]
    p = ldlib.params(n_theta=NT, top_k=4, border=1)
    q = ldlib.proposal_params(0.2, p_fallback, 2)
    pk, npk, st, fb, act = (t.cpu().numpy() for t in ctx.detect_batch_proposal(dev, p, net, q))
    assert (st == 0).all()
    assert (act >= 1).all() and (act <= NT // 2).all() and ((fb == 0) | (act == NT // 2)).all()
    checked = 0
    for i in sorted({0, 1, n // 2, n - 2, n - 1}):
        dec = _oracle_rows(ora, params, raw[i], 0.2, p_fallback, 2)
        if dec is None:
            continue
        rows, n_pairs, fell_back = dec
        assert fb[i] == fell_back and act[i] == n_pairs, i
        e = ora.edge_list(ora.binarize(ora.sobel_mag(raw[i], border=1), 128))
        acc = ora.hough(e, W, H, NT)
        acc[~rows] = 0
        ref = ora.peaks(acc, 4)
        assert npk[i] == len(ref), i
        np.testing.assert_array_equal(pk[i, : npk[i]], ref)
        checked += 1
    assert checked >= 2


@pytest.mark.parametrize("always_k,rel", [(4, 0.0), (4, 0.4), (0, 0.6), (16, 1.0)])
def test_targets_kernel_matches_oracle(ctx, ldlib, always_k, rel):
    raw, dev = _frames([4200, 4201, 4202, 4203])
    p = ldlib.params(n_theta=NT, top_k=16, border=1)
    pk, npk, st = ctx.detect_batch(dev, p)
    tgt = torch.empty((4, 44), dtype=torch.float32, device="cuda")
    ldlib.ld_proposal_targets(pk.data_ptr(), npk.data_ptr(), 4, 16, W, H, NT, always_k, rel, tgt.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    pkc, nc, tg = pk.cpu().numpy(), npk.cpu().numpy(), tgt.cpu().numpy()
    for i in range(4):
        peaks = pkc[i, : nc[i]]
        keep = [k for k in range(len(peaks)) if k < always_k or peaks[k, 2] >= np.float32(rel) * np.float32(peaks[0, 2])]
        sel = peaks[keep]
        np.testing.assert_array_equal(tg[i, :36], cnn.theta_band_targets(sel, NT))
        np.testing.assert_array_equal(tg[i, 36:], cnn.row_band_targets(sel, W, H, NT))
