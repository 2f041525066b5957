"""ld_detect_batch_host: Steps 1-4 with frames and results in host memory.

The call uploads the frames into one of two staging areas of the context on
a copy stream, detects on the caller's stream and copies the outputs back.
Checked against the oracle and against ld_detect_batch on device frames:
pinned and pageable frames, one [n][h][pitch] tensor (one upload) and a
list of separate tensors, padded pitches, several calls in flight at once
(alternating areas, the later ones larger so that an area grows), and
argument errors reported before anything runs.
"""
import numpy as np
import pytest
import torch

from paper_2212_09460_gb300 import synth

pytestmark = pytest.mark.gpu

SIZES = [(320, 240), (640, 480), (197, 101)]


def _frames(seed0, sizes):
    out = []
    for i, (w, h) in enumerate(sizes):
        out.append(synth.road_frame(seed0 + i, w, h, synth.THROUGHPUT_1080P))
    return out


def _padded(raw, pin):
    """[h][pitch] CPU tensors with pitch rounded up to 16 (padding bytes 0x5A)."""
    ts = []
    for r in raw:
        h, w = r.shape
        pitch = (w + 15) // 16 * 16
        t = torch.full((h, pitch), 0x5A, dtype=torch.uint8)
        t[:, :w] = torch.from_numpy(r)
        ts.append(t.pin_memory() if pin else t)
    return ts


def _check(ora, raw, p, res):
    pk, n, st = (x.numpy() for x in res)
    assert (st == 0).all(), st
    for i, r in enumerate(raw):
        ref = ora.detect(r, p.n_theta, p.top_k)
        assert n[i] == len(ref), (i, n[i], len(ref))
        np.testing.assert_array_equal(pk[i, : n[i]], ref)


@pytest.mark.parametrize("pin", [True, False])
def test_host_batch_matches_oracle(ldlib, ora, pin):
    raw = _frames(500, SIZES)
    host = _padded(raw, pin)
    p = ldlib.params(n_theta=180, top_k=3)
    with ldlib.Context(0) as c:
        res = c.detect_batch_host(host, p, widths=[r.shape[1] for r in raw])
    _check(ora, raw, p, res)


def test_host_batch_one_tensor_equals_device_batch(ldlib, ora):
    raw = [synth.road_frame(900 + i, 640, 480, synth.THROUGHPUT_1080P) for i in range(6)]
    host = torch.from_numpy(np.stack(raw)).pin_memory()          # adjacent frames: one upload
    p = ldlib.params(n_theta=360, top_k=4)
    with ldlib.Context(0) as c:
        got = c.detect_batch_host(host, p)
        dev = c.detect_batch([host[i].cuda() for i in range(len(raw))], p)
        torch.cuda.synchronize()
    for a, b in zip(got, dev):
        np.testing.assert_array_equal(a.numpy(), b.cpu().numpy())
    _check(ora, raw, p, got)


def test_host_calls_in_flight_alternate_and_grow(ldlib, ora):
    """Four calls enqueued before one synchronisation; each later pair of
    calls has more frames, so both staging areas grow between uses."""
    p = ldlib.params(n_theta=180, top_k=2)
    batches = [_frames(700 + 10 * k, SIZES[: 1 + (k // 2)] * (1 + k)) for k in range(4)]
    hosts = [_padded(b, True) for b in batches]
    outs = []
    with ldlib.Context(0) as c:
        for b, h in zip(batches, hosts):
            outs.append(c.detect_batch_host(h, p, widths=[r.shape[1] for r in b], sync=False))
        torch.cuda.current_stream().synchronize()
    for b, o in zip(batches, outs):
        _check(ora, b, p, o)


def test_host_batch_rejects_bad_arguments(ldlib):
    p = ldlib.params(n_theta=180, top_k=2)
    good = _padded(_frames(1, [(64, 48)]), True)
    with ldlib.Context(0) as c:
        bad_pitch = [(good[0].data_ptr(), 64, 48, 72)]        # pitch not a multiple of 16
        with pytest.raises(ldlib.LdError):
            c.detect_batch_host(ldlib._frames_array(bad_pitch), p)
        with pytest.raises(ldlib.LdError):                     # NULL outputs
            ldlib.ld_detect_batch_host(c.handle, [(good[0].data_ptr(), 64, 48, 64)], p, None, None, None,
                                       torch.cuda.current_stream().cuda_stream)
        res = c.detect_batch_host(good, p)                    # the context still works
    assert int(res[2][0]) == 0
