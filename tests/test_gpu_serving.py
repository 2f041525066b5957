"""The serving loop on the GPU: frames served in the mix (8 Poisson cameras at
20x their nominal rate, so that launches hold many frames of mixed sizes)
give the same peaks, status and fallback decision as the same frame detected
alone, and plain-class frames equal the oracle."""
import numpy as np
import pytest
import torch

from paper_2212_09460_gb300 import ld, synth
from paper_2212_09460_gb300.serving import PROPOSAL_SIZE, Server, summarize

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def served(ldlib):
    srv = Server(workers=2, max_batch=32, budget_bytes=1 << 30, autotune=False)
    st = srv.serve(0.5, rate_scale=20.0, keep_peaks=True)
    yield srv, st
    srv.close()


def test_all_frames_served_ok(served):
    srv, st = served
    s = summarize(st)
    assert s["frames"] > 1500 and s["status_nonzero"] == 0
    assert s["max_batch_seen"] > 1                                  # launches did batch
    assert srv.executor.net is not None
    assert any(f.fallback >= 0 for f in st.frames)                  # the proposal path served 1080p


def _sample(st, per_size=4):
    out, rng = [], np.random.default_rng(0)
    sizes = sorted({f.size for f in st.frames})
    batch_n = {}
    for f in st.frames:
        batch_n[f.batch] = batch_n.get(f.batch, 0) + 1
    for s in sizes:
        fs = [f for f in st.frames if f.size == s and batch_n[f.batch] > 1]
        out += [fs[i] for i in rng.choice(len(fs), min(per_size, len(fs)), replace=False)]
    return out


def test_alone_equals_in_the_mix(served):
    srv, st = served
    ex = srv.executor
    for f in _sample(st):
        bufs, keep = ld.synth_frames_device([(f.seed, f.w, f.h, synth.THROUGHPUT_1080P)], 0)
        with ld.Context(0) as ctx:
            if f.size == PROPOSAL_SIZE:
                pk, npk, stt, fb, _ = ctx.detect_batch_proposal(bufs, ex.p, ex.net, ex.q, widths=[f.w])
                torch.cuda.synchronize()
                assert int(fb[0]) == f.fallback
            else:
                pk, npk, stt = ctx.detect_batch(bufs, ex.p, widths=[f.w])
                torch.cuda.synchronize()
        assert int(stt[0]) == f.status == 0
        np.testing.assert_array_equal(pk[0, : int(npk[0])].cpu().numpy(), f.peaks)


def test_plain_frames_in_the_mix_equal_the_oracle(served, ora):
    srv, st = served
    p = srv.executor.p
    fs = [f for f in _sample(st, 2) if f.size == (1280, 720)]
    assert fs
    for f in fs:
        img = synth.road_frame(f.seed, f.w, f.h, synth.THROUGHPUT_1080P)
        ref = ora.detect(img, p.n_theta, p.top_k, border=ora.BORDER_CLEAR)
        np.testing.assert_array_equal(f.peaks, ref)
