"""The voting kernels' bounded waits, made to run out on the GPU.

Every wait of the voting kernels for a streamed edge chunk is bounded.  With
the context's wait limit set to 0 polls (ld_ctx_set_wait_limit), every such
wait gives up at once; no copy has to fail.  A CTA whose wait gave up flags
its frame, waits for the copies it issued itself and stops, so the call
completes, the frames report LD_ERR_TIMEOUT, and the context stays usable:
the next call with the default limit returns LD_OK and the oracle's peaks.
Covers both voting kernels (the interleaved-column kernel for 1080p frames,
the packed-pair kernel for min_votes 0, and the 8-slot interleaved tiles of
4K frames).
"""
import numpy as np
import pytest
import torch

from paper_2212_09460_gb300 import synth

pytestmark = pytest.mark.gpu


def _run(c, ld, frames, p):
    pk, n, st = c.detect_batch(frames, p)
    torch.cuda.synchronize()
    return pk.cpu().numpy(), n.cpu().numpy(), st.cpu().numpy()


@pytest.mark.parametrize("case", ["cols_1080p", "pairs_min_votes_0", "cols8_4k"])
def test_wait_timeout_reports_status_and_context_recovers(ldlib, ora, case):
    if case == "cols8_4k":
        raw = [synth.road_frame(2080, 3840, 2160, synth.THROUGHPUT_1080P)]
        kw = dict(n_theta=360, top_k=4)
    else:
        raw = [synth.road_frame(1000 + i, 1920, 1080, synth.THROUGHPUT_1080P) for i in range(2)]
        kw = dict(n_theta=360, top_k=4, min_votes=0 if case == "pairs_min_votes_0" else 1)
    frames = [torch.from_numpy(r).cuda() for r in raw]
    p = ldlib.params(**kw)
    with ldlib.Context(0) as c:
        c.set_wait_limit(0)
        _, _, st = _run(c, ldlib, frames, p)
        assert (st == ldlib.LD_ERR_TIMEOUT).all(), st
        c.set_wait_limit(-1)
        pk, n, st = _run(c, ldlib, frames, p)
    assert (st == 0).all(), st
    for i, r in enumerate(raw):
        ref = ora.detect(r, kw["n_theta"], kw["top_k"], min_votes=kw.get("min_votes", 1))
        assert n[i] == len(ref)
        np.testing.assert_array_equal(pk[i, : n[i]], ref)


def test_wait_limit_rejects_too_many_polls(ldlib):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    with ldlib.Context(0) as c:
        with pytest.raises(ldlib.LdError):
            c.set_wait_limit((1 << 26) + 1)
