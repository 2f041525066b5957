"""ld_detect_batch captured in a CUDA graph and replayed.

After ld_ctx_reserve (scratch) and one ordinary call (Q16 table, kernel
attributes), the call enqueues only memsets and kernel launches, so it can be
captured once and replayed on new frame contents written into the same
device buffers."""
import numpy as np
import pytest
import torch

from paper_2212_09460_gb300 import synth

pytestmark = pytest.mark.gpu


def _ref(ora, frames, n_theta, top_k):
    return [ora.detect(f, n_theta, top_k) for f in frames]


@pytest.mark.parametrize("sizes,n_theta,top_k", [
    ([(640, 480)], 180, 2),
    ([(640, 480), (1280, 720), (1920, 1080), (333, 200)], 360, 4),
])
def test_graph_replay_matches_oracle(ctx, ldlib, ora, sizes, n_theta, top_k):
    p = ldlib.params(n_theta=n_theta, top_k=top_k)
    bufs = [torch.empty((h, (w + 15) // 16 * 16), dtype=torch.uint8, device="cuda") for w, h in sizes]
    widths = [w for w, h in sizes]
    n = len(sizes)
    out = (torch.zeros((n, top_k, 3), dtype=torch.int32, device="cuda"),
           torch.zeros(n, dtype=torch.int32, device="cuda"),
           torch.zeros(n, dtype=torch.int32, device="cuda"))
    ctx.reserve(sum(w * h for w, h in sizes), n, 0, p)

    def load(seed0):
        raw = [synth.road_frame(seed0 + i, w, h, synth.THROUGHPUT_1080P) for i, (w, h) in enumerate(sizes)]
        for b, r in zip(bufs, raw):
            b.copy_(torch.from_numpy(synth.pitched(r, b.shape[1], fill=0)))
        return raw

    load(500)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx.detect_batch(bufs, p, widths=widths, out=out)      # warm-up outside the capture
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ctx.detect_batch(bufs, p, widths=widths, out=out)
    for seed0 in (600, 700):
        raw = load(seed0)
        g.replay()
        torch.cuda.synchronize()
        pk, npk, st = (t.cpu().numpy() for t in out)
        for i, ref in enumerate(_ref(ora, raw, n_theta, top_k)):
            assert st[i] == 0 and npk[i] == len(ref)
            np.testing.assert_array_equal(pk[i, : npk[i]], ref)
