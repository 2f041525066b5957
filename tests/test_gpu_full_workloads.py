"""Every frame of the two benchmark workloads against the oracle.

  * the headline batch: 64 seeded 1920x1080 dashed-lane frames (seeds
    1000-1063), 360 theta, top-4, in one ld_detect_batch call with the tile
    plans the benchmark tunes (autotuned on the first 16 frames);
  * the batching workload: 96 frames in one call, 24 each of 640x480,
    1280x720, 1920x1080 and 3840x2160 (seeds 2000-2095), 360 theta, top-4,
    after ld_ctx_reserve and ld_autotune on all of them, replayed from a
    CUDA graph as the benchmark times it.

The oracle (oracle.detect) runs on a spawn process pool over the host cores
(tests/oracle_pool.py); the peaks must match bit for bit for every frame.
"""
import numpy as np
import pytest
import torch

import oracle_pool

pytestmark = pytest.mark.gpu

MIXED_SIZES = [(640, 480), (1280, 720), (1920, 1080), (3840, 2160)]


def _compare(pk, n, st, refs, names):
    bad = []
    for i, ref in enumerate(refs):
        if st[i] != 0 or n[i] != len(ref) or not np.array_equal(pk[i, : n[i]], ref):
            bad.append((names[i], int(st[i]), pk[i, : n[i]].tolist(), ref.tolist()))
    assert not bad, f"{len(bad)} of {len(refs)} frames differ, first: {bad[:3]}"


def test_headline_batch_every_frame(ldlib):
    jobs = [(1000 + i, 1920, 1080, 360, 4) for i in range(64)]
    res = oracle_pool.run(jobs)
    frames = [torch.from_numpy(f).cuda() for f, _ in res]
    p = ldlib.params(n_theta=360, top_k=4)
    with ldlib.Context(0) as c:
        c.autotune(frames[:16], p, iters=2)
        pk, n, st = c.detect_batch(frames, p)
        torch.cuda.synchronize()
    _compare(pk.cpu().numpy(), n.cpu().numpy(), st.cpu().numpy(), [r for _, r in res],
             [f"seed {j[0]}" for j in jobs])


def test_batching_workload_every_frame(ldlib):
    jobs = [(2000 + i, *MIXED_SIZES[i // 24], 360, 4) for i in range(96)]
    res = oracle_pool.run(jobs)
    frames = [torch.from_numpy(f).cuda() for f, _ in res]
    p = ldlib.params(n_theta=360, top_k=4)
    n_f = len(frames)
    with ldlib.Context(0) as c:
        c.reserve(sum(f.numel() for f in frames), n_f, 0, p)
        c.autotune(frames, p, iters=2)
        out = (torch.full((n_f, 4, 3), -1, dtype=torch.int32, device="cuda"),
               torch.full((n_f,), -1, dtype=torch.int32, device="cuda"),
               torch.full((n_f,), -1, dtype=torch.int32, device="cuda"))
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            c.detect_batch(frames, p, out=out)   # warm-up outside the capture
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            c.detect_batch(frames, p, out=out)
        for t in out:
            t.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        pk, n, st = (t.cpu().numpy() for t in out)
    _compare(pk, n, st, [r for _, r in res], [f"seed {j[0]} {j[1]}x{j[2]}" for j in jobs])
