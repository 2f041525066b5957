"""Frames and their oracle peaks computed in a process pool (test helper).

Each job generates one seeded frame and runs the CPU oracle's whole path on
it (oracle.detect), so a full workload of 64-96 frames is checked in the time
of a few frames.  The pool uses the spawn start method, which is safe after
the parent process has initialised CUDA (a forked child of such a process
can hang); this module imports neither torch nor the CUDA binding.
"""
from __future__ import annotations

import multiprocessing as mp
import os


def frame_and_peaks(job):
    """job = (seed, w, h, n_theta, top_k) -> (frame uint8 [h][w], peaks [n][3])."""
    seed, w, h, n_theta, top_k = job
    import oracle
    from paper_2212_09460_gb300 import synth
    img = synth.road_frame(seed, w, h, synth.THROUGHPUT_1080P)
    return img, oracle.detect(img, n_theta, top_k)


def run(jobs):
    """The jobs' (frame, peaks) in order, over up to 16 host cores."""
    import oracle
    oracle.build()   # once, before the workers load it
    n = max(1, min(16, os.cpu_count() or 1, len(jobs)))
    with mp.get_context("spawn").Pool(n) as pool:
        return pool.map(frame_and_peaks, jobs, chunksize=1)
