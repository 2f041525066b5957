"""Host logic of the serving loop, without a GPU: Poisson arrivals, memory
admission (including injected allocation failures), continuous batching,
dropped and late cameras.  The executor here is a fake that "runs" a batch
for a simulated time on a virtual clock and computes each frame's peaks with
the oracle from the frame's slot buffer at completion time, so a frame whose
slot were reused too early, or whose result were attached to the wrong frame,
would fail the comparison with the frame's own peaks."""
import numpy as np
import pytest

from paper_2212_09460_gb300 import synth
from paper_2212_09460_gb300.serving import (Admission, AdmissionError, Frame, Scheduler, frame_seed, pitch_of,
                                            poisson_arrivals, summarize)

SMALL = [(64, 48)] * 3 + [(96, 64)] * 3 + [(128, 96)] * 2
PROPOSAL = (96, 64)          # the class the fake sends down its "proposal" path


class VirtualClock:
    def __init__(self, quantum=5e-5):
        self.t, self.q = 0.0, quantum

    def now(self):
        return self.t

    def idle(self, until, busy):
        nxt = self.t + self.q
        self.t = min(until, nxt) if until is not None and until > self.t else nxt


class FakeExecutor:
    """Service time a + b * pixels per batch; peaks by the oracle at completion."""

    def __init__(self, ora, clock, n_workers=2, a=2e-4, b=2e-9, fail_seed=None):
        self.ora, self.clock, self.n_workers = ora, clock, n_workers
        self.a, self.b, self.fail_seed = a, b, fail_seed
        self.jobs = [None] * n_workers
        self.loads = 0
        self.max_concurrent = 0

    def batch_class(self, f):
        return "proposal" if f.size == PROPOSAL else "plain"

    def load(self, frames):
        self.loads += 1
        for f in frames:
            f.buf[:, : f.w] = synth.road_frame(f.seed, f.w, f.h, synth.LATENCY_640x480)
            f.ready = True

    def busy(self, wi):
        return self.jobs[wi] is not None

    def submit(self, wi, frames, seq):
        assert self.jobs[wi] is None
        assert all(f.ready for f in frames)
        assert len({self.batch_class(f) for f in frames}) == 1
        t_end = self.clock.now() + self.a + self.b * sum(f.w * f.h for f in frames)
        self.jobs[wi] = (frames, t_end)
        self.max_concurrent = max(self.max_concurrent, sum(j is not None for j in self.jobs))

    def poll(self, wi):
        frames, t_end = self.jobs[wi]
        if self.clock.now() < t_end:
            return None
        self.jobs[wi] = None
        n = len(frames)
        pk = np.zeros((n, 2, 3), np.int32)
        npk = np.zeros(n, np.int32)
        for k, f in enumerate(frames):
            got = self.ora.detect(np.ascontiguousarray(f.buf[:, : f.w]), 180, 2)
            pk[k, : len(got)] = got
            npk[k] = len(got)
        status = np.array([5 if f.seed == self.fail_seed else 0 for f in frames], np.int32)
        fb = np.array([0 if self.batch_class(f) == "proposal" else -1 for f in frames], np.int32)
        return frames, pk, npk, status, fb


def _alloc(w, h):
    return np.zeros((h, pitch_of(w)), np.uint8)


def _expected(ora, f):
    return ora.detect(synth.road_frame(f.seed, f.w, f.h, synth.LATENCY_640x480), 180, 2)


def _serve(ora, arrivals, budget=1 << 20, workers=2, max_batch=8, min_slots=2, **kw):
    clock = VirtualClock()
    adm = Admission(SMALL, budget, _alloc, min_slots=min_slots)
    ex = FakeExecutor(ora, clock, workers, **kw)
    st = Scheduler(adm, ex, max_batch, clock).run(arrivals, keep_peaks=True)
    return st, adm, ex


# ------------------------------------------------------------------ arrivals
def test_poisson_arrivals_rate_seeds_and_order():
    arr = poisson_arrivals(SMALL, 60.0, fps=30.0, seed=42)
    assert all(a.t_arrival <= b.t_arrival for a, b in zip(arr, arr[1:]))
    for s in range(len(SMALL)):
        fs = [f for f in arr if f.stream == s]
        assert abs(len(fs) - 1800) < 4 * np.sqrt(1800)          # Poisson count, 4 sigma
        assert [f.index for f in fs] == list(range(len(fs)))
        assert all(f.seed == 10_000_000 * (s + 1) + f.index for f in fs)
        gaps = np.diff([0.0] + [f.t_arrival for f in fs])
        assert abs(gaps.mean() - 1 / 30) < 4 * (1 / 30) / np.sqrt(len(gaps))
        assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1       # exponential: cv = 1
    assert frame_seed(2, 7) == 30_000_007
    assert len(poisson_arrivals(SMALL, 60.0, seed=42)) == len(arr)        # deterministic
    assert [f.t_arrival for f in poisson_arrivals(SMALL, 60.0, seed=43)][:5] != [f.t_arrival for f in arr][:5]


def test_dropped_camera_leaves_the_others_unchanged():
    full = poisson_arrivals(SMALL, 5.0)
    cut = poisson_arrivals(SMALL, 5.0, stop_at={3: 1.0})
    assert max(f.t_arrival for f in cut if f.stream == 3) < 1.0
    key = lambda fs: [(f.stream, f.index, f.t_arrival) for f in fs if f.stream != 3]
    assert key(full) == key(cut)


# ------------------------------------------------------------------ admission
def test_admission_slots_follow_offered_bytes():
    budget = 1 << 20
    adm = Admission(SMALL, budget, _alloc)
    offered = {(64, 48): 3 * 48 * 64, (96, 64): 3 * 64 * 96, (128, 96): 2 * 96 * 128}
    tot = sum(offered.values())
    for s, b in offered.items():
        assert adm.slots(s) == int(budget * b / tot) // (s[1] * pitch_of(s[0]))
    assert adm.bytes_reserved <= budget
    f = Frame(0.0, 0, 0, 1, 64, 48)
    assert adm.admit(f) and f.buf is adm.bufs[(64, 48)][f.slot] and adm.in_use == 1
    adm.release(f)
    assert adm.in_use == 0 and f.buf is None
    with pytest.raises(AdmissionError):
        adm.admit(Frame(0.0, 0, 0, 1, 32, 32))


def test_admission_with_injected_allocation_failure():
    calls = {"n": 0}

    def flaky(w, h):                     # the 4th allocation of the 96x64 pool fails
        if (w, h) == (96, 64):
            calls["n"] += 1
            if calls["n"] == 4:
                raise RuntimeError("CUDA out of memory (injected)")
        return _alloc(w, h)

    adm = Admission(SMALL, 1 << 20, flaky)
    assert adm.slots((96, 64)) == 3 and adm.alloc_failed == {(96, 64): True}
    assert adm.slots((64, 48)) > 3

    def dead(w, h):
        if (w, h) == (128, 96):
            raise MemoryError("injected")
        return _alloc(w, h)

    with pytest.raises(AdmissionError):
        Admission(SMALL, 1 << 20, dead)


# ------------------------------------------------------------------ the loop
def _check_served(ora, arrivals, st, adm, max_batch, workers):
    assert len(st.frames) == len(arrivals)
    assert {(f.stream, f.index) for f in st.frames} == {(f.stream, f.index) for f in arrivals}
    for f in st.frames:
        assert f.t_arrival <= f.t_admit <= f.t_launch <= f.t_done
        np.testing.assert_array_equal(f.peaks, _expected(ora, f))
    assert max(st.batch_sizes) <= max_batch and st.launches == len(st.batch_sizes)
    assert st.max_inflight <= workers
    for s in adm.bufs:
        assert len(adm.free[s]) == adm.slots(s)                 # every slot back
    assert st.max_slots_in_use <= sum(adm.slots(s) for s in adm.bufs)
    # one camera's frames launch in arrival order
    for s in {f.stream for f in st.frames}:
        b = [f.batch for f in sorted((f for f in st.frames if f.stream == s), key=lambda f: f.index)]
        assert b == sorted(b)


def test_light_load_serves_every_frame_alone(ora):
    arr = poisson_arrivals(SMALL, 0.5, fps=30.0)
    st, adm, ex = _serve(ora, arr)
    _check_served(ora, arr, st, adm, 8, 2)
    assert np.mean(st.batch_sizes) < 1.5                        # arrivals rarely coincide
    s = summarize(st, adm)
    assert s["frames"] == len(arr) and 0 < s["latency_ms_p50"] <= s["latency_ms_p99"] <= s["latency_ms_max"]
    assert s["bytes_reserved"] == sum(adm.slots(z) * z[1] * pitch_of(z[0]) for z in adm.bufs)
    assert s["budget_bytes"] == 1 << 20 and s["over_budget"] == (s["bytes_reserved"] > s["budget_bytes"])
    # stall attribution: the loop's longest gap and its longest call of each phase
    ph = s["max_phase_ms"]
    assert {"load", "poll", "submit", "idle"} <= set(ph) and ph["idle"] > 0
    assert s["max_loop_gap_ms"] >= max(ph.values()) - 1e-9


def test_heavy_load_batches_and_backpressure(ora):
    # offered 8 x 30 x 40 = 9600 frames/s against ~0.2 ms + 2 ns/px per batch
    # on two workers, with two slots per size: frames wait for slots and
    # launches fill up to max_batch
    arr = poisson_arrivals(SMALL, 0.25, fps=30.0, rate_scale=40.0)
    st, adm, ex = _serve(ora, arr, budget=0, max_batch=4, min_slots=4)
    _check_served(ora, arr, st, adm, 4, 2)
    assert st.max_waiting > 0 and max(st.batch_sizes) == 4 and ex.max_concurrent == 2
    assert all(adm.slots(s) == 4 for s in adm.bufs)
    assert summarize(st, adm)["over_budget"]   # the min_slots floor exceeds a zero budget, and says so


def test_proposal_class_is_batched_apart_and_fallback_reported(ora):
    arr = poisson_arrivals(SMALL, 0.2, fps=30.0, rate_scale=20.0)
    st, adm, ex = _serve(ora, arr)
    _check_served(ora, arr, st, adm, 8, 2)
    for f in st.frames:
        assert f.fallback == (0 if f.size == PROPOSAL else -1)
    assert summarize(st)["proposal_fallback_rate"] == 0.0


def test_late_camera_burst_and_dropped_camera(ora):
    arr = poisson_arrivals(SMALL, 1.0, fps=30.0, rate_scale=2.0, stop_at={5: 0.3})
    # camera 1 is late: everything it captured in [0.2, 0.6) reaches the host at 0.6
    for f in arr:
        if f.stream == 1 and 0.2 <= f.t_arrival < 0.6:
            f.t_arrival = 0.6
    arr.sort(key=lambda f: (f.t_arrival, f.stream, f.index))
    st, adm, ex = _serve(ora, arr, max_batch=4)
    _check_served(ora, arr, st, adm, 4, 2)
    assert not [f for f in st.frames if f.stream == 5 and f.t_arrival >= 0.3]


def test_failed_frame_status_is_reported_and_serving_continues(ora):
    arr = poisson_arrivals(SMALL, 0.3, fps=30.0, rate_scale=4.0)
    bad = arr[len(arr) // 2].seed
    st, adm, ex = _serve(ora, arr, fail_seed=bad)
    assert len(st.frames) == len(arr)
    assert [f.seed for f in st.frames if f.status != 0] == [bad]
    assert summarize(st)["status_nonzero"] == 1
