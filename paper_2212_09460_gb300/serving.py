"""Multi-camera serving loop with continuous batching.

The paper has no serving layer; this is the runtime around the detection
path.  The loop is split so that its host logic runs without a GPU:

* ``poisson_arrivals``: per-camera Poisson arrival times (seeded); frame i of
  camera s has the generator seed 10^7 (s + 1) + i.
* ``Admission``: device frame slots, sized from a byte budget in proportion to
  each resolution's offered bytes.  A frame is admitted when a slot of its
  size is free (memory-based admission); until then it waits in its size's
  host queue.  A failed slot allocation shrinks that size's pool; a size left
  with no slot at all is an error at start-up.
* ``Scheduler``: the event loop.  Arrivals -> admission -> the executor
  loads admitted frames into their slots -> whenever a worker is idle, the
  batch class (see ``GpuExecutor.batch_class``) of the oldest admitted frame
  forms the next launch from up to ``max_batch`` admitted frames of that class,
  oldest first (continuous batching: a launch takes whatever has arrived,
  while earlier launches are still running on other workers).  Completion
  frees the slots and records each frame's latency (arrival -> peaks on the
  host).
* ``GpuExecutor``: one ld context, CUDA stream and pinned result buffers per
  worker, so that in-flight batches never share scratch.  A frame is loaded
  by the device generator (ld_synth_frames, in place of a camera's DMA) on a
  loader stream; a launch waits on that load's event.  Plain launches take
  frames of any size together (ld_detect_batch packs mixed sizes); 1920x1080
  frames take the learned-proposal path (ld_detect_batch_proposal, with its
  full-vote fallback) when a trained network is given.  The Q16 tables, the
  edge lists and candidate buffers stay resident in each context from
  start-up (ld_ctx_reserve plus one warm launch per batch class).

No kernel mixes frames, so a frame's peaks are the same alone and in any
batch; a GPU test checks this on frames served in the mix.
"""
from __future__ import annotations

import ctypes
import gc
import os
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

DEFAULT_STREAMS = [(1280, 720)] * 3 + [(1920, 1080)] * 3 + [(3840, 2160)] * 2
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "proposal_1080p.npz")
PROPOSAL_SIZE = (1920, 1080)


def pitch_of(w: int) -> int:
    return (w + 15) // 16 * 16


@dataclass
class Frame:
    t_arrival: float
    stream: int
    index: int
    seed: int
    w: int
    h: int
    slot: int = -1
    buf: object = None
    ready: object = None        # executor's handle for "loaded into its slot"
    t_admit: float = -1.0
    t_launch: float = -1.0
    t_done: float = -1.0
    batch: int = -1             # sequence number of the launch that served it
    peaks: np.ndarray | None = None
    status: int = -1
    fallback: int = -1

    @property
    def size(self):
        return (self.w, self.h)


def frame_seed(stream: int, index: int) -> int:
    return 10_000_000 * (stream + 1) + index


def poisson_arrivals(streams, duration_s: float, fps: float = 30.0, seed: int = 42, rate_scale: float = 1.0,
                     stop_at: dict | None = None) -> list[Frame]:
    """Frames arriving in [0, duration_s): camera s delivers a Poisson process
    of rate fps * rate_scale (exponential gaps from a generator seeded by
    (seed, s), so cameras are independent of one another).  stop_at[s] = t
    ends camera s at time t (a dropped camera).  Returned in arrival order."""
    lam = fps * rate_scale
    out = []
    for s, (w, h) in enumerate(streams):
        rng = np.random.default_rng([seed, s])
        t_end = duration_s if stop_at is None or s not in stop_at else min(duration_s, stop_at[s])
        t, i = 0.0, 0
        while True:
            t += rng.exponential(1.0 / lam)
            if t >= t_end:
                break
            out.append(Frame(t, s, i, frame_seed(s, i), w, h))
            i += 1
    out.sort(key=lambda f: (f.t_arrival, f.stream))
    return out


class AdmissionError(RuntimeError):
    pass


class Admission:
    """Device frame slots per resolution, sized by bytes.

    A w x h frame takes h * pitch bytes (pitch = w rounded up to 16).  Size s
    gets max(min_slots, budget * share_s // bytes_s) slots, share_s being its
    fraction of the offered bytes (frames/s x bytes); alloc(w, h) makes one
    slot's buffer.  An allocation that fails (MemoryError or RuntimeError,
    which covers the CUDA allocator's out-of-memory error) ends that size's
    pool; a size with no slot raises AdmissionError.  The min_slots floor can
    take the reservation past the budget: bytes_reserved and budget_bytes are
    both kept, and the serving stats report them side by side."""

    def __init__(self, streams, budget_bytes: int, alloc, min_slots: int = 2):
        self.budget_bytes = int(budget_bytes)
        sizes = sorted(set(map(tuple, streams)))
        offered = {s: sum(1 for t in streams if tuple(t) == s) * s[1] * pitch_of(s[0]) for s in sizes}
        total = sum(offered.values())
        self.bufs, self.free, self.alloc_failed = {}, {}, {}
        self.bytes_reserved = 0
        for s in sizes:
            nbytes = s[1] * pitch_of(s[0])
            want = max(min_slots, int(budget_bytes * offered[s] / total) // nbytes)
            bufs = []
            for _ in range(want):
                try:
                    bufs.append(alloc(*s))
                except (MemoryError, RuntimeError):
                    self.alloc_failed[s] = True
                    break
            if not bufs:
                raise AdmissionError(f"no device slot could be allocated for {s[0]}x{s[1]} frames")
            self.bufs[s] = bufs
            self.free[s] = deque(range(len(bufs)))
            self.bytes_reserved += len(bufs) * nbytes
        self.in_use = 0
        self.max_in_use = 0

    def slots(self, size) -> int:
        return len(self.bufs[size])

    def admit(self, f: Frame) -> bool:
        pool = self.free.get(f.size)
        if pool is None:
            raise AdmissionError(f"no slot pool for {f.w}x{f.h} frames")
        if not pool:
            return False
        f.slot = pool.popleft()
        f.buf = self.bufs[f.size][f.slot]
        self.in_use += 1
        self.max_in_use = max(self.max_in_use, self.in_use)
        return True

    def release(self, f: Frame) -> None:
        self.free[f.size].append(f.slot)
        self.in_use -= 1
        f.buf = None


class RealClock:
    def __init__(self):
        self.t0 = time.perf_counter()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def idle(self, until: float | None, busy: bool) -> None:
        """Nothing to do: spin while batches are in flight (completion is
        polled), else sleep towards the next arrival."""
        if busy:
            return
        if until is not None:
            dt = until - self.now()
            if dt > 0:
                time.sleep(min(dt, 1e-3))


@dataclass
class ServeStats:
    frames: list = field(default_factory=list)
    launches: int = 0
    batch_sizes: list = field(default_factory=list)
    max_inflight: int = 0
    max_waiting: int = 0
    max_slots_in_use: int = 0
    wall_s: float = 0.0
    batch_device_ms: list = field(default_factory=list)   # (device ms, batch class, frames) per batch
    max_loop_gap_ms: float = 0.0   # longest time between two scheduler iterations
    max_phase_ms: dict = field(default_factory=dict)   # longest single load / poll / submit / idle call

    def phase(self, name: str, t0: float, t1: float) -> None:
        ms = (t1 - t0) * 1e3
        if name not in self.max_phase_ms or ms > self.max_phase_ms[name]:
            self.max_phase_ms[name] = ms


class Scheduler:
    """Arrivals -> admission -> load -> continuous batching -> completion.

    The executor provides: n_workers; batch_class(frame); load(frames) (start
    putting admitted frames in their slots); submit(worker, frames, seq)
    (launch one batch); poll(worker) -> None while the worker's batch runs,
    else (frames, peaks[n][k][3], n_peaks[n], status[n], fallback[n]) with
    fallback -1 on plain launches; busy(worker); optionally device_ms(worker)
    -> (device ms, batch class) of the batch poll just returned."""

    def __init__(self, admission: Admission, executor, max_batch: int = 64, clock=None):
        self.adm, self.ex, self.max_batch = admission, executor, max_batch
        self.clock = clock or RealClock()

    def run(self, arrivals: list[Frame], keep_peaks: bool = False) -> ServeStats:
        """Serve the arrivals (with Python's cyclic garbage collector paused,
        so that no collection stalls the loop)."""
        gc_was = gc.isenabled()
        gc.disable()
        try:
            return self._run(arrivals, keep_peaks)
        finally:
            if gc_was:
                gc.enable()

    def _run(self, arrivals: list[Frame], keep_peaks: bool) -> ServeStats:
        adm, ex, clock = self.adm, self.ex, self.clock
        st = ServeStats()
        waiting = {s: deque() for s in adm.bufs}      # arrived, no slot yet
        admitted = {}                                  # batch class -> deque of loaded frames
        total, ai, done, seq = len(arrivals), 0, 0, 0
        t_start = clock.now()
        t_prev = t_start
        dev_ms = getattr(ex, "device_ms", None)
        while done < total:
            now = clock.now()
            st.max_loop_gap_ms = max(st.max_loop_gap_ms, (now - t_prev) * 1e3)
            t_prev = now
            progressed = False
            while ai < total and arrivals[ai].t_arrival <= now:
                f = arrivals[ai]
                waiting[f.size].append(f)
                ai += 1
            st.max_waiting = max(st.max_waiting, sum(len(q) for q in waiting.values()))
            # memory-based admission
            newly = []
            for q in waiting.values():
                while q and adm.admit(q[0]):
                    f = q.popleft()
                    f.t_admit = now
                    newly.append(f)
            if newly:
                newly.sort(key=lambda f: f.t_arrival)
                t0 = clock.now()
                ex.load(newly)
                st.phase("load", t0, clock.now())
                for f in newly:
                    admitted.setdefault(ex.batch_class(f), deque()).append(f)
                progressed = True
            # completions
            inflight = 0
            for wi in range(ex.n_workers):
                if not ex.busy(wi):
                    continue
                t0 = clock.now()
                res = ex.poll(wi)
                st.phase("poll", t0, clock.now())
                if res is None:
                    inflight += 1
                    continue
                frames, pk, npk, status, fb = res
                if dev_ms is not None:
                    ms, cls = dev_ms(wi)
                    st.batch_device_ms.append((ms, cls, len(frames)))
                t_done = clock.now()
                for k, f in enumerate(frames):
                    f.t_done = t_done
                    f.status, f.fallback = int(status[k]), int(fb[k])
                    if keep_peaks:
                        f.peaks = np.array(pk[k, : npk[k]], copy=True)
                    adm.release(f)
                    st.frames.append(f)
                done += len(frames)
                progressed = True
            st.max_inflight = max(st.max_inflight, inflight)
            # continuous batching: each idle worker takes the oldest class
            for wi in range(ex.n_workers):
                if ex.busy(wi):
                    continue
                heads = [(q[0].t_arrival, c) for c, q in admitted.items() if q]
                if not heads:
                    break
                _, c = min(heads)
                q = admitted[c]
                frames = [q.popleft() for _ in range(min(self.max_batch, len(q)))]
                t_launch = clock.now()
                for f in frames:
                    f.t_launch, f.batch = t_launch, seq
                t0 = clock.now()
                ex.submit(wi, frames, seq)
                st.phase("submit", t0, clock.now())
                st.launches += 1
                st.batch_sizes.append(len(frames))
                seq += 1
                progressed = True
            st.max_slots_in_use = max(st.max_slots_in_use, adm.max_in_use)
            if not progressed:
                busy = any(ex.busy(wi) for wi in range(ex.n_workers))
                t0 = clock.now()
                clock.idle(arrivals[ai].t_arrival if ai < total else None, busy)
                st.phase("idle", t0, clock.now())
        st.wall_s = clock.now() - t_start
        return st


def summarize(st: ServeStats, adm: "Admission | None" = None) -> dict:
    """Latency percentiles (ms, arrival -> peaks on the host) and throughput;
    with adm, also the device bytes its slots reserve against its budget."""
    fr = st.frames
    mem = {} if adm is None else {"bytes_reserved": adm.bytes_reserved, "budget_bytes": adm.budget_bytes,
                                  "over_budget": adm.bytes_reserved > adm.budget_bytes}
    if not fr:
        return {"frames": 0}
    lat = np.array([(f.t_done - f.t_arrival) * 1e3 for f in fr])
    span = max(f.t_done for f in fr) - min(f.t_arrival for f in fr)
    fb = [f.fallback for f in fr if f.fallback >= 0]
    by_size = {}
    for f in fr:
        by_size.setdefault(f"{f.w}x{f.h}", []).append((f.t_done - f.t_arrival) * 1e3)
    return {"frames": len(fr), "frames_per_s": len(fr) / span if span > 0 else None,
            "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
            "latency_ms_max": float(lat.max()),
            "latency_ms_p99_by_size": {k: float(np.percentile(v, 99)) for k, v in sorted(by_size.items())},
            "launches": st.launches, "mean_batch": float(np.mean(st.batch_sizes)),
            "max_batch_seen": int(max(st.batch_sizes)), "max_inflight_batches": st.max_inflight,
            "max_waiting_for_slot": st.max_waiting, "max_slots_in_use": st.max_slots_in_use,
            "proposal_fallback_rate": float(np.mean(fb)) if fb else None,
            "status_nonzero": int(sum(1 for f in fr if f.status != 0)),
            "max_loop_gap_ms": st.max_loop_gap_ms,
            "max_phase_ms": dict(st.max_phase_ms),
            **_device_summary(st.batch_device_ms), **mem}


def _device_summary(bd: list) -> dict:
    """Device time per batch (launch to results on the host side of the
    stream): p50, p99 and the slowest batch."""
    if not bd:
        return {}
    ms = np.array([b[0] for b in bd])
    worst = max(bd, key=lambda b: b[0])
    return {"batch_device_ms_p50": float(np.percentile(ms, 50)), "batch_device_ms_p99": float(np.percentile(ms, 99)),
            "batch_device_ms_max": float(worst[0]), "slowest_batch": {"class": str(worst[1]), "frames": worst[2]}}


class GpuExecutor:
    """Workers on one CUDA device (see the module docstring)."""

    def __init__(self, admission: Admission, sizes, p=None, net=None, q=None, workers: int = 3,
                 max_batch: int = 64, device: int = 0, autotune: bool = True):
        import torch

        from . import ld, synth
        self.torch, self.ld, self.synth = torch, ld, synth
        self.dev = torch.device("cuda", device)
        self.p = p if p is not None else ld.params(n_theta=360, top_k=4, border=ld.LD_BORDER_CLEAR)
        self.net, self.q = net, (q if q is not None else ld.proposal_params())
        self.style = synth.THROUGHPUT_1080P
        self.n_workers, self.max_batch = workers, max_batch
        self.loader = torch.cuda.Stream(self.dev)
        # frame descriptors go to the device through a ring of pinned buffers
        # allocated here, so that no load allocates pinned memory (which can
        # stall the host for milliseconds)
        max_load = sum(admission.slots(sz) for sz in admission.bufs)
        desc_bytes = ctypes.sizeof(ld.ld_synth_frame) * max_load
        self.desc_ring = 8
        self.desc_host = torch.empty((self.desc_ring, desc_bytes), dtype=torch.uint8, pin_memory=True)
        self.desc_dev = torch.empty((self.desc_ring, desc_bytes), dtype=torch.uint8, device=self.dev)
        self.desc_ev = [None] * self.desc_ring
        self.desc_next = 0
        max_px = max(w * h for w, h in sizes) * max_batch
        k = self.p.top_k
        self.w = []
        for _ in range(workers):
            ctx = ld.Context(device)
            ctx.reserve(max_px, max_batch, 0, self.p)
            dev_out = (torch.zeros((max_batch, k, 3), dtype=torch.int32, device=self.dev),) + tuple(
                torch.zeros(max_batch, dtype=torch.int32, device=self.dev) for _ in range(4))
            host_out = tuple(torch.zeros(t.shape, dtype=t.dtype, pin_memory=True) for t in dev_out[:4])
            self.w.append({"ctx": ctx, "stream": torch.cuda.Stream(self.dev), "dev": dev_out, "host": host_out,
                           "frames": None, "event": None, "proposal": False})
        self._warm(admission, sizes, autotune)

    def close(self) -> None:
        for w in self.w:
            w["ctx"].close()

    def batch_class(self, f: Frame):
        return "proposal" if self.net is not None and f.size == PROPOSAL_SIZE else "plain"

    def _warm(self, adm: Admission, sizes, autotune: bool) -> None:
        """Tune and allocate every worker's scratch before serving: one launch
        per batch class at the largest batch the slots allow."""
        torch = self.torch
        for s in sizes:
            n = min(self.max_batch, adm.slots(s))
            frames = [Frame(0.0, -1, i, 1 + i, s[0], s[1], slot=i, buf=adm.bufs[s][i]) for i in range(n)]
            self.load(frames)
            self.loader.synchronize()
            for wi in range(self.n_workers):
                ctx = self.w[wi]["ctx"]
                if autotune:
                    ctx.autotune([f.buf for f in frames[:8]], self.p, widths=[s[0]] * min(8, n),
                                 stream=self.w[wi]["stream"])
                self.submit(wi, frames, -1)
                self.w[wi]["event"].synchronize()
                self.w[wi]["frames"] = None
        torch.cuda.synchronize(self.dev)

    def load(self, frames) -> None:
        """Generate the frames into their slots on the loader stream (one launch)."""
        torch, ld = self.torch, self.ld
        specs = [(f.seed, f.w, f.h, self.style) for f in frames]
        arr = ld.synth_descriptors(specs, [f.buf for f in frames])
        nbytes = ctypes.sizeof(arr)
        k = self.desc_next
        self.desc_next = (k + 1) % self.desc_ring
        if self.desc_ev[k] is not None:
            self.desc_ev[k].synchronize()   # the copy that last used this buffer (long done)
        host, dev = self.desc_host[k], self.desc_dev[k]
        ctypes.memmove(host.data_ptr(), ctypes.addressof(arr), nbytes)
        with torch.cuda.stream(self.loader):
            dev[:nbytes].copy_(host[:nbytes], non_blocking=True)
            ld.ld_synth_frames(dev.data_ptr(), len(frames), self.loader.cuda_stream)
            ev = torch.cuda.Event()
            ev.record(self.loader)
        self.desc_ev[k] = ev
        for f in frames:
            f.ready = ev

    def busy(self, wi: int) -> bool:
        return self.w[wi]["frames"] is not None

    def submit(self, wi: int, frames, seq: int) -> None:
        torch = self.torch
        w = self.w[wi]
        s = w["stream"]
        n = len(frames)
        waited = set()
        for f in frames:
            if f.ready is not None and id(f.ready) not in waited:
                s.wait_event(f.ready)
                waited.add(id(f.ready))
        out = tuple(t[:n] for t in w["dev"])
        cls = self.batch_class(frames[0])
        proposal = cls == "proposal"
        ev0 = torch.cuda.Event(enable_timing=True)
        ev0.record(s)
        bufs, widths = [f.buf for f in frames], [f.w for f in frames]
        if proposal:
            w["ctx"].detect_batch_proposal(bufs, self.p, self.net, self.q, widths=widths, out=out, stream=s)
        else:
            w["ctx"].detect_batch(bufs, self.p, widths=widths, out=out[:3], stream=s)
        with torch.cuda.stream(s):
            for h_t, d_t in zip(w["host"], out[:4]):
                h_t[:n].copy_(d_t, non_blocking=True)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(s)
        w["frames"], w["event"], w["proposal"] = frames, ev, proposal
        w["ev0"], w["class"] = ev0, cls + " " + "+".join(sorted({f"{f.w}x{f.h}" for f in frames}))

    def poll(self, wi: int):
        w = self.w[wi]
        if w["frames"] is None or not w["event"].query():
            return None
        frames, n = w["frames"], len(w["frames"])
        w["frames"] = None
        pk, npk, st, fb = (t[:n].numpy() for t in w["host"])
        fb = fb.copy() if w["proposal"] else np.full(n, -1, np.int32)
        return frames, pk.copy(), npk.copy(), st.copy(), fb

    def device_ms(self, wi: int):
        """(device ms, batch class) of the worker's last completed batch."""
        w = self.w[wi]
        return w["ev0"].elapsed_time(w["event"]), w["class"]


class Server:
    """Admission + GpuExecutor + Scheduler with the defaults of the 8-camera
    workload (3 x 1280x720, 3 x 1920x1080, 2 x 3840x2160 at 30 frames/s)."""

    def __init__(self, streams=None, workers: int = 3, max_batch: int = 64, budget_bytes: int = 2 << 30,
                 use_proposal: bool = True, device: int = 0, autotune: bool = True):
        import torch
        self.streams = list(streams or DEFAULT_STREAMS)
        dev = torch.device("cuda", device)
        self.admission = Admission(self.streams, budget_bytes,
                                   lambda w, h: torch.empty((h, pitch_of(w)), dtype=torch.uint8, device=dev))
        net = None
        if use_proposal and os.path.exists(WEIGHTS) and PROPOSAL_SIZE in set(map(tuple, self.streams)):
            from .proposal import ProposalNet
            net = ProposalNet.load(WEIGHTS, device)
        self.executor = GpuExecutor(self.admission, sorted(set(map(tuple, self.streams))), net=net,
                                    workers=workers, max_batch=max_batch, device=device, autotune=autotune)
        self.max_batch = max_batch

    def serve(self, duration_s: float, fps: float = 30.0, seed: int = 42, rate_scale: float = 1.0,
              keep_peaks: bool = False) -> ServeStats:
        arr = poisson_arrivals(self.streams, duration_s, fps, seed, rate_scale)
        return Scheduler(self.admission, self.executor, self.max_batch).run(arr, keep_peaks)

    def close(self) -> None:
        self.executor.close()


def main():
    import argparse
    import json
    ap = argparse.ArgumentParser(description="8-camera serving loop")
    ap.add_argument("--seconds", type=float, default=60.0)
    ap.add_argument("--rate-scale", type=float, default=1.0)
    ap.add_argument("--workers", type=int, default=3)
    ap.add_argument("--max-batch", type=int, default=64)
    ap.add_argument("--no-proposal", action="store_true")
    a = ap.parse_args()
    from . import build
    build.build()
    srv = Server(workers=a.workers, max_batch=a.max_batch, use_proposal=not a.no_proposal)
    try:
        st = srv.serve(a.seconds, rate_scale=a.rate_scale)
        print(json.dumps({"seconds": a.seconds, "rate_scale": a.rate_scale, **summarize(st, srv.admission)}))
    finally:
        srv.close()


if __name__ == "__main__":
    main()
