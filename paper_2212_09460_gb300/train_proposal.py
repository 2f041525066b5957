"""Train the theta-band proposal network on the GPU, and evaluate it.

Training data: seeded synthetic 1920x1080 dashed-lane frames (the throughput
frame style) generated on the device, labelled by the plain path with the
1-pixel frame border cleared (so that the labels are the lane lines, not the
image border): 360 theta bins, 5x5 suppression, top-16 peaks, of which the
first 4 and every peak with at least 40% of the first one's votes count.
The counted set holds every band the top-4 peaks the proposal must find lie
in, plus the bands of other strong lane lines (a frame's 4th and 5th lane
edges often differ by a few votes, so which of them is in the top 4 is not
predictable from the image; restricted voting is exact for any superset).  Input: the 8x8 edge-count map of the same binary image.  Every step
(generation, Sobel, voting, targets, network forward/backward, Adam) runs in
libld.so's kernels.

  python -m paper_2212_09460_gb300.train_proposal --steps 25000 --batch 64 \
      --lr 3e-3 --out paper_2212_09460_gb300/weights/proposal_1080p.npz
  python -m paper_2212_09460_gb300.train_proposal --eval FILE --frames 10000

Training seeds: 1_000_000 + (i mod 200_000) (25000 steps of 64 = 8 epochs over
the 200k training frames); held-out evaluation seeds: 9_000_000 + i.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import ld, synth
from .proposal import ProposalNet

W, H, N_THETA, TOP_K = 1920, 1080, 360, 4
LABEL_TOP_K, LABEL_ALWAYS, LABEL_REL = 16, 4, 0.4
TRAIN_SEED0, EVAL_SEED0 = 1_000_000, 9_000_000
TRAIN_FRAMES = 200_000


class FrameSource:
    """Batches of device-generated frames (fixed buffers, reused)."""

    def __init__(self, torch, device, batch):
        self.torch, self.device, self.batch = torch, device, batch
        self.bufs = [torch.empty((H, W), dtype=torch.uint8, device=device) for _ in range(batch)]

    def fill(self, seeds):
        specs = [(int(s), W, H, synth.THROUGHPUT_1080P) for s in seeds]
        arr = ld.synth_descriptors(specs, self.bufs[: len(specs)])
        desc = self.torch.frombuffer(bytearray(bytes(arr)), dtype=self.torch.uint8).to(self.device)
        ld.ld_synth_frames(desc.data_ptr(), len(specs), self.torch.cuda.current_stream(self.device).cuda_stream)
        self._keep = desc
        return self.bufs[: len(specs)]


def labelled_batch(torch, ctx, src, seeds, p):
    frames = src.fill(seeds)
    pool = ctx.edge_pool(frames, p)
    p_lab = ld.params(n_theta=p.n_theta, top_k=LABEL_TOP_K, border=p.border)
    pk, npk, st = ctx.detect_batch(frames, p_lab)
    tgt = torch.empty((len(frames), 44), dtype=torch.float32, device=src.device)
    ld.ld_proposal_targets(pk.data_ptr(), npk.data_ptr(), len(frames), LABEL_TOP_K, W, H, N_THETA, LABEL_ALWAYS,
                           LABEL_REL, tgt.data_ptr(), torch.cuda.current_stream(src.device).cuda_stream)
    return frames, pool, tgt


def train(steps: int, batch: int, lr: float, out: str, seed: int = 0, log_every: int = 100,
          checkpoint_every: int = 0, resume: str | None = None, train_frames: int = TRAIN_FRAMES):
    """Train for `steps` steps of `batch` device-generated frames drawn from the
    train_frames training frames in order (step k uses frames
    TRAIN_SEED0 + (k*batch mod train_frames) ..., so more steps are more
    epochs over the same frames).  Every checkpoint_every steps the network
    and Adam's state go to out + ".ckpt.npz"; resume continues from such a
    file at its step, reproducing the uninterrupted run bit for bit."""
    import torch
    dev = torch.device("cuda", 0)
    p = ld.params(n_theta=N_THETA, top_k=TOP_K, border=ld.LD_BORDER_CLEAR)
    net = ProposalNet.load(resume, 0) if resume else ProposalNet(device=0, seed=seed)
    src = FrameSource(torch, dev, batch)
    log = []
    t0 = time.time()
    with ld.Context(0) as ctx:
        for step in range(net.step_count, steps):
            seeds = TRAIN_SEED0 + (step * batch + np.arange(batch)) % train_frames
            _, pool, tgt = labelled_batch(torch, ctx, src, seeds, p)
            cur_lr = lr * 0.5 * (1 + math.cos(math.pi * step / steps))      # cosine decay
            loss = net.train_step(pool, tgt, cur_lr)
            if step % log_every == 0 or step == steps - 1:
                log.append((step, float(loss.item())))
                print(json.dumps({"step": step, "loss": log[-1][1], "lr": cur_lr,
                                  "elapsed_s": round(time.time() - t0, 1)}), flush=True)
            if checkpoint_every and (step + 1) % checkpoint_every == 0:
                net.save(out + ".ckpt.npz", with_optimizer=True)
    net.save(out)
    return net, log


def evaluate(weights: str, frames: int, batch: int = 64, p_band=0.2, p_fallback=0.5, margin=2):
    """Proposal vs plain on held-out frames: peak agreement, fallback rate,
    voted fraction, and device time of both paths (frames resident)."""
    import torch
    dev = torch.device("cuda", 0)
    net = ProposalNet.load(weights, 0)
    p = ld.params(n_theta=N_THETA, top_k=TOP_K, border=ld.LD_BORDER_CLEAR)
    q = ld.proposal_params(p_band, p_fallback, margin)
    src = FrameSource(torch, dev, batch)
    agree = total = fallbacks = 0
    active = 0
    ms_plain = ms_prop = 0.0
    with ld.Context(0) as ctx:
        ctx.autotune(src.fill(EVAL_SEED0 + np.arange(batch)), p, iters=2)
        for b0 in range(0, frames, batch):
            n = min(batch, frames - b0)
            fr = src.fill(EVAL_SEED0 + b0 + np.arange(n))
            prep = ctx.prepare(fr)
            ctx.detect_batch(prep, p)
            ctx.detect_batch_proposal(prep, p, net, q)             # warm (first batch: scratch)
            e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            e[0].record()
            plain = ctx.detect_batch(prep, p)
            e[1].record()
            e[2].record()
            prop = ctx.detect_batch_proposal(prep, p, net, q)
            e[3].record()
            torch.cuda.synchronize()
            ms_plain += e[0].elapsed_time(e[1])
            ms_prop += e[2].elapsed_time(e[3])
            ppk, pn, pst = (t.cpu().numpy() for t in plain)
            qpk, qn, qst, qfb, qact = (t.cpu().numpy() for t in prop)
            assert (pst == 0).all() and (qst == 0).all()
            for i in range(n):
                total += 1
                agree += int(pn[i] == qn[i] and np.array_equal(ppk[i, : pn[i]], qpk[i, : qn[i]]))
            fallbacks += int(qfb.sum())
            active += int(qact.sum())
    return {"frames": total, "agreement": agree / total, "fallback_rate": fallbacks / total,
            "voted_theta_fraction": active / total / (N_THETA // 2),
            "plain_frames_per_s": total / (ms_plain / 1e3), "proposal_frames_per_s": total / (ms_prop / 1e3),
            "p_band": p_band, "p_fallback": p_fallback, "margin": margin}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=25000)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--out", default="proposal_1080p.npz")
    ap.add_argument("--eval", default=None, help="weights file to evaluate instead of training")
    ap.add_argument("--frames", type=int, default=10000)
    ap.add_argument("--p-band", type=float, default=0.2)
    ap.add_argument("--p-fallback", type=float, default=0.5)
    ap.add_argument("--margin", type=int, default=2)
    ap.add_argument("--checkpoint-every", type=int, default=0, help="steps between resumable checkpoints")
    ap.add_argument("--resume", default=None, help="checkpoint (network + Adam state) to continue from")
    a = ap.parse_args()
    from . import build
    build.build()
    if a.eval:
        print(json.dumps(evaluate(a.eval, a.frames, a.batch, a.p_band, a.p_fallback, a.margin)))
    else:
        train(a.steps, a.batch, a.lr, a.out, checkpoint_every=a.checkpoint_every, resume=a.resume)


if __name__ == "__main__":
    main()
