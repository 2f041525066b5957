"""The learned theta-band proposal network: parameters, forward, backward,
Adam, checkpoints.  Every computation runs in libld.so's kernels; this module
only owns the device buffers and orders the calls.

The paper has no learned stage.  The network predicts, from the 8x8
edge-count map of a frame (edge pixels per block), which 5-degree theta bands hold the frame's
top Hough peaks (36 logits) and which of 8 row bands their lines cross
(8 logits).  Voting restricted to the predicted bands finds exactly the
peaks of the full vote whenever the bands contain them (ld_detect_batch_
proposal), with the full vote as fallback when the network is unsure.
"""
from __future__ import annotations

import io
from dataclasses import dataclass

import numpy as np

from . import ld

LAYERS = [(1, 16, 1), (16, 32, 2), (32, 32, 2), (32, 32, 2)]   # (Cin, Cout, stride)
N_FEAT, N_OUT, N_THETA_BANDS, N_ROW_BANDS = 1024, 44, 36, 8


def conv_out(n: int, stride: int) -> int:
    return (n + 2 - 3) // stride + 1


def init_numpy(seed: int = 0) -> dict:
    """He-uniform conv weights, zero biases, small head (float32, numpy)."""
    rng = np.random.default_rng(seed)
    p = {}
    for i, (ci, co, _) in enumerate(LAYERS):
        bound = np.sqrt(6.0 / (9 * ci))
        p[f"w{i}"] = rng.uniform(-bound, bound, size=(co, 3, 3, ci)).astype(np.float32)
        p[f"b{i}"] = np.zeros(co, np.float32)
    bound = np.sqrt(1.0 / N_FEAT)
    p["wh"] = rng.uniform(-bound, bound, size=(N_OUT, N_FEAT)).astype(np.float32)
    p["bh"] = np.zeros(N_OUT, np.float32)
    return p


@dataclass
class Acts:
    ys: list        # conv outputs (bf16 NHWC) per layer
    shapes: list    # (h, w) of each conv output
    feat: object
    logits: object


class ProposalNet:
    """Parameters (fp32 masters, bf16 conv copies), Adam state and gradients on one device."""

    def __init__(self, params: dict | None = None, device=0, seed: int = 0):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device) if isinstance(device, int) else device
        src = params if params is not None else init_numpy(seed)
        ref = init_numpy(0)   # the shapes the kernels read (a wrong head size would be read out of bounds)
        if set(src) != set(ref) or any(np.shape(src[k]) != ref[k].shape for k in ref):
            raise ValueError("proposal network parameters do not have the expected names and shapes "
                             f"(head {N_OUT} x {N_FEAT})")
        self.p = {k: torch.tensor(np.asarray(v, np.float32), device=self.device).contiguous() for k, v in src.items()}
        self.g = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.m = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.v = {k: torch.zeros_like(v) for k, v in self.p.items()}
        self.w16 = {f"w{i}": self.p[f"w{i}"].to(torch.bfloat16).contiguous() for i in range(4)}
        self.step_count = 0

    # ---------------------------------------------------------------- io
    def state_numpy(self) -> dict:
        return {k: v.detach().cpu().numpy() for k, v in self.p.items()}

    def save(self, path: str, with_optimizer: bool = False) -> None:
        """Weights and the step count; with_optimizer also stores Adam's moments,
        so that training resumed from the file continues bit for bit."""
        buf = io.BytesIO()
        extra = {}
        if with_optimizer:
            for k in self.p:
                extra["adam_m_" + k] = self.m[k].detach().cpu().numpy()
                extra["adam_v_" + k] = self.v[k].detach().cpu().numpy()
        np.savez(buf, step=np.array(self.step_count), **self.state_numpy(), **extra)
        with open(path, "wb") as f:
            f.write(buf.getvalue())

    @classmethod
    def load(cls, path: str, device=0) -> "ProposalNet":
        z = np.load(path)
        net = cls({k: z[k] for k in z.files if k != "step" and not k.startswith("adam_")}, device)
        net.step_count = int(z["step"])
        for k in net.p:
            if "adam_m_" + k in z.files:
                net.m[k].copy_(net.torch.from_numpy(z["adam_m_" + k]))
                net.v[k].copy_(net.torch.from_numpy(z["adam_v_" + k]))
        return net

    def c_struct(self) -> "ld.ld_proposal_net":
        """Device pointers of the current weights, for ld_detect_batch_proposal."""
        s = ld.ld_proposal_net()
        for i in range(4):
            s.w[i] = self.w16[f"w{i}"].data_ptr()
            s.b[i] = self.p[f"b{i}"].data_ptr()
        s.wh, s.bh = self.p["wh"].data_ptr(), self.p["bh"].data_ptr()
        return s

    # ---------------------------------------------------------------- passes
    def _stream(self):
        return self.torch.cuda.current_stream(self.device).cuda_stream

    def forward(self, pool) -> Acts:
        """pool: uint8 [n][h][w] edge counts (0..64) on the device -> activations and logits [n][44]."""
        torch = self.torch
        n, h, w = pool.shape
        s = self._stream()
        x, ys, shapes = pool, [], []
        for i, (ci, co, st) in enumerate(LAYERS):
            oh, ow = conv_out(h, st), conv_out(w, st)
            y = torch.empty((n, oh, ow, co), dtype=torch.bfloat16, device=self.device)
            ld.ld_conv3x3_forward(x.data_ptr(), n, h, w, ci, co, st, self.w16[f"w{i}"].data_ptr(),
                                  self.p[f"b{i}"].data_ptr(), y.data_ptr(), s)
            ys.append(y)
            shapes.append((oh, ow))
            x, h, w = y, oh, ow
        feat = torch.empty((n, N_FEAT), dtype=torch.float32, device=self.device)
        logits = torch.empty((n, N_OUT), dtype=torch.float32, device=self.device)
        ld.ld_pool_head_forward(x.data_ptr(), n, h, w, self.p["wh"].data_ptr(), self.p["bh"].data_ptr(),
                                feat.data_ptr(), logits.data_ptr(), s)
        return Acts(ys, shapes, feat, logits)

    def backward(self, pool, acts: Acts, dlogits) -> None:
        """Accumulate dL/dparam into self.g for the loss gradient dlogits."""
        torch = self.torch
        s = self._stream()
        n, h0, w0 = pool.shape
        h4, w4 = acts.shapes[3]
        dy = torch.empty_like(acts.ys[3])
        ld.ld_pool_head_backward(acts.feat.data_ptr(), dlogits.data_ptr(), self.p["wh"].data_ptr(), n, h4, w4,
                                 self.g["wh"].data_ptr(), self.g["bh"].data_ptr(), dy.data_ptr(), s)
        for i in range(3, -1, -1):
            ci, co, st = LAYERS[i]
            x = pool if i == 0 else acts.ys[i - 1]
            h, w = (h0, w0) if i == 0 else acts.shapes[i - 1]
            dx = None if i == 0 else torch.empty_like(acts.ys[i - 1])
            ld.ld_conv3x3_backward(x.data_ptr(), n, h, w, ci, co, st, self.w16[f"w{i}"].data_ptr(),
                                   acts.ys[i].data_ptr(), dy.data_ptr(), dx.data_ptr() if dx is not None else None,
                                   self.g[f"w{i}"].data_ptr(), self.g[f"b{i}"].data_ptr(), s)
            dy = dx

    def loss(self, logits, target):
        """Mean BCE with logits -> (loss [1], dlogits) on the device."""
        torch = self.torch
        n, k = logits.shape
        out = torch.empty(1, dtype=torch.float32, device=self.device)
        dl = torch.empty_like(logits)
        ld.ld_bce_loss(logits.data_ptr(), target.data_ptr(), n, k, out.data_ptr(), dl.data_ptr(), self._stream())
        return out, dl

    def zero_grad(self) -> None:
        for v in self.g.values():
            v.zero_()

    def adam(self, lr: float = 2e-3, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8) -> None:
        self.step_count += 1
        s = self._stream()
        for k, v in self.p.items():
            p16 = self.w16[k].data_ptr() if k in self.w16 else None
            ld.ld_adam_step(v.data_ptr(), self.g[k].data_ptr(), self.m[k].data_ptr(), self.v[k].data_ptr(),
                            v.numel(), lr, b1, b2, eps, self.step_count, p16, s)

    def train_step(self, pool, target, lr: float = 2e-3):
        """One forward + backward + Adam step; returns the loss tensor [1]."""
        self.zero_grad()
        acts = self.forward(pool)
        loss, dl = self.loss(acts.logits, target)
        self.backward(pool, acts, dl)
        self.adam(lr)
        return loss
