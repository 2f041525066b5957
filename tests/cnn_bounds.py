"""Element-wise tolerances of the proposal network's bf16 kernels.

The GPU stores activations and activation gradients in bf16 (8 significant
bits, round to nearest: unit roundoff u = 2^-8) and accumulates in fp32.  The
oracle (oracle/cnn.py) runs in float64 on the same bf16 conv weights.  For
every tensor the GPU produces, this module propagates, element by element,
the standard deviation sigma of |gpu - oracle| under the usual model of
rounding errors as independent and uniform within half an ulp:

  storage rounding       bf16(v) - v has variance <= u^2 v^2 / 3
  fp32 sums of n terms   error <= gamma(n) * sum |terms|, gamma(n) = n u32 /
                         (1 - n u32), u32 = 2^-23 (twice fp32's 2^-24, which
                         also covers accumulators that truncate), counted as a
                         uniform error of that half-width
  conv / linear layers   input variances pass through W^2 (sums of
                         independent errors)
  average pool           variance / area^2 (the smallest bin, conservative)
  ReLU                   forward, the error passes where z > -K sigma(z);
                         backward, where |z| <= K sigma(z) the GPU's mask (read
                         from its own output) may differ from the oracle's, so
                         that element's gradient counts as an error of |dy|

A worst case over rounding directions compounds through |W| layer after
layer and grows far beyond the errors seen (about 10^5 times the measured
error on the logits), so the tests use K_SIGMA = 8 standard deviations per
element instead.  An error of one element that is wrong by more than a few
u times the magnitude its terms justify lands outside.  `emulate` runs the same
network in fp32 with bf16 storage on the CPU; the CPU tests check that it
stays inside K_SIGMA sigma and that planted slips do not.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

U16 = 2.0 ** -8
V16 = U16 * U16 / 3.0     # variance of a bf16 rounding error, relative to the value squared
U32 = 2.0 ** -23
K_SIGMA = 8.0             # tests accept |gpu - oracle| <= K_SIGMA * sigma per element
POOL_H, POOL_W = 4, 8


def gamma(n: int) -> float:
    return n * U32 / (1.0 - n * U32)


def _t(a):
    return torch.as_tensor(np.asarray(a, np.float64))


def _conv(x, w, s):         # x NCHW, w [Cout][3][3][Cin]
    return F.conv2d(x, w.permute(0, 3, 1, 2), stride=s, padding=1)


def _conv_t(g, w, s, shape):   # input gradient of _conv
    return torch.nn.grad.conv2d_input(shape, w.permute(0, 3, 1, 2), g, stride=s, padding=1)


def _corr(x, g, s, wshape):    # weight gradient of _conv, as [Cout][3][3][Cin]
    co, kh, kw, ci = wshape
    return torch.nn.grad.conv2d_weight(x, (co, ci, kh, kw), g, stride=s, padding=1).permute(0, 2, 3, 1)


def _pool(a):
    g = F.adaptive_avg_pool2d(a, (POOL_H, POOL_W))
    return g.permute(0, 2, 3, 1).reshape(g.shape[0], -1)


def _bin_areas(h4, w4):
    ys = [(i * h4 // POOL_H, -(-(i + 1) * h4 // POOL_H)) for i in range(POOL_H)]
    xs = [(j * w4 // POOL_W, -(-(j + 1) * w4 // POOL_W)) for j in range(POOL_W)]
    return min((b - a) * (d - c) for a, b in ys for c, d in xs)   # smallest bin: the larger variance


def forward_sigma(params, x, layers, ref):
    """Standard deviations of the GPU's forward values about the oracle's:
    dict with 'a' [4 x NCHW], 'z' (pre-activations), 'feat', 'logits'.
    x: [N][H][W] inputs (counts / 64, exact); ref: oracle.cnn.intermediates."""
    a_prev, v_prev = _t(x)[:, None], torch.zeros_like(_t(x)[:, None])
    out = {"a": [], "z": []}
    for i, (ci, co, s) in enumerate(layers):
        W, b = _t(params[f"w{i}"]), _t(params[f"b{i}"])
        mag = _conv(a_prev.abs(), W.abs(), s) + b.abs()[None, :, None, None]
        vz = _conv(v_prev, W * W, s) + (gamma(9 * ci + 2) * mag) ** 2 / 3.0
        a = _t(ref["a"][i])
        z = _t(ref["z"][i])
        # ReLU passes the error where z > 0; near 0 it passes part of it
        va = vz * (z > -K_SIGMA * vz.sqrt()).double() + V16 * a * a
        out["z"].append(vz.sqrt())
        out["a"].append(va.sqrt())
        a_prev, v_prev = a, va
    h4, w4 = a_prev.shape[2:]
    area = _bin_areas(h4, w4)
    feat = _t(ref["feat"])
    vfeat = _pool(v_prev) / area + (gamma(area + 1) * _pool(a_prev.abs())) ** 2 / 3.0
    wh, bh = _t(params["wh"]), _t(params["bh"])
    vl = vfeat @ (wh * wh).T + (gamma(feat.shape[1] + 2) * (feat.abs() @ wh.abs().T + bh.abs())) ** 2 / 3.0
    out["feat"], out["logits"] = vfeat.sqrt(), vl.sqrt()
    return out


def backward_sigma(params, x, layers, ref, fs):
    """Standard deviations of the GPU's backward values about the oracle's,
    given the forward ones fs: 'g' (parameter gradients), 'dy' (d loss / d ReLU
    output per layer), 'dlogits'.  Where |z| <= K_SIGMA sigma(z) the GPU's ReLU
    mask may differ from the oracle's: such an element's gradient counts as an
    error of up to |dy| (variance dy^2)."""
    nk = ref["logits"].size
    dl = _t(ref["dlogits"])
    vdl = (fs["logits"] / (4.0 * nk)) ** 2 + (8 * U32 / nk) ** 2
    feat, vfeat = _t(ref["feat"]), fs["feat"] ** 2
    n = feat.shape[0]
    g = {}
    g["wh"] = vdl.T @ (feat * feat) + (dl * dl).T @ vfeat + (gamma(n) * (dl.abs().T @ feat.abs())) ** 2 / 3.0
    g["bh"] = vdl.sum(0) + (gamma(n) * dl.abs().sum(0)) ** 2 / 3.0
    wh = _t(params["wh"])
    a4 = _t(ref["a"][3])
    n_, c4, h4, w4 = a4.shape
    area = _bin_areas(h4, w4)
    vdfeat = vdl @ (wh * wh) + (gamma(wh.shape[0] + 2) * (dl.abs() @ wh.abs())) ** 2 / 3.0

    def spread(v):   # adjoint of the average pool: sum over covering bins of v / area
        t = torch.zeros((n_, c4, h4, w4), dtype=torch.float64, requires_grad=True)
        (_pool(t) * v).sum().backward()
        return t.grad

    dy = _t(ref["dy"][3])
    vdy = spread(vdfeat) / area + V16 * dy * dy
    out_dy = [None] * len(layers)
    out_dy[3] = vdy.sqrt()
    for i in range(len(layers) - 1, -1, -1):
        ci, co, s = layers[i]
        W = _t(params[f"w{i}"])
        z, sz = _t(ref["z"][i]), fs["z"][i]
        amb = (z.abs() <= K_SIGMA * sz).double()
        dz = dy * (z > 0).double()
        vdz = vdy * (z > -K_SIGMA * sz).double() + amb * dy * dy
        a_in = _t(x)[:, None] if i == 0 else _t(ref["a"][i - 1])
        v_in = torch.zeros_like(a_in) if i == 0 else fs["a"][i - 1] ** 2
        m = dz.shape[0] * dz.shape[2] * dz.shape[3]
        wshape = tuple(W.shape)
        g[f"w{i}"] = (_corr(a_in * a_in, vdz, s, wshape) + _corr(v_in, dz * dz, s, wshape)
                      + (gamma(m + 2) * _corr(a_in.abs(), dz.abs(), s, wshape)) ** 2 / 3.0)
        g[f"b{i}"] = vdz.sum((0, 2, 3)) + (gamma(m + 2) * dz.abs().sum((0, 2, 3))) ** 2 / 3.0
        if i > 0:
            shape = a_in.shape
            dy_prev = _t(ref["dy"][i - 1])
            v = _conv_t(vdz, W * W, s, shape) + (gamma(9 * co + 2) * _conv_t(dz.abs(), W.abs(), s, shape)) ** 2 / 3.0
            vdy = v + V16 * dy_prev * dy_prev
            dy = dy_prev
            out_dy[i - 1] = vdy.sqrt()
    return {"g": {k: v.sqrt() for k, v in g.items()}, "dy": out_dy, "dlogits": vdl.sqrt()}


def loss_sigma(ref, fs):
    """sigma of the loss: |d loss / d logit| <= 1 / nk per logit."""
    nk = ref["logits"].size
    return float(np.sqrt((fs["logits"] ** 2).sum()) / nk + gamma(nk + 8) * (np.abs(ref["logits"]).mean() + 1.0))


def _bf16(t):
    return t.to(torch.bfloat16).to(torch.float32)


def emulate(params, x, target, layers):
    """The network computed the way the GPU kernels do, on the CPU: fp32
    arithmetic, bf16 storage of activations and activation gradients, ReLU
    masks read from the stored outputs.  Returns the same keys as the oracle's
    intermediates (NCHW activations) plus the parameter gradients."""
    f32 = lambda a: torch.as_tensor(np.asarray(a, np.float32))
    h = f32(x)[:, None]
    acts, ins = [], []
    for i, (ci, co, s) in enumerate(layers):
        ins.append(h)
        z = _conv(h, f32(params[f"w{i}"]), s) + f32(params[f"b{i}"])[None, :, None, None]
        h = _bf16(torch.relu(z))
        acts.append(h)
    feat = _pool(h)
    logits = feat @ f32(params["wh"]).T + f32(params["bh"])
    t = f32(target)
    nk = logits.numel()
    dl = (torch.sigmoid(logits) - t) / nk
    g = {"wh": dl.T @ feat, "bh": dl.sum(0)}
    n_, c4, h4, w4 = h.shape
    dfeat = dl @ f32(params["wh"])
    t4 = torch.zeros((n_, c4, h4, w4), dtype=torch.float32, requires_grad=True)
    (_pool(t4) * dfeat).sum().backward()
    dy = _bf16(t4.grad)
    dys = [None] * len(layers)
    dys[3] = dy
    for i in range(len(layers) - 1, -1, -1):
        ci, co, s = layers[i]
        W = f32(params[f"w{i}"])
        dz = dy * (acts[i] > 0).float()
        g[f"w{i}"] = _corr(ins[i], dz, s, tuple(W.shape))
        g[f"b{i}"] = dz.sum((0, 2, 3))
        if i > 0:
            dy = _bf16(_conv_t(dz, W, s, ins[i].shape))
            dys[i - 1] = dy
    ce = F.binary_cross_entropy_with_logits(logits, t, reduction="mean")
    return {"a": [a.numpy() for a in acts], "feat": feat.detach().numpy(), "logits": logits.detach().numpy(),
            "dy": [d.numpy() for d in dys], "g": {k: v.detach().numpy() for k, v in g.items()},
            "loss": float(ce)}


def worst(got, ref, bound):
    """max |got - ref| / bound over the elements (<= 1 means inside the bound)."""
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    b = np.asarray(bound, np.float64)
    return float(np.max(np.abs(got - ref) / np.maximum(b, 1e-300)))
