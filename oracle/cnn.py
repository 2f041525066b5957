"""CPU oracle of the learned theta-band proposal network (TEST INFRASTRUCTURE).

Only the tests, the smoke check and the benchmark's CPU baseline use this
module.  It is a plain float64 PyTorch-CPU statement of the network the
CUDA kernels train and run, with gradients from autograd:

  input   x [N, 1, 135, 240]: the binary edge map, box-downsampled 8x8: the
          number of edge pixels in each block divided by 64
  conv1   3x3, stride 1, pad 1, 1 -> 16, + bias, ReLU      -> [N, 16, 135, 240]
  conv2   3x3, stride 2, pad 1, 16 -> 32, + bias, ReLU     -> [N, 32, 68, 120]
  conv3   3x3, stride 2, pad 1, 32 -> 32, + bias, ReLU     -> [N, 32, 34, 60]
  conv4   3x3, stride 2, pad 1, 32 -> 32, + bias, ReLU     -> [N, 32, 17, 30]
  pool    adaptive average to 4 x 8 (bin i covers rows floor(i*17/4) ..
          ceil((i+1)*17/4) - 1, likewise columns)           -> 1024 features,
          ordered (bin row, bin column, channel)
  head    linear 1024 -> 44 logits: 36 theta bands of 5 degrees, 8 row bands
  loss    binary cross-entropy with logits, mean over the batch and the 44
          outputs

The paper has no learned component; this network is the proposal stage the
project adds in front of the Hough vote (it predicts which theta bands hold
the top peaks, so that voting can skip the others).
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

IN_H, IN_W = 135, 240
CHANNELS = [(1, 16, 1), (16, 32, 2), (32, 32, 2), (32, 32, 2)]   # (Cin, Cout, stride)
POOL_H, POOL_W = 4, 8
N_FEAT = 32 * POOL_H * POOL_W
N_THETA_BANDS, N_ROW_BANDS = 36, 8
N_OUT = N_THETA_BANDS + N_ROW_BANDS


def conv_out(n: int, stride: int) -> int:
    return (n + 2 - 3) // stride + 1


def init_params(seed: int = 0) -> dict:
    """He-uniform conv weights, zero biases, small head; float64 numpy arrays.
    Conv weights are [Cout][3][3][Cin] (the layout the kernels use)."""
    rng = np.random.default_rng(seed)
    p = {}
    for i, (ci, co, _) in enumerate(CHANNELS):
        bound = np.sqrt(6.0 / (9 * ci))
        p[f"w{i}"] = rng.uniform(-bound, bound, size=(co, 3, 3, ci))
        p[f"b{i}"] = np.zeros(co)
    bound = np.sqrt(1.0 / N_FEAT)
    p["wh"] = rng.uniform(-bound, bound, size=(N_OUT, N_FEAT))
    p["bh"] = np.zeros(N_OUT)
    return p


def _t(a, grad=False):
    return torch.tensor(np.asarray(a, dtype=np.float64), dtype=torch.float64, requires_grad=grad)


def forward(params: dict, x: np.ndarray, keep: bool = False):
    """Logits [N, 44] (and the activations if keep) for inputs x [N, 135, 240]."""
    with torch.no_grad():
        out, acts = _forward_t({k: _t(v) for k, v in params.items()}, _t(x))
    return (out.numpy(), [a.numpy() for a in acts]) if keep else out.numpy()


def _conv3x3_relu_t(h: torch.Tensor, w: torch.Tensor, b: torch.Tensor, stride: int) -> torch.Tensor:
    """One conv layer on NCHW: 3x3 cross-correlation, zero padding 1, the given
    stride, + bias, ReLU; w is [Cout][3][3][Cin] (the kernels' layout)."""
    return F.relu(F.conv2d(h, w.permute(0, 3, 1, 2), b, stride=stride, padding=1))


def conv3x3_relu(x: np.ndarray, w: np.ndarray, b: np.ndarray, stride: int) -> np.ndarray:
    """One conv layer of the network on NHWC input x [N][H][W][Cin] (float64):
    y[n, i, j, co] = relu(b[co] + sum_{ky, kx, ci} w[co, ky, kx, ci] *
    x[n, i*stride + ky - 1, j*stride + kx - 1, ci]) with x = 0 outside the input;
    returns NHWC [N][(H-1)//stride+1][(W-1)//stride+1][Cout]."""
    with torch.no_grad():
        y = _conv3x3_relu_t(_t(x).permute(0, 3, 1, 2), _t(w), _t(b), stride)
    return y.permute(0, 2, 3, 1).numpy()


def _forward_t(P: dict, x: torch.Tensor):
    h = x[:, None, :, :]
    acts = []
    for i, (_, _, s) in enumerate(CHANNELS):
        h = _conv3x3_relu_t(h, P[f"w{i}"], P[f"b{i}"], s)
        acts.append(h)
    g = F.adaptive_avg_pool2d(h, (POOL_H, POOL_W))    # [N, 32, 4, 8]
    feat = g.permute(0, 2, 3, 1).reshape(g.shape[0], -1)   # (bin row, bin col, channel)
    return feat @ P["wh"].T + P["bh"], acts + [feat]


def loss_and_grads(params: dict, x: np.ndarray, target: np.ndarray):
    """Mean BCE-with-logits loss and d loss / d param for every parameter."""
    P = {k: _t(v, grad=True) for k, v in params.items()}
    logits, _ = _forward_t(P, _t(x))
    loss = F.binary_cross_entropy_with_logits(logits, _t(target), reduction="mean")
    loss.backward()
    return float(loss.detach()), {k: v.grad.numpy() for k, v in P.items()}


def intermediates(params: dict, x: np.ndarray, target: np.ndarray) -> dict:
    """Every value of one forward and backward pass, for element-wise checks:
    z[i] (layer i's pre-activation, NCHW), a[i] (its ReLU output), dy[i] (d loss
    / d a[i]), feat, logits, dlogits (d loss / d logits), loss, and the
    parameter gradients g[name]."""
    P = {k: _t(v, grad=True) for k, v in params.items()}
    h = _t(x)[:, None, :, :]
    zs, acts = [], []
    for i, (_, _, s) in enumerate(CHANNELS):
        z = F.conv2d(h, P[f"w{i}"].permute(0, 3, 1, 2), P[f"b{i}"], stride=s, padding=1)
        h = F.relu(z)
        h.retain_grad()
        zs.append(z)
        acts.append(h)
    g = F.adaptive_avg_pool2d(h, (POOL_H, POOL_W))
    feat = g.permute(0, 2, 3, 1).reshape(g.shape[0], -1)
    logits = feat @ P["wh"].T + P["bh"]
    logits.retain_grad()
    loss = F.binary_cross_entropy_with_logits(logits, _t(target), reduction="mean")
    loss.backward()
    return {"z": [z.detach().numpy() for z in zs], "a": [a.detach().numpy() for a in acts],
            "dy": [a.grad.numpy() for a in acts], "feat": feat.detach().numpy(),
            "logits": logits.detach().numpy(), "dlogits": logits.grad.numpy(), "loss": float(loss.detach()),
            "g": {k: v.grad.numpy() for k, v in P.items()}}


def pool_bins(n_in: int, n_out: int):
    """Adaptive-pooling bins [start, end) along one axis."""
    return [(i * n_in // n_out, -(-(i + 1) * n_in // n_out)) for i in range(n_out)]


def count_pool8(binary: np.ndarray) -> np.ndarray:
    """Edge pixels per 8x8 block of a 0/255 map (ragged last blocks), uint8."""
    h, w = binary.shape
    ph, pw = -(-h // 8), -(-w // 8)
    pad = np.zeros((ph * 8, pw * 8), np.int64)
    pad[:h, :w] = binary == 255
    return pad.reshape(ph, 8, pw, 8).sum(axis=(1, 3)).astype(np.uint8)


def theta_band_targets(peaks: np.ndarray, n_theta: int = 360) -> np.ndarray:
    """Multi-hot [36]: the 5-degree bands that hold any of the peaks."""
    t = np.zeros(N_THETA_BANDS)
    for th, _, _ in peaks:
        t[int(th) * N_THETA_BANDS // n_theta] = 1.0
    return t


def row_band_targets(peaks: np.ndarray, w: int, h: int, n_theta: int = 360) -> np.ndarray:
    """Multi-hot [8]: the 135-row bands of the image that each peak's line
    rho = x cos(theta) + y sin(theta) crosses inside the frame."""
    D = int(np.ceil(np.hypot(w, h)))
    t = np.zeros(N_ROW_BANDS)
    ys = np.arange(h)
    for th, ri, _ in peaks:
        ang = np.pi * int(th) / n_theta
        rho = int(ri) - D
        c, s = np.cos(ang), np.sin(ang)
        if abs(c) > 1e-9:
            xs = (rho - ys * s) / c
            rows = ys[(xs >= 0) & (xs <= w - 1)]
        else:
            y0 = rho / s
            rows = ys[np.abs(ys - y0) <= 0.5] if 0 <= y0 <= h - 1 else ys[:0]
        for y in rows:
            t[min(int(y) * N_ROW_BANDS // h, N_ROW_BANDS - 1)] = 1.0
    return t
