"""The proposal network's GPU kernels against the CPU oracle (oracle/cnn.py).

The GPU stores activations and activation gradients in bf16 and accumulates
in fp32, so values are compared within a bf16 tolerance: relative L2 error
below 2e-2 per tensor for the forward pass, 3e-2 for gradients.  Derivation:
bf16 unit roundoff u = 2^-9; an element of a conv weight gradient carries
about sqrt(5) u = 0.0044 relative error from the roundings along its
backward chain (activation, its gradient, the next layer's gradient ...), and
the weight-gradient sums cancel (sum of |terms| / |sum| of 3-7), giving
0.013-0.031.  The oracle runs in float64 on the same bf16-rounded
conv weights.  Also checked: the edge-count input map (bit-exact), and that a
frame's logits are bitwise the same alone and inside a batch."""
import numpy as np
import pytest
import torch

import oracle.cnn as cnn
from paper_2212_09460_gb300 import synth

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def _bf16_params(seed):
    p = cnn.init_params(seed)
    for i in range(4):
        p[f"w{i}"] = torch.tensor(p[f"w{i}"], dtype=torch.float32).to(torch.bfloat16).double().numpy()
        p[f"b{i}"] = np.random.default_rng(seed + i).uniform(-0.05, 0.1, size=p[f"b{i}"].shape)
    p["bh"] = np.random.default_rng(seed + 9).uniform(-0.1, 0.1, size=p["bh"].shape)
    return p


def _counts(seed, n):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 24, size=(n, 135, 240)).astype(np.uint8) * (rng.random((n, 135, 240)) < 0.5)


def _net(ld_mod, params):
    from paper_2212_09460_gb300.proposal import ProposalNet
    return ProposalNet({k: np.asarray(v, np.float32) for k, v in params.items()}, 0)


def test_edge_count_map_matches_oracle(ctx, ldlib, ora):
    frames = [synth.road_frame(1000 + i, 1920, 1080, synth.THROUGHPUT_1080P) for i in range(2)] + \
             [synth.road_frame(5, 333, 201, synth.LATENCY_640x480)]
    for f in frames:
        h, w = f.shape
        p = ldlib.params(n_theta=360, border=1)
        got = ctx.edge_pool([torch.from_numpy(synth.pitched(f)).cuda()], p, widths=[w])
        torch.cuda.synchronize()
        ref = cnn.count_pool8(ora.binarize(ora.sobel_mag(f, border=1), 128))
        np.testing.assert_array_equal(got.cpu().numpy()[0], ref)


def test_forward_matches_oracle(ldlib):
    params = _bf16_params(11)
    x = _counts(3, 3)
    net = _net(ldlib, params)
    acts = net.forward(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    assert ldlib.ld_conv_faults(0) == 0          # no tensor-core wait gave up
    ref_logits, ref_acts = cnn.forward(params, x.astype(np.float64) / 64.0, keep=True)
    for i in range(4):
        got = acts.ys[i].float().cpu().numpy().transpose(0, 3, 1, 2)
        assert _rel(got, ref_acts[i]) < 2e-2, i
    assert _rel(acts.feat.cpu().numpy(), ref_acts[4]) < 2e-2
    assert _rel(acts.logits.cpu().numpy(), ref_logits) < 2e-2


def test_backward_matches_oracle(ldlib):
    params = _bf16_params(12)
    x = _counts(4, 2)
    tgt = (np.random.default_rng(5).random((2, 44)) < 0.25).astype(np.float32)
    net = _net(ldlib, params)
    xd = torch.from_numpy(x).cuda()
    net.zero_grad()
    acts = net.forward(xd)
    loss, dl = net.loss(acts.logits, torch.from_numpy(tgt).cuda())
    net.backward(xd, acts, dl)
    torch.cuda.synchronize()
    ref_loss, ref_g = cnn.loss_and_grads(params, x.astype(np.float64) / 64.0, tgt.astype(np.float64))
    assert float(loss.item()) == pytest.approx(ref_loss, rel=1e-2)
    errs = {k: _rel(net.g[k].cpu().numpy(), ref_g[k]) for k in ["wh", "bh", "w3", "b3", "w2", "b2", "w1", "b1",
                                                                  "w0", "b0"]}
    assert max(errs.values()) < 3e-2, errs


def test_logits_are_batch_invariant(ldlib):
    params = _bf16_params(13)
    x = _counts(6, 4)
    net = _net(ldlib, params)
    full = net.forward(torch.from_numpy(x).cuda()).logits.cpu().numpy()
    for i in range(4):
        alone = net.forward(torch.from_numpy(x[i:i + 1]).cuda()).logits.cpu().numpy()
        np.testing.assert_array_equal(alone[0], full[i])
    mixed = net.forward(torch.from_numpy(x[[2, 0]]).cuda()).logits.cpu().numpy()
    np.testing.assert_array_equal(mixed, full[[2, 0]])


def test_training_reduces_loss(ldlib):
    # a few Adam steps on one fixed batch lower the loss (the optimiser and all
    # gradients point the right way)
    params = _bf16_params(14)
    x = torch.from_numpy(_counts(7, 8)).cuda()
    tgt = torch.from_numpy((np.random.default_rng(8).random((8, 44)) < 0.2).astype(np.float32)).cuda()
    net = _net(ldlib, params)
    first = float(net.train_step(x, tgt, lr=3e-3).item())
    for _ in range(40):
        last = float(net.train_step(x, tgt, lr=3e-3).item())
    assert last < 0.7 * first


@pytest.mark.parametrize("cin,stride,h,w", [(16, 2, 37, 41), (32, 2, 20, 23), (16, 1, 19, 13), (32, 1, 17, 18),
                                            (32, 2, 135, 240)])
def test_tensor_core_conv_matches_oracle(ldlib, cin, stride, h, w):
    # every (channels, stride) form of the tcgen05 forward convolution, at
    # sizes with ragged 16 x 8 output tiles, against float64 conv + ReLU
    rng = np.random.default_rng(cin * 100 + stride * 10 + h)
    x = torch.from_numpy(rng.standard_normal((2, h, w, cin)).astype(np.float32)).to(torch.bfloat16)
    wt = torch.from_numpy(rng.uniform(-0.2, 0.2, (32, 3, 3, cin)).astype(np.float32)).to(torch.bfloat16)
    b = torch.from_numpy(rng.uniform(-0.1, 0.1, 32).astype(np.float32))
    oh, ow = (h - 1) // stride + 1, (w - 1) // stride + 1
    y = torch.empty((2, oh, ow, 32), dtype=torch.bfloat16, device="cuda")
    xd, wd, bd = x.cuda().contiguous(), wt.cuda().contiguous(), b.cuda()
    ldlib.ld_conv3x3_forward(xd.data_ptr(), 2, h, w, cin, 32, stride, wd.data_ptr(), bd.data_ptr(), y.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert ldlib.ld_conv_faults(0) == 0
    ref = torch.nn.functional.conv2d(x.double().permute(0, 3, 1, 2), wt.double().permute(0, 3, 1, 2),
                                     b.double(), stride=stride, padding=1).relu().permute(0, 2, 3, 1).numpy()
    assert _rel(y.float().cpu().numpy(), ref) < 1e-2


@pytest.mark.parametrize("hw", [(135, 240), (70, 100)])
def test_fused_inference_equals_layer_calls(ctx, ldlib, hw):
    # ld_proposal_logits (conv1 fused into the tensor-core conv2) gives the
    # same bits as the separate layer calls the trainer uses
    params = _bf16_params(21)
    rng = np.random.default_rng(hw[0])
    x = (rng.integers(0, 40, size=(3,) + hw) * (rng.random((3,) + hw) < 0.4)).astype(np.uint8)
    net = _net(ldlib, params)
    xd = torch.from_numpy(x).cuda()
    ref = net.forward(xd).logits
    got = ctx.proposal_logits(xd, net)
    torch.cuda.synchronize()
    assert ldlib.ld_conv_faults(0) == 0
    np.testing.assert_array_equal(got.cpu().numpy(), ref.cpu().numpy())


def test_training_is_reproducible_and_resumes_exactly(ldlib, tmp_path):
    # gradients are reduced in a fixed order, so two runs give the same bits,
    # and a checkpoint with Adam's moments resumes the same trajectory
    params = _bf16_params(15)
    x = [torch.from_numpy(_counts(30 + i, 4)).cuda() for i in range(4)]
    tg = [torch.from_numpy((np.random.default_rng(40 + i).random((4, 44)) < 0.2).astype(np.float32)).cuda()
          for i in range(4)]

    def run(net, steps):
        return [float(net.train_step(x[i], tg[i], lr=2e-3).item()) for i in steps]

    a = _net(ldlib, params)
    la = run(a, range(4))
    b = _net(ldlib, params)
    lb = run(b, range(4))
    assert la == lb
    for k in a.p:
        assert torch.equal(a.p[k], b.p[k]), k
    c = _net(ldlib, params)
    lc = run(c, range(2))
    ck = str(tmp_path / "ck.npz")
    c.save(ck, with_optimizer=True)
    from paper_2212_09460_gb300.proposal import ProposalNet
    d = ProposalNet.load(ck, 0)
    assert d.step_count == 2
    lc += run(d, range(2, 4))
    assert lc == la
    for k in a.p:
        assert torch.equal(a.p[k], d.p[k]) and torch.equal(a.m[k], d.m[k]) and torch.equal(a.v[k], d.v[k]), k
