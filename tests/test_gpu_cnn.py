"""The proposal network's GPU kernels against the CPU oracle (oracle/cnn.py).

The GPU stores activations and activation gradients in bf16 and accumulates
in fp32; the oracle runs in float64 on the same bf16-rounded conv weights.
Values are compared element by element.  A single tensor-core layer is held
to its worst-case rounding bound, |gpu - ref| <= u |ref| + (1 + u) gamma(K)
sum |terms| (bf16 unit roundoff u = 2^-8, fp32 sums of K terms).  Through the
whole network worst-case bounds compound far beyond the errors seen, so
there each element must lie within K_SIGMA = 8 standard deviations of the
rounding-error model that tests/cnn_bounds.py propagates (a faithful CPU
emulation of the kernels' arithmetic stays within 4 sigma at these sizes:
tests/test_cnn_bounds.py).  Also checked: the edge-count input map
(bit-exact), and that a frame's logits are bitwise the same alone and inside
a batch."""
import numpy as np
import pytest
import torch

import cnn_bounds as cb
import oracle.cnn as cnn
from paper_2212_09460_gb300 import synth

pytestmark = pytest.mark.gpu


def _within(name, got, ref, sigma):
    r = cb.worst(got, ref, sigma) / cb.K_SIGMA
    assert r <= 1.0, f"{name}: worst element at {r * cb.K_SIGMA:.2f} sigma (limit {cb.K_SIGMA})"
    return r * cb.K_SIGMA


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
    xf = x.astype(np.float64) / 64.0
    tgt = np.zeros((x.shape[0], 44))
    ref = cnn.intermediates(params, xf, tgt)
    sig = cb.forward_sigma(params, xf, cnn.CHANNELS, ref)
    seen = {}
    for i in range(4):
        got = acts.ys[i].float().cpu().numpy().transpose(0, 3, 1, 2)
        seen[f"a{i}"] = _within(f"conv{i + 1}", got, ref["a"][i], sig["a"][i])
    seen["feat"] = _within("features", acts.feat.cpu().numpy(), ref["feat"], sig["feat"])
    seen["logits"] = _within("logits", acts.logits.cpu().numpy(), ref["logits"], sig["logits"])
    print("forward, worst element in sigma:", {k: round(v, 2) for k, v in seen.items()})


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
    xf = x.astype(np.float64) / 64.0
    ref = cnn.intermediates(params, xf, tgt.astype(np.float64))
    fs = cb.forward_sigma(params, xf, cnn.CHANNELS, ref)
    bs = cb.backward_sigma(params, xf, cnn.CHANNELS, ref, fs)
    seen = {"loss": _within("loss", float(loss.item()), ref["loss"], cb.loss_sigma(ref, fs)),
            "dlogits": _within("dlogits", dl.cpu().numpy(), ref["dlogits"], bs["dlogits"])}
    for k in ["wh", "bh", "w3", "b3", "w2", "b2", "w1", "b1", "w0", "b0"]:
        seen[k] = _within("grad " + k, net.g[k].cpu().numpy(), ref["g"][k], bs["g"][k])
    print("backward, worst element in sigma:", {k: round(v, 2) for k, v in seen.items()})


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
    # sizes with ragged 16 x 8 output tiles, against the oracle's layer
    # (oracle.cnn.conv3x3_relu) on the same bf16 inputs and weights.  The only
    # errors are the fp32 sum of K = 9 cin + 1 terms and the bf16 rounding of
    # the output, so each element obeys the worst-case bound
    # |gpu - ref| <= u |ref| + (1 + u) gamma(K) sum |terms|.
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
    x64, w64, b64 = x.double().numpy(), wt.double().numpy(), b.double().numpy()
    ref = cnn.conv3x3_relu(x64, w64, b64, stride)
    terms = cnn.conv3x3_relu(np.abs(x64), np.abs(w64), np.abs(b64), stride)   # sum |terms| (all >= 0)
    bound = cb.U16 * np.abs(ref) + (1 + cb.U16) * cb.gamma(9 * cin + 1) * terms
    err = np.abs(y.float().cpu().numpy().astype(np.float64) - ref)
    assert (err <= bound).all(), float((err / np.maximum(bound, 1e-300)).max())


@pytest.mark.parametrize("cin,stride,h,w", [(16, 2, 37, 41), (32, 2, 20, 23), (16, 1, 19, 13), (32, 1, 17, 18),
                                            (32, 2, 68, 120)])
def test_tensor_core_conv_backward_matches_reference(ldlib, cin, stride, h, w):
    # every (channels, stride) form of the tcgen05 weight and input gradients,
    # at ragged sizes, against float64 sums of the same bf16 values.  The ReLU
    # mask is the GPU forward's own output (y > 0), applied on both sides, so
    # the only errors are fp32 sums (within a CTA on the tensor core, then of
    # the CTAs' partials in a fixed order) and, for dx, the bf16 rounding:
    # |gpu - ref| <= u |ref| + (1 + u) gamma(K) sum |terms| per element.
    rng = np.random.default_rng(cin * 1000 + stride * 100 + h)
    n = 2
    x = torch.from_numpy(rng.standard_normal((n, h, w, cin)).astype(np.float32)).to(torch.bfloat16)
    wt = torch.from_numpy(rng.uniform(-0.2, 0.2, (32, 3, 3, cin)).astype(np.float32)).to(torch.bfloat16)
    b = torch.from_numpy(rng.uniform(-0.1, 0.1, 32).astype(np.float32))
    oh, ow = (h - 1) // stride + 1, (w - 1) // stride + 1
    dy = torch.from_numpy(rng.standard_normal((n, oh, ow, 32)).astype(np.float32)).to(torch.bfloat16)
    xd, wd, bd, dyd = x.cuda().contiguous(), wt.cuda().contiguous(), b.cuda(), dy.cuda().contiguous()
    y = torch.empty((n, oh, ow, 32), dtype=torch.bfloat16, device="cuda")
    dx = torch.empty((n, h, w, cin), dtype=torch.bfloat16, device="cuda")
    dw = torch.zeros((32, 3, 3, cin), dtype=torch.float32, device="cuda")
    db = torch.zeros(32, dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    ldlib.ld_conv3x3_forward(xd.data_ptr(), n, h, w, cin, 32, stride, wd.data_ptr(), bd.data_ptr(), y.data_ptr(), s)
    ldlib.ld_conv3x3_backward(xd.data_ptr(), n, h, w, cin, 32, stride, wd.data_ptr(), y.data_ptr(), dyd.data_ptr(),
                              dx.data_ptr(), dw.data_ptr(), db.data_ptr(), s)
    torch.cuda.synchronize()
    assert ldlib.ld_conv_faults(0) == 0
    mask = (y.float().cpu() > 0).double()
    dz = (dy.double() * mask).permute(0, 3, 1, 2)             # NCHW
    x64 = x.double().permute(0, 3, 1, 2)
    w64 = wt.double().permute(0, 3, 1, 2)                     # [co][ci][3][3]
    gw = torch.nn.grad.conv2d_weight(x64, w64.shape, dz, stride=stride, padding=1)
    gw_abs = torch.nn.grad.conv2d_weight(x64.abs(), w64.shape, dz.abs(), stride=stride, padding=1)
    gx = torch.nn.grad.conv2d_input(x64.shape, w64, dz, stride=stride, padding=1)
    gx_abs = torch.nn.grad.conv2d_input(x64.shape, w64.abs(), dz.abs(), stride=stride, padding=1)
    ctas = ((oh * ow + 2047) // 2048) * n
    k_w = n * oh * ow + ctas                                   # terms of a weight-gradient sum
    got_w = dw.cpu().double().permute(0, 3, 1, 2)
    bound_w = (1 + cb.U16) * cb.gamma(k_w) * gw_abs
    assert ((got_w - gw).abs() <= bound_w).all(), float(((got_w - gw).abs() / bound_w.clamp_min(1e-300)).max())
    got_b, ref_b = db.cpu().double(), dz.sum(dim=(0, 2, 3))
    bound_b = (1 + cb.U16) * cb.gamma(k_w) * dz.abs().sum(dim=(0, 2, 3))
    assert ((got_b - ref_b).abs() <= bound_b).all()
    got_x = dx.float().cpu().double().permute(0, 3, 1, 2)
    bound_x = cb.U16 * gx.abs() + (1 + cb.U16) * cb.gamma(9 * 32) * gx_abs
    assert ((got_x - gx).abs() <= bound_x).all(), float(((got_x - gx).abs() / bound_x.clamp_min(1e-300)).max())


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
