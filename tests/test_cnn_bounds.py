"""The element-wise error bounds the GPU network tests use (tests/cnn_bounds.py),
checked on the CPU: a faithful bf16 emulation of the kernels' arithmetic stays
inside them, and plausible slips (a dropped tap, a lost ReLU mask, a
transposed weight) land outside them.  Also pins oracle.cnn.intermediates to
oracle.cnn.loss_and_grads and to the closed-form BCE gradient."""
import numpy as np
import pytest
import torch

import oracle.cnn as cnn
import cnn_bounds as cb


def _setup(seed, n=2, h=37, w=45):
    p = cnn.init_params(seed)
    rng = np.random.default_rng(seed + 100)
    for i in range(4):
        p[f"w{i}"] = torch.tensor(p[f"w{i}"], dtype=torch.float32).to(torch.bfloat16).double().numpy()
        p[f"b{i}"] = rng.uniform(-0.05, 0.1, size=p[f"b{i}"].shape)
    p["bh"] = rng.uniform(-0.1, 0.1, size=p["bh"].shape)
    counts = rng.integers(0, 40, size=(n, h, w)) * (rng.random((n, h, w)) < 0.5)
    x = counts.astype(np.float64) / 64.0
    t = (rng.random((n, 44)) < 0.25).astype(np.float64)
    return p, x, t


def _nchw(a):
    return np.asarray(a)


def _check_all(p, x, t, emu):
    ref = cnn.intermediates(p, x, t)
    fb = cb.forward_sigma(p, x, cnn.CHANNELS, ref)
    bb = cb.backward_sigma(p, x, cnn.CHANNELS, ref, fb)
    ratios = {}
    for i in range(4):
        ratios[f"a{i}"] = cb.worst(emu["a"][i], ref["a"][i], fb["a"][i])
    ratios["feat"] = cb.worst(emu["feat"], ref["feat"], fb["feat"])
    ratios["logits"] = cb.worst(emu["logits"], ref["logits"], fb["logits"])
    for i in range(4):
        ratios[f"dy{i}"] = cb.worst(emu["dy"][i], ref["dy"][i], bb["dy"][i])
    for k in ref["g"]:
        ratios["g_" + k] = cb.worst(emu["g"][k], ref["g"][k], bb["g"][k])
    ratios["loss"] = abs(emu["loss"] - ref["loss"]) / cb.loss_sigma(ref, fb)
    return {k: v / cb.K_SIGMA for k, v in ratios.items()}


def test_intermediates_agree_with_loss_and_grads():
    p, x, t = _setup(1)
    ref = cnn.intermediates(p, x, t)
    loss, g = cnn.loss_and_grads(p, x, t)
    assert ref["loss"] == pytest.approx(loss, rel=1e-14)
    for k in g:
        np.testing.assert_allclose(ref["g"][k], g[k], rtol=1e-12, atol=1e-15)
    # d mean-BCE / d logits = (sigmoid(l) - t) / (N * 44)
    sig = 1.0 / (1.0 + np.exp(-ref["logits"]))
    np.testing.assert_allclose(ref["dlogits"], (sig - t) / t.size, rtol=1e-12, atol=1e-18)
    # the ReLU outputs are relu of the pre-activations
    for z, a in zip(ref["z"], ref["a"]):
        np.testing.assert_array_equal(a, np.maximum(z, 0.0))


@pytest.mark.parametrize("seed", [2, 3])
def test_bf16_emulation_inside_bounds(seed):
    p, x, t = _setup(seed)
    emu = cb.emulate(p, x, t, cnn.CHANNELS)
    ratios = _check_all(p, x, t, emu)
    print({k: round(v * cb.K_SIGMA, 2) for k, v in ratios.items()})   # in units of sigma
    assert max(ratios.values()) <= 1.0, ratios


def test_slips_fall_outside_bounds():
    p, x, t = _setup(4)
    # a dropped tap in conv2 (its centre weight zeroed in the computation only)
    q = {k: v.copy() for k, v in p.items()}
    q["w1"][:, 1, 1, :] = 0.0
    r = _check_all(p, x, t, cb.emulate(q, x, t, cnn.CHANNELS))
    assert r["a1"] > 1.0
    # transposed kernel taps in conv3
    q = {k: v.copy() for k, v in p.items()}
    q["w2"] = np.ascontiguousarray(q["w2"].transpose(0, 2, 1, 3))
    r = _check_all(p, x, t, cb.emulate(q, x, t, cnn.CHANNELS))
    assert r["a2"] > 1.0
    # a wrong bias in the head
    q = {k: v.copy() for k, v in p.items()}
    q["bh"][7] += 0.01
    r = _check_all(p, x, t, cb.emulate(q, x, t, cnn.CHANNELS))
    assert r["logits"] > 1.0
