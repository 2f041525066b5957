"""ld_hough_peaks_static, the peak search for callers that may not allocate.

A frame loop with a fixed deadline, or a host thread that must never block on
the GPU, cannot call cudaMalloc while it runs (cudaMalloc can synchronise the
device and has no latency bound).  ld_hough_peaks_static keeps its candidates
in a fixed array inside the library instead of a context buffer.  These tests
call it through the C ABI and check that it returns exactly what
ld_hough_peaks returns, on two calls in a row (the array keeps the previous
call's contents, which must not leak into the next result), and that it
refuses accumulators whose candidates would not fit the array.

This file is named so that pytest collects it after every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2212_09460_gb300 import synth

pytestmark = pytest.mark.gpu


def _static_peaks(ld, acc_dev, p, top_k=None):
    n_theta, n_rho = acc_dev.shape
    peaks = torch.full((p.top_k if p is not None else top_k, 3), -7, dtype=torch.int32, device=acc_dev.device)
    n = torch.full((1,), -7, dtype=torch.int32, device=acc_dev.device)
    ld.ld_hough_peaks_static(acc_dev.data_ptr(), n_theta, n_rho, p, peaks.data_ptr(), n.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    k = int(n.item())
    return peaks.cpu().numpy()[:k]


def _ctx_peaks(ctx, acc_dev, p):
    pk, n = ctx.hough_peaks(acc_dev, p)
    torch.cuda.synchronize()
    return pk.cpu().numpy()[: int(n.item())]


def _accumulators(ora):
    img = synth.road_frame(1001, 1920, 1080, synth.THROUGHPUT_1080P)
    real = ora.hough(ora.edge_list(ora.binarize(ora.sobel_mag(img))), 1920, 1080, 360)
    rng = np.random.default_rng(4)
    ties = rng.integers(0, 4, size=(180, 1601)).astype(np.int32)
    return real, ties


def test_static_peaks_match_context_peaks_twice(ctx, ldlib, ora):
    # both entry points, and the oracle's greedy (Sec. 2.3 "Hough Peak"), agree
    real, ties = _accumulators(ora)
    for acc, kw in ((real, dict(top_k=4)), (ties, dict(top_k=16, nms_theta=3, nms_rho=7, min_votes=2))):
        p = ldlib.params(**kw)
        acc_dev = torch.from_numpy(acc).cuda()
        ref = _ctx_peaks(ctx, acc_dev, p)
        np.testing.assert_array_equal(ref, ora.peaks(acc, p.top_k, p.nms_theta, p.nms_rho, p.min_votes))
        first = _static_peaks(ldlib, acc_dev, p)
        second = _static_peaks(ldlib, acc_dev, p)
        np.testing.assert_array_equal(first, ref)
        np.testing.assert_array_equal(second, ref)


def test_static_peaks_null_params_are_the_defaults(ctx, ldlib, ora):
    # p = NULL means the defaults (top_k 4, 5 x 5, min_votes 1), as for ld_hough_peaks
    real, _ = _accumulators(ora)
    acc_dev = torch.from_numpy(real).cuda()
    got = _static_peaks(ldlib, acc_dev, None, top_k=4)
    np.testing.assert_array_equal(got, ora.peaks(real, 4, 5, 5, 1))
    np.testing.assert_array_equal(got, _ctx_peaks(ctx, acc_dev, ldlib.params()))


def test_static_peaks_rejects_reserved_field(ldlib):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    p = ldlib.params()
    p.reserved = 1
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    peaks = torch.zeros((4, 3), dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(ldlib.LdError) as ei:
        ldlib.ld_hough_peaks_static(dummy.data_ptr(), 4, 4, p, peaks.data_ptr(), n.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert ei.value.status == ldlib.LD_ERR_INVALID


def test_static_peaks_alternating_inputs(ctx, ldlib, ora):
    # a small accumulator after a large one: stale candidates of the first
    # call sit in the array and must not show up in the second result
    real, ties = _accumulators(ora)
    small = ties[:7, :50].copy()
    p = ldlib.params(top_k=4)
    for acc in (real, small, real, small):
        acc_dev = torch.from_numpy(acc).cuda()
        np.testing.assert_array_equal(_static_peaks(ldlib, acc_dev, p), _ctx_peaks(ctx, acc_dev, p))


def test_static_peaks_rejects_oversize(ldlib):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    p = ldlib.params(top_k=16, nms_theta=5, nms_rho=5)     # M = 376
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    peaks = torch.zeros((16, 3), dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    # 4096 x 65535 cells -> 16384 chunks x 376 slots, far above the 131072 the array holds;
    # rejected on the host before anything is launched
    with pytest.raises(ldlib.LdError) as ei:
        ldlib.ld_hough_peaks_static(dummy.data_ptr(), 4096, 65535, p, peaks.data_ptr(), n.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert ei.value.status == ldlib.LD_ERR_INVALID
    assert "static buffer" in str(ei.value)
    assert ctypes.sizeof(ldlib.ld_params) == 40
