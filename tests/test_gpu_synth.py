"""The device-side frame generator reproduces synth.road_frame byte for byte."""
import numpy as np
import pytest
import torch

from paper_2212_09460_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("specs", [
    [(0, 640, 480, synth.LATENCY_640x480), (1000, 1920, 1080, synth.THROUGHPUT_1080P)],
    [(7, 97, 61, synth.THROUGHPUT_1080P), (3, 3840, 2160, synth.THROUGHPUT_1080P), (11, 3, 3, synth.LATENCY_640x480),
     (12, 1280, 720, synth.THROUGHPUT_1080P)],
])
def test_device_generator_matches_host(ldlib, specs):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    bufs, _keep = ldlib.synth_frames_device(specs, torch.device("cuda", 0))
    torch.cuda.synchronize()
    for (seed, w, h, style), b in zip(specs, bufs):
        np.testing.assert_array_equal(b.cpu().numpy()[:, :w], synth.road_frame(seed, w, h, style),
                                      err_msg=f"seed {seed} {w}x{h}")
