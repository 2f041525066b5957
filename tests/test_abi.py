"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every function include/ld.h declares, and its pure
host logic (defaults, size rules, errors) behaves as documented."""
import ctypes
import os

import pytest

from paper_2212_09460_gb300 import build as ldbuild


@pytest.fixture(scope="module")
def ld():
    ldbuild.build()
    from paper_2212_09460_gb300 import ld as ldmod
    ldmod.load()
    return ldmod


def test_library_exports_every_header_symbol(ld):
    names = ld.header_functions()
    assert len(names) >= 10
    lib = ld.load()
    for n in names:
        assert hasattr(lib, n), n
    # and the binding exposes the same names
    for n in names:
        assert hasattr(ld, n), n


def test_struct_layouts_match_header(ld):
    assert ctypes.sizeof(ld.ld_params) == 40
    assert ctypes.sizeof(ld.ld_peak) == 12
    assert ctypes.sizeof(ld.ld_frame) == 24
    assert ctypes.sizeof(ld.ld_lines_params) == 16
    assert ctypes.sizeof(ld.ld_segment) == 24
    assert ctypes.sizeof(ld.ld_canny_params) == 16
    assert ctypes.sizeof(ld.ld_synth_stripe) == 64
    assert ctypes.sizeof(ld.ld_synth_frame) == 328


def test_params_default(ld):
    p = ld.ld_params_default()
    assert (p.n_theta, p.threshold, p.border, p.top_k, p.nms_theta, p.nms_rho, p.min_votes,
            p.reserved, p.edge_capacity) == (180, 128, 0, 4, 5, 5, 1, 0, 0)


@pytest.mark.parametrize("w,h,nt,D", [(640, 480, 180, 800), (1920, 1080, 360, 2203), (3840, 2160, 360, 4406),
                                      (512, 512, 180, 725), (3, 3, 2, 5)])
def test_query_sizes(ld, w, h, nt, D):
    acc, edges, d = ld.ld_query_sizes(w, h, ld.params(n_theta=nt))
    assert d == D and acc == nt * (2 * D + 1) and edges == w * h


@pytest.mark.parametrize("w,h", [(2, 10), (10, 2), (20000, 12768), (0, 5)])
def test_query_sizes_rejects_bad_sizes(ld, w, h):
    with pytest.raises(ld.LdError) as ei:
        ld.ld_query_sizes(w, h, ld.params())
    assert ei.value.status == ld.LD_ERR_INVALID
    assert "size" in str(ei.value) or "fit" in str(ei.value)


@pytest.mark.parametrize("kw", [dict(n_theta=181), dict(n_theta=0), dict(n_theta=8192), dict(threshold=0),
                                dict(threshold=256), dict(top_k=0), dict(top_k=17), dict(nms_theta=4),
                                dict(nms_rho=0), dict(border=2), dict(edge_capacity=-1)])
def test_bad_params_rejected(ld, kw):
    with pytest.raises(ld.LdError):
        ld.ld_query_sizes(64, 64, ld.params(**kw))


def test_ctx_create_without_gpu_fails_cleanly(ld):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(ld.LdError) as ei:
        ld.ld_ctx_create(0)
    assert ei.value.status in (ld.LD_ERR_CUDA, ld.LD_ERR_INVALID)
    assert ld.ld_last_error()


def test_header_documents_each_entry_point():
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "ld.h")).read()
    for sec in ("Eq. 1", "Eq. 3", "Eqs. 4-5", "Sec. 2.2", "Sec. 2.3"):
        assert sec in hdr
