"""hmfsr_merge_static, the merge entry point that allocates nothing (its scratch is a
fixed array inside the library), gives bit for bit the image hmfsr_merge gives with a
caller workspace, on calls in a row (the shared scratch keeps the previous call's
contents, here a larger burst's), and rejects bursts too large for its scratch.  The
binding's wrapper checks its tensors before anything reaches the library.  Collected
last on purpose."""
import ctypes

import pytest
import torch

import burstgen
import paper_1905_03277_gb300 as hm
from paper_1905_03277_gb300 import _lib

pytestmark = pytest.mark.gpu
WL = 4095


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hm.build()
    return torch.device("cuda:0")


def call_static(L, burst, motion, params, scale):
    n, h, w = burst.shape
    desc = _lib.BurstDesc(n, h, w, w, 0, 0, WL, 0)
    ho, wo = hm.out_size(h, w, scale)
    rgb = torch.full((3, ho, wo), float("nan"), dtype=torch.float32, device=burst.device)
    pc = params.c()
    st = L.hmfsr_merge_static(ctypes.c_void_p(burst.data_ptr()), ctypes.byref(desc),
                              ctypes.c_void_p(motion.data_ptr()), ctypes.byref(pc), scale[0], scale[1],
                              ctypes.c_void_p(rgb.data_ptr()), None,
                              ctypes.c_void_p(torch.cuda.current_stream(burst.device).cuda_stream))
    return st, rgb


def test_static_merge_matches_workspace_merge(dev):
    L = _lib.load()
    # the first call fills most of the shared scratch with a larger burst, so the smaller
    # calls after it run over stale contents; the static path runs the same kernels on the
    # same launches as hmfsr_merge with a workspace, so every output must be bit-identical
    big = burstgen.make_burst(dict(n=8, h=512, w=768, gain=1.5, read=3.0, motion="global", scale=(1, 1)), seed=30)
    bursts = [(big, (2, 1)),
              (burstgen.make_burst(dict(n=6, h=192, w=256, gain=1.0, read=3.0, motion="global", scale=(1, 1)),
                                   seed=31), (3, 2)),
              (burstgen.make_burst(dict(n=4, h=128, w=160, gain=2.0, read=4.0, motion="global", scale=(1, 1)),
                                   seed=32), (2, 1))]
    for b, scale in bursts:   # calls in a row, different bursts
        raw = b["raw"].to(dev)
        p = hm.MergeParams(noise_a=b["gain"], noise_b=b["read"] ** 2)
        motion = hm.align(raw, 0, hm.AlignParams())
        ref = hm.merge(raw, motion, p, scale)
        st, got = call_static(L, raw, motion, p, scale)
        torch.cuda.synchronize()
        assert st == 0, L.hmfsr_status_string(st)
        assert torch.isfinite(got).all()
        assert torch.equal(got, ref), f"max |diff| {(got - ref).abs().max().item()}"
        # the binding's wrapper gives the same image
        assert torch.equal(hm.merge_static(raw, motion, p, scale), ref)


def test_static_merge_wrapper_checks_before_any_launch(dev):
    raw = torch.zeros((4, 64, 96), dtype=torch.uint16, device=dev)
    good = torch.zeros((4, 4, 6, 2), dtype=torch.float32, device=dev)
    with pytest.raises(ValueError):
        hm.merge_static(raw, good.cpu())                       # motion on the host
    with pytest.raises(ValueError):
        hm.merge_static(raw.cpu(), good)                       # burst on the host
    with pytest.raises(ValueError):
        hm.merge_static(raw, good[:, :3].contiguous())         # too few tile rows
    with pytest.raises(ValueError):
        hm.merge_static(raw, good.double())                    # wrong dtype
    with pytest.raises(ValueError):
        hm.merge_static(raw, good.transpose(1, 2).contiguous().transpose(1, 2))   # not contiguous


def test_static_merge_rejects_too_large(dev):
    L = _lib.load()
    raw = torch.zeros((8, 3024, 4032), dtype=torch.uint16, device=dev)
    motion = torch.zeros((8, 189, 252, 2), dtype=torch.float32, device=dev)
    st, _ = call_static(L, raw, motion, hm.MergeParams(), (1, 1))
    assert st == -3
