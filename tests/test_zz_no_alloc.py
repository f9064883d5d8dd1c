"""hmfsr_merge_static, the merge entry point that allocates nothing (its scratch is a
fixed array inside the library), gives the same image as hmfsr_merge with a caller
workspace, on two calls in a row (the shared scratch keeps the previous call's
contents), and rejects bursts too large for its scratch.  Collected last on purpose."""
import ctypes

import numpy as np
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
    bursts = [burstgen.make_burst(dict(n=6, h=192, w=256, gain=1.0, read=3.0, motion="global", scale=(1, 1)), seed=31),
              burstgen.make_burst(dict(n=4, h=128, w=160, gain=2.0, read=4.0, motion="global", scale=(1, 1)), seed=32)]
    for b, scale in zip(bursts, [(3, 2), (2, 1)]):   # two calls in a row, different bursts
        raw = b["raw"].to(dev)
        p = hm.MergeParams(noise_a=b["gain"], noise_b=b["read"] ** 2)
        motion = hm.align(raw, 0, hm.AlignParams())
        ref = hm.merge(raw, motion, p, scale)
        st, got = call_static(L, raw, motion, p, scale)
        torch.cuda.synchronize()
        assert st == 0, L.hmfsr_status_string(st)
        err = (got - ref).abs().cpu().numpy().reshape(3, -1)
        assert np.isfinite(got.cpu().numpy()).all()
        assert (err.max(axis=1) <= 1e-4 * WL).all() and (err.mean(axis=1) <= 1e-6 * WL).all()


def test_static_merge_rejects_too_large(dev):
    L = _lib.load()
    raw = torch.zeros((8, 3024, 4032), dtype=torch.uint16, device=dev)
    motion = torch.zeros((8, 189, 252, 2), dtype=torch.float32, device=dev)
    st, _ = call_static(L, raw, motion, hm.MergeParams(), (1, 1))
    assert st == -3
