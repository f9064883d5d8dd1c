"""The checked build (the library compiled with -DHMFSR_CHECKED): every global load and
store of the alignment and merge kernels is checked against the buffers of its call.
The tiny, ragged and edge-case parity inputs run through it: the device error word stays
0 and every output is bit-identical to the default build's.  The checker itself is
tested by shrinking the registered workspace (the kernels still touch only real memory,
but their last workspace accesses then count as outside, are not made, and must be
recorded)."""
import ctypes

import numpy as np
import pytest
import torch

import burstgen
import oracle
import paper_1905_03277_gb300 as hm
from paper_1905_03277_gb300 import _lib

pytestmark = pytest.mark.gpu
WL = 4095


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hm.build(checked=True)
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def C(dev):
    return _lib.open_library(_lib.CHECKED_LIB_PATH)


def ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def stream(dev):
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def ws_of(L, op, d, tile, scale, dev):
    n = L.hmfsr_workspace_size(op, ctypes.byref(d), tile, scale[0], scale[1])
    buf = torch.empty(n + 256, dtype=torch.uint8, device=dev)
    off = (-buf.data_ptr()) % 256
    return buf, buf[off:off + n]


def desc_of(raw, ref):
    n, h, w = raw.shape
    return _lib.BurstDesc(n, h, w, w, ref, 0, WL, 0)


def align_checked(C, raw, ref, ap, dev, quadfit=False):
    n, h, w = raw.shape
    d = desc_of(raw, ref)
    ty, tx = hm.n_tiles(h, w, ap.tile)
    motion = torch.empty((n, ty, tx, 2), dtype=torch.float32, device=dev)
    mint = torch.empty((n, ty, tx, 2), dtype=torch.int32, device=dev)
    _, ws = ws_of(C, _lib.OP_ALIGN, d, ap.tile, (1, 1), dev)
    fn = C.hmfsr_align_quadfit if quadfit else C.hmfsr_align
    pc = ap.c()
    _lib.check(fn(ptr(raw), ctypes.byref(d), ctypes.byref(pc), ptr(motion), ptr(mint), ptr(ws), ws.numel(),
                  stream(dev)), "checked align")
    return motion, mint


def merge_checked(C, raw, motion, p, scale, ref, dev, with_den=False, opts=None, table=None):
    n, h, w = raw.shape
    d = desc_of(raw, ref)
    ho, wo = hm.out_size(h, w, scale)
    rgb = torch.full((3, ho, wo), float("nan"), dtype=torch.float32, device=dev)
    den = torch.full((3, ho, wo), float("nan"), dtype=torch.float32, device=dev) if with_den else None
    _, ws = ws_of(C, _lib.OP_MERGE, d, p.tile, scale, dev)
    pc = p.c()
    if opts is not None:
        st = C.hmfsr_merge_ex(ptr(raw), ctypes.byref(d), ptr(motion), ctypes.byref(pc), ctypes.byref(opts), scale[0],
                              scale[1], ptr(rgb), ptr(den), ptr(ws), ws.numel(), stream(dev))
    elif table is not None:
        st = C.hmfsr_merge_noise(ptr(raw), ctypes.byref(d), ptr(motion), ctypes.byref(pc), ptr(table), scale[0],
                                 scale[1], ptr(rgb), ptr(den), ptr(ws), ws.numel(), stream(dev))
    else:
        st = C.hmfsr_merge(ptr(raw), ctypes.byref(d), ptr(motion), ctypes.byref(pc), scale[0], scale[1], ptr(rgb),
                           ptr(den), ptr(ws), ws.numel(), stream(dev))
    _lib.check(st, "checked merge")
    return (rgb, den) if with_den else rgb


def status(C, reset=True):
    torch.cuda.synchronize()
    line = ctypes.c_int(-1)
    _lib.check(C.hmfsr_check_status(int(reset), ctypes.byref(line)), "hmfsr_check_status")
    return line.value


def test_checked_alignment_stays_in_bounds(dev, C, tiny_burst):
    status(C)
    b = burstgen.make_burst(dict(n=4, h=136, w=200, gain=1.0, read=2.0, motion="global", scale=(1, 1)), seed=21)
    cases = [(tiny_burst["raw"], 0, hm.AlignParams()), (b["raw"], 2, hm.AlignParams()),
             (b["raw"], 0, hm.AlignParams(tile=32, radius=(2, 3, 4, 4))),
             (b["raw"], 1, hm.AlignParams(tile=8, n_levels=2, lk_iters=5)),
             (b["raw"], 3, hm.AlignParams(tile=64, n_levels=3, radius=(0, 7, 5, 4), lk_iters=1))]
    for raw, ref, ap in cases:
        raw = raw.to(dev)
        for quadfit in (False, True):
            got_m, got_i = align_checked(C, raw, ref, ap, dev, quadfit)
            want_m, want_i = hm.align(raw, ref, ap, with_int=True, subpixel="quadfit" if quadfit else "lk")
            assert status(C) == 0, (raw.shape, ref, ap, quadfit)
            assert torch.equal(got_i, want_i) and torch.equal(got_m, want_m)


def test_checked_merge_stays_in_bounds(dev, C, tiny_burst):
    status(C)
    raw = tiny_burst["raw"]
    mv = torch.from_numpy(oracle.align(raw.numpy())[1].astype(np.float32)).to(dev)
    raw = raw.to(dev)
    p = hm.MergeParams(noise_a=tiny_burst["gain"], noise_b=tiny_burst["read"] ** 2)
    for scale in [(1, 1), (3, 2), (2, 1)]:
        got, gden = merge_checked(C, raw, mv, p, scale, 0, dev, with_den=True)
        want, wden = hm.merge(raw, mv, p, scale, with_den=True)
        assert status(C) == 0, scale
        assert torch.equal(got, want) and torch.equal(gden, wden)
    # windows partly or wholly outside the frame, rejected tiles, ref != 0, one frame,
    # the smallest frame
    b = burstgen.make_burst(dict(n=5, h=136, w=200, gain=2.0, read=4.0, motion="global", scale=(1, 1)), seed=22)
    r2 = b["raw"].to(dev)
    p2 = hm.MergeParams(noise_a=b["gain"], noise_b=b["read"] ** 2)
    ty, tx = hm.n_tiles(136, 200, 16)
    rng = np.random.default_rng(0)
    m2 = rng.uniform(-3, 3, size=(5, ty, tx, 2)).astype(np.float32)
    m2[3, :3, :4] = (41.25, -37.5)
    m2[4, -2:, -3:] = (-250.0, 180.0)
    m2 = torch.from_numpy(m2).to(dev)
    for ref in (0, 3):
        for scale in [(1, 1), (3, 2), (2, 1)]:
            got = merge_checked(C, r2, m2, p2, scale, ref, dev)
            assert status(C) == 0, (ref, scale)
            assert torch.equal(got, hm.merge(r2, m2, p2, scale, ref))
    one = merge_checked(C, r2[:1].contiguous(), m2[:1].contiguous(), p2, (2, 1), 0, dev)
    assert status(C) == 0 and torch.equal(one, hm.merge(r2[:1].contiguous(), m2[:1].contiguous(), p2, (2, 1)))
    small = r2[:3, :4, :6].contiguous()
    sm = torch.zeros((3, 1, 1, 2), dtype=torch.float32, device=dev)
    got = merge_checked(C, small, sm, p2, (3, 2), 0, dev)
    assert status(C) == 0 and torch.equal(got, hm.merge(small, sm, p2, (3, 2)))


def test_checked_merge_options_stay_in_bounds(dev, C, tiny_burst):
    status(C)
    raw = tiny_burst["raw"].to(dev)
    mv = torch.from_numpy(oracle.align(tiny_burst["raw"].numpy())[1].astype(np.float32)).to(dev)
    p = hm.MergeParams(noise_a=tiny_burst["gain"], noise_b=tiny_burst["read"] ** 2)
    table = hm.noise_table(p.noise_a, p.noise_b, device=dev)
    got = merge_checked(C, raw, mv, p, (3, 2), 0, dev, table=table)
    assert status(C) == 0 and torch.equal(got, hm.merge_noise(raw, mv, table, p, (3, 2)))
    opts = _lib.MergeOptionsC(table.data_ptr(), 0.03)
    got = merge_checked(C, raw, mv, p, (2, 1), 0, dev, opts=opts)
    assert status(C) == 0 and torch.equal(got, hm.merge_ex(raw, mv, p, (2, 1), noise_table=table, hf_loss=0.03))


def test_checked_chunked_merge_stays_in_bounds(dev, C, tiny_burst):
    status(C)
    raw = tiny_burst["raw"].to(dev)
    mv = torch.from_numpy(oracle.align(tiny_burst["raw"].numpy())[1].astype(np.float32)).to(dev)
    p = hm.MergeParams(noise_a=tiny_burst["gain"], noise_b=tiny_burst["read"] ** 2)
    for scale, k, ref in [((1, 1), 3, 0), ((3, 2), 2, 5), ((2, 1), 7, 7)]:
        d = desc_of(raw, ref)
        ho, wo = hm.out_size(raw.shape[1], raw.shape[2], scale)
        rgb = torch.full((3, ho, wo), float("nan"), dtype=torch.float32, device=dev)
        n = C.hmfsr_merge_chunked_workspace_size(ctypes.byref(d), p.tile, scale[0], scale[1], k)
        buf = torch.empty(n + 256, dtype=torch.uint8, device=dev)
        off = (-buf.data_ptr()) % 256
        ws = buf[off:off + n]
        pc = p.c()
        _lib.check(C.hmfsr_merge_chunked(ptr(raw), ctypes.byref(d), ptr(mv), ctypes.byref(pc), scale[0], scale[1], k,
                                         ptr(rgb), None, ptr(ws), ws.numel(), stream(dev)), "checked chunked merge")
        assert status(C) == 0, (scale, k, ref)
        assert torch.equal(rgb, hm.merge(raw, mv, p, scale, ref))


def test_checked_one_call_path_stays_in_bounds(dev, C, tiny_burst):
    # hmfsr_align_merge: the alignment on the library's side stream, the preparation beside it
    status(C)
    raw = tiny_burst["raw"].to(dev)
    for scale, ref in [((1, 1), 0), ((3, 2), 4), ((2, 1), 7)]:
        ap = hm.AlignParams()
        p = hm.MergeParams(noise_a=tiny_burst["gain"], noise_b=tiny_burst["read"] ** 2)
        d = desc_of(raw, ref)
        n, h, w = raw.shape
        ty, tx = hm.n_tiles(h, w, p.tile)
        ho, wo = hm.out_size(h, w, scale)
        motion = torch.empty((n, ty, tx, 2), dtype=torch.float32, device=dev)
        rgb = torch.full((3, ho, wo), float("nan"), dtype=torch.float32, device=dev)
        _, ws = ws_of(C, _lib.OP_ALIGN_MERGE, d, p.tile, scale, dev)
        a, m = ap.c(), p.c()
        _lib.check(C.hmfsr_align_merge(ptr(raw), ctypes.byref(d), ctypes.byref(a), ctypes.byref(m), scale[0], scale[1],
                                       ptr(motion), None, ptr(rgb), None, ptr(ws), ws.numel(), stream(dev)),
                   "checked align_merge")
        assert status(C) == 0, (scale, ref)
        want_m = hm.align(raw, ref, ap)
        assert torch.equal(motion, want_m)
        assert torch.equal(rgb, hm.merge(raw, want_m, p, scale, ref))


def test_checker_records_an_access_outside_the_registered_workspace(dev, C, tiny_burst):
    status(C)
    raw = tiny_burst["raw"].to(dev)
    mv = torch.zeros((8, 16, 16, 2), dtype=torch.float32, device=dev)
    p = hm.MergeParams(noise_a=tiny_burst["gain"], noise_b=tiny_burst["read"] ** 2)
    _lib.check(C.hmfsr_check_shrink(1 << 20), "hmfsr_check_shrink")
    try:
        merge_checked(C, raw, mv, p, (1, 1), 0, dev)
        line = status(C)
    finally:
        _lib.check(C.hmfsr_check_shrink(0), "hmfsr_check_shrink")
    assert line > 0
    merge_checked(C, raw, mv, p, (1, 1), 0, dev)
    assert status(C) == 0
