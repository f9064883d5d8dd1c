"""The C-ABI library builds, loads, exports what include/hmfsr.h declares, and rejects bad
arguments on the host before any launch.  No GPU needed (no compute call is made)."""
import ctypes
import os
import re

import pytest

import paper_1905_03277_gb300 as hm
from paper_1905_03277_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    hm.build()
    return _lib.load()


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(hmfsr_[a-z0-9_]+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert {"hmfsr_align", "hmfsr_merge", "hmfsr_workspace_size"} <= names
    for n in names:
        assert hasattr(L, n), n
    assert set(_lib.EXPORTS) <= names


def test_default_build_has_no_checker(L):
    # the checker's entry points answer "unsupported" outside the checked build
    line = ctypes.c_int(0)
    assert L.hmfsr_check_status(0, ctypes.byref(line)) == -2
    assert L.hmfsr_check_shrink(0) == -2


def test_status_strings(L):
    assert L.hmfsr_status_string(0) == b"ok"
    assert b"workspace" in L.hmfsr_status_string(-3)
    assert L.hmfsr_version().startswith(b"0.")


def desc(n=8, h=256, w=256, pitch=None, ref=0, cfa=0, wl=4095, bl=0):
    return _lib.BurstDesc(n, h, w, pitch or w, ref, cfa, wl, bl)


def test_workspace_size_queries(L):
    d = desc()
    ws_m = L.hmfsr_workspace_size(_lib.OP_MERGE, ctypes.byref(d), 16, 1, 1)
    ws_a = L.hmfsr_workspace_size(_lib.OP_ALIGN, ctypes.byref(d), 16, 1, 1)
    hw = 128 * 128
    # sums 8 B + kernel 16 B + Rhat 4 B per half-res pixel per frame, plus base stats
    assert ws_m >= 8 * hw * 28 + 16 * hw
    assert ws_a >= 8 * hw * 2
    assert L.hmfsr_workspace_size(_lib.OP_MERGE, ctypes.byref(d), 16, 1, 2) == 0      # scale < 1
    assert L.hmfsr_workspace_size(_lib.OP_MERGE, ctypes.byref(d), 12, 1, 1) == 0      # unsupported tile
    assert L.hmfsr_workspace_size(_lib.OP_MERGE, ctypes.byref(desc(h=255)), 16, 1, 1) == 0
    assert L.hmfsr_workspace_size(99, ctypes.byref(d), 16, 1, 1) == 0


def _merge_call(L, d, params=None, snum=1, sden=1, burst=16, motion=16, rgb=16, ws=256, ws_bytes=1 << 40):
    p = params or hm.MergeParams().c()
    return L.hmfsr_merge(ctypes.c_void_p(burst) if burst else None, ctypes.byref(d) if d else None,
                         ctypes.c_void_p(motion) if motion else None, ctypes.byref(p), snum, sden,
                         ctypes.c_void_p(rgb) if rgb else None, None, ctypes.c_void_p(ws) if ws else None,
                         ws_bytes, None)


def test_merge_rejects_bad_arguments_on_host(L):
    # every case returns before any launch, so fake (never dereferenced) pointers are safe
    assert _merge_call(L, None) == -1
    assert _merge_call(L, desc(h=7)) == -1
    assert _merge_call(L, desc(ref=8)) == -1
    assert _merge_call(L, desc(pitch=100)) == -1
    assert _merge_call(L, desc(wl=9000)) == -1
    assert _merge_call(L, desc(cfa=1)) == -2
    assert _merge_call(L, desc(bl=64)) == -2
    assert _merge_call(L, desc(), burst=0) == -1
    assert _merge_call(L, desc(), burst=17) == -1          # misaligned burst pointer
    assert _merge_call(L, desc(), rgb=0) == -1
    assert _merge_call(L, desc(), snum=1, sden=2) == -1
    assert _merge_call(L, desc(), snum=9, sden=1) == -1
    bad = hm.MergeParams(k_detail=0.0).c()
    assert _merge_call(L, desc(), params=bad) == -1
    bad = hm.MergeParams(noise_a=float("nan")).c()
    assert _merge_call(L, desc(), params=bad) == -1
    bad = hm.MergeParams(tile=24).c()
    assert _merge_call(L, desc(), params=bad) == -1
    assert _merge_call(L, desc(), ws=0) == -3
    assert _merge_call(L, desc(), ws=128) == -3             # misaligned workspace
    assert _merge_call(L, desc(), ws_bytes=1000) == -3     # too small


def test_merge_rejects_empty_and_oversized_bursts_on_host(L):
    # sizes the 32-bit in-frame offsets and 16-bit guide sums cannot hold, and empty or
    # degenerate bursts: all rejected before any launch
    assert _merge_call(L, desc(n=0)) == -1
    assert _merge_call(L, desc(n=4097)) == -1
    assert _merge_call(L, desc(h=2)) == -1
    assert _merge_call(L, desc(w=0)) == -1
    assert _merge_call(L, desc(h=-256)) == -1
    assert _merge_call(L, desc(w=65538)) == -1              # wider than 65536
    assert _merge_call(L, desc(h=32768, w=65536)) == -1     # 2^31 samples in one frame
    assert _merge_call(L, desc(h=4096, w=4096, pitch=524288)) == -1
    assert _merge_call(L, desc(ref=-1)) == -1
    assert _merge_call(L, desc(wl=0)) == -1
    assert _merge_call(L, desc(wl=7282)) == -1              # 9 x WL must fit 16 bits
    assert L.hmfsr_workspace_size(_lib.OP_MERGE, ctypes.byref(desc(w=65538)), 16, 1, 1) == 0
    assert L.hmfsr_workspace_size(_lib.OP_MERGE, ctypes.byref(desc(n=0)), 16, 1, 1) == 0


def test_align_rejects_bad_arguments_on_host(L):
    d = desc()

    def call(p, motion=16, ws_bytes=1 << 40):
        pc = p.c()
        return L.hmfsr_align(ctypes.c_void_p(16), ctypes.byref(d), ctypes.byref(pc),
                             ctypes.c_void_p(motion) if motion else None, None, ctypes.c_void_p(256), ws_bytes, None)

    assert call(hm.AlignParams(tile=12)) == -1
    assert call(hm.AlignParams(n_levels=0)) == -1
    assert call(hm.AlignParams(n_levels=5)) == -1
    assert call(hm.AlignParams(radius=(1, 9, 4, 4))) == -1
    assert call(hm.AlignParams(lk_iters=-1)) == -1
    assert call(hm.AlignParams(), motion=0) == -1
    assert call(hm.AlignParams(), ws_bytes=10) == -3


def test_align_merge_rejects_bad_arguments_on_host(L):
    d = desc()
    ws_a = L.hmfsr_workspace_size(_lib.OP_ALIGN, ctypes.byref(d), 16, 1, 1)
    ws_m = L.hmfsr_workspace_size(_lib.OP_MERGE, ctypes.byref(d), 16, 2, 1)
    assert L.hmfsr_workspace_size(_lib.OP_ALIGN_MERGE, ctypes.byref(d), 16, 2, 1) == ws_a + ws_m
    assert L.hmfsr_workspace_size(_lib.OP_ALIGN_MERGE, ctypes.byref(d), 16, 1, 2) == 0

    def call(ap=None, mp=None, snum=1, sden=1, motion=16, rgb=16, ws_bytes=1 << 40, dd=d):
        a, m = (ap or hm.AlignParams()).c(), (mp or hm.MergeParams()).c()
        v = lambda x: ctypes.c_void_p(x) if x else None
        return L.hmfsr_align_merge(v(16), ctypes.byref(dd), ctypes.byref(a), ctypes.byref(m), snum, sden, v(motion),
                                   None, v(rgb), None, v(256), ws_bytes, None)

    # every case returns before any CUDA call (fake pointers, never dereferenced)
    assert call(ap=hm.AlignParams(tile=32)) == -1            # alignment and merge tiles differ
    assert call(ap=hm.AlignParams(tile=32), mp=hm.MergeParams(tile=16)) == -1
    assert call(ap=hm.AlignParams(n_levels=0)) == -1
    assert call(mp=hm.MergeParams(k_shrink=-1.0)) == -1
    assert call(snum=1, sden=2) == -1
    assert call(motion=0) == -1
    assert call(motion=20) == -1                              # motion not 8-byte aligned
    assert call(rgb=0) == -1
    assert call(dd=desc(cfa=1)) == -2
    assert call(ws_bytes=ws_a + ws_m - 1) == -3


def test_chunked_workspace_does_not_grow_with_the_frame_count(L):
    # the bounded-memory merge's workspace depends on the chunk size and the output size,
    # not on the frame count (Sec. 6, Table 2)
    size = lambda n, k, sc=(1, 1): L.hmfsr_merge_chunked_workspace_size(ctypes.byref(desc(n=n, h=512, w=768)), 16,
                                                                        sc[0], sc[1], k)
    assert size(8, 2) == size(40, 2) == size(4096, 2) > 0
    assert size(3, 2) == size(8, 2) and size(2, 2) < size(3, 2)
    assert size(8, 1) < size(8, 2) < size(8, 4)
    assert size(8, 2, (2, 1)) > size(8, 2)
    resident = lambda n: L.hmfsr_workspace_size(_lib.OP_MERGE, ctypes.byref(desc(n=n, h=512, w=768)), 16, 1, 1)
    assert size(40, 2) < resident(40)
    assert size(8, 0) == 0 and size(8, 4097) == 0 and size(8, 2, (1, 2)) == 0


def test_chunked_merge_rejects_bad_arguments_on_host(L):
    d = desc()
    p = hm.MergeParams().c()

    def call(k=2, ws_bytes=1 << 40, motion=16):
        v = lambda x: ctypes.c_void_p(x) if x else None
        return L.hmfsr_merge_chunked(v(16), ctypes.byref(d), v(motion), ctypes.byref(p), 1, 1, k, v(16), None, v(256),
                                     ws_bytes, None)

    need = L.hmfsr_merge_chunked_workspace_size(ctypes.byref(d), 16, 1, 1, 2)
    assert call(k=0) == -1 and call(k=-3) == -1 and call(k=5000) == -1
    assert call(motion=0) == -1
    assert call(ws_bytes=need - 1) == -3


def test_product_path_does_not_use_the_oracle():
    src_dir = os.path.join(ROOT, "paper_1905_03277_gb300")
    for fn in os.listdir(src_dir):
        if fn.endswith(".py"):
            txt = open(os.path.join(src_dir, fn)).read()
            assert "import oracle" not in txt and "from oracle" not in txt, fn


def test_load_fails_loudly_without_library(tmp_path):
    saved = _lib._lib
    _lib._lib = None
    try:
        with pytest.raises(RuntimeError, match="libhmfsr.so not found"):
            _lib.load(str(tmp_path / "missing.so"))
    finally:
        _lib._lib = saved


def test_batch_plan_validation_on_host(L):
    # plan creation is host work only
    p = hm.BatchPlan([(4, 64, 96), (3, 128, 128)], hm.MergeParams(), [(1, 1), (3, 2)], [0, 2])
    assert p.ws_bytes > 0
    with pytest.raises(RuntimeError, match="invalid argument"):
        hm.BatchPlan([(4, 63, 96)])                       # odd height
    with pytest.raises(RuntimeError, match="invalid argument"):
        hm.BatchPlan([(4, 64, 96)], hm.MergeParams(tile=32))  # batches use tile 16
    with pytest.raises(RuntimeError, match="invalid argument"):
        hm.BatchPlan([(4, 64, 96)], refs=4)                # ref out of range
    with pytest.raises(RuntimeError, match="invalid argument"):
        p.configure(merge_tile_w=48)                       # must divide 128


def test_batch_vectors_rejects_bad_arguments(L):
    # fake, never dereferenced pointers: every case returns before any copy
    p = hm.BatchPlan([(4, 64, 96)])
    ws, dst = ctypes.c_void_p(256), ctypes.c_void_p(512)
    assert L.hmfsr_batch_vectors(None, ws, 0, dst, None) == -1
    assert L.hmfsr_batch_vectors(p._h, None, 0, dst, None) == -1
    assert L.hmfsr_batch_vectors(p._h, ws, 0, None, None) == -1
    assert L.hmfsr_batch_vectors(p._h, ws, 1, dst, None) == -1        # burst index outside the plan
    assert L.hmfsr_batch_vectors(p._h, ws, -1, dst, None) == -1
    assert L.hmfsr_batch_vectors(p._h, ws, 0, ctypes.c_void_p(514), None) == -1   # misaligned
    with pytest.raises(RuntimeError):
        p.vectors(0)                                                 # not run yet
    out = (ctypes.c_ulonglong * 42)()
    assert L.hmfsr_batch_stage_profile(None, ws, out, 42, None) == -1
    assert L.hmfsr_batch_stage_profile(p._h, None, out, 42, None) == -1
    assert L.hmfsr_batch_stage_profile(p._h, ws, out, 41, None) == -1     # too short
    assert L.hmfsr_batch_set_profile(None, 1) == -1


def test_snr_tuning_through_the_abi_matches_the_oracle(L):
    # host-only entry point: no GPU needed
    import oracle
    # (sum, count): whole means and a 12-MP frame's ragged quotient
    for (ssum, cnt), a, b in [((200, 4), 4.0, 36.0), ((700, 1), 2.0, 9.0), ((6000, 4), 4.0, 36.0),
                              ((3240, 1), 10.0, 0.0), ((4000, 1), 0.5, 4.0), ((800, 1), 0.0, 0.0),
                              ((0, 7), 1.0, 1.0), ((17_654_321_987, 12_192_768), 4.0, 36.0)]:
        mean = ssum / cnt
        mp, ap, snr = hm.snr_tuning(ssum, cnt, a, b)
        want = oracle.snr_tuning(mean, a, b)
        assert snr == want["snr"]
        assert mp.tile == ap.tile == want["tile"]
        for k in ("k_detail", "k_denoise", "d_th", "d_tr", "k_stretch", "k_shrink", "t", "s1", "s2", "m_th"):
            assert getattr(mp, k) == pytest.approx(want[k], rel=1e-7, abs=1e-12), k
        assert (mp.noise_a, mp.noise_b) == (a, b)
        assert (ap.n_levels, ap.radius, ap.lk_iters) == (4, (1, 4, 4, 4), 3)


def test_tuning_entry_points_reject_bad_arguments(L):
    mp, ap = _lib.MergeParamsC(), _lib.AlignParamsC()
    assert L.hmfsr_snr_tuning(10, 0, 1.0, 1.0, ctypes.byref(mp), ctypes.byref(ap), None) == -1       # no samples
    assert L.hmfsr_snr_tuning(1 << 53, 1, 1.0, 1.0, ctypes.byref(mp), ctypes.byref(ap), None) == -1  # sum not exact
    assert L.hmfsr_snr_tuning(10, 1, float("nan"), 1.0, ctypes.byref(mp), ctypes.byref(ap), None) == -1
    assert L.hmfsr_snr_tuning(10, 1, -1.0, 1.0, ctypes.byref(mp), ctypes.byref(ap), None) == -1
    assert L.hmfsr_snr_tuning(10, 1, 1.0, 1.0, None, ctypes.byref(ap), None) == -1
    d = desc(n=2)
    # fake, never dereferenced pointers: every case returns before any launch
    assert L.hmfsr_frame_sum(ctypes.c_void_p(16), ctypes.byref(d), 2, ctypes.c_void_p(256), None) == -1
    assert L.hmfsr_frame_sum(ctypes.c_void_p(16), ctypes.byref(d), -1, ctypes.c_void_p(256), None) == -1
    assert L.hmfsr_frame_sum(ctypes.c_void_p(16), ctypes.byref(d), 0, ctypes.c_void_p(260), None) == -1
    assert L.hmfsr_frame_sum(None, ctypes.byref(d), 0, ctypes.c_void_p(256), None) == -1


def test_noise_table_entry_points_reject_bad_arguments(L):
    # fake, never dereferenced pointers: every case returns before any launch
    assert L.hmfsr_noise_table(1.0, 4.0, 4095, None, None) == -1
    assert L.hmfsr_noise_table(1.0, 4.0, 4095, ctypes.c_void_p(264), None) == -1      # not 16-byte aligned
    assert L.hmfsr_noise_table(-1.0, 4.0, 4095, ctypes.c_void_p(256), None) == -1
    assert L.hmfsr_noise_table(1.0, float("inf"), 4095, ctypes.c_void_p(256), None) == -1
    assert L.hmfsr_noise_table(1.0, 4.0, 0, ctypes.c_void_p(256), None) == -1
    d, p = desc(), hm.MergeParams().c()

    def call(table):
        return L.hmfsr_merge_noise(ctypes.c_void_p(16), ctypes.byref(d), ctypes.c_void_p(16), ctypes.byref(p),
                                   table, 1, 1, ctypes.c_void_p(16), None, ctypes.c_void_p(256), 1 << 40, None)

    assert call(None) == -1
    assert call(ctypes.c_void_p(264)) == -1


def test_merge_ex_rejects_bad_options(L):
    d, p = desc(), hm.MergeParams().c()

    def call(opts):
        return L.hmfsr_merge_ex(ctypes.c_void_p(16), ctypes.byref(d), ctypes.c_void_p(16), ctypes.byref(p),
                                ctypes.byref(opts) if opts is not None else None, 1, 1, ctypes.c_void_p(16), None,
                                ctypes.c_void_p(256), 1 << 40, None)

    assert call(None) == -1
    assert call(_lib.MergeOptionsC(264, 0.0)) == -1          # misaligned table
    assert call(_lib.MergeOptionsC(None, -0.1)) == -1
    assert call(_lib.MergeOptionsC(None, float("nan"))) == -1
