"""CUDA path vs the FP64 oracle, element by element, through the C-ABI.

Bars (stated by the task and derived in the design notes):
  * integer alignment (block-matching vectors): bit-exact;
  * Lucas-Kanade motion: within 1e-3 px on well-conditioned tiles;
  * merge: per channel, max |gpu - oracle| <= 1e-4 * WL and mean <= 1e-6 * WL, with both
    sides given the same float32 motion field (the oracle's own alignment).
"""
import numpy as np
import pytest
import torch

import burstgen
import oracle
import paper_1905_03277_gb300 as hm
from _parity import assert_merge_close, assert_motion_matches_oracle, oparams

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hm.build()
    return torch.device("cuda:0")


def params_of(b, **kw):
    return hm.MergeParams(noise_a=b["gain"], noise_b=b["read"] ** 2, **kw)


def check_align(raw, dev, ref=0, tile=16, white_level=4095, **kw):
    raw_np = raw.numpy()
    ap = hm.AlignParams(tile=tile, **kw)
    g_motion, g_int = hm.align(raw.to(dev), ref, ap, with_int=True, white_level=white_level)
    return assert_motion_matches_oracle(g_int.cpu().numpy(), g_motion.cpu().numpy(), raw_np, ref, tile,
                                        n_levels=ap.n_levels, radius=ap.radius, lk_iters=ap.lk_iters)


# --------------------------------------------------------------------------------------
# alignment
# --------------------------------------------------------------------------------------
def test_align_tiny(dev, tiny_burst):
    check_align(tiny_burst["raw"], dev)


def test_align_ragged_sizes_and_ref(dev):
    b = burstgen.make_burst(dict(n=4, h=136, w=200, gain=1.0, read=2.0, motion="global", scale=(1, 1)), seed=21)
    check_align(b["raw"], dev, ref=2)
    check_align(b["raw"], dev, ref=0, tile=32, radius=(2, 3, 4, 4))
    check_align(b["raw"], dev, ref=1, tile=8, n_levels=2, lk_iters=5)
    check_align(b["raw"], dev, ref=3, tile=64, n_levels=3, radius=(0, 7, 5, 4), lk_iters=1)
    check_align(b["raw"], dev, ref=0, radius=(3, 6, 2, 0), lk_iters=0)


def test_align_full_swing_13_bit(dev):
    # 13-bit frames of black and white 16-px blocks: a misaligned level-0 tile row sums
    # 8 squared differences of ~29000, beyond 2^32; the search must stay exact
    rng = np.random.default_rng(1905_03277 + 31)
    n, h, w, wl = 4, 128, 192, 7281
    img = np.kron((rng.random((h // 16, w // 16)) > 0.5) * float(wl), np.ones((16, 16)))
    frames = [np.roll(img, tuple(rng.integers(-6, 7, size=2)), axis=(0, 1)) for _ in range(n)]
    raw = np.clip(np.stack(frames) + rng.normal(0.0, 20.0, (n, h, w)), 0, wl).astype(np.uint16)
    check_align(torch.from_numpy(raw), dev, white_level=wl)



# --------------------------------------------------------------------------------------
# merge stages
# --------------------------------------------------------------------------------------
def test_merge_stages_tiny(dev, tiny_burst):
    raw = tiny_burst["raw"]
    raw_np = raw.numpy()
    _, mf, _, _ = oracle.align(raw_np)
    mv = mf.astype(np.float32)
    p = params_of(tiny_burst)
    om, rh = hm.merge_stages(raw.to(dev), torch.from_numpy(mv).to(dev), p)
    om = om.cpu().numpy()
    rh = rh.cpu().numpy()
    op = oparams(p)
    for f in range(raw_np.shape[0]):
        ref_om = oracle.omega_plane(raw_np[f], op)
        scale = np.abs(ref_om[0]) + np.abs(ref_om[2])
        assert (np.abs(om[f] - ref_om) <= 2e-6 * scale[None]).all(), f"Omega frame {f}"
        if f == 0:
            assert np.all(rh[f] == 1.0)
            continue
        _, ref_rh = oracle.robustness(raw_np[0], raw_np[f], mv[f], 16, op)
        assert np.abs(rh[f] - ref_rh).max() <= 2e-5, f"Rhat frame {f}: {np.abs(rh[f] - ref_rh).max()}"


def test_identical_frames_robustness_is_one(dev, tiny_burst):
    raw = tiny_burst["raw"][:1].repeat(4, 1, 1).contiguous()
    mv = torch.zeros((4, 16, 16, 2), dtype=torch.float32, device=dev)
    _, rh = hm.merge_stages(raw.to(dev), mv, params_of(tiny_burst))
    assert bool((rh == 1.0).all())


# --------------------------------------------------------------------------------------
# merge
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("scale", [(1, 1), (3, 2), (2, 1)])
def test_merge_tiny(dev, tiny_burst, scale):
    raw = tiny_burst["raw"]
    raw_np = raw.numpy()
    _, mf, _, _ = oracle.align(raw_np)
    mv = mf.astype(np.float32)
    p = params_of(tiny_burst)
    rgb = hm.merge(raw.to(dev), torch.from_numpy(mv).to(dev), p, scale).cpu().numpy()
    ref = oracle.merge(raw_np, mv, oparams(p), scale=scale)
    assert rgb.shape == ref.shape
    assert_merge_close(rgb, ref, f"scale {scale}")


def test_merge_denominator(dev, tiny_burst):
    raw = tiny_burst["raw"]
    raw_np = raw.numpy()
    _, mf, _, _ = oracle.align(raw_np)
    mv = mf.astype(np.float32)
    p = params_of(tiny_burst)
    _, den = hm.merge(raw.to(dev), torch.from_numpy(mv).to(dev), p, (1, 1), with_den=True)
    _, oden = oracle.merge(raw_np, mv, oparams(p), with_den=True)
    assert np.abs(den.cpu().numpy() - np.log2(oden)).max() <= 1e-3


def test_merge_edge_cases(dev):
    b = burstgen.make_burst(dict(n=5, h=136, w=200, gain=2.0, read=4.0, motion="global", scale=(1, 1)), seed=22)
    raw = b["raw"]
    raw_np = raw.numpy()
    p = params_of(b)
    ty, tx = hm.n_tiles(136, 200, 16)
    rng = np.random.default_rng(0)
    # large and odd motion: windows partly or wholly outside the frame, some tiles rejected
    mv = rng.uniform(-3, 3, size=(5, ty, tx, 2)).astype(np.float32)
    mv[3, :3, :4] = (41.25, -37.5)
    mv[4, -2:, -3:] = (-250.0, 180.0)
    mv[2] = np.round(mv[2] * 4) / 4   # quarter-pixel values: exact window-centre ties
    for ref in (0, 3):
        for scale in [(1, 1), (3, 2), (2, 1)]:
            rgb = hm.merge(raw.to(dev), torch.from_numpy(mv).to(dev), p, scale, ref=ref).cpu().numpy()
            oref = oracle.merge(raw_np, mv, oparams(p), scale=scale, ref=ref)
            assert_merge_close(rgb, oref, f"ref {ref} scale {scale}")
    # a single frame
    one = hm.merge(raw[:1].to(dev), torch.from_numpy(mv[:1]).to(dev), p, (2, 1)).cpu().numpy()
    assert_merge_close(one, oracle.merge(raw_np[:1], mv[:1], oparams(p), scale=(2, 1)), "single frame")
    # the smallest frame
    small = raw[:3, :4, :6].contiguous()
    smv = np.zeros((3, 1, 1, 2), np.float32)
    smv[1] = (0.3, -0.7)
    got = hm.merge(small.to(dev), torch.from_numpy(smv).to(dev), p, (3, 2)).cpu().numpy()
    assert_merge_close(got, oracle.merge(small.numpy(), smv, oparams(p), scale=(3, 2)), "4x6 frame")


def test_merge_rejects_bad_arguments(dev, tiny_burst):
    raw = tiny_burst["raw"].to(dev)
    mv = torch.zeros((8, 16, 16, 2), dtype=torch.float32, device=dev)
    with pytest.raises(RuntimeError, match="invalid argument"):
        hm.merge(raw, mv, hm.MergeParams(k_detail=-1.0))
    with pytest.raises(RuntimeError, match="invalid argument"):
        hm.merge(raw, mv, scale=(1, 2))


# --------------------------------------------------------------------------------------
# full-size workloads, whole images
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("config", ["12mp", "sr15"])
def test_full_size_whole_image(dev, config):
    # 12 MP x 8 at 1x and 12 MP x 15 at 2x (48.8 M output pixels): every output pixel of
    # the GPU merge against the oracle's, given the same float32 motion
    b = burstgen.make_burst(config, device=dev)
    raw = b["raw"]
    raw_np = raw.cpu().numpy()
    mv = check_align(raw.cpu(), dev)          # bit-exact integer stage on every tile
    p = params_of(b)
    scale = b["scale"]
    rgb = hm.merge(raw, torch.from_numpy(mv).to(dev), p, scale).cpu().numpy()
    ref = oracle.merge(raw_np, mv, oparams(p), scale=scale)
    assert_merge_close(rgb, ref, config)


# --------------------------------------------------------------------------------------
# noise-dependent tuning: the base frame's exact sum and the parameters it selects
# --------------------------------------------------------------------------------------
def test_frame_sum_exact(dev, tiny_burst):
    raw = tiny_burst["raw"]
    for f in range(raw.shape[0]):
        assert hm.frame_sum(raw.to(dev), f) == int(raw[f].numpy().astype(np.int64).sum())
    # ragged rows, a row stride beyond the width, widths below one 8-sample load
    rng = np.random.default_rng(1905_03277 + 52)
    for n, h, w, pitch in [(3, 10, 6, 6), (2, 37, 101, 104), (2, 64, 250, 256), (1, 5, 4, 12)]:
        full = rng.integers(0, 65536, size=(n, h, pitch), dtype=np.uint16)
        t = torch.from_numpy(full).to(dev)[:, :, :w]
        for f in range(n):
            assert hm.frame_sum(t, f) == int(full[f, :, :w].astype(np.int64).sum())
    # a full-size frame of 12-bit samples
    big = rng.integers(0, 4096, size=(1, 3024, 4032), dtype=np.uint16)
    assert hm.frame_sum(torch.from_numpy(big).to(dev), 0) == int(big.astype(np.int64).sum())


def test_auto_params_match_the_oracle(dev, tiny_burst):
    raw = tiny_burst["raw"]
    for ref in (0, 3):
        mp, ap, snr = hm.auto_params(raw.to(dev), tiny_burst["gain"], tiny_burst["read"] ** 2, ref=ref)
        want = oracle.snr_tuning(oracle.frame_mean(raw[ref].numpy()), tiny_burst["gain"], tiny_burst["read"] ** 2)
        assert snr == pytest.approx(want["snr"], rel=1e-12)
        assert mp.tile == ap.tile == want["tile"]
        for k in ("k_detail", "k_denoise", "d_th", "d_tr"):
            assert getattr(mp, k) == pytest.approx(want[k], rel=1e-7)
    # the selected parameters drive a merge that stays at parity with the oracle
    motion = oracle.align(raw.numpy(), ref=0, tile=mp.tile)[1].astype(np.float32)
    rgb = hm.merge(raw.to(dev), torch.from_numpy(motion).to(dev), mp).cpu().numpy()
    assert_merge_close(rgb, oracle.merge(raw.numpy(), motion, oparams(mp), tile=mp.tile), "auto parameters")


# --------------------------------------------------------------------------------------
# Monte-Carlo noise statistics (Sec. 5.2.2)
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("a,b,wl", [(4.0, 36.0, 4095), (0.5, 4.0, 4095), (8.0, 100.0, 7281), (0.0, 0.0, 4095)])
def test_noise_table_matches_the_oracle(dev, a, b, wl):
    got = hm.noise_table(a, b, wl, device=dev).cpu().numpy()
    want = oracle.noise_table(a, b, wl)
    # the same per-trial values on both sides; only the order of the FP64 sums differs
    assert np.allclose(got, want.astype(np.float32), rtol=1e-6, atol=1e-9)


def test_merge_with_noise_table(dev):
    # a bright burst: its highlights reach the white point, where the simulated
    # statistics depart from the closed form
    b = burstgen.make_burst("tiny")
    raw = np.minimum(b["raw"].numpy().astype(np.int64) * 3, 4095).astype(np.uint16)
    rt = torch.from_numpy(raw)
    a_, b_ = b["gain"], b["read"] ** 2
    p = hm.MergeParams(noise_a=a_, noise_b=b_)
    motion = oracle.align(raw, ref=0, tile=16)[1].astype(np.float32)
    mv = torch.from_numpy(motion).to(dev)
    table = hm.noise_table(a_, b_, 4095, device=dev)
    otab = oracle.noise_table(a_, b_, 4095)
    for scale in [(1, 1), (3, 2)]:
        got = hm.merge_noise(rt.to(dev), mv, table, p, scale).cpu().numpy()
        want = oracle.merge(raw, motion, oparams(p), scale=scale, noise_table=otab)
        assert_merge_close(got, want, f"noise table, scale {scale}")
    closed = hm.merge(rt.to(dev), mv, p).cpu().numpy()
    assert not np.array_equal(closed, hm.merge_noise(rt.to(dev), mv, table, p).cpu().numpy())


# --------------------------------------------------------------------------------------
# quadratic-fit subpixel alignment (Sec. 3.2): exact SSDs and FP64 vertex on both sides
# --------------------------------------------------------------------------------------
def test_align_quadfit_bit_exact(dev, tiny_burst):
    b = burstgen.make_burst(dict(n=4, h=136, w=200, gain=1.0, read=2.0, motion="global", scale=(1, 1)), seed=21)
    for raw, ref, tile in [(tiny_burst["raw"], 0, 16), (b["raw"], 2, 16), (b["raw"], 1, 32), (b["raw"], 3, 8)]:
        g_motion, g_int = hm.align(raw.to(dev), ref, hm.AlignParams(tile=tile), with_int=True, subpixel="quadfit")
        mi, mf = oracle.align_quadfit(raw.numpy(), ref=ref, tile=tile)
        assert np.array_equal(g_int.cpu().numpy(), mi)
        assert np.array_equal(g_motion.cpu().numpy(), mf)


# --------------------------------------------------------------------------------------
# high-frequency artifact rejection (supplement, High Frequency Artifacts Removal)
# --------------------------------------------------------------------------------------
def test_merge_with_high_frequency_rejection(dev):
    # four noisy frames of a scene half Nyquist pattern, half ramp, under a motion field
    # whose tiles alternate by 1 px (every tile's motion span exceeds m_th)
    rng = np.random.default_rng(1905_03277 + 57)
    h, w, n = 96, 128, 4
    y, x = np.mgrid[0:h, 0:w]
    scene = np.where(x < w // 2, 2000 + 1500 * np.where(((x // 2) + (y // 2)) % 2 == 0, 1, -1), 500 + 20 * x + 10 * y)
    raw = np.clip(scene[None] + rng.normal(0, 8, size=(n, h, w)), 0, 4095).astype(np.uint16)
    ty, tx = h // 16, w // 16
    motion = np.zeros((n, ty, tx, 2), np.float32)
    motion[1:, ..., 0] = np.where((np.add.outer(np.arange(ty), np.arange(tx)) % 2) == 0, 0.5, -0.5)
    p = hm.MergeParams(noise_a=1.0, noise_b=64.0)
    rt, mv = torch.from_numpy(raw).to(dev), torch.from_numpy(motion).to(dev)
    assert oracle.hf_loss_map(raw[0], 0.03).any()
    for scale in [(1, 1), (2, 1)]:
        got = hm.merge_ex(rt, mv, p, scale, hf_loss=0.03).cpu().numpy()
        want = oracle.merge(raw, motion, oparams(p), scale=scale, hf_loss=0.03)
        assert_merge_close(got, want, f"high-frequency rejection, scale {scale}")
        off = hm.merge_ex(rt, mv, p, scale).cpu().numpy()
        assert np.array_equal(off, hm.merge(rt, mv, p, scale).cpu().numpy())   # no options: hmfsr_merge
        assert not np.array_equal(off, got)
