"""Pins for the FP64 oracle: each check compares it with something other than itself
(closed forms, hand-worked values, invariants the paper states, textbook special cases,
NumPy/SciPy routines and brute force on tiny inputs).  CPU only."""
import json
import math
import os

import numpy as np
import pytest
from scipy import ndimage

import oracle
from oracle import MergeParams

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
WL = 4095


def smooth_texture(h, w, seed=0, sigma=3.0, mean=2000.0, std=700.0, pad=64):
    rng = np.random.default_rng(seed)
    big = ndimage.gaussian_filter(rng.normal(size=(h + 2 * pad, w + 2 * pad)), sigma)
    return mean + std * big / big.std(), pad


def shifted_burst(shifts, h=128, w=128, seed=0, sigma=3.0):
    """Grey smooth texture seen with raw-px shifts (base -> frame displacement)."""
    big, pad = smooth_texture(h, w, seed, sigma)
    yy, xx = np.mgrid[0:h, 0:w].astype(float)
    frames = [ndimage.map_coordinates(big, [yy + pad - ty, xx + pad - tx], order=3) for tx, ty in shifts]
    return np.clip(np.round(np.stack(frames)), 0, WL).astype(np.uint16)


# --------------------------------------------------------------------------------------
# luminance, structure tensor (Sec. 5.1.2, Eq. 3)
# --------------------------------------------------------------------------------------
def test_luma_is_quad_sum():
    rng = np.random.default_rng(1)
    raw = rng.integers(0, WL + 1, size=(12, 18)).astype(np.uint16)
    lq = oracle.luma(raw)
    r = raw.astype(np.int64)
    assert np.array_equal(lq, r[0::2, 0::2] + r[0::2, 1::2] + r[1::2, 0::2] + r[1::2, 1::2])


def test_tensor_of_linear_ramp_closed_form():
    # raw(x, y) = g x in every channel -> Lq(u) = 8 g u + 2 g; each sub-square's forward
    # gradient = 2 * 8 g = 16 g, no y gradient: a = 4 (16 g)^2, b = c = 0 (interior)
    g = 3
    xs = np.arange(40)
    raw = np.tile(g * xs, (20, 1)).astype(np.uint16)
    a, b, c = oracle.structure_tensor(raw, 7, 4)
    assert (a, b, c) == (4 * (16 * g) ** 2, 0, 0)
    # diagonal ramp raw = g (x + y): gx = gy = 16 g, so a = b = c
    yy, xx = np.mgrid[0:20, 0:20]
    raw2 = (g * (xx + yy)).astype(np.uint16)
    assert oracle.structure_tensor(raw2, 5, 5) == (4 * 256 * g * g,) * 3


def test_tensor_of_step_edges():
    raw = np.zeros((16, 16), np.uint16)
    raw[:, 8:] = 1000          # vertical edge at raw x = 8 (half-res u = 4)
    a, b, c = oracle.structure_tensor(raw, 4, 4)
    assert a > 0 and b == 0 and c == 0
    a, b, c = oracle.structure_tensor(raw.T.copy(), 4, 4)
    assert a == 0 and b == 0 and c > 0
    # flat -> zero tensor
    assert oracle.structure_tensor(np.full((8, 8), 77, np.uint16), 2, 2) == (0, 0, 0)


# --------------------------------------------------------------------------------------
# kernel shape (Eq. 4 + supplement S.1)
# --------------------------------------------------------------------------------------
def _golden_params(js):
    p = js["params"]
    return MergeParams(k_detail=p["k_detail"], k_denoise=p["k_denoise"], d_th=p["d_th"], d_tr=p["d_tr"],
                       k_stretch=p["k_stretch"], k_shrink=p["k_shrink"])


def test_kernel_shape_hand_worked_cases():
    js = json.load(open(os.path.join(GOLDEN, "kernel_shape_cases.json")))
    params = _golden_params(js)
    for case in js["cases"]:
        got = oracle.kernel_from_tensor(*case["tensor"], params, js["params"]["white_level"])
        for k, v in case["expect"].items():
            assert got[k] == pytest.approx(v, rel=1e-12, abs=1e-12), (case["name"], k, got[k], v)


def test_kernel_eigen_matches_numpy_eigh():
    rng = np.random.default_rng(2)
    params = MergeParams()
    for _ in range(200):
        gx = rng.integers(-3000, 3000, size=4)
        gy = rng.integers(-3000, 3000, size=4)
        a, b, c = int((gx * gx).sum()), int((gx * gy).sum()), int((gy * gy).sum())
        got = oracle.kernel_from_tensor(a, b, c, params)
        lam, vec = np.linalg.eigh(np.array([[a, b], [b, c]], float))
        assert got["l1"] == pytest.approx(lam[1], rel=1e-9, abs=1e-6)
        assert got["l2"] == pytest.approx(lam[0], rel=1e-9, abs=1e-3)
        e1 = vec[:, 1]
        om = np.array([[got["Oxx"], got["Oxy"]], [got["Oxy"], got["Oyy"]]])
        # Omega has eigenvalue k_across along the dominant gradient e1, k_along along e2
        assert om @ e1 == pytest.approx(got["k_across"] * e1, rel=1e-9, abs=1e-12)
        e2 = np.array([-e1[1], e1[0]])
        assert om @ e2 == pytest.approx(got["k_along"] * e2, rel=1e-9, abs=1e-12)
        assert got["A"] == pytest.approx(1 + math.sqrt((lam[1] - lam[0]) / (lam[1] + lam[0])), rel=1e-9)


def test_kernel_isotropic_when_no_stretch_and_isotropic_tensor():
    p = MergeParams(k_stretch=1.0, k_shrink=1.0, d_th=0.0, d_tr=0.001)
    got = oracle.kernel_from_tensor(900000, 0, 900000, p)     # lambda1 == lambda2 -> A = 1
    assert got["A"] == 1.0
    assert got["Oxx"] == pytest.approx(got["Oyy"], rel=1e-15) and got["Oxy"] == 0.0
    assert got["Oxx"] == pytest.approx((0.29 * float(np.float32(0.29)) / 0.29) ** 2, rel=1e-6)


def test_kernel_denoise_limits():
    p = MergeParams()
    flat = oracle.kernel_from_tensor(0, 0, 0, p)
    kd = float(np.float32(0.29)) * 4.0
    assert flat["D"] == 1.0 and flat["k_along"] == pytest.approx(kd * kd) and flat["k_across"] == pytest.approx(kd * kd)
    sharp = oracle.kernel_from_tensor(10 ** 12, 0, 0, p)
    kdet = float(np.float32(0.29))
    assert sharp["D"] == 0.0
    assert sharp["k_along"] == pytest.approx((kdet * 4 * 2) ** 2, rel=1e-12)
    assert sharp["k_across"] == pytest.approx((kdet / (2 * 2)) ** 2, rel=1e-12)


# --------------------------------------------------------------------------------------
# motion prior (Eq. 7-8) and robustness (Eq. 5, 6, 9)
# --------------------------------------------------------------------------------------
def test_motion_prior_uniform_and_outlier():
    p = MergeParams()
    mv = np.zeros((6, 7, 2), np.float32)
    mv[...] = (1.25, -0.5)
    M, s = oracle.tile_strength(mv, p)
    assert np.all(M == 0) and np.all(s == np.float32(2.0))
    mv[3, 4] += (0.6, 0.8)          # span (0.6, 0.8) -> M = 1.0 > 0.8 in the 3x3 around it
    M, s = oracle.tile_strength(mv, p)
    near = np.zeros((6, 7), bool)
    near[2:5, 3:6] = True
    assert np.allclose(M[near], 1.0, atol=1e-6) and np.all(M[~near] == 0)
    assert np.all(s[near] == 12.0) and np.all(s[~near] == 2.0)
    mv[3, 4] = (1.25 + 0.3, -0.5 + 0.4)   # M = 0.5 < 0.8 -> s2 everywhere
    _, s = oracle.tile_strength(mv, p)
    assert np.all(s == 2.0)


def test_robustness_identical_frames_is_one(tiny_burst):
    raw = tiny_burst["raw"].numpy()
    p = MergeParams(noise_a=0.5, noise_b=4.0)
    ty, tx = oracle.n_tiles(256, 256, 16)
    R, Rh = oracle.robustness(raw[0], raw[0], np.zeros((ty, tx, 2), np.float32), 16, p)
    assert np.all(R == 1.0) and np.all(Rh == 1.0)


def test_robustness_large_difference_rejects(tiny_burst):
    raw = tiny_burst["raw"].numpy()
    alt = np.clip(raw[0].astype(np.int32) + 1500, 0, WL).astype(np.uint16)
    p = MergeParams(noise_a=0.5, noise_b=4.0)
    ty, tx = oracle.n_tiles(256, 256, 16)
    R, Rh = oracle.robustness(raw[0], alt, np.zeros((ty, tx, 2), np.float32), 16, p)
    assert np.all(Rh == 0.0)


def test_robustness_constant_patches_closed_form():
    # base and alt are flat (sigma_ms = 0) with per-channel offsets; noise var = b only.
    # sigma_c^2 = var_c (G: var/2), d_md,c^2 = 2 var_c / 9, d_c = d^3 / (d^2 + d_md^2),
    # ratio = sum d_c^2 / sum sigma_c^2, R = clamp(s2 exp(-ratio) - t, 0, 1).
    h = w = 32
    base = np.zeros((h, w), np.uint16)
    base[0::2, 0::2] = 1000     # R
    base[0::2, 1::2] = 1200     # G1
    base[1::2, 0::2] = 1200     # G2
    base[1::2, 1::2] = 900      # B
    off = {"R": 5, "G": 4, "B": -6}
    alt = base.astype(np.int32).copy()
    alt[0::2, 0::2] += off["R"]
    alt[0::2, 1::2] += off["G"]
    alt[1::2, 0::2] += off["G"]
    alt[1::2, 1::2] += off["B"]
    alt = alt.astype(np.uint16)
    B = 16.0
    p = MergeParams(noise_a=0.0, noise_b=B, t=0.125, s2=2.0, s1=12.0)
    ty, tx = oracle.n_tiles(h, w, 16)
    R, Rh = oracle.robustness(base, alt, np.zeros((ty, tx, 2), np.float32), 16, p)
    var = {"R": B, "G": B / 2, "B": B}
    dd = 0.0
    ss = 0.0
    for ch in "RGB":
        dms = -off[ch]
        dmd2 = 2 * var[ch] / 9
        d = dms ** 3 / (dms ** 2 + dmd2)
        dd += d * d
        ss += var[ch]
    expect = min(1.0, max(0.0, 2.0 * math.exp(-dd / ss) - 0.125))
    assert 0.0 < expect < 1.0
    assert np.allclose(R, expect, rtol=1e-12, atol=0)
    assert np.allclose(Rh, expect, rtol=1e-12, atol=0)


def test_robustness_min5_is_sliding_minimum(tiny_burst):
    raw = tiny_burst["raw"].numpy()
    p = MergeParams(noise_a=0.5, noise_b=4.0)
    ty, tx = oracle.n_tiles(256, 256, 16)
    mv = np.zeros((ty, tx, 2), np.float32)
    mv[..., 0] = 0.7
    mv[3:6, 3:6] = (5.0, -3.0)   # misaligned patch -> low R there
    R, Rh = oracle.robustness(raw[0], raw[1], mv, 16, p)
    assert R.min() < 0.5 < R.max()
    ref = ndimage.minimum_filter(R, size=5, mode="constant", cval=np.inf)
    assert np.array_equal(Rh, ref)


# --------------------------------------------------------------------------------------
# merge (Eq. 1-2)
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("scale", [(1, 1), (3, 2), (2, 1)])
def test_merge_constant_scene_is_constant(scale):
    n, h, w = 3, 24, 20
    burst = np.full((n, h, w), 1234, np.uint16)
    ty, tx = oracle.n_tiles(h, w, 16)
    rng = np.random.default_rng(3)
    mv = rng.uniform(-2.5, 2.5, size=(n, ty, tx, 2)).astype(np.float32)
    out = oracle.merge(burst, mv, MergeParams(), scale=scale)
    assert out.shape == (3,) + oracle.out_size(h, w, scale)
    assert np.allclose(out, 1234.0, rtol=1e-12, atol=0)


def test_merge_identical_frames_equals_single_frame(tiny_burst):
    raw = tiny_burst["raw"].numpy()
    p = MergeParams(noise_a=0.5, noise_b=4.0)
    ty, tx = oracle.n_tiles(256, 256, 16)
    one = oracle.merge(raw[:1], np.zeros((1, ty, tx, 2), np.float32), p)
    four = oracle.merge(np.repeat(raw[:1], 4, axis=0), np.zeros((4, ty, tx, 2), np.float32), p)
    assert np.allclose(four, one, rtol=1e-12, atol=1e-9)


def test_merge_even_integer_shift_equals_single_frame():
    # frame n is the base moved by an even number of raw px (Bayer phase kept) and the
    # motion field says exactly that: every frame then contributes identical samples at
    # identical offsets, robustness is 1, and the merge equals the base-only merge away
    # from the border.  A wrong sign or axis of v breaks this.
    h, w = 96, 112
    big = np.random.default_rng(4).integers(200, 3800, size=(h + 40, w + 40)).astype(np.uint16)
    shifts = [(0, 0), (4, -2), (-6, 2), (2, 6)]
    frames = [big[20 - sy:20 - sy + h, 20 - sx:20 - sx + w] for sx, sy in shifts]
    burst = np.stack(frames)
    ty, tx = oracle.n_tiles(h, w, 16)
    mv = np.zeros((4, ty, tx, 2), np.float32)
    for k, (sx, sy) in enumerate(shifts):
        mv[k] = (sx, sy)
    p = MergeParams(noise_a=1.0, noise_b=4.0)
    for scale in [(1, 1), (2, 1)]:
        all4 = oracle.merge(burst, mv, p, scale=scale)
        one = oracle.merge(burst[:1], mv[:1], p, scale=scale)
        s = scale[0] / scale[1]
        m = int(16 * s)
        assert np.allclose(all4[:, m:-m, m:-m], one[:, m:-m, m:-m], rtol=1e-10, atol=1e-9)


def test_merge_isotropic_is_normalized_gaussian_convolution():
    # With k_stretch = k_shrink = 1 and D = 1 everywhere (huge D_th), Omega = (k_d k_dn)^2 I.
    # One frame at 1x, zero motion: each channel is the normalized convolution of its
    # Bayer samples with the 3x3 Gaussian exp(-|d|^2 / 2k) (Eq. 1-2), computed here with
    # scipy.ndimage.
    rng = np.random.default_rng(5)
    raw = rng.integers(0, WL + 1, size=(1, 20, 24)).astype(np.uint16)
    p = MergeParams(k_stretch=1.0, k_shrink=1.0, d_th=1000.0, d_tr=1.0, k_detail=0.5, k_denoise=1.5)
    k = float(np.float32(0.5)) * float(np.float32(1.5))
    k = k * k
    out = oracle.merge(raw, np.zeros((1, 2, 2, 2), np.float32), p)
    yy, xx = np.mgrid[-1:2, -1:2]
    K = np.exp(-(xx ** 2 + yy ** 2) / (2 * k))
    r = raw[0].astype(float)
    py, px = np.mgrid[0:20, 0:24]
    ch = (px & 1) + (py & 1)
    for c in range(3):
        mask = (ch == c).astype(float)
        num = ndimage.convolve(r * mask, K, mode="constant", cval=0.0)
        den = ndimage.convolve(mask, K, mode="constant", cval=0.0)
        assert np.allclose(out[c], num / den, rtol=1e-12, atol=1e-9)


def test_merge_wide_kernel_is_window_average_at_2x():
    # Omega = (k_d k_dn)^2 I with a huge variance: every weight -> 1, so each channel is
    # the plain mean of its samples in the 3x3 window centred on round(x0), with
    # x0 = (X + 1/2)/2 - 1/2 at 2x.
    rng = np.random.default_rng(6)
    h, w = 12, 14
    raw = rng.integers(0, WL + 1, size=(1, h, w)).astype(np.uint16)
    p = MergeParams(k_stretch=1.0, k_shrink=1.0, d_th=1000.0, d_tr=1.0, k_detail=64.0, k_denoise=64.0)
    out = oracle.merge(raw, np.zeros((1, 1, 1, 2), np.float32), p, scale=(2, 1))
    r = raw[0].astype(float)
    for Y in range(2 * h):
        for X in range(2 * w):
            kx = math.floor((X + 0.5) / 2 - 0.5 + 0.5)
            ky = math.floor((Y + 0.5) / 2 - 0.5 + 0.5)
            sums = np.zeros(3)
            cnt = np.zeros(3)
            for j in (-1, 0, 1):
                for i in (-1, 0, 1):
                    qx, qy = kx + i, ky + j
                    if 0 <= qx < w and 0 <= qy < h:
                        c = (qx & 1) + (qy & 1)
                        sums[c] += r[qy, qx]
                        cnt[c] += 1
            assert np.allclose(out[:, Y, X], sums / cnt, rtol=1e-6)


def test_merge_output_is_convex_combination(tiny_burst):
    raw = tiny_burst["raw"].numpy()
    _, mf, _, _ = oracle.align(raw)
    p = MergeParams(noise_a=0.5, noise_b=4.0)
    out, den = oracle.merge(raw, mf.astype(np.float32), p, with_den=True)
    assert np.all(den > 0)
    assert out.min() >= raw.min() - 1e-9 and out.max() <= raw.max() + 1e-9


def test_merge_pixels_matches_rows(tiny_burst):
    raw = tiny_burst["raw"].numpy()
    _, mf, _, _ = oracle.align(raw)
    mv = mf.astype(np.float32)
    p = MergeParams(noise_a=0.5, noise_b=4.0)
    for scale in [(1, 1), (3, 2)]:
        full = oracle.merge(raw, mv, p, scale=scale)
        rng = np.random.default_rng(7)
        ho, wo = full.shape[1:]
        xy = np.stack([rng.integers(0, wo, 50), rng.integers(0, ho, 50)], axis=1)
        xy[:4] = [(0, 0), (wo - 1, ho - 1), (0, ho - 1), (wo - 1, 0)]
        pix = oracle.merge_pixels(raw, mv, p, xy, scale=scale)
        assert np.array_equal(pix, full[:, xy[:, 1], xy[:, 0]].T)
        band = oracle.merge(raw, mv, p, scale=scale, rows=(37, 61))
        assert np.array_equal(band, full[:, 37:61])


def test_merge_beats_single_frame_demosaic():
    import burstgen
    import torch
    b = burstgen.make_burst(dict(n=8, h=128, w=128, gain=0.5, read=2.0, motion="global", scale=(1, 1)),
                            seed=11, with_gt=True)
    raw = b["raw"].numpy()
    gt = b["gt"].numpy().astype(float)
    _, mf, _, _ = oracle.align(raw)
    p = MergeParams(noise_a=0.5, noise_b=4.0)
    merged = oracle.merge(raw, mf.astype(np.float32), p)
    # bilinear demosaic of the base frame
    r = raw[0].astype(float)
    py, px = np.mgrid[0:128, 0:128]
    ch = (px & 1) + (py & 1)
    K = np.array([[0.25, 0.5, 0.25], [0.5, 1.0, 0.5], [0.25, 0.5, 0.25]])
    dem = np.stack([ndimage.convolve(r * (ch == c), K, mode="mirror") / ndimage.convolve((ch == c) * 1.0, K, mode="mirror")
                    for c in range(3)])
    sl = (slice(None), slice(8, -8), slice(8, -8))
    mse_merge = np.mean((merged[sl] - gt[sl]) ** 2)
    mse_dem = np.mean((dem[sl] - gt[sl]) ** 2)
    assert mse_merge < mse_dem
    del torch


# --------------------------------------------------------------------------------------
# alignment (Sec. 3.2)
# --------------------------------------------------------------------------------------
def test_align_even_integer_shift_is_exact():
    shifts = [(0, 0), (2, -4), (-6, 2), (4, 4)]
    h = w = 128
    big, pad = smooth_texture(h, w, seed=8)
    big = np.clip(np.round(big), 0, WL)
    frames = [big[pad - sy:pad - sy + h, pad - sx:pad - sx + w] for sx, sy in shifts]
    burst = np.stack(frames).astype(np.uint16)
    mi, mf, fl, nl = oracle.align(burst)
    assert nl >= 2
    for k, (sx, sy) in enumerate(shifts):
        # interior tiles (away from the clamped border by more than the shift)
        inner_i = mi[k, 1:-1, 1:-1]
        inner_f = mf[k, 1:-1, 1:-1]
        assert np.all(inner_i[..., 0] == sx // 2) and np.all(inner_i[..., 1] == sy // 2)
        assert np.all(inner_f[..., 0] == sx) and np.all(inner_f[..., 1] == sy)


def _brute_search(Lr, La, t, tx, ty, cx, cy, rad):
    H, W = Lr.shape
    xs = np.clip(np.arange(tx * t, tx * t + t), 0, W - 1)
    ys = np.clip(np.arange(ty * t, ty * t + t), 0, H - 1)
    ref = Lr[np.ix_(ys, xs)]
    cands = []
    for dy in range(-rad, rad + 1):
        for dx in range(-rad, rad + 1):
            xa = np.clip(np.arange(tx * t, tx * t + t) + cx + dx, 0, W - 1)
            ya = np.clip(np.arange(ty * t, ty * t + t) + cy + dy, 0, H - 1)
            ssd = int(((ref - La[np.ix_(ya, xa)]) ** 2).sum())
            cands.append((ssd, abs(dx) + abs(dy), dy, dx))
    best = min(cands)
    return cx + best[3], cy + best[2]


def test_align_single_level_equals_exhaustive_search():
    rng = np.random.default_rng(9)
    burst = rng.integers(0, WL + 1, size=(3, 32, 48)).astype(np.uint16)
    burst[1] = np.roll(burst[0], (2, -4), axis=(0, 1))
    mi, _, _, nl = oracle.align(burst, n_levels=1, radius=(12,), lk_iters=0)
    assert nl == 1
    L = [oracle.luma(f).astype(np.int64) for f in burst]
    t = 8
    for k in range(3):
        for ty in range(mi.shape[1]):
            for tx in range(mi.shape[2]):
                if k == 0:
                    assert tuple(mi[k, ty, tx]) == (0, 0)
                    continue
                assert tuple(mi[k, ty, tx]) == _brute_search(L[0], L[k], t, tx, ty, 0, 0, 12)


def test_align_pyramid_matches_restatement():
    # coarse-to-fine restated with NumPy: level sizes, floor-mean decimation, parent
    # lookup and search; integer vectors must agree exactly
    rng = np.random.default_rng(10)
    big, pad = smooth_texture(160, 200, seed=10, sigma=2.0)
    frames = [big[pad:pad + 160, pad:pad + 200]]
    for sx, sy in [(3, -2), (-5, 1)]:
        frames.append(big[pad - sy:pad - sy + 160, pad - sx:pad - sx + 200])
    burst = np.clip(np.round(np.stack(frames)) + rng.integers(-20, 20, size=(3, 160, 200)), 0, WL).astype(np.uint16)
    mi, _, _, nl = oracle.align(burst, lk_iters=0)
    t = 8
    facs = [2, 4, 4]
    radius = [1, 4, 4, 4]

    def pyramid(f):
        lv = [oracle.luma(f).astype(np.int64)]
        for l in range(3):
            fct = facs[l]
            H, W = lv[-1].shape[0] // fct, lv[-1].shape[1] // fct
            if H < 16 or W < 16:
                break
            lv.append(lv[-1][:H * fct, :W * fct].reshape(H, fct, W, fct).sum(axis=(1, 3)) // (fct * fct))
        return lv

    pr = pyramid(burst[0])
    assert len(pr) == nl
    for k in (1, 2):
        pa = pyramid(burst[k])
        vec = None
        for l in range(nl - 1, -1, -1):
            H, W = pr[l].shape
            lty, ltx = -(-H // t), -(-W // t)
            cur = np.zeros((lty, ltx, 2), np.int64)
            for ty in range(lty):
                for tx in range(ltx):
                    cx = cy = 0
                    if vec is not None:
                        f = facs[l]
                        px = min((tx * t + t // 2) // f // t, vec.shape[1] - 1)
                        py = min((ty * t + t // 2) // f // t, vec.shape[0] - 1)
                        cx, cy = vec[py, px] * f
                    cur[ty, tx] = _brute_search(pr[l], pa[l], t, tx, ty, int(cx), int(cy), radius[l])
            vec = cur
        assert np.array_equal(mi[k], vec)


def test_lk_recovers_subpixel_shift():
    shifts = [(0.0, 0.0), (1.3, -0.7), (-2.2, 0.45), (0.5, 1.9)]
    burst = shifted_burst(shifts, seed=12)
    _, mf, fl, _ = oracle.align(burst)
    for k, (sx, sy) in enumerate(shifts):
        err = np.abs(mf[k, 1:-1, 1:-1] - np.array([sx, sy]))
        assert np.median(err) < 0.05 and err.max() < 0.25
        assert fl[k].sum() == 0


# --------------------------------------------------------------------------------------
# noise-dependent tuning (supplement: "Noise-dependent Tuning", "Tuning Procedure and
# Parameters"): the range ends printed there, and the reading's linearity in SNR
# --------------------------------------------------------------------------------------
def test_frame_mean_is_the_plain_average():
    rng = np.random.default_rng(1905_03277 + 51)
    f = rng.integers(0, 4096, size=(6, 10), dtype=np.uint16)
    total = 0
    for row in f.tolist():
        for v in row:
            total += v
    assert oracle.frame_mean(f) == total / 60


def test_snr_closed_form():
    # a flat frame at 1000 DN under var = 4 x + 36 has SNR 1000 / sqrt(4036)
    f = np.full((8, 8), 1000, dtype=np.uint16)
    assert oracle.snr_of(oracle.frame_mean(f), 4.0, 36.0) == pytest.approx(1000.0 / 4036.0 ** 0.5, rel=1e-15)


def test_tuning_range_ends_are_the_printed_values():
    low = oracle.snr_tuning(100.0, 256.0, 0.0)        # SNR 0.625: below the range
    high = oracle.snr_tuning(4000.0, 1.0, 0.0)        # SNR 63: above the range
    assert (low["k_detail"], low["k_denoise"], low["d_th"], low["d_tr"]) == (0.33, 5.0, 0.010, 0.020)
    assert (high["k_detail"], high["k_denoise"], high["d_th"], high["d_tr"]) == (0.25, 3.0, 0.001, 0.006)
    assert low["tile"] == 64 and high["tile"] == 16
    for k, v in {"k_stretch": 4, "k_shrink": 2, "t": 0.12, "s1": 12, "s2": 2, "m_th": 0.8}.items():
        assert low[k] == v and high[k] == v
    free = oracle.snr_tuning(500.0, 0.0, 0.0)           # noise-free model: the detail end
    assert free["snr"] == float("inf") and free["k_detail"] == 0.25 and free["tile"] == 16


def test_tuning_midpoint_and_monotone():
    # mean 3240 under var = 10 x gives SNR 3240 / 180 = 18, the middle of [6, 30]
    mid = oracle.snr_tuning(3240.0, 10.0, 0.0)
    assert mid["snr"] == pytest.approx(18.0, rel=1e-15)
    assert mid["k_detail"] == pytest.approx(0.29, abs=1e-15)
    assert mid["k_denoise"] == pytest.approx(4.0, abs=1e-15)
    assert mid["d_th"] == pytest.approx(0.0055, abs=1e-15)
    assert mid["d_tr"] == pytest.approx(0.013, abs=1e-15)
    prev = None
    for mean in np.linspace(10.0, 4000.0, 200):
        cur = oracle.snr_tuning(float(mean), 4.0, 36.0)
        if prev is not None:
            assert cur["snr"] > prev["snr"]
            for k in ("k_detail", "k_denoise", "d_th", "d_tr"):
                assert cur[k] <= prev[k]
            assert cur["tile"] <= prev["tile"]
        prev = cur


@pytest.mark.parametrize("snr,tile", [(6.0, 64), (9.999, 64), (10.0, 32), (13.999, 32), (14.0, 16), (29.0, 16)])
def test_tuning_tile_steps(snr, tile):
    # b = 0: SNR = sqrt(mean / a), so mean = a SNR^2 hits the SNR exactly
    assert oracle.snr_tuning(snr * snr, 1.0, 0.0)["tile"] == tile


# --------------------------------------------------------------------------------------
# Monte-Carlo noise statistics (Sec. 5.2.2: sigma_md and d_md simulated per brightness,
# with sensor clipping): the simulation against closed forms where they exist
# --------------------------------------------------------------------------------------
def _unclipped(var):
    # rounding to whole DN adds 1/12 (Sheppard); a 3x3 population variance expects 8/9
    # of the sample variance; two independent 9-sample means differ by 2 var / 9
    v = var + 1.0 / 12.0
    return np.array([8.0 / 9.0 * v, 8.0 / 9.0 * (var / 2.0 + 1.0 / 24.0), 2.0 * v / 9.0, (var / 2.0 + 1.0 / 24.0) * 2.0 / 9.0])


def test_noise_table_matches_closed_forms_away_from_clipping():
    a, b, wl = 4.0, 36.0, 4095
    tab = oracle.noise_table(a, b, wl)
    trials = oracle.NOISE_TRIALS
    # 4 standard errors: a 3x3 population variance has relative spread sqrt(2 / 8), a
    # squared difference of means sqrt(2)
    tol = 4.0 * np.array([0.5, 0.5, 2 ** 0.5, 2 ** 0.5]) / trials ** 0.5
    for i in (32, 48, 64, 80, 96):
        x = i * wl / (oracle.NOISE_LEVELS - 1)
        want = _unclipped(a * x + b)
        assert np.all(np.abs(tab[i] / want - 1.0) < tol), (i, tab[i], want)


def test_noise_table_clips_at_the_white_point():
    # at x = WL half the samples clip: a normal censored at its mean keeps
    # 1/2 - 1/(2 pi) of its variance (sigma there is 128 DN, so rounding is negligible)
    a, b, wl = 4.0, 36.0, 4095
    tab = oracle.noise_table(a, b, wl)
    var = a * wl + b
    ratio = tab[-1, 0] / (8.0 / 9.0 * var)
    assert abs(ratio - (0.5 - 1.0 / (2.0 * np.pi))) < 0.03  # ~4 standard errors of the trial mean
    # and the clipped end is far below the unclipped model
    assert tab[-1, 0] < 0.4 * _unclipped(var)[0]


def test_noise_table_noise_free_and_deterministic():
    assert np.array_equal(oracle.noise_table(0.0, 0.0), np.zeros((oracle.NOISE_LEVELS, 4)))
    t1, t2 = oracle.noise_table(1.5, 9.0), oracle.noise_table(1.5, 9.0)
    assert np.array_equal(t1, t2)
    # the generator: distinct counters give distinct words, and its bits are balanced
    words = np.array([oracle.philox((c, 7, 3, 0), (0x19050327, 0x5EED0001)) for c in range(2000)], dtype=np.uint64)
    assert len({tuple(w) for w in words.tolist()}) == 2000
    bits = np.unpackbits(words.astype(np.uint32).view(np.uint8))
    assert abs(bits.mean() - 0.5) < 4.0 * 0.5 / bits.size ** 0.5


def test_philox_matches_the_published_known_answers():
    # Philox-4x32-10 (Salmon et al., SC'11) known-answer vectors of the Random123
    # distribution: (counter, key) -> output words
    kat = [((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
           ((0xFFFFFFFF,) * 4, (0xFFFFFFFF, 0xFFFFFFFF), (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
           ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
            (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1))]
    for ctr, key, want in kat:
        assert tuple(oracle.philox(ctr, key)) == want


def test_robustness_with_noise_table_keeps_identical_frames():
    # identical frames have no colour difference, whatever the noise statistics
    rng = np.random.default_rng(1905_03277 + 53)
    frame = rng.integers(0, 4096, size=(48, 64), dtype=np.uint16)
    mv = np.zeros((3, 4, 2), dtype=np.float32)
    p = MergeParams(noise_a=4.0, noise_b=36.0)
    R, _ = oracle.robustness(frame, frame, mv, 16, p, noise_table=oracle.noise_table(4.0, 36.0))
    assert np.all(R == 1.0)


# --------------------------------------------------------------------------------------
# quadratic-fit subpixel alignment (Sec. 3.2): the parabola vertex and the tile SSDs
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("d", [-0.4, -0.125, 0.0, 0.2, 0.375])
def test_parabola_vertex_of_an_exact_parabola(d):
    e = lambda x: 6.0 * (x - d) ** 2 + 11.0
    assert oracle.parabola_vertex(e(-1), e(0), e(1)) == pytest.approx(d, abs=1e-15)


def test_parabola_vertex_degenerate_and_clamped():
    assert oracle.parabola_vertex(5, 5, 5) == 0.0                 # flat: no curvature
    assert oracle.parabola_vertex(3, 5, 3) == 0.0                 # concave
    assert oracle.parabola_vertex(100, 0, 0) == 0.5               # vertex beyond the sample: clamped
    assert oracle.parabola_vertex(0, 0, 100) == -0.5


def test_tile_ssd_is_the_plain_sum():
    rng = np.random.default_rng(1905_03277 + 54)
    a = rng.integers(0, 16000, size=(20, 24))
    b = rng.integers(0, 16000, size=(20, 24))
    # the last two tiles overhang the 20 x 24 level: the base reads its edge pixel, the
    # other frame the clamped displaced position
    for (x0, y0, ox, oy) in [(0, 0, 1, -1), (16, 12, 3, 5), (8, 16, -9, 2), (20, 16, -3, -2)]:
        tot = 0
        for j in range(8):
            for i in range(8):
                y, x = min(y0 + j, 19), min(x0 + i, 23)
                ya, xa = min(max(y0 + j + oy, 0), 19), min(max(x0 + i + ox, 0), 23)
                tot += (int(a[y, x]) - int(b[ya, xa])) ** 2
        assert oracle.tile_ssd(a, b, x0, y0, 8, ox, oy) == tot


def test_quadfit_recovers_subpixel_shifts_of_a_smooth_scene():
    # a smooth scene shifted by known subpixel amounts: the fit lands near them, and, as
    # the paper found, less accurately than three Lucas-Kanade iterations
    from scipy import ndimage
    rng = np.random.default_rng(1905_03277 + 55)
    base = ndimage.gaussian_filter(rng.random((160, 160)), 4.0) * 12000 + 800
    shifts = (0.0, 0.5, 1.25)  # half-res px along x (0.6 of it along y)
    frames = [np.clip(ndimage.shift(base, (0.6 * s, s), order=3, mode="nearest"), 0, 4 * 4095 - 1) for s in shifts]
    raw = np.stack([np.kron(f / 4.0, np.ones((2, 2))) for f in frames]).astype(np.uint16)[:, :128, :128]
    _, mq = oracle.align_quadfit(raw, ref=0, tile=32, n_levels=1, radius=(4,))
    _, ml, _, _ = oracle.align(raw, ref=0, tile=32, n_levels=1, radius=(4,), lk_iters=3)
    err_q, err_l = [], []
    for f in (1, 2):
        # content moved by +s half-res px: the base -> frame displacement is +2 s raw px
        want = np.array([2.0 * shifts[f], 1.2 * shifts[f]])
        q = np.median(mq[f, 1:-1, 1:-1].reshape(-1, 2), axis=0)
        lk = np.median(ml[f, 1:-1, 1:-1].reshape(-1, 2), axis=0)
        assert np.all(np.abs(q - want) < 0.35), (q, want)
        err_q.append(np.abs(q - want).max())
        err_l.append(np.abs(lk - want).max())
    assert max(err_l) < max(err_q)


# --------------------------------------------------------------------------------------
# high-frequency artifact rejection (supplement, High Frequency Artifacts Removal)
# --------------------------------------------------------------------------------------
def _hf_scene(h=64, w=96):
    # left: a pattern at the guide's Nyquist frequency (4 raw px period); right: a smooth ramp
    y, x = np.mgrid[0:h, 0:w]
    hf = 2000 + 1500 * np.where(((x // 2) + (y // 2)) % 2 == 0, 1, -1)
    smooth = 500 + 20 * x + 10 * y
    return np.where(x < w // 2, hf, smooth).astype(np.uint16)


def test_hf_loss_map_flags_nyquist_content_only():
    m = oracle.hf_loss_map(_hf_scene(), 0.03)
    hh, wh = m.shape
    assert m[2:-2, 2:wh // 2 - 2].all()          # the pattern lost its variance to the 3x3 means
    assert not m[:, wh // 2 + 2:].any()          # a ramp keeps it
    assert not oracle.hf_loss_map(_hf_scene(), 0.0).any()


def test_hf_rejection_in_the_robustness_matches_the_restatement():
    base = _hf_scene()
    rng = np.random.default_rng(1905_03277 + 56)
    alt = np.clip(base.astype(np.int64) + rng.integers(-3, 4, size=base.shape), 0, 4095).astype(np.uint16)
    ty, tx = 4, 6
    p = MergeParams(noise_a=1.0, noise_b=4.0)
    # checkerboard of +-0.5 px tile vectors: every tile's motion span exceeds m_th
    mv = np.zeros((ty, tx, 2), np.float32)
    mv[..., 0] = np.where((np.add.outer(np.arange(ty), np.arange(tx)) % 2) == 0, 0.5, -0.5)
    R_off, _ = oracle.robustness(base, alt, mv, 16, p)
    R_on, _ = oracle.robustness(base, alt, mv, 16, p, hf_loss=0.03)
    flag = oracle.hf_loss_map(base, 0.03)
    assert flag.any()
    assert np.all(R_on[flag] == 0.0)
    assert np.array_equal(R_on[~flag], R_off[~flag])
    # with no motion span nothing is rejected, whatever the content
    R_still, _ = oracle.robustness(base, alt, np.zeros_like(mv), 16, p, hf_loss=0.03)
    R_still_off, _ = oracle.robustness(base, alt, np.zeros_like(mv), 16, p)
    assert np.array_equal(R_still, R_still_off)
