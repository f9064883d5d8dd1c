"""The oracle's analytic adjoint of the merge against FP64 central finite differences of
the oracle's own forward, at points where no discrete decision (window centre, motion
prior, clamp, 5x5 argmin, bilinear cell) changes between the two evaluations."""
import math

import numpy as np
import pytest

import burstgen
import oracle
from oracle import MergeParams

FIELDS = ("k_detail", "k_denoise", "d_th", "d_tr", "k_stretch", "k_shrink", "s2", "t")


def f32(x):
    return float(np.float32(x))


def setup_case(scale, seed=41):
    b = burstgen.make_burst(dict(n=4, h=48, w=64, gain=1.0, read=3.0, motion="global", scale=(1, 1)), seed=seed)
    raw = b["raw"].numpy()
    _, mf, _, _ = oracle.align(raw)
    mv = mf.astype(np.float32)
    rng = np.random.default_rng(seed)
    mv[2, 1, 2] += np.float32(0.9)      # a misaligned tile: robustness below 1 around it
    mv[3, 2, 0] += np.float32(-0.7)
    # wide denoise transition so D is strictly inside (0, 1) for many pixels
    # and a low-noise model with s2 near 1, so the robustness R lies strictly inside (0, 1)
    p = MergeParams(k_detail=0.3, k_denoise=3.0, d_th=0.004, d_tr=0.05, k_stretch=3.0, k_shrink=1.8,
                    t=0.12, s1=12.0, s2=1.1, m_th=3.0, noise_a=0.02, noise_b=0.5)
    ho, wo = oracle.out_size(48, 64, scale)
    g = rng.normal(size=(3, ho, wo))
    return raw, mv, p, g


def loss(raw, mv, p, g, scale):
    return float((oracle.merge(raw, mv, p, scale=scale) * g).sum())


@pytest.mark.parametrize("scale", [(1, 1), (3, 2)])
def test_param_gradients_match_central_differences(scale):
    raw, mv, p, g = setup_case(scale)
    gp, _ = oracle.merge_backward(raw, mv, p, g, scale=scale)
    fp0 = oracle.merge_fingerprint(raw, mv, p, scale=scale)
    checked = 0
    for k, name in enumerate(FIELDS):
        base = getattr(p, name)
        hrel = 1e-4
        hp = MergeParams(**{**p.__dict__, name: f32(base * (1 + hrel))})
        hm = MergeParams(**{**p.__dict__, name: f32(base * (1 - hrel))})
        if oracle.merge_fingerprint(raw, mv, hp, scale=scale) != fp0 or oracle.merge_fingerprint(raw, mv, hm, scale=scale) != fp0:
            continue
        step = getattr(hp, name) - getattr(hm, name)
        fd = (loss(raw, mv, hp, g, scale) - loss(raw, mv, hm, g, scale)) / step
        assert gp[k] == pytest.approx(fd, rel=1e-3, abs=1e-6 * (abs(fd) + 1)), (name, gp[k], fd)
        checked += 1
    assert checked >= 6
    assert all(abs(x) > 0 for x in gp), gp


def test_motion_gradients_match_central_differences():
    scale = (1, 1)
    raw, mv, p, g = setup_case(scale, seed=42)
    _, gm = oracle.merge_backward(raw, mv, p, g, scale=scale)
    fp0 = oracle.merge_fingerprint(raw, mv, p, scale=scale)
    rng = np.random.default_rng(3)
    checked = 0
    n, ty, tx, _ = mv.shape
    for _ in range(40):
        f, y, x, c = int(rng.integers(1, n)), int(rng.integers(0, ty)), int(rng.integers(0, tx)), int(rng.integers(0, 2))
        v0 = float(mv[f, y, x, c])
        mp, mm = mv.copy(), mv.copy()
        mp[f, y, x, c] = np.float32(v0 + 1e-3)
        mm[f, y, x, c] = np.float32(v0 - 1e-3)
        if oracle.merge_fingerprint(raw, mp, p, scale=scale) != fp0 or oracle.merge_fingerprint(raw, mm, p, scale=scale) != fp0:
            continue
        step = float(mp[f, y, x, c]) - float(mm[f, y, x, c])
        fd = (loss(raw, mp, p, g, scale) - loss(raw, mm, p, g, scale)) / step
        # per element, 1e-3 relative (the gradient bar); the FP64 differences agree to ~3e-6
        assert gm[f, y, x, c] == pytest.approx(fd, rel=1e-3, abs=1e-12), (f, y, x, c, gm[f, y, x, c], fd)
        checked += 1
    assert checked >= 15
    assert np.all(gm[0] == 0)


def test_adjoint_of_constant_scene_is_zero():
    # a constant scene merges to the constant for any parameters and motion: zero gradient
    burst = np.full((3, 32, 32), 777, np.uint16)
    mv = np.random.default_rng(1).uniform(-1, 1, size=(3, 2, 2, 2)).astype(np.float32)
    g = np.random.default_rng(2).normal(size=(3, 32, 32))
    gp, gm = oracle.merge_backward(burst, mv, MergeParams(), g)
    assert np.abs(gp).max() < 1e-9 and np.abs(gm).max() < 1e-9
