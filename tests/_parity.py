"""Shared helpers of the GPU parity tests: the merge bars and the conditioning test for
Lucas-Kanade tiles.  The bars: integer alignment bit-exact; Lucas-Kanade within 1e-3 px
on well-conditioned tiles; merge per channel max |gpu - oracle| <= 1e-4 * WL and mean
<= 1e-6 * WL."""
import numpy as np

import oracle

WL = 4095
MAX_ABS = 1e-4 * WL
MEAN_ABS = 1e-6 * WL


def oparams(p) -> oracle.MergeParams:
    """The oracle's parameter set with the values of a binding MergeParams."""
    return oracle.MergeParams(**{k: getattr(p, k) for k in oracle.MergeParams.__dataclass_fields__})


def merge_errors(gpu, ref):
    err = np.abs(gpu.astype(np.float64) - ref)
    return err.reshape(3, -1).max(axis=1), err.reshape(3, -1).mean(axis=1)


def assert_merge_close(gpu, ref, what=""):
    assert gpu.shape == ref.shape, (what, gpu.shape, ref.shape)
    assert np.isfinite(gpu).all(), what
    mx, mn = merge_errors(gpu, ref)
    assert (mx <= MAX_ABS).all() and (mn <= MEAN_ABS).all(), f"{what}: max {mx}, mean {mn}"


def lk_conditioned(raw_np, ref, tile, floor=1e-6):
    """Tiles whose level-0 normal matrix is well conditioned (lambda_min / lambda_max)."""
    lq = oracle.luma(raw_np[ref]).astype(np.float64)
    gx = np.zeros_like(lq)
    gy = np.zeros_like(lq)
    gx[:, 1:-1] = lq[:, 2:] - lq[:, :-2]
    gx[:, 0] = lq[:, 1] - lq[:, 0]
    gx[:, -1] = lq[:, -1] - lq[:, -2]
    gy[1:-1] = lq[2:] - lq[:-2]
    gy[0] = lq[1] - lq[0]
    gy[-1] = lq[-1] - lq[-2]
    t = tile // 2
    H, W = lq.shape
    ty, tx = -(-H // t), -(-W // t)
    pad = lambda a: np.pad(a, ((0, ty * t - H), (0, tx * t - W)), mode="edge")
    sxx = (pad(gx * gx)).reshape(ty, t, tx, t).sum(axis=(1, 3))
    syy = (pad(gy * gy)).reshape(ty, t, tx, t).sum(axis=(1, 3))
    sxy = (pad(gx * gy)).reshape(ty, t, tx, t).sum(axis=(1, 3))
    tr = sxx + syy
    det = sxx * syy - sxy * sxy
    disc = np.sqrt(np.maximum(tr * tr / 4 - det, 0))
    lmin, lmax = tr / 2 - disc, tr / 2 + disc
    return lmin > floor * np.maximum(lmax, 1e-30) * 1e3


def assert_motion_matches_oracle(g_int, g_motion, raw_np, ref, tile=16, **align_kw):
    """Integer vectors bit-exact against the oracle's; skipped (ill-conditioned) tiles
    exactly 2u on both sides; Lucas-Kanade within 1e-3 px on conditioned tiles.  Returns
    the oracle's float32 motion."""
    mi, mf, fl, _ = oracle.align(raw_np, ref=ref, tile=tile, **align_kw)
    assert np.array_equal(g_int, mi), "integer block matching differs"
    sk = fl.astype(bool)
    assert np.array_equal(g_motion[sk], (2 * mi[sk]).astype(np.float32))
    good = lk_conditioned(raw_np, ref, tile)[None].repeat(raw_np.shape[0], 0) & ~sk
    err = np.abs(g_motion - mf).max(axis=-1)
    if good.any():
        assert err[good].max() <= 1e-3, f"LK max err {err[good].max()} on conditioned tiles"
    return mf.astype(np.float32)
