"""An independent restatement of the merge, checked against the C oracle (CPU only).

The restatement below evaluates Eq. 1-9 and supplement S.1 in FP64 from the paper and
the readings the oracle documents.  It is written differently from the oracle, so that a
slip in either (an index, a clamp, a transposed operand, a dropped term) shows up as a
mismatch:
- it works on whole half-resolution planes, with edge padding for clamped reads and array
  slicing for the Bayer channels; the oracle walks pixel by pixel with clamped indices;
- it rounds the window centre with exact rationals (Python Fractions); the oracle uses
  integer floor division.

The tiny bursts are built so that every branch is taken: anisotropic and isotropic
kernels, the detail/denoise blend strictly inside (0, 1), robustness values of 0, 1 and
in between, both motion-prior strengths, window centres near the frame border, and a
base frame other than frame 0.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import MergeParams

WL = 4095


def _f32(p: MergeParams) -> dict:
    """The parameters as the merge sees them (single precision, widened)."""
    return {k: float(np.float32(v)) for k, v in p.__dict__.items()}


# ----------------------------------------------------------------------------------------
# half-resolution planes (Sec. 5.1.2, Sec. 5.2.2)
# ----------------------------------------------------------------------------------------
def _quads(raw):
    r = raw.astype(np.int64)
    return r[0::2, 0::2], r[0::2, 1::2], r[1::2, 0::2], r[1::2, 1::2]


def _shift(P, dx, dy, hh, wh, pad):
    """View of the padded plane P offset by (dx, dy) texels."""
    return P[pad + dy:pad + dy + hh, pad + dx:pad + dx + wh]


# ----------------------------------------------------------------------------------------
# kernel covariance (Eq. 3, Eq. 4, supplement S.1)
# ----------------------------------------------------------------------------------------
def omega_planes(raw, p: MergeParams, wl: int = WL):
    """(Oxx, Oxy, Oyy) planes of one frame."""
    q = _f32(p)
    R, G1, G2, B = _quads(raw)
    Lq = R + G1 + G2 + B
    hh, wh = Lq.shape
    P = np.pad(Lq, 1, mode="edge")
    a = np.zeros_like(Lq)
    b = np.zeros_like(Lq)
    c = np.zeros_like(Lq)
    # Eq. 3: four 2x2 sub-squares of the 3x3 window, one forward-difference gradient each
    for j in (-1, 0):
        for i in (-1, 0):
            tl, tr_ = _shift(P, i, j, hh, wh, 1), _shift(P, i + 1, j, hh, wh, 1)
            bl, br = _shift(P, i, j + 1, hh, wh, 1), _shift(P, i + 1, j + 1, hh, wh, 1)
            gx = (tr_ - tl) + (br - bl)
            gy = (bl - tl) + (br - tr_)
            a += gx * gx
            b += gx * gy
            c += gy * gy
    # Eq. 4: eigen-analysis of [[a, b], [b, c]] without trigonometry
    trace = (a + c).astype(np.float64)
    disc = np.sqrt((a - c).astype(np.float64) ** 2 + 4.0 * b.astype(np.float64) ** 2)
    lam1 = 0.5 * (trace + disc)
    tie = (a == c) & (b == 0)
    with np.errstate(invalid="ignore", divide="ignore"):
        cos2 = np.where(tie, 1.0, (a - c) / disc)
        sin2 = np.where(tie, 0.0, 2.0 * b / disc)
        A = np.where(a + c == 0, 1.0, 1.0 + np.sqrt(disc / trace))
    # S.1: detail/denoise blend and the stretched / shrunk extents
    lam1n = lam1 / (4.0 * (8.0 * wl) ** 2)
    D = np.clip(1.0 - np.sqrt(lam1n) / q["d_tr"] + q["d_th"], 0.0, 1.0)
    kd = q["k_detail"] * q["k_denoise"]
    k_along = ((1.0 - D) * q["k_detail"] * q["k_stretch"] * A + D * kd) ** 2
    k_across = ((1.0 - D) * q["k_detail"] / (q["k_shrink"] * A) + D * kd) ** 2
    # Omega = k_across e1 e1^T + k_along e2 e2^T (stretch along the edge)
    e1 = np.stack([0.5 * (1.0 + cos2), 0.5 * sin2, 0.5 * (1.0 - cos2)])
    e2 = np.stack([1.0 - e1[0], -e1[1], 1.0 - e1[2]])
    om = k_across * e1 + k_along * e2
    return om, {"A": A, "D": D}


# ----------------------------------------------------------------------------------------
# robustness (Eq. 5-9)
# ----------------------------------------------------------------------------------------
def _guide(raw):
    R, G1, G2, B = _quads(raw)
    return [R.astype(np.float64), 0.5 * (G1 + G2).astype(np.float64), B.astype(np.float64)]


def _box(plane):
    """3x3 sum with clamped reads."""
    hh, wh = plane.shape
    P = np.pad(plane, 1, mode="edge")
    return sum(_shift(P, i, j, hh, wh, 1) for j in (-1, 0, 1) for i in (-1, 0, 1))


def _bilinear(img, fx, fy):
    """Bilinear sample of img at continuous (fx, fy), reads clamped to the image."""
    hh, wh = img.shape
    x0, y0 = np.floor(fx), np.floor(fy)
    ax, ay = fx - x0, fy - y0
    ix, iy = x0.astype(np.int64), y0.astype(np.int64)
    at = lambda x, y: img[np.clip(y, 0, hh - 1), np.clip(x, 0, wh - 1)]
    return ((1 - ay) * ((1 - ax) * at(ix, iy) + ax * at(ix + 1, iy))
            + ay * ((1 - ax) * at(ix, iy + 1) + ax * at(ix + 1, iy + 1)))


def tile_strength(mv, p: MergeParams):
    """Eq. 7-8: s1 where the motion span of the 3x3 tile neighbourhood exceeds M_th."""
    q = _f32(p)
    ty, tx = mv.shape[:2]
    v = mv.astype(np.float64)
    s = np.empty((ty, tx))
    for y in range(ty):
        for x in range(tx):
            nb = v[max(y - 1, 0):y + 2, max(x - 1, 0):x + 2].reshape(-1, 2)
            span = nb.max(axis=0) - nb.min(axis=0)
            s[y, x] = q["s1"] if math.sqrt(span[0] ** 2 + span[1] ** 2) > q["m_th"] else q["s2"]
    return s


def robustness(base, alt, mv, tile: int, p: MergeParams, wl: int = WL):
    """R and Rhat of frame `alt` on the base frame's half-res grid."""
    q = _f32(p)
    gb, ga = _guide(base), _guide(alt)
    hh, wh = gb[0].shape
    v, u = np.mgrid[0:hh, 0:wh]
    ty, tx = mv.shape[:2]
    tyi, txi = np.minimum(2 * v // tile, ty - 1), np.minimum(2 * u // tile, tx - 1)
    vt = mv.astype(np.float64)[tyi, txi]
    fx, fy = u + 0.5 * vt[..., 0], v + 0.5 * vt[..., 1]
    dd = np.zeros((hh, wh))
    ss = np.zeros((hh, wh))
    for ch in range(3):
        mu = _box(gb[ch]) / 9.0
        var_ms = np.maximum(_box(gb[ch] ** 2) / 9.0 - mu ** 2, 0.0)  # base frame
        mu_n = _bilinear(_box(ga[ch]) / 9.0, fx, fy)                    # aligned frame
        d_ms = mu - mu_n
        var_md = q["noise_a"] * np.clip(mu, 0.0, wl) + q["noise_b"]
        if ch == 1:
            var_md = var_md / 2.0  # the green guide averages two samples
        var_md = np.maximum(var_md, 0.0)
        dmd2 = 2.0 * var_md / 9.0
        sigma2 = np.maximum(var_ms, var_md)                               # Eq. 6
        den = d_ms ** 2 + dmd2
        with np.errstate(invalid="ignore", divide="ignore"):
            d = np.where(den > 0, d_ms ** 3 / den, 0.0)                   # Eq. 6
        dd += d * d
        ss += sigma2
    s = tile_strength(mv, p)[tyi, txi]
    R = np.clip(s * np.exp(-dd / np.maximum(ss, 1e-12 * wl * wl)) - q["t"], 0.0, 1.0)  # Eq. 5
    Rp = np.pad(R, 2, mode="edge")  # the minimum over a clamped window = over valid pixels
    Rhat = np.min([_shift(Rp, i, j, hh, wh, 2) for j in range(-2, 3) for i in range(-2, 3)], axis=0)  # Eq. 9
    return R, Rhat


# ----------------------------------------------------------------------------------------
# accumulation and normalisation (Eq. 1-2)
# ----------------------------------------------------------------------------------------
def merge(burst, motion, p: MergeParams, scale=(1, 1), ref: int = 0, tile: int = 16, wl: int = WL):
    n, h, w = burst.shape
    num_s, den_s = scale
    ho, wo = h * num_s // den_s, w * num_s // den_s
    ty, tx = motion.shape[1:3]
    Y, X = np.mgrid[0:ho, 0:wo]
    s = Fraction(num_s, den_s)
    # output pixel centres on the raw grid (pixel centres at integers on both grids)
    x0f = [[(Fraction(int(xx)) + Fraction(1, 2)) / s - Fraction(1, 2) for xx in row] for row in X]
    y0f = [[(Fraction(int(yy)) + Fraction(1, 2)) / s - Fraction(1, 2) for yy in row] for row in Y]
    x0 = np.array([[float(v) for v in row] for row in x0f])
    y0 = np.array([[float(v) for v in row] for row in y0f])
    tyi = np.clip(np.array([[math.floor(v / tile) for v in row] for row in y0f]), 0, ty - 1)
    txi = np.clip(np.array([[math.floor(v / tile) for v in row] for row in x0f]), 0, tx - 1)
    num = np.zeros((3, ho, wo))
    den = np.zeros((3, ho, wo))
    gx, gy = (x0 - 0.5) / 2.0, (y0 - 0.5) / 2.0  # base half-res position of the pixel
    for f in range(n):
        om, _ = omega_planes(burst[f], p, wl)
        if f == ref:
            vx, vy = np.zeros((ho, wo)), np.zeros((ho, wo))
            rh = np.ones((ho, wo))
        else:
            mv = motion[f].astype(np.float64)
            vx, vy = mv[tyi, txi, 0], mv[tyi, txi, 1]
            _, Rhat = robustness(burst[ref], burst[f], motion[f], tile, p, wl)
            rh = _bilinear(Rhat, gx, gy)
        # window centre: the raw pixel nearest to x0 + v, ties up (exact rationals)
        kx = np.array([[math.floor(x0f[i][j] + Fraction(float(vx[i, j])) + Fraction(1, 2)) for j in range(wo)]
                       for i in range(ho)])
        ky = np.array([[math.floor(y0f[i][j] + Fraction(float(vy[i, j])) + Fraction(1, 2)) for j in range(wo)]
                       for i in range(ho)])
        px, py = x0 + vx, y0 + vy
        hx, hy = (px - 0.5) / 2.0, (py - 0.5) / 2.0  # frame f's half-res position
        oxx, oxy, oyy = (_bilinear(om[k], hx, hy) for k in range(3))
        det = oxx * oyy - oxy * oxy
        for j in (-1, 0, 1):
            for i in (-1, 0, 1):
                qx, qy = kx + i, ky + j
                inside = (qx >= 0) & (qx < w) & (qy >= 0) & (qy < h)
                dx, dy = qx - px, qy - py
                quad = (oyy * dx * dx - 2.0 * oxy * dx * dy + oxx * dy * dy) / det  # d^T Omega^-1 d
                wgt = np.where(inside, np.exp(-0.5 * quad) * rh, 0.0)             # Eq. 2
                val = burst[f][np.clip(qy, 0, h - 1), np.clip(qx, 0, w - 1)].astype(np.float64)
                ch = (qx & 1) + (qy & 1)  # RGGB: 0 R, 1 G, 2 B
                for c in range(3):
                    m = ch == c
                    num[c] += np.where(m, wgt * val, 0.0)
                    den[c] += np.where(m, wgt, 0.0)
    return num / den                                                              # Eq. 1


# ----------------------------------------------------------------------------------------
# tiny bursts
# ----------------------------------------------------------------------------------------
def _scene(h, w, rng):
    """An edge at an angle, a grating and a smooth ramp, 12-bit."""
    y, x = np.mgrid[0:h, 0:w].astype(np.float64)
    img = 600.0 + 4.0 * x + 2.5 * y
    img += np.where(x * 0.8 + y * 0.6 > 0.45 * (w + h), 1500.0, 0.0)
    img += 400.0 * np.sin(2 * np.pi * x / 3.1) * (y < h / 3)
    return img


def _burst(n, h, w, seed, mismatch=True):
    rng = np.random.default_rng(seed)
    base = _scene(h, w, rng)
    frames = []
    for f in range(n):
        img = base.copy()
        if f and mismatch:
            img[2:8, w - 10:w - 2] += 1800.0  # a moved object: rejected outright
            img[0:12, 8:20] += 45.0 * f        # a small change: partial robustness
        img = img + rng.normal(0.0, 6.0, img.shape)
        img[h // 2:, : w // 4] = 2000.0  # a noise-free flat patch: a zero structure tensor
        frames.append(np.clip(np.round(img), 0, WL).astype(np.uint16))
    return np.stack(frames)


def _motion(n, h, w, tile, seed, ref):
    rng = np.random.default_rng(seed)
    ty, tx = oracle.n_tiles(h, w, tile)
    mv = rng.uniform(-0.15, 0.15, (n, ty, tx, 2)).astype(np.float32)
    mv[:, 0, 0] = (2.7, -1.3)     # a large vector: the motion prior's s1 around it
    mv[:, -1, -1] = (-1.8, 2.2)   # and a window centre pushed past the frame border
    mv[ref] = 0.0
    return mv


P = MergeParams(k_detail=0.3, k_denoise=3.0, d_th=0.004, d_tr=0.015, k_stretch=4.0, k_shrink=2.0, t=0.12,
                s1=12.0, s2=2.0, m_th=0.8, noise_a=1.0, noise_b=36.0)


def test_omega_planes_match_the_oracle():
    raw = _burst(1, 24, 32, 1)[0]
    om, aux = omega_planes(raw, P)
    ref = oracle.omega_plane(raw, P)
    np.testing.assert_allclose(om, ref, rtol=1e-12, atol=1e-15)
    # the burst exercises the blend strictly inside (0, 1) and anisotropic kernels
    assert np.any((aux["D"] > 0.05) & (aux["D"] < 0.95))
    assert aux["A"].max() > 1.5 and aux["A"].min() == 1.0


def test_robustness_matches_the_oracle():
    burst = _burst(2, 24, 32, 2)
    mv = _motion(2, 24, 32, 8, 3, ref=0)[1]
    R, Rhat = robustness(burst[0], burst[1], mv, 8, P)
    Ro, Rho = oracle.robustness(burst[0], burst[1], mv, 8, P)
    np.testing.assert_allclose(R, Ro, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(Rhat, Rho, rtol=1e-10, atol=1e-12)
    assert (R == 0).any() and (R == 1).any() and ((R > 0.05) & (R < 0.95)).any()
    s = tile_strength(mv, P)
    assert (s == np.float32(P.s1)).any() and (s == np.float32(P.s2)).any()


@pytest.mark.parametrize("scale,ref", [((1, 1), 0), ((3, 2), 1), ((2, 1), 2)])
def test_merge_matches_the_oracle(scale, ref):
    n, h, w, tile = 3, 16, 24, 8
    burst = _burst(n, h, w, 4)
    mv = _motion(n, h, w, tile, 5, ref)
    out = merge(burst, mv, P, scale=scale, ref=ref, tile=tile)
    got = oracle.merge(burst, mv, P, scale=scale, ref=ref, tile=tile)
    assert out.shape == got.shape
    np.testing.assert_allclose(got, out, rtol=1e-9, atol=1e-9 * WL)
