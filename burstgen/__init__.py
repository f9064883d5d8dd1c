"""Seeded synthetic raw bursts for tests and benchmarks.

This module renders RGGB Bayer bursts of a procedural scene.  It holds none of the
merge or alignment arithmetic; it only produces inputs (and, for the fitting workload,
a ground-truth RGB image of the base frame).  Both the CUDA path and the FP64 oracle
consume its output, so both see bit-identical uint16 frames.

Scene (a stand-in for the Kodak / McMaster bursts of the paper's synthetic experiment,
Sec. 7.1, which are not available here): a sum of randomly oriented sinusoid gratings
(periods 1.5-20 px, so the finest ones alias on the Bayer grid, as super-resolution
needs, Sec. 4) under randomly placed convex polygons with flat colours, all clipped to
[0.05, 0.95].  Each raw pixel is the box average of the scene over 4x4 sub-positions of
its footprint, warped into the frame, then Bayer-sampled, scaled by the white level and
given Poisson-Gaussian noise (gain * Poisson(x / gain) + N(0, read^2)), rounded and
clipped.  Frame `ref` (always 0) sees the scene unwarped.

Random numbers for the scene and motion come from NumPy's Philox; the noise comes from
a seeded torch.Generator on the rendering device.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

WHITE_LEVEL = 4095
SEED_BASE = 1905_03277

# Workloads: 'tiny' (8 x 256x256, 1x), '12mp' (8 x 3024x4032, 1x),
# 'sr15' (15 x 3024x4032, 2x, two moving objects), 'fit' (8 x 1024x1024, 1.5x, with
# ground truth).  'ragged' bursts are produced by `make_ragged_batch`.
CONFIGS = {
    "tiny": dict(index=0, n=8, h=256, w=256, gain=0.5, read=2.0, motion="global", scale=(1, 1)),
    "12mp": dict(index=1, n=8, h=3024, w=4032, gain=4.0, read=6.0, motion="tremor", scale=(1, 1)),
    "sr15": dict(index=2, n=15, h=3024, w=4032, gain=1.0, read=3.0, motion="objects", scale=(2, 1)),
    "fit": dict(index=3, n=8, h=1024, w=1024, gain=1.0, read=3.0, motion="global", scale=(3, 2)),
}


@dataclass
class Scene:
    """Parameters of one procedural scene (all in base-frame raw pixel units).

    Background: a flat colour plus low-frequency gratings.  On top, convex polygons in
    order; each is either flat-coloured or filled with its own fine grating (period
    1.5-20 px), so that fine, aliasing detail sits inside bounded patches with edges.
    """
    base: np.ndarray            # [3]
    grat_k: np.ndarray          # [G, 2] background wave vectors (cycles / px)
    grat_phase: np.ndarray      # [G]
    grat_amp: np.ndarray        # [G, 3]
    poly_xy: list = field(default_factory=list)     # list of [V, 2] CCW vertex arrays
    poly_col: list = field(default_factory=list)    # list of [3]
    poly_grat: list = field(default_factory=list)   # list of None or (kx, ky, phase, amp[3])


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def make_scene(rng: np.random.Generator, h: int, w: int, n_grat: int = 3, n_poly: int | None = None,
               margin: float = 0.0) -> Scene:
    if n_poly is None:
        n_poly = int(np.clip(10 + (h * w) // 200_000, 10, 80))
    base = rng.uniform(0.3, 0.7, size=3)
    theta = rng.uniform(0, math.pi, size=n_grat)
    period = rng.uniform(40.0, 200.0, size=n_grat)
    k = np.stack([np.cos(theta), np.sin(theta)], axis=1) / period[:, None]
    phase = rng.uniform(0, 2 * math.pi, size=n_grat)
    amp = rng.uniform(0.03, 0.1, size=(n_grat, 1)) * rng.uniform(0.3, 1.0, size=(n_grat, 3))
    sc = Scene(base=base, grat_k=k, grat_phase=phase, grat_amp=amp)
    m = min(h, w)
    for _ in range(n_poly):
        cx = rng.uniform(-margin, w + margin)
        cy = rng.uniform(-margin, h + margin)
        rad = rng.uniform(0.03, 0.18) * m
        nv = int(rng.integers(3, 7))
        ang = np.sort(rng.uniform(0, 2 * math.pi, size=nv))
        rr = rad * rng.uniform(0.6, 1.0, size=nv)
        xy = np.stack([cx + rr * np.cos(ang), cy + rr * np.sin(ang)], axis=1)
        sc.poly_xy.append(xy)
        sc.poly_col.append(rng.uniform(0.15, 0.85, size=3))
        if rng.uniform() < 0.5:
            th = rng.uniform(0, math.pi)
            per = rng.uniform(1.5, 20.0)
            sc.poly_grat.append((math.cos(th) / per, math.sin(th) / per, rng.uniform(0, 2 * math.pi),
                                 rng.uniform(0.08, 0.3) * rng.uniform(0.3, 1.0, size=3)))
        else:
            sc.poly_grat.append(None)
    return sc


def scene_eval(sc: Scene, x: torch.Tensor, y: torch.Tensor, ch: torch.Tensor | int) -> torch.Tensor:
    """Scene value in [0.05, 0.95] at points (x, y) for colour channel `ch` (0 R, 1 G, 2 B).

    `ch` is an int or an integer tensor broadcastable to x.
    """
    dev, dt = x.device, x.dtype
    if isinstance(ch, int):
        chs = torch.full_like(x, ch, dtype=torch.long)
    else:
        chs = ch.expand_as(x).to(torch.long)
    base = torch.as_tensor(sc.base, device=dev, dtype=dt)
    out = base[chs].clone()
    two_pi = 2 * math.pi
    for g in range(sc.grat_k.shape[0]):
        kx, ky = float(sc.grat_k[g, 0]), float(sc.grat_k[g, 1])
        amp = torch.as_tensor(sc.grat_amp[g], device=dev, dtype=dt)
        out = out + amp[chs] * torch.cos(two_pi * (kx * x + ky * y) + float(sc.grat_phase[g]))
    for xy, col, gr in zip(sc.poly_xy, sc.poly_col, sc.poly_grat):
        x_lo, y_lo = xy.min(axis=0)
        x_hi, y_hi = xy.max(axis=0)
        inside = (x >= float(x_lo)) & (x <= float(x_hi)) & (y >= float(y_lo)) & (y <= float(y_hi))
        if not bool(inside.any()):
            continue
        nv = xy.shape[0]
        for i in range(nv):
            x0, y0 = float(xy[i, 0]), float(xy[i, 1])
            x1, y1 = float(xy[(i + 1) % nv, 0]), float(xy[(i + 1) % nv, 1])
            inside &= ((x1 - x0) * (y - y0) - (y1 - y0) * (x - x0)) >= 0
        c = torch.as_tensor(col, device=dev, dtype=dt)
        val = c[chs]
        if gr is not None:
            gkx, gky, gph, gamp = gr
            ga = torch.as_tensor(gamp, device=dev, dtype=dt)
            val = val + ga[chs] * torch.cos(two_pi * (gkx * x + gky * y) + gph)
        out = torch.where(inside, val, out)
    return out.clamp(0.05, 0.95)


@dataclass
class Motion:
    """Warp of one frame: frame pixel q sees scene point S(q).

    S(q) = c + Rot(-rot) (q - c) - shift - warp(q), so a scene point at base pixel x is
    seen in the frame near x + shift (+ rotation, + warp): `shift` is the base -> frame
    displacement in raw px.
    """
    shift: tuple = (0.0, 0.0)
    rot: float = 0.0                                   # radians
    warp: list = field(default_factory=list)           # [(ax, ay, fx, fy, phase)]


def _apply_motion(m: Motion, qx: torch.Tensor, qy: torch.Tensor, cx: float, cy: float):
    c, s = math.cos(-m.rot), math.sin(-m.rot)
    dx, dy = qx - cx, qy - cy
    sx = cx + c * dx - s * dy - m.shift[0]
    sy = cy + s * dx + c * dy - m.shift[1]
    for ax, ay, fx, fy, ph in m.warp:
        arg = 2 * math.pi * (fx * qx + fy * qy) + ph
        sn = torch.sin(arg)
        sx = sx - ax * sn
        sy = sy - ay * sn
    return sx, sy


@dataclass
class MovingObject:
    """A textured square moving linearly over the burst (for the local-motion workload)."""
    centre: tuple
    half: float
    disp: tuple                  # displacement at the last frame (base -> frame)
    scene: Scene
    occluded_frames: tuple = ()  # frames in which a flat occluder covers the square
    occluder_col: tuple = (0.1, 0.1, 0.1)


def _render_frame(sc: Scene, m: Motion, objects: list, n: int, n_frames: int, h: int, w: int,
                  device, ss: int = 4, rows_per_chunk: int = 128) -> torch.Tensor:
    """Noise-free Bayer mosaic of frame n in [0, 1] (float32 [h, w])."""
    out = torch.empty((h, w), dtype=torch.float32, device=device)
    cx, cy = (w - 1) / 2.0, (h - 1) / 2.0
    sub = (torch.arange(ss, dtype=torch.float32, device=device) + 0.5) / ss - 0.5
    xs = torch.arange(w, dtype=torch.float32, device=device)
    chunk = max(1, min(rows_per_chunk, (1 << 22) // max(1, w * ss * ss) + 1))
    for r0 in range(0, h, chunk):
        r1 = min(h, r0 + chunk)
        ys = torch.arange(r0, r1, dtype=torch.float32, device=device)
        # channel by RGGB parity: (even, even) R, (odd, odd) B, otherwise G
        py = (torch.arange(r0, r1, device=device) & 1)[:, None]
        px = (torch.arange(w, device=device) & 1)[None, :]
        ch = (px + py)                       # 0 R, 1 G, 2 B
        qx = xs[None, :, None, None] + sub[None, None, None, :]
        qy = ys[:, None, None, None] + sub[None, None, :, None]
        qx, qy = torch.broadcast_tensors(qx, qy)
        sx, sy = _apply_motion(m, qx, qy, cx, cy)
        chb = ch[:, :, None, None].expand_as(sx)
        val = scene_eval(sc, sx, sy, chb)
        for ob in objects:
            t = n / max(1, n_frames - 1)
            ox = ob.centre[0] + t * ob.disp[0]
            oy = ob.centre[1] + t * ob.disp[1]
            inside = ((sx - ox).abs() <= ob.half) & ((sy - oy).abs() <= ob.half)
            if inside.any():
                tv = scene_eval(ob.scene, sx - ox, sy - oy, chb)
                val = torch.where(inside, tv, val)
            if n in ob.occluded_frames:
                occ = ((sx - ob.centre[0]).abs() <= ob.half * 1.15) & ((sy - ob.centre[1]).abs() <= ob.half * 1.15)
                oc = torch.as_tensor(ob.occluder_col, device=device, dtype=torch.float32)
                val = torch.where(occ, oc[chb], val)
        out[r0:r1] = val.mean(dim=(2, 3))
    return out


def _motions(kind: str, rng: np.random.Generator, n: int, h: int, w: int) -> list:
    ms = [Motion()]
    if kind == "global":
        for _ in range(1, n):
            ms.append(Motion(shift=tuple(rng.uniform(-2, 2, size=2)),
                             rot=math.radians(rng.uniform(-0.5, 0.5))))
    elif kind in ("tremor", "objects"):
        pos = np.zeros(2)
        for _ in range(1, n):
            pos = np.clip(pos + rng.normal(0, 1.2, size=2), -4, 4)
            warp = []
            for _k in range(3):
                f = rng.uniform(0.3, 1.5, size=2) / np.array([w, h])
                a = rng.uniform(-0.1, 0.1, size=2)
                warp.append((float(a[0]), float(a[1]), float(f[0]), float(f[1]),
                             float(rng.uniform(0, 2 * math.pi))))
            ms.append(Motion(shift=(float(pos[0]), float(pos[1])),
                             rot=math.radians(rng.uniform(-0.05, 0.05)), warp=warp))
    else:
        raise ValueError(kind)
    return ms


def _add_noise(clean: torch.Tensor, gain: float, read: float, gen: torch.Generator) -> torch.Tensor:
    x = clean * WHITE_LEVEL
    shot = torch.poisson(x / gain, generator=gen) * gain
    rd = torch.randn(x.shape, generator=gen, device=x.device, dtype=torch.float32) * read
    return torch.round(shot + rd).clamp(0, WHITE_LEVEL).to(torch.int32).to(torch.uint16)


def make_burst(config: str | dict, seed: int | None = None, device: str | torch.device = "cpu",
               with_gt: bool = False, **overrides) -> dict:
    """Render one synthetic burst.

    Returns a dict with 'raw' (torch.uint16 [N, H, W] on `device`), 'ref' (0),
    'white_level', 'gain', 'read', 'scale' ((num, den)), 'motions' (list of Motion)
    and, if `with_gt`, 'gt' (float32 [3, Ho, Wo] in DN: the base-frame scene
    box-averaged over each output pixel with 8x8 sub-samples).
    """
    cfg = dict(CONFIGS[config]) if isinstance(config, str) else dict(config)
    cfg.update(overrides)
    n, h, w = int(cfg["n"]), int(cfg["h"]), int(cfg["w"])
    if h % 2 or w % 2:
        raise ValueError("frame sides must be even")
    if seed is None:
        seed = SEED_BASE + int(cfg.get("index", 0))
    rng = _rng(seed)
    objects = []
    motion_kind = cfg.get("motion", "global")
    sc = make_scene(rng, h, w, margin=40.0)
    ms = _motions("tremor" if motion_kind == "objects" else motion_kind, rng, n, h, w)
    if motion_kind == "objects":
        half = min(200.0, 0.12 * min(h, w))
        for k in range(2):
            osc = make_scene(rng, int(2 * half), int(2 * half), n_grat=2, n_poly=6, margin=0.0)
            ang = rng.uniform(0, 2 * math.pi)
            dist = rng.uniform(15, 30)
            centre = (float(rng.uniform(0.25, 0.75) * w), float(rng.uniform(0.25, 0.75) * h))
            occl = tuple(range(n // 3, (2 * n) // 3)) if k == 1 else ()
            objects.append(MovingObject(centre=centre, half=half,
                                        disp=(dist * math.cos(ang), dist * math.sin(ang)),
                                        scene=osc, occluded_frames=occl))
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    raw = torch.empty((n, h, w), dtype=torch.uint16, device=device)
    for i in range(n):
        clean = _render_frame(sc, ms[i], objects, i, n, h, w, device, ss=int(cfg.get("ss", 4)))
        raw[i] = _add_noise(clean, float(cfg["gain"]), float(cfg["read"]), gen)
    out = dict(raw=raw, ref=0, white_level=WHITE_LEVEL, gain=float(cfg["gain"]),
               read=float(cfg["read"]), scale=tuple(cfg.get("scale", (1, 1))), motions=ms,
               seed=seed, scene=sc)
    if with_gt:
        out["gt"] = render_gt(sc, h, w, out["scale"], device)
    return out


def render_gt(sc: Scene, h: int, w: int, scale: tuple, device, ss: int = 8) -> torch.Tensor:
    """Base-frame scene in DN, box-averaged over each output pixel (float32 [3, Ho, Wo]).

    Output pixel X spans raw-centre coordinates [X / s - 1/2, (X + 1) / s - 1/2].
    """
    num, den = scale
    ho, wo = (h * num) // den, (w * num) // den
    out = torch.empty((3, ho, wo), dtype=torch.float32, device=device)
    sub = (torch.arange(ss, dtype=torch.float32, device=device) + 0.5) / ss
    xs = torch.arange(wo, dtype=torch.float32, device=device)
    rows = max(1, (1 << 21) // (wo * ss * ss))
    for c in range(3):
        for r0 in range(0, ho, rows):
            r1 = min(ho, r0 + rows)
            ys = torch.arange(r0, r1, dtype=torch.float32, device=device)
            qx = (xs[None, :, None, None] + sub[None, None, None, :]) * den / num - 0.5
            qy = (ys[:, None, None, None] + sub[None, None, :, None]) * den / num - 0.5
            qx, qy = torch.broadcast_tensors(qx, qy)
            out[c, r0:r1] = scene_eval(sc, qx, qy, c).mean(dim=(2, 3)) * WHITE_LEVEL
    return out


def make_ragged_batch(n_bursts: int = 64, seed: int | None = None, device="cpu",
                      mp_range=(0.5, 12.0), max_frames: int = 15, ss: int = 4) -> list:
    """Ragged batch: per burst MP ~ U[mp_range], aspect 4:3 or 16:9 (sides even),
    frame count ~ U{4..max_frames}, scale in {1, 1.5, 2}, gain ~ U[0.5, 8]; `ss` is
    the per-axis supersampling of the rendering."""
    if seed is None:
        seed = SEED_BASE + 4
    rng = _rng(seed)
    out = []
    for b in range(n_bursts):
        mp = rng.uniform(*mp_range) * 1e6
        ar = (4, 3) if rng.uniform() < 0.5 else (16, 9)
        unit = math.sqrt(mp / (ar[0] * ar[1]))
        w = max(32, 2 * int(round(unit * ar[0] / 2)))
        h = max(32, 2 * int(round(unit * ar[1] / 2)))
        n = int(rng.integers(4, max_frames + 1))
        scale = [(1, 1), (3, 2), (2, 1)][int(rng.integers(0, 3))]
        gain = float(rng.uniform(0.5, 8.0))
        cfg = dict(index=4, n=n, h=h, w=w, gain=gain, read=2.0 + gain, motion="global", scale=scale, ss=ss)
        out.append(make_burst(cfg, seed=seed * 1000 + b, device=device))
    return out


def tile_motion_from_warp(m: Motion, h: int, w: int, tile: int) -> np.ndarray:
    """Approximate base -> frame displacement of each tile centre (float32 [TY, TX, 2]),
    from the warp used to render the frame (first-order inverse).  For sanity checks of
    alignment only; the method never sees it."""
    ty, tx = -(-h // tile), -(-w // tile)
    cy = (np.arange(ty) * tile + tile / 2 - 0.5)
    cx = (np.arange(tx) * tile + tile / 2 - 0.5)
    X, Y = np.meshgrid(cx, cy)
    qx = torch.as_tensor(X, dtype=torch.float64)
    qy = torch.as_tensor(Y, dtype=torch.float64)
    sx, sy = _apply_motion(m, qx, qy, (w - 1) / 2.0, (h - 1) / 2.0)
    return np.stack([(qx - sx).numpy(), (qy - sy).numpy()], axis=-1).astype(np.float32)
