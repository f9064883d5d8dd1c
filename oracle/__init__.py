"""Python access to the FP64 oracle (hmfsr_oracle.c).

TEST INFRASTRUCTURE ONLY: the oracle is a plain CPU restatement of the paper's method,
used by the tests, the smoke check and the benchmark's CPU-baseline leg to check and
time the CUDA path.  The product path never imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, fields

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hmfsr_oracle.c")
_HDR = os.path.join(_HERE, "hmfsr_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction, OpenMP)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def build_sanitized(path: str) -> str:
    """Compile the oracle with AddressSanitizer and UndefinedBehaviorSanitizer (every
    report fatal) into `path`; a test runs the oracle's pins against it in a process
    that preloads the ASan runtime and points HMFSR_ORACLE_LIB at it."""
    cmd = ["gcc", "-O1", "-g", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer",
           "-shared", "-o", str(path), _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    return str(path)


class _Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "k_detail", "k_denoise", "d_th", "d_tr", "k_stretch", "k_shrink",
        "t", "s1", "s2", "m_th", "noise_a", "noise_b")] + [("noise_table", ctypes.c_void_p),
                                                            ("hf_loss", ctypes.c_double)]


@dataclass
class MergeParams:
    """Merge tuning parameters (supplement S.2 ranges; mid-range defaults)."""
    k_detail: float = 0.29
    k_denoise: float = 4.0
    d_th: float = 0.005
    d_tr: float = 0.012
    k_stretch: float = 4.0
    k_shrink: float = 2.0
    t: float = 0.12
    s1: float = 12.0
    s2: float = 2.0
    m_th: float = 0.8
    noise_a: float = 1.0
    noise_b: float = 4.0

    def c(self, noise_table=None, hf_loss: float = 0.0) -> _Params:
        """The C struct; `noise_table` (NOISE_LEVELS x 4, from noise_table()) replaces the
        closed-form noise statistics; `hf_loss` > 0 switches on the high-frequency
        rejection with that threshold."""
        # promote the float32 values the CUDA path sees
        p = _Params(*[float(np.float32(getattr(self, f.name))) for f in fields(self)], None,
                    float(np.float32(hf_loss)))
        if noise_table is not None:
            tab = np.ascontiguousarray(noise_table, dtype=np.float64)
            if tab.shape != (NOISE_LEVELS, 4):
                raise ValueError(f"noise table must be [{NOISE_LEVELS}, 4]")
            p.noise_table = tab.ctypes.data
            p._keep = tab  # the array outlives the struct's use
        return p


def lib():
    global _lib
    if _lib is None:
        # HMFSR_ORACLE_LIB: an oracle built elsewhere (the sanitizer build of the tests)
        path = os.environ.get("HMFSR_ORACLE_LIB") or build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        u16p, i32p, f32p, f64p = P(ctypes.c_uint16), P(ctypes.c_int32), P(ctypes.c_float), P(ctypes.c_double)
        ci = ctypes.c_int
        L.orc_luma.argtypes = [u16p, ci, ci, i32p]
        L.orc_structure_tensor.argtypes = [u16p, ci, ci, ci, ci, P(ctypes.c_int64)]
        L.orc_kernel_from_tensor.argtypes = [ctypes.c_int64] * 3 + [P(_Params), ci, f64p]
        L.orc_omega_plane.argtypes = [u16p, ci, ci, P(_Params), ci, f64p]
        L.orc_tile_strength.argtypes = [f32p, ci, ci, P(_Params), f64p, f64p]
        L.orc_robustness.argtypes = [u16p, u16p, ci, ci, f32p, ci, P(_Params), ci, f64p, f64p]
        L.orc_merge_rows.argtypes = [u16p, ci, ci, ci, ci, f32p, ci, P(_Params), ci, ci, ci, ci, ci,
                                     f64p, f64p, ci]
        L.orc_merge_pixels.argtypes = [u16p, ci, ci, ci, ci, f32p, ci, P(_Params), ci, ci, ci, i32p, ci,
                                       f64p, ci]
        L.orc_align.argtypes = [u16p, ci, ci, ci, ci, ci, ci, i32p, ci, i32p, f64p, i32p, ci]
        L.orc_merge_backward.argtypes = [u16p, ci, ci, ci, ci, f32p, ci, P(_Params), ci, ci, ci, f64p, f64p, f64p, ci]
        L.orc_merge_fingerprint.argtypes = [u16p, ci, ci, ci, ci, f32p, ci, P(_Params), ci, ci, ci]
        L.orc_merge_fingerprint.restype = ctypes.c_ulonglong
        L.orc_noise_table.argtypes = [ctypes.c_double, ctypes.c_double, ci, f64p]
        L.orc_noise_table.restype = None
        L.orc_philox.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
        L.orc_philox.restype = None
        for name in ("orc_luma", "orc_structure_tensor", "orc_kernel_from_tensor", "orc_omega_plane",
                     "orc_tile_strength", "orc_robustness", "orc_merge_rows", "orc_merge_pixels", "orc_align",
                     "orc_merge_backward"):
            getattr(L, name).restype = ci
        _lib = L
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _u16(a) -> np.ndarray:
    a = np.asarray(a)
    if a.dtype != np.uint16:
        a = a.astype(np.uint16)
    return np.ascontiguousarray(a)


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise ValueError(f"oracle {what} failed with {rc}")
    return rc


def n_tiles(h: int, w: int, tile: int):
    return -(-h // tile), -(-w // tile)


def luma(raw) -> np.ndarray:
    raw = _u16(raw)
    h, w = raw.shape
    out = np.empty((h // 2, w // 2), np.int32)
    _check(lib().orc_luma(_ptr(raw, ctypes.c_uint16), h, w, _ptr(out, ctypes.c_int32)), "luma")
    return out


def structure_tensor(raw, u: int, v: int) -> tuple:
    raw = _u16(raw)
    out = np.zeros(3, np.int64)
    _check(lib().orc_structure_tensor(_ptr(raw, ctypes.c_uint16), raw.shape[0], raw.shape[1], u, v,
                                      _ptr(out, ctypes.c_int64)), "structure_tensor")
    return tuple(int(x) for x in out)


def kernel_from_tensor(a: int, b: int, c: int, params: MergeParams, wl: int = 4095) -> dict:
    out = np.zeros(11, np.float64)
    p = params.c()
    _check(lib().orc_kernel_from_tensor(a, b, c, ctypes.byref(p), wl, _ptr(out, ctypes.c_double)), "kernel")
    keys = ("Oxx", "Oxy", "Oyy", "l1", "l2", "A", "D", "k_along", "k_across", "cos2t", "sin2t")
    return dict(zip(keys, out.tolist()))


def omega_plane(raw, params: MergeParams, wl: int = 4095) -> np.ndarray:
    raw = _u16(raw)
    h, w = raw.shape
    out = np.empty((3, h // 2, w // 2), np.float64)
    p = params.c()
    _check(lib().orc_omega_plane(_ptr(raw, ctypes.c_uint16), h, w, ctypes.byref(p), wl,
                                 _ptr(out, ctypes.c_double)), "omega_plane")
    return out


def tile_strength(motion_frame, params: MergeParams):
    mv = np.ascontiguousarray(motion_frame, dtype=np.float32)
    ty, tx = mv.shape[:2]
    M = np.empty((ty, tx), np.float64)
    s = np.empty((ty, tx), np.float64)
    p = params.c()
    _check(lib().orc_tile_strength(_ptr(mv, ctypes.c_float), ty, tx, ctypes.byref(p),
                                   _ptr(M, ctypes.c_double), _ptr(s, ctypes.c_double)), "tile_strength")
    return M, s


def robustness(base, alt, motion_alt, tile: int, params: MergeParams, wl: int = 4095, noise_table=None, hf_loss: float = 0.0):
    base, alt = _u16(base), _u16(alt)
    h, w = base.shape
    mv = np.ascontiguousarray(motion_alt, dtype=np.float32)
    R = np.empty((h // 2, w // 2), np.float64)
    Rh = np.empty((h // 2, w // 2), np.float64)
    p = params.c(noise_table, hf_loss)
    _check(lib().orc_robustness(_ptr(base, ctypes.c_uint16), _ptr(alt, ctypes.c_uint16), h, w,
                                _ptr(mv, ctypes.c_float), tile, ctypes.byref(p), wl,
                                _ptr(R, ctypes.c_double), _ptr(Rh, ctypes.c_double)), "robustness")
    return R, Rh


def out_size(h: int, w: int, scale) -> tuple:
    num, den = scale
    return (h * num) // den, (w * num) // den


def merge(burst, motion, params: MergeParams, scale=(1, 1), ref: int = 0, tile: int = 16, wl: int = 4095,
          rows=None, with_den: bool = False, n_threads: int = 0, noise_table=None, hf_loss: float = 0.0):
    """Oracle merge of output rows [y0, y1) (all rows by default): double [3, rows, Wo]."""
    burst = _u16(burst)
    n, h, w = burst.shape
    mv = np.ascontiguousarray(motion, dtype=np.float32)
    ty, tx = n_tiles(h, w, tile)
    if mv.shape != (n, ty, tx, 2):
        raise ValueError(f"motion must be [{n},{ty},{tx},2], got {mv.shape}")
    ho, wo = out_size(h, w, scale)
    y0, y1 = (0, ho) if rows is None else rows
    out = np.empty((3, y1 - y0, wo), np.float64)
    den = np.empty((3, y1 - y0, wo), np.float64) if with_den else None
    p = params.c(noise_table, hf_loss)
    _check(lib().orc_merge_rows(_ptr(burst, ctypes.c_uint16), n, h, w, ref, _ptr(mv, ctypes.c_float), tile,
                                ctypes.byref(p), wl, scale[0], scale[1], y0, y1, _ptr(out, ctypes.c_double),
                                _ptr(den, ctypes.c_double) if den is not None else None, n_threads), "merge")
    return (out, den) if with_den else out


def merge_pixels(burst, motion, params: MergeParams, xy, scale=(1, 1), ref: int = 0, tile: int = 16,
                 wl: int = 4095, n_threads: int = 0, noise_table=None, hf_loss: float = 0.0) -> np.ndarray:
    """Oracle merge of the output pixels xy[k] = (X, Y): double [k, 3]."""
    burst = _u16(burst)
    n, h, w = burst.shape
    mv = np.ascontiguousarray(motion, dtype=np.float32)
    xy = np.ascontiguousarray(xy, dtype=np.int32)
    out = np.empty((xy.shape[0], 3), np.float64)
    p = params.c(noise_table, hf_loss)
    _check(lib().orc_merge_pixels(_ptr(burst, ctypes.c_uint16), n, h, w, ref, _ptr(mv, ctypes.c_float), tile,
                                  ctypes.byref(p), wl, scale[0], scale[1], _ptr(xy, ctypes.c_int32),
                                  xy.shape[0], _ptr(out, ctypes.c_double), n_threads), "merge_pixels")
    return out


def align(burst, ref: int = 0, tile: int = 16, n_levels: int = 4, radius=(1, 4, 4, 4), lk_iters: int = 3,
          n_threads: int = 0):
    """Oracle alignment: (motion_int int32 [n,ty,tx,2] half-res px, motion float64
    [n,ty,tx,2] raw px, lk_skipped int32 [n,ty,tx], n_levels_used)."""
    burst = _u16(burst)
    n, h, w = burst.shape
    ty, tx = n_tiles(h, w, tile)
    mi = np.empty((n, ty, tx, 2), np.int32)
    mf = np.empty((n, ty, tx, 2), np.float64)
    fl = np.empty((n, ty, tx), np.int32)
    rad = np.zeros(4, np.int32)
    rad[:len(radius)] = radius
    nl = _check(lib().orc_align(_ptr(burst, ctypes.c_uint16), n, h, w, ref, tile, n_levels,
                                _ptr(rad, ctypes.c_int32), lk_iters, _ptr(mi, ctypes.c_int32),
                                _ptr(mf, ctypes.c_double), _ptr(fl, ctypes.c_int32), n_threads), "align")
    return mi, mf, fl, nl


PARAM_NAMES = ("k_detail", "k_denoise", "d_th", "d_tr", "k_stretch", "k_shrink", "s2", "t")


def merge_backward(burst, motion, params: MergeParams, grad_out, scale=(1, 1), ref: int = 0, tile: int = 16,
                   wl: int = 4095, n_threads: int = 0):
    """Oracle adjoint: (dL/dparams double [8] in PARAM_NAMES order, dL/dmotion double
    [n, ty, tx, 2]) for the upstream gradient grad_out = dL/dC (double [3, Ho, Wo])."""
    burst = _u16(burst)
    n, h, w = burst.shape
    mv = np.ascontiguousarray(motion, dtype=np.float32)
    ty, tx = n_tiles(h, w, tile)
    g = np.ascontiguousarray(grad_out, dtype=np.float64)
    gp = np.zeros(8, np.float64)
    gm = np.zeros((n, ty, tx, 2), np.float64)
    p = params.c()
    _check(lib().orc_merge_backward(_ptr(burst, ctypes.c_uint16), n, h, w, ref, _ptr(mv, ctypes.c_float), tile,
                                    ctypes.byref(p), wl, scale[0], scale[1], _ptr(g, ctypes.c_double),
                                    _ptr(gp, ctypes.c_double), _ptr(gm, ctypes.c_double), n_threads), "merge_backward")
    return gp, gm


def merge_fingerprint(burst, motion, params: MergeParams, scale=(1, 1), ref: int = 0, tile: int = 16,
                      wl: int = 4095) -> int:
    """Hash of every discrete decision of the merge (equal hashes: same branches)."""
    burst = _u16(burst)
    n, h, w = burst.shape
    mv = np.ascontiguousarray(motion, dtype=np.float32)
    p = params.c()
    return int(lib().orc_merge_fingerprint(_ptr(burst, ctypes.c_uint16), n, h, w, ref, _ptr(mv, ctypes.c_float),
                                           tile, ctypes.byref(p), wl, scale[0], scale[1]))


# ---------------------------------------------------------------------------------------
# Noise-dependent tuning (supplement: "Noise-dependent Tuning"; "Tuning Procedure and
# Parameters").  The SNR of the base frame (one raw sample, one frame) is the mean
# brightness over its noise standard deviation under var(x) = a x + b; the parameters
# that trade resolution against denoising are piecewise linear in SNR over [6, 30],
# running from the denoising end of the printed ranges (low SNR) to the detail end; the
# tile is 16 px and grows to 32 and 64 px in very low light.
# ---------------------------------------------------------------------------------------
SNR_RANGE = (6.0, 30.0)
# parameter: (value at SNR <= 6, value at SNR >= 30)
SNR_RAMPS = {"k_detail": (0.33, 0.25), "k_denoise": (5.0, 3.0), "d_th": (0.010, 0.001), "d_tr": (0.020, 0.006)}
FIXED_TUNING = {"k_stretch": 4.0, "k_shrink": 2.0, "t": 0.12, "s1": 12.0, "s2": 2.0, "m_th": 0.8}


def frame_mean(frame) -> float:
    """Mean sample value of one raw frame, from its exact integer sum."""
    f = np.asarray(frame)
    return int(f.astype(np.int64).sum()) / f.size


def snr_of(mean: float, noise_a: float, noise_b: float) -> float:
    var = noise_a * mean + noise_b
    return mean / np.sqrt(var) if var > 0 else float("inf")


def snr_tuning(mean: float, noise_a: float, noise_b: float) -> dict:
    """Every tuned value for a base frame of mean brightness `mean` (DN)."""
    snr = snr_of(mean, noise_a, noise_b)
    lo, hi = SNR_RANGE
    s = hi if np.isinf(snr) else snr
    frac = min(max((s - lo) / (hi - lo), 0.0), 1.0)
    out = {k: (1.0 - frac) * a + frac * b for k, (a, b) in SNR_RAMPS.items()}
    out.update(FIXED_TUNING)
    # very low light: the lowest third of the range, split in two
    out["tile"] = 64 if s < 10.0 else (32 if s < 14.0 else 16)
    out["snr"] = snr
    return out



# ---------------------------------------------------------------------------------------
# Monte-Carlo noise statistics (Sec. 5.2.2): sigma_md^2 and d_md^2 per brightness level
# ---------------------------------------------------------------------------------------
NOISE_LEVELS = 129
NOISE_TRIALS = 4096


def noise_table(noise_a: float, noise_b: float, wl: int = 4095) -> np.ndarray:
    """double [NOISE_LEVELS, 4]: per brightness level i WL / (NOISE_LEVELS - 1), the trial
    means of {3x3 population variance red/blue, green; squared difference of two patch
    means red/blue, green} (orc_noise_table).  noise_a / noise_b are promoted from float32,
    as the CUDA path sees them."""
    L = lib()
    out = np.empty((NOISE_LEVELS, 4), dtype=np.float64)
    L.orc_noise_table(float(np.float32(noise_a)), float(np.float32(noise_b)), int(wl),
                      _ptr(out, ctypes.c_double))
    return out


def philox(ctr, key) -> tuple:
    """Philox-4x32-10 of the 4-word counter under the 2-word key (orc_philox)."""
    L = lib()
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    L.orc_philox(c, k, o)
    return tuple(o)


# ---------------------------------------------------------------------------------------
# Subpixel alignment by a quadratic fit to the block-matching error (Sec. 3.2: the variant
# the paper explored before settling on Lucas-Kanade)
# ---------------------------------------------------------------------------------------
def parabola_vertex(em: int, e0: int, ep: int) -> float:
    """Vertex offset of the parabola through (-1, em), (0, e0), (1, ep): (em - ep) /
    (2 (em - 2 e0 + ep)), 0 when the curvature is not positive, clamped to [-1/2, 1/2]."""
    den = 2 * (em - 2 * e0 + ep)
    if den <= 0:
        return 0.0
    return min(max(float(em - ep) / float(den), -0.5), 0.5)


def tile_ssd(lq_ref: np.ndarray, lq_alt: np.ndarray, x0: int, y0: int, t: int, ox: int, oy: int) -> int:
    """Exact SSD of the t x t tile at (x0, y0) of the base level against the other frame
    displaced by (ox, oy), reads clamped as in the block-matching search: the base at the
    clamped tile pixel, the other frame at the clamped displaced (unclamped) pixel."""
    lh, lw = lq_ref.shape
    ys, xs = np.arange(y0, y0 + t), np.arange(x0, x0 + t)
    r = lq_ref[np.ix_(np.minimum(ys, lh - 1), np.minimum(xs, lw - 1))].astype(np.int64)
    a = lq_alt[np.ix_(np.clip(ys + oy, 0, lh - 1), np.clip(xs + ox, 0, lw - 1))].astype(np.int64)
    return int(((r - a) ** 2).sum())


def align_quadfit(burst, ref: int = 0, tile: int = 16, n_levels: int = 4, radius=(1, 4, 4, 4)):
    """(motion_int int32 [n,ty,tx,2], motion float32 [n,ty,tx,2] raw px): the pyramid
    search's integer vectors, refined per axis by the vertex of the parabola through the
    level-0 SSD at the vector and its two neighbours on that axis (FP64, then float32)."""
    burst = _u16(burst)
    n, h, w = burst.shape
    mi, _, _, _ = align(burst, ref, tile, n_levels, radius, lk_iters=0)
    lq = [luma(burst[f]) for f in range(n)]
    t = tile // 2
    ty, tx = n_tiles(h, w, tile)
    mf = np.zeros((n, ty, tx, 2), np.float32)
    for f in range(n):
        if f == ref:
            continue
        for j in range(ty):
            for i in range(tx):
                ux, uy = int(mi[f, j, i, 0]), int(mi[f, j, i, 1])
                e = lambda dx, dy: tile_ssd(lq[ref], lq[f], i * t, j * t, t, ux + dx, uy + dy)
                e0 = e(0, 0)
                dx = parabola_vertex(e(-1, 0), e0, e(1, 0))
                dy = parabola_vertex(e(0, -1), e0, e(0, 1))
                mf[f, j, i, 0] = np.float32(2.0 * (ux + dx))
                mf[f, j, i, 1] = np.float32(2.0 * (uy + dy))
    return mi, mf



def hf_loss_map(base, kappa: float) -> np.ndarray:
    """bool [H/2, W/2]: the high-frequency test of every base texel, restated in NumPy from
    exact integer sums (the variance of the 3x3 local means against kappa times the 3x3
    variance, R and B at full weight, green at a quarter)."""
    base = _u16(base).astype(np.int64)
    q = {0: base[0::2, 0::2], 1: base[0::2, 1::2] + base[1::2, 0::2], 2: base[1::2, 1::2]}
    hh, wh = q[0].shape
    pad = lambda a: np.pad(a, 1, mode="edge")
    def box(a):
        p = pad(a)
        return sum(p[j:j + hh, i:i + wh] for j in range(3) for i in range(3))
    A = np.zeros((hh, wh), np.int64)
    B = np.zeros((hh, wh), np.int64)
    for c, wgt in ((0, 4), (1, 1), (2, 4)):
        s1, s2 = box(q[c]), box(q[c] * q[c])
        B += wgt * (9 * s2 - s1 * s1)
        A += wgt * (9 * box(s1 * s1) - box(s1) ** 2)
    return (B > 0) & (A.astype(np.float64) < float(np.float32(kappa)) * (81.0 * B.astype(np.float64)))
