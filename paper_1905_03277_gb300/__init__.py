"""Handheld multi-frame super-resolution (Wronski et al. 2019) on one sm_103a GPU.

Thin Python binding over the C-ABI library libhmfsr.so (include/hmfsr.h).  PyTorch
provides device memory and streams; every step of the method runs in the library's
hand-written CUDA kernels.  The calls follow the paper's statement of the problem:

    motion = align(burst, ref)                           # Sec. 3.2
    rgb = merge(burst, motion, params, scale)            # Sec. 5, Eq. 1-9

`burst` is a torch.uint16 tensor [n_frames, height, width] of RGGB Bayer frames.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, fields

import torch

from . import _lib
from ._lib import build  # noqa: F401  (re-exported)

__all__ = ["MergeParams", "AlignParams", "align", "merge", "merge_stages", "align_merge", "AlignMergePipeline", "build",
           "workspace_size", "out_size", "n_tiles", "frame_sum", "snr_tuning", "auto_params", "noise_table", "merge_noise", "merge_ex"]


@dataclass
class MergeParams:
    """Merge tuning (supplement S.2 ranges; mid-range defaults) and the noise model
    var(x) = noise_a * x + noise_b in DN^2 (Sec. 5.2.2)."""
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
    tile: int = 16

    def c(self) -> _lib.MergeParamsC:
        vals = [getattr(self, f.name) for f in fields(self) if f.name != "tile"]
        return _lib.MergeParamsC(*[float(v) for v in vals], int(self.tile))


@dataclass
class AlignParams:
    """Pyramid block matching + Lucas-Kanade (Sec. 3.2)."""
    tile: int = 16
    n_levels: int = 4
    radius: tuple = (1, 4, 4, 4)
    lk_iters: int = 3

    def c(self) -> _lib.AlignParamsC:
        r = (ctypes.c_int * 4)(*list(self.radius) + [0] * (4 - len(self.radius)))
        return _lib.AlignParamsC(int(self.tile), int(self.n_levels), r, int(self.lk_iters))


def n_tiles(h: int, w: int, tile: int):
    return -(-h // tile), -(-w // tile)


def out_size(h: int, w: int, scale) -> tuple:
    num, den = scale
    return (h * num) // den, (w * num) // den


def _desc(burst: torch.Tensor, ref: int, white_level: int) -> _lib.BurstDesc:
    if burst.dtype != torch.uint16 or burst.dim() != 3:
        raise TypeError("burst must be a torch.uint16 tensor [n_frames, height, width]")
    if burst.stride(2) != 1 or burst.stride(0) != burst.shape[1] * burst.stride(1):
        raise ValueError("burst rows must be contiguous with frames packed back to back")
    n, h, w = burst.shape
    return _lib.BurstDesc(n, h, w, burst.stride(1), ref, 0, white_level, 0)


def _merge_inputs(burst: torch.Tensor, motion: torch.Tensor, params: MergeParams, ref: int, white_level: int,
                  *others: torch.Tensor | None) -> _lib.BurstDesc:
    """The checks every merge-family call makes before handing pointers to the library:
    burst and motion (and any other given tensors) on one CUDA device, the burst's layout,
    and motion contiguous float32 [n, TY, TX, 2] for the params' tile.  Raises before any
    launch; returns the burst descriptor."""
    if not (burst.is_cuda and motion.is_cuda) or motion.device != burst.device:
        raise ValueError("burst and motion must be on the same CUDA device")
    for t in others:
        if t is not None and (not t.is_cuda or t.device != burst.device):
            raise ValueError("every tensor argument must be on the burst's CUDA device")
    d = _desc(burst, ref, white_level)
    n, h, w = burst.shape
    ty, tx = n_tiles(h, w, params.tile)
    if motion.dtype != torch.float32 or tuple(motion.shape) != (n, ty, tx, 2) or not motion.is_contiguous():
        raise ValueError(f"motion must be contiguous float32 [{n},{ty},{tx},2]")
    return d


def _ptr(t: torch.Tensor | None):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(device, stream):
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return ctypes.c_void_p(s.cuda_stream)


_ws_cache: dict = {}


def _workspace(device: torch.device, nbytes: int, stream=None) -> torch.Tensor:
    """A reusable, 256-byte aligned scratch buffer per (device, stream), grown on demand.
    Calls on one stream run in order and share it; calls on different streams get their
    own, so concurrent calls never race on scratch.  The buffer is allocated on that
    stream, so the caching allocator orders its reuse after the stream's work."""
    s = stream if stream is not None else torch.cuda.current_stream(device)
    key = (device.type, device.index, s.cuda_stream)
    buf = _ws_cache.get(key)
    if buf is None or buf.numel() < nbytes + 256:
        with torch.cuda.stream(s):
            _ws_cache[key] = buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    off = (-buf.data_ptr()) % 256
    return buf[off:off + max(nbytes, 1)]


def workspace_size(op: int, burst_shape, tile: int, scale=(1, 1), white_level: int = 4095) -> int:
    n, h, w = burst_shape
    d = _lib.BurstDesc(n, h, w, w, 0, 0, white_level, 0)
    return int(_lib.load().hmfsr_workspace_size(op, ctypes.byref(d), tile, scale[0], scale[1]))


def align(burst: torch.Tensor, ref: int = 0, params: AlignParams | None = None, with_int: bool = False,
          white_level: int = 4095, stream=None, subpixel: str = "lk"):
    """Tile motion field float32 [n, TY, TX, 2] in raw px (base -> frame), computed by
    hmfsr_align (subpixel="lk") or hmfsr_align_quadfit (subpixel="quadfit").  With
    `with_int`, also the integer block-matching vectors (half-res px)."""
    L = _lib.load()
    params = params or AlignParams()
    if not burst.is_cuda:
        raise ValueError("burst must be on a CUDA device")
    d = _desc(burst, ref, white_level)
    n, h, w = burst.shape
    ty, tx = n_tiles(h, w, params.tile)
    motion = torch.empty((n, ty, tx, 2), dtype=torch.float32, device=burst.device)
    mint = torch.empty((n, ty, tx, 2), dtype=torch.int32, device=burst.device) if with_int else None
    nbytes = L.hmfsr_workspace_size(_lib.OP_ALIGN, ctypes.byref(d), params.tile, 1, 1)
    ws = _workspace(burst.device, nbytes, stream)
    pc = params.c()
    if subpixel not in ("lk", "quadfit"):
        raise ValueError("subpixel must be 'lk' (Lucas-Kanade) or 'quadfit' (quadratic fit to the matching error)")
    fn = L.hmfsr_align if subpixel == "lk" else L.hmfsr_align_quadfit
    _lib.check(fn(_ptr(burst), ctypes.byref(d), ctypes.byref(pc), _ptr(motion), _ptr(mint), _ptr(ws), ws.numel(),
                  _stream(burst.device, stream)), "hmfsr_align")
    return (motion, mint) if with_int else motion


def _own_workspace(workspace: torch.Tensor, nbytes: int, device) -> torch.Tensor:
    """A caller's workspace tensor checked for the library: uint8 on the device, at least
    nbytes, 256-byte aligned."""
    if (workspace.dtype != torch.uint8 or not workspace.is_cuda or workspace.device != device
            or not workspace.is_contiguous() or workspace.numel() < nbytes or workspace.data_ptr() % 256):
        raise ValueError(f"workspace must be a contiguous, 256-byte aligned uint8 tensor of at least {nbytes} "
                         "bytes on the burst's device")
    return workspace


def backward_workspace(burst_shape, tile: int = 16, scale=(1, 1), device=None, white_level: int = 4095):
    """A workspace for `merge` followed by `merge_backward(..., prepared=True)`: sized for
    the adjoint, 256-byte aligned."""
    nbytes = workspace_size(_lib.OP_MERGE_BACKWARD, burst_shape, tile, scale, white_level)
    if nbytes == 0:
        raise ValueError("unsupported burst shape, tile or scale")
    buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=device or "cuda")
    off = (-buf.data_ptr()) % 256
    return buf[off:off + nbytes]


def merge(burst: torch.Tensor, motion: torch.Tensor, params: MergeParams | None = None, scale=(1, 1), ref: int = 0,
          with_den: bool = False, white_level: int = 4095, stream=None, workspace: torch.Tensor | None = None):
    """Merged RGB float32 [3, Ho, Wo] in DN (hmfsr_merge).  With `with_den`, also the
    per-channel log2 of Eq. 1's denominator.  `workspace`: the caller's scratch (e.g. from
    `backward_workspace`, so that `merge_backward(..., prepared=True)` reuses its planes)."""
    L = _lib.load()
    params = params or MergeParams()
    d = _merge_inputs(burst, motion, params, ref, white_level)
    n, h, w = burst.shape
    ho, wo = out_size(h, w, scale)
    rgb = torch.empty((3, ho, wo), dtype=torch.float32, device=burst.device)
    den = torch.empty((3, ho, wo), dtype=torch.float32, device=burst.device) if with_den else None
    nbytes = L.hmfsr_workspace_size(_lib.OP_MERGE, ctypes.byref(d), params.tile, scale[0], scale[1])
    ws = _own_workspace(workspace, nbytes, burst.device) if workspace is not None else \
        _workspace(burst.device, nbytes, stream)
    pc = params.c()
    _lib.check(L.hmfsr_merge(_ptr(burst), ctypes.byref(d), _ptr(motion), ctypes.byref(pc), scale[0], scale[1],
                             _ptr(rgb), _ptr(den), _ptr(ws), ws.numel(), _stream(burst.device, stream)),
               "hmfsr_merge")
    return (rgb, den) if with_den else rgb


def merge_chunked(burst: torch.Tensor, motion: torch.Tensor, params: MergeParams | None = None, scale=(1, 1),
                  ref: int = 0, chunk_frames: int = 2, with_den: bool = False, white_level: int = 4095, stream=None):
    """hmfsr_merge_chunked: the same RGB as `merge`, bit for bit, from a workspace that does
    not grow with the frame count (chunk_frames non-base frames at a time; the running
    sums stay in the workspace between chunks)."""
    L = _lib.load()
    params = params or MergeParams()
    d = _merge_inputs(burst, motion, params, ref, white_level)
    n, h, w = burst.shape
    ho, wo = out_size(h, w, scale)
    rgb = torch.empty((3, ho, wo), dtype=torch.float32, device=burst.device)
    den = torch.empty((3, ho, wo), dtype=torch.float32, device=burst.device) if with_den else None
    nbytes = L.hmfsr_merge_chunked_workspace_size(ctypes.byref(d), params.tile, scale[0], scale[1], int(chunk_frames))
    if nbytes == 0:
        raise ValueError("unsupported burst shape, tile, scale or chunk size")
    ws = _workspace(burst.device, nbytes, stream)
    pc = params.c()
    _lib.check(L.hmfsr_merge_chunked(_ptr(burst), ctypes.byref(d), _ptr(motion), ctypes.byref(pc), scale[0], scale[1],
                                     int(chunk_frames), _ptr(rgb), _ptr(den), _ptr(ws), ws.numel(),
                                     _stream(burst.device, stream)), "hmfsr_merge_chunked")
    return (rgb, den) if with_den else rgb


def chunked_workspace_size(burst_shape, tile: int = 16, scale=(1, 1), chunk_frames: int = 2,
                           white_level: int = 4095) -> int:
    n, h, w = burst_shape
    d = _lib.BurstDesc(n, h, w, w, 0, 0, white_level, 0)
    return int(_lib.load().hmfsr_merge_chunked_workspace_size(ctypes.byref(d), tile, scale[0], scale[1],
                                                              int(chunk_frames)))


def merge_stages(burst: torch.Tensor, motion: torch.Tensor, params: MergeParams | None = None, ref: int = 0,
                 white_level: int = 4095, stream=None):
    """Per-frame merge stages: Omega entries float32 [n, 3, H/2, W/2] (Eq. 4) and the
    final robustness Rhat float32 [n, H/2, W/2] on the base grid (Eq. 9)."""
    L = _lib.load()
    params = params or MergeParams()
    d = _merge_inputs(burst, motion, params, ref, white_level)
    n, h, w = burst.shape
    omega = torch.empty((n, 3, h // 2, w // 2), dtype=torch.float32, device=burst.device)
    rhat = torch.empty((n, h // 2, w // 2), dtype=torch.float32, device=burst.device)
    nbytes = L.hmfsr_workspace_size(_lib.OP_MERGE_STAGES, ctypes.byref(d), params.tile, 1, 1)
    ws = _workspace(burst.device, nbytes, stream)
    pc = params.c()
    _lib.check(L.hmfsr_merge_stages(_ptr(burst), ctypes.byref(d), _ptr(motion), ctypes.byref(pc), _ptr(omega),
                                    _ptr(rhat), _ptr(ws), ws.numel(), _stream(burst.device, stream)),
               "hmfsr_merge_stages")
    return omega, rhat


def align_merge(burst: torch.Tensor, params: MergeParams | None = None, scale=(1, 1), ref: int = 0,
                align_params: AlignParams | None = None, device=None, out=None, white_level: int = 4095,
                stream=None, with_motion: bool = False):
    """The whole path in one call (hmfsr_align_merge): align, then merge, with the merge's
    motion-free preparation overlapping the alignment.  A device `burst` gives a device RGB
    (written into `out` when given); a host `burst` (ideally pinned) is copied to the
    device first and the RGB copied back into `out` (or a new pinned host tensor).  With
    `with_motion`, also the motion field (on the device)."""
    L = _lib.load()
    params = params or MergeParams()
    align_params = align_params or AlignParams(tile=params.tile)
    if align_params.tile != params.tile:
        raise ValueError("the alignment tile and the merge tile must match")
    host = not burst.is_cuda
    dev_burst = burst.to(device or "cuda", non_blocking=True) if host else burst
    d = _desc(dev_burst, ref, white_level)
    n, h, w = dev_burst.shape
    ty, tx = n_tiles(h, w, params.tile)
    ho, wo = out_size(h, w, scale)
    dv = dev_burst.device
    motion = torch.empty((n, ty, tx, 2), dtype=torch.float32, device=dv)
    if not host and out is not None:
        if not out.is_cuda or out.device != dv or out.dtype != torch.float32 or tuple(out.shape) != (3, ho, wo) \
                or not out.is_contiguous():
            raise ValueError(f"out must be contiguous float32 [3,{ho},{wo}] on the burst's device")
        rgb = out
    else:
        rgb = torch.empty((3, ho, wo), dtype=torch.float32, device=dv)
    nbytes = L.hmfsr_workspace_size(_lib.OP_ALIGN_MERGE, ctypes.byref(d), params.tile, scale[0], scale[1])
    if nbytes == 0:
        raise ValueError("unsupported burst shape, tile or scale")
    ws = _workspace(dv, nbytes, stream)
    ap, mp = align_params.c(), params.c()
    _lib.check(L.hmfsr_align_merge(_ptr(dev_burst), ctypes.byref(d), ctypes.byref(ap), ctypes.byref(mp), scale[0],
                                   scale[1], _ptr(motion), None, _ptr(rgb), None, _ptr(ws), ws.numel(),
                                   _stream(dv, stream)), "hmfsr_align_merge")
    if host:
        if out is None:
            out = torch.empty(rgb.shape, dtype=rgb.dtype, pin_memory=True)
        out.copy_(rgb, non_blocking=True)
        rgb = out
    return (rgb, motion) if with_motion else rgb


class AlignMergePipeline:
    """The whole path over a stream of host bursts of one shape, with the copies of one
    burst overlapped with the compute of another.

    `depth` device slots each hold a burst, its motion field and its RGB result.  Per
    `submit`, the host burst is copied in on a copy stream, aligned and merged (through
    hmfsr_align_merge) on a compute stream, and the RGB copied back into the
    caller's host tensor on a second copy stream; CUDA events order the three, so burst
    k + 1 travels in and burst k - 1 travels out while burst k is merged.  Host buffers
    should be pinned; the caller keeps a submitted burst and its output untouched until
    `synchronize` (or a later submit of the same slot) says the copies are done.  Every
    device buffer is allocated once, here."""

    def __init__(self, shape, params: MergeParams | None = None, scale=(1, 1), ref: int = 0,
                 align_params: AlignParams | None = None, device=None, white_level: int = 4095, depth: int = 2):
        L = _lib.load()
        self.params = params or MergeParams()
        self.align_params = align_params or AlignParams(tile=self.params.tile)
        self.scale, self.ref, self.white_level, self.depth = tuple(scale), ref, white_level, depth
        self.device = torch.device(device or "cuda")
        n, h, w = shape
        self.shape = (n, h, w)
        ty, tx = n_tiles(h, w, self.params.tile)
        ho, wo = out_size(h, w, scale)
        mk = lambda *a, **k: torch.empty(*a, device=self.device, **k)
        self.bursts = [mk((n, h, w), dtype=torch.uint16) for _ in range(depth)]
        self.motions = [mk((n, ty, tx, 2), dtype=torch.float32) for _ in range(depth)]
        self.rgbs = [mk((3, ho, wo), dtype=torch.float32) for _ in range(depth)]
        self.desc = _desc(self.bursts[0], ref, white_level)
        if self.align_params.tile != self.params.tile:
            raise ValueError("the alignment tile and the merge tile must match")
        nb = L.hmfsr_workspace_size(_lib.OP_ALIGN_MERGE, ctypes.byref(self.desc), self.params.tile, scale[0],
                                    scale[1])
        if nb == 0:
            raise ValueError("unsupported burst shape, tile or scale")
        self._ws_raw = mk(nb + 256, dtype=torch.uint8)  # one compute stream: the slots share it
        base = (-self._ws_raw.data_ptr()) % 256
        self.ws = self._ws_raw[base:base + nb]
        self.h2d, self.compute, self.d2h = (torch.cuda.Stream(self.device) for _ in range(3))
        self.ev_in = [torch.cuda.Event() for _ in range(depth)]
        self.ev_done = [torch.cuda.Event() for _ in range(depth)]
        self.ev_out = [torch.cuda.Event() for _ in range(depth)]
        self.used = [False] * depth
        self.k = 0
        self._ap, self._mp = self.align_params.c(), self.params.c()

    def submit(self, host_burst: torch.Tensor, host_out: torch.Tensor) -> None:
        L = _lib.load()
        if tuple(host_burst.shape) != self.shape or host_burst.dtype != torch.uint16:
            raise ValueError(f"burst must be uint16 {self.shape}")
        i = self.k % self.depth
        self.k += 1
        b, mv, rgb = self.bursts[i], self.motions[i], self.rgbs[i]
        with torch.cuda.stream(self.h2d):
            if self.used[i]:
                self.h2d.wait_event(self.ev_done[i])  # the slot's previous burst has been merged
            b.copy_(host_burst, non_blocking=True)
            self.ev_in[i].record(self.h2d)
        self.compute.wait_event(self.ev_in[i])
        if self.used[i]:
            self.compute.wait_event(self.ev_out[i])  # the slot's previous RGB has been read out
        cs = ctypes.c_void_p(self.compute.cuda_stream)
        _lib.check(L.hmfsr_align_merge(_ptr(b), ctypes.byref(self.desc), ctypes.byref(self._ap),
                                       ctypes.byref(self._mp), self.scale[0], self.scale[1], _ptr(mv), None, _ptr(rgb),
                                       None, _ptr(self.ws), self.ws.numel(), cs), "hmfsr_align_merge")
        self.ev_done[i].record(self.compute)
        with torch.cuda.stream(self.d2h):
            self.d2h.wait_event(self.ev_done[i])
            host_out.copy_(rgb, non_blocking=True)
            self.ev_out[i].record(self.d2h)
        self.used[i] = True

    def synchronize(self) -> None:
        """Wait until every submitted burst's result is in its host tensor."""
        for st in (self.h2d, self.compute, self.d2h):
            st.synchronize()


def frame_sum(burst: torch.Tensor, frame: int = 0, stream=None, out: torch.Tensor | None = None):
    """Exact sum of one frame's samples (hmfsr_frame_sum), read back to the host; with
    `out` (a one-element int64 device tensor) the sum stays there and the call returns
    without waiting."""
    L = _lib.load()
    d = _desc(burst, 0, 4095)
    dst = out if out is not None else torch.empty(1, dtype=torch.int64, device=burst.device)  # < 2^63
    _lib.check(L.hmfsr_frame_sum(_ptr(burst), ctypes.byref(d), frame, _ptr(dst), _stream(burst.device, stream)),
               "hmfsr_frame_sum")
    return dst if out is not None else int(dst.item())


def snr_tuning(sample_sum: int, sample_count: int, noise_a: float, noise_b: float):
    """(MergeParams, AlignParams, snr) for a base frame whose samples sum to `sample_sum`
    over `sample_count` samples (mean brightness in DN = their quotient, taken in C) and
    the noise model var = noise_a * x + noise_b (hmfsr_snr_tuning; host arithmetic)."""
    L = _lib.load()
    mp, ap, snr = _lib.MergeParamsC(), _lib.AlignParamsC(), ctypes.c_double()
    _lib.check(L.hmfsr_snr_tuning(int(sample_sum), int(sample_count), float(noise_a), float(noise_b),
                                  ctypes.byref(mp), ctypes.byref(ap), ctypes.byref(snr)), "hmfsr_snr_tuning")
    m = MergeParams(**{f.name: getattr(mp, f.name) for f in fields(MergeParams)})
    a = AlignParams(tile=ap.tile, n_levels=ap.n_levels, radius=tuple(ap.radius), lk_iters=ap.lk_iters)
    return m, a, snr.value


def auto_params(burst: torch.Tensor, noise_a: float, noise_b: float, ref: int = 0, stream=None):
    """The paper's automatic parameter choice for this burst: the base frame's mean
    brightness (one device reduction and an 8-byte read back) and the noise model give
    the SNR, and the SNR every parameter.  Returns (MergeParams, AlignParams, snr)."""
    n, h, w = burst.shape
    return snr_tuning(frame_sum(burst, ref, stream), h * w, noise_a, noise_b)


def noise_table(noise_a: float, noise_b: float, white_level: int = 4095, device=None, stream=None) -> torch.Tensor:
    """Monte-Carlo noise statistics (hmfsr_noise_table): float32 [129, 4] on the device,
    per brightness level {sigma_md^2 red/blue, green; d_md^2 red/blue, green}."""
    L = _lib.load()
    dev = torch.device(device or "cuda")
    tab = torch.empty((_lib.NOISE_LEVELS, 4), dtype=torch.float32, device=dev)
    _lib.check(L.hmfsr_noise_table(float(noise_a), float(noise_b), int(white_level), _ptr(tab), _stream(dev, stream)),
               "hmfsr_noise_table")
    return tab


def merge_noise(burst: torch.Tensor, motion: torch.Tensor, table: torch.Tensor, params: MergeParams | None = None,
                scale=(1, 1), ref: int = 0, with_den: bool = False, white_level: int = 4095, stream=None):
    """`merge` with the robustness's noise statistics from a `noise_table` (hmfsr_merge_noise)."""
    L = _lib.load()
    params = params or MergeParams()
    d = _merge_inputs(burst, motion, params, ref, white_level, table)
    if table.dtype != torch.float32 or tuple(table.shape) != (_lib.NOISE_LEVELS, 4) or not table.is_contiguous():
        raise ValueError(f"noise table must be contiguous float32 [{_lib.NOISE_LEVELS},4]")
    n, h, w = burst.shape
    ho, wo = out_size(h, w, scale)
    rgb = torch.empty((3, ho, wo), dtype=torch.float32, device=burst.device)
    den = torch.empty((3, ho, wo), dtype=torch.float32, device=burst.device) if with_den else None
    nbytes = L.hmfsr_workspace_size(_lib.OP_MERGE, ctypes.byref(d), params.tile, scale[0], scale[1])
    ws = _workspace(burst.device, nbytes, stream)
    pc = params.c()
    _lib.check(L.hmfsr_merge_noise(_ptr(burst), ctypes.byref(d), _ptr(motion), ctypes.byref(pc), _ptr(table), scale[0],
                                   scale[1], _ptr(rgb), _ptr(den), _ptr(ws), ws.numel(), _stream(burst.device, stream)),
               "hmfsr_merge_noise")
    return (rgb, den) if with_den else rgb


def merge_ex(burst: torch.Tensor, motion: torch.Tensor, params: MergeParams | None = None, scale=(1, 1), ref: int = 0,
             noise_table: torch.Tensor | None = None, hf_loss: float = 0.0, with_den: bool = False,
             white_level: int = 4095, stream=None):
    """`merge` with the options of hmfsr_merge_ex: Monte-Carlo noise statistics from
    `noise_table` (from noise_table()) and the high-frequency rejection with threshold
    `hf_loss` (0: off)."""
    L = _lib.load()
    params = params or MergeParams()
    d = _merge_inputs(burst, motion, params, ref, white_level, noise_table)
    if noise_table is not None and (noise_table.dtype != torch.float32 or not noise_table.is_contiguous()
                                    or tuple(noise_table.shape) != (_lib.NOISE_LEVELS, 4)):
        raise ValueError(f"noise table must be contiguous float32 [{_lib.NOISE_LEVELS},4]")
    n, h, w = burst.shape
    ho, wo = out_size(h, w, scale)
    rgb = torch.empty((3, ho, wo), dtype=torch.float32, device=burst.device)
    den = torch.empty((3, ho, wo), dtype=torch.float32, device=burst.device) if with_den else None
    nbytes = L.hmfsr_workspace_size(_lib.OP_MERGE, ctypes.byref(d), params.tile, scale[0], scale[1])
    ws = _workspace(burst.device, nbytes, stream)
    pc = params.c()
    opts = _lib.MergeOptionsC(noise_table.data_ptr() if noise_table is not None else None, float(hf_loss))
    _lib.check(L.hmfsr_merge_ex(_ptr(burst), ctypes.byref(d), _ptr(motion), ctypes.byref(pc), ctypes.byref(opts),
                                scale[0], scale[1], _ptr(rgb), _ptr(den), _ptr(ws), ws.numel(),
                                _stream(burst.device, stream)), "hmfsr_merge_ex")
    return (rgb, den) if with_den else rgb


def merge_prepare(burst: torch.Tensor, motion: torch.Tensor, params: MergeParams | None = None, ref: int = 0,
                  white_level: int = 4095, stream=None, workspace: torch.Tensor | None = None) -> torch.Tensor:
    """First half of `merge` (hmfsr_merge_prepare): per-frame planes into a workspace,
    returned for `merge_accumulate` to read.  By default the planes get a buffer of their
    own (from PyTorch's caching allocator, on the call's stream), so no later call of this
    module can overwrite them; a caller may pass its own `workspace` instead (uint8,
    contiguous, 256-byte aligned, at least workspace_size(OP_MERGE_STAGES, ...) bytes)."""
    L = _lib.load()
    params = params or MergeParams()
    d = _merge_inputs(burst, motion, params, ref, white_level, workspace)
    nbytes = L.hmfsr_workspace_size(_lib.OP_MERGE_STAGES, ctypes.byref(d), params.tile, 1, 1)
    if workspace is None:
        s = stream if stream is not None else torch.cuda.current_stream(burst.device)
        with torch.cuda.stream(s):
            buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=burst.device)
        off = (-buf.data_ptr()) % 256
        ws = buf[off:off + nbytes]
    else:
        if (workspace.dtype != torch.uint8 or workspace.device != burst.device or workspace.numel() < nbytes
                or workspace.data_ptr() % 256 or not workspace.is_contiguous()):
            raise ValueError(f"workspace must be a contiguous, 256-byte aligned uint8 tensor of >= {nbytes} bytes "
                             "on the burst's device")
        ws = workspace
    pc = params.c()
    _lib.check(L.hmfsr_merge_prepare(_ptr(burst), ctypes.byref(d), _ptr(motion), ctypes.byref(pc), _ptr(ws),
                                     ws.numel(), _stream(burst.device, stream)), "hmfsr_merge_prepare")
    return ws


def merge_accumulate(burst: torch.Tensor, motion: torch.Tensor, ws: torch.Tensor, params: MergeParams | None = None,
                     scale=(1, 1), ref: int = 0, out: torch.Tensor | None = None, den: torch.Tensor | None = None,
                     white_level: int = 4095, stream=None) -> torch.Tensor:
    """Second half of `merge` (hmfsr_merge_accumulate) from the planes in `ws`."""
    L = _lib.load()
    params = params or MergeParams()
    d = _merge_inputs(burst, motion, params, ref, white_level, ws, out, den)
    n, h, w = burst.shape
    ho, wo = out_size(h, w, scale)
    nbytes = L.hmfsr_workspace_size(_lib.OP_MERGE_STAGES, ctypes.byref(d), params.tile, 1, 1)
    if ws.dtype != torch.uint8 or ws.numel() < nbytes or ws.data_ptr() % 256 or not ws.is_contiguous():
        raise ValueError(f"ws must be the planes merge_prepare returned (>= {nbytes} aligned bytes)")
    for t, what in ((out, "out"), (den, "den")):
        if t is not None and (t.dtype != torch.float32 or tuple(t.shape) != (3, ho, wo) or not t.is_contiguous()):
            raise ValueError(f"{what} must be contiguous float32 [3,{ho},{wo}]")
    if out is None:
        out = torch.empty((3, ho, wo), dtype=torch.float32, device=burst.device)
    pc = params.c()
    _lib.check(L.hmfsr_merge_accumulate(_ptr(burst), ctypes.byref(d), _ptr(motion), ctypes.byref(pc), scale[0],
                                        scale[1], _ptr(out), _ptr(den), _ptr(ws), ws.numel(),
                                        _stream(burst.device, stream)), "hmfsr_merge_accumulate")
    return out


def pyramid_levels(h: int, w: int, n_levels_max: int = 4) -> int:
    """Number of alignment pyramid levels for a frame (factors 2, 4, 4; sides >= 16)."""
    lh, lw, nl = h // 2, w // 2, 1
    for f in (2, 4, 4)[: max(0, min(n_levels_max, 4) - 1)]:
        lh, lw = lh // f, lw // f
        if lh < 16 or lw < 16:
            break
        nl += 1
    return nl


def launches_per_call(n_frames: int, h: int, w: int, n_levels_max: int = 4, tile: int = 16,
                      radius0: int = 1) -> dict:
    """Kernel launches made by one hmfsr_align / hmfsr_merge_prepare / accumulate call."""
    nl = pyramid_levels(h, w, n_levels_max)
    # align: levels 0 and 1 in one launch, levels 2 and 3 in one, one search per level, LK;
    # with tiles of 16 px or less and radius 1 at level 0, that level's search runs inside
    # the Lucas-Kanade launch
    fused = tile <= 16 and radius0 == 1
    return {"align": 1 + (1 if nl > 2 else 0) + nl + (0 if fused else 1),
            "merge_prepare": 3 if n_frames > 1 else 2, "merge_accumulate": 2}


def merge_static(burst: torch.Tensor, motion: torch.Tensor, params: MergeParams | None = None, scale=(1, 1),
                 ref: int = 0, white_level: int = 4095, stream=None) -> torch.Tensor:
    """`merge` through hmfsr_merge_static: the library's fixed in-module scratch instead
    of a workspace (for callers that cannot allocate; small bursts only, and calls that
    overlap on the GPU race)."""
    L = _lib.load()
    params = params or MergeParams()
    d = _merge_inputs(burst, motion, params, ref, white_level)
    n, h, w = burst.shape
    ho, wo = out_size(h, w, scale)
    rgb = torch.empty((3, ho, wo), dtype=torch.float32, device=burst.device)
    pc = params.c()
    _lib.check(L.hmfsr_merge_static(_ptr(burst), ctypes.byref(d), _ptr(motion), ctypes.byref(pc), scale[0], scale[1],
                                    _ptr(rgb), None, _stream(burst.device, stream)), "hmfsr_merge_static")
    return rgb


PARAM_NAMES = ("k_detail", "k_denoise", "d_th", "d_tr", "k_stretch", "k_shrink", "s2", "t")


def merge_backward(burst: torch.Tensor, motion: torch.Tensor, params: MergeParams, rgb: torch.Tensor,
                   den: torch.Tensor, grad_rgb: torch.Tensor, scale=(1, 1), ref: int = 0, white_level: int = 4095,
                   stream=None, workspace: torch.Tensor | None = None, prepared: bool = False):
    """Adjoint of `merge` (hmfsr_merge_backward): (dL/dparams float32 [8] in PARAM_NAMES
    order, dL/dmotion float32 [n, TY, TX, 2]) for grad_rgb = dL/drgb, given the forward's
    rgb and den (merge(..., with_den=True)).  With `prepared`, `workspace` is the one the
    forward `merge` used with these arguments (hmfsr_merge_backward_prepared: its planes
    are reused, not recomputed)."""
    if prepared and workspace is None:
        raise ValueError("prepared=True needs the forward's workspace")
    L = _lib.load()
    d = _merge_inputs(burst, motion, params, ref, white_level, rgb, den, grad_rgb)
    n, h, w = burst.shape
    ty, tx = n_tiles(h, w, params.tile)
    ho, wo = out_size(h, w, scale)
    for t, what in ((rgb, "rgb"), (den, "den"), (grad_rgb, "grad_rgb")):
        if tuple(t.shape) != (3, ho, wo):
            raise ValueError(f"{what} must be [3,{ho},{wo}]")
    for t, what in ((rgb, "rgb"), (den, "den")):
        if t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError(f"{what} must be contiguous float32 (the forward's output)")
    gp = torch.empty(8, dtype=torch.float32, device=burst.device)
    gm = torch.empty((n, ty, tx, 2), dtype=torch.float32, device=burst.device)
    grad_rgb = grad_rgb.contiguous().float()
    nbytes = L.hmfsr_workspace_size(_lib.OP_MERGE_BACKWARD, ctypes.byref(d), params.tile, scale[0], scale[1])
    ws = _own_workspace(workspace, nbytes, burst.device) if workspace is not None else \
        _workspace(burst.device, nbytes, stream)
    pc = params.c()
    fn = L.hmfsr_merge_backward_prepared if prepared else L.hmfsr_merge_backward
    _lib.check(fn(_ptr(burst), ctypes.byref(d), _ptr(motion), ctypes.byref(pc), scale[0], scale[1], _ptr(rgb),
                  _ptr(den), _ptr(grad_rgb), _ptr(gp), _ptr(gm), _ptr(ws), ws.numel(), _stream(burst.device, stream)),
               "hmfsr_merge_backward")
    return gp, gm


class MergeFn(torch.autograd.Function):
    """rgb = merge(burst, motion, params) as a differentiable function of the eight tuning
    parameters (a float tensor in PARAM_NAMES order) and of the motion field; gradients
    come from the hand-written adjoint (hmfsr_merge_backward).  `values`, when given, are
    theta's values already on the host (the launch takes the parameters by value), which
    spares a device-to-host read per call."""

    @staticmethod
    def forward(ctx, theta, motion, burst, base: MergeParams, scale=(1, 1), ref: int = 0, values=None):
        vals = [float(x) for x in (values if values is not None else theta.detach().cpu().tolist())]
        p = MergeParams(**{**base.__dict__, **dict(zip(PARAM_NAMES, vals))})
        motion_c = motion.detach().contiguous()
        # the forward's planes stay in a workspace of the adjoint's size, which the
        # backward reuses instead of preparing them again
        ws = backward_workspace(tuple(burst.shape), p.tile, scale, burst.device)
        rgb, den = merge(burst, motion_c, p, scale, ref, with_den=True, workspace=ws)
        ctx.save_for_backward(motion_c, rgb, den)
        ctx.burst, ctx.p, ctx.scale, ctx.ref, ctx.ws = burst, p, scale, ref, ws
        ctx.theta_device = theta.device
        return rgb

    @staticmethod
    def backward(ctx, grad_rgb):
        motion_c, rgb, den = ctx.saved_tensors
        gp, gm = merge_backward(ctx.burst, motion_c, ctx.p, rgb, den, grad_rgb, ctx.scale, ctx.ref, workspace=ctx.ws,
                                prepared=True)
        ctx.ws = None
        return gp.to(ctx.theta_device), gm, None, None, None, None, None


class BatchPlan:
    """A ragged batch of bursts aligned and merged by one persistent, graph-captured
    launch (hmfsr_batch_*).  `shapes`: list of (n_frames, height, width); `params`,
    `scales`, `refs`: per burst (or one value for all)."""

    def __init__(self, shapes, params=None, scales=(1, 1), refs=0, align_params: AlignParams | None = None,
                 white_level: int = 4095):
        L = _lib.load()
        nb = len(shapes)
        params = params if isinstance(params, (list, tuple)) else [params or MergeParams()] * nb
        scales = scales if (isinstance(scales, (list, tuple)) and isinstance(scales[0], (list, tuple))) else [scales] * nb
        refs = refs if isinstance(refs, (list, tuple)) else [refs] * nb
        ap = align_params or AlignParams()
        self.shapes, self.scales = [tuple(s) for s in shapes], [tuple(s) for s in scales]
        self._descs = (_lib.BurstDesc * nb)(*[_lib.BurstDesc(n, h, w, w, r, 0, white_level, 0)
                                             for (n, h, w), r in zip(shapes, refs)])
        self._mp = (_lib.MergeParamsC * nb)(*[p.c() for p in params])
        self._ap = (_lib.AlignParamsC * nb)(*[ap.c() for _ in range(nb)])
        self._num = (ctypes.c_int * nb)(*[s[0] for s in scales])
        self._den = (ctypes.c_int * nb)(*[s[1] for s in scales])
        h = ctypes.c_void_p()
        _lib.check(L.hmfsr_batch_plan_create(self._descs, nb, self._mp, self._ap, self._num, self._den,
                                             ctypes.byref(h)), "hmfsr_batch_plan_create")
        self._h = h
        self._L = L
        self.n = nb
        self.ws_bytes = int(L.hmfsr_batch_workspace_size(h))
        self.ws = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._L.hmfsr_batch_free(h)
            self._h = None

    def outputs(self, device):
        return [torch.empty((3,) + out_size(h, w, sc), dtype=torch.float32, device=device)
                for (n, h, w), sc in zip(self.shapes, self.scales)]

    def _arrays(self, bursts, rgbs, motions):
        VP = ctypes.c_void_p * self.n
        b = VP(*[t.data_ptr() for t in bursts])
        r = VP(*[t.data_ptr() for t in rgbs])
        m = VP(*[t.data_ptr() for t in motions]) if motions is not None else None
        return b, m, r

    def _workspace(self, device):
        if self.ws is None or self.ws.device != device:
            buf = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=device)
            off = (-buf.data_ptr()) % 256
            self._ws_buf, self.ws = buf, buf[off:off + self.ws_bytes]
        return self.ws

    def run(self, bursts, rgbs, motions=None, stream=None, wait: bool = False):
        """Enqueue the whole batch; with `wait`, synchronise and raise on a device error."""
        dev = bursts[0].device
        ws = self._workspace(dev)
        b, m, r = self._arrays(bursts, rgbs, motions)
        st = _stream(dev, stream)
        _lib.check(self._L.hmfsr_batch_run(self._h, b, m, r, _ptr(ws), ws.numel(), st), "hmfsr_batch_run")
        if wait:
            self.wait(stream)
        return rgbs

    STAGES = ("luminance", "preparation", "pyramid 1", "pyramid 2", "pyramid 3", "matching 3", "matching 2",
              "matching 1", "matching 0", "lucas-kanade", "motion prior", "robustness", "accumulation")

    def set_profile(self, enable: bool = True):
        """Per-stage cycle counters in the persistent kernel (hmfsr_batch_set_profile)."""
        _lib.check(self._L.hmfsr_batch_set_profile(self._h, int(enable)), "hmfsr_batch_set_profile")

    def stage_profile(self, stream=None) -> dict:
        """{stage: (wait cycles, run cycles, items)} of the last profiled persistent run."""
        if self.ws is None:
            raise RuntimeError("run the plan first")
        n = 3 * 14
        out = (ctypes.c_ulonglong * n)()
        _lib.check(self._L.hmfsr_batch_stage_profile(self._h, _ptr(self.ws), out, n, _stream(self.ws.device, stream)),
                   "hmfsr_batch_stage_profile")
        return {name: (int(out[3 * s]), int(out[3 * s + 1]), int(out[3 * s + 2])) for s, name in enumerate(self.STAGES)}

    def vectors(self, k: int, stream=None) -> torch.Tensor:
        """Integer block-matching vectors (level 0, half-res px) of burst k from the last
        run: int32 [n, TY, TX, 2] (hmfsr_batch_vectors)."""
        if self.ws is None:
            raise RuntimeError("run the plan first")
        n, h, w = self.shapes[k]
        out = torch.empty((n,) + n_tiles(h, w, 16) + (2,), dtype=torch.int32, device=self.ws.device)
        _lib.check(self._L.hmfsr_batch_vectors(self._h, _ptr(self.ws), k, _ptr(out), _stream(self.ws.device, stream)),
                   "hmfsr_batch_vectors")
        return out

    def wait(self, stream=None) -> int:
        st = self._L.hmfsr_batch_wait(self._h, _ptr(self.ws), _stream(self.ws.device, stream))
        _lib.check(st, "batch")
        return st

    def configure(self, merge_tile_w: int = 32, ctas_per_sm: int = 0, regs_variant: int = 1, queue_order: int = 0,
                  spin_limit: int = 1 << 22, inject_stall: bool = False):
        _lib.check(self._L.hmfsr_batch_configure(self._h, merge_tile_w, ctas_per_sm, regs_variant, queue_order,
                                                 spin_limit, int(inject_stall)), "hmfsr_batch_configure")

    TUNE_CANDIDATES = ("persistent 32x4 128reg", "persistent 16x8 128reg", "persistent 32x4 80reg",
                       "persistent 32x4 64reg", "persistent 32x4 128reg wavefront", "graph 2 branches",
                       "graph 4 branches", "graph 8 branches")

    def set_mode(self, streams: int):
        """0: the one persistent kernel; k > 0: graph of per-burst kernels on k branches."""
        _lib.check(self._L.hmfsr_batch_set_mode(self._h, streams), "hmfsr_batch_set_mode")

    def tune(self, bursts, rgbs, motions=None, stream=None):
        """Autotune on these buffers; returns (best ms, {candidate: ms})."""
        dev = bursts[0].device
        ws = self._workspace(dev)
        b, m, r = self._arrays(bursts, rgbs, motions)
        best = ctypes.c_float()
        log = (ctypes.c_float * 8)()
        _lib.check(self._L.hmfsr_batch_tune(self._h, b, m, r, _ptr(ws), ws.numel(), _stream(dev, stream),
                                            ctypes.byref(best), log), "hmfsr_batch_tune")
        return float(best.value), dict(zip(self.TUNE_CANDIDATES, [float(x) for x in log]))
