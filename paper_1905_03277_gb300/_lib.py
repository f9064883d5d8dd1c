"""Build and load libhmfsr.so (the C-ABI library of hand-written sm_103a kernels)."""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB_PATH = os.path.join(PKG, "libhmfsr.so")
SOURCES = ("api.cu", "align.cu", "align_t4.cu", "align_t8.cu", "align_t16.cu", "align_t32.cu", "merge.cu",
           "merge_bwd.cu", "batch.cu", "merge_static.cu", "tuning.cu", "probe.cu")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fmad=false: no automatic FMA contraction, so a device function gives the same bits in
# every kernel it is inlined into (fused multiply-adds are written out with fmaf)
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC", "-I" + INCLUDE]


def _nvcc() -> str:
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(home, "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _inputs():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return files


CHECKED_LIB_PATH = os.path.join(PKG, "libhmfsr_checked.so")
# the units whose kernels the checked build checks (alignment and merge entry points);
# the others link unchanged from the default build
CHECKED_SOURCES = ("api.cu", "align.cu", "align_t4.cu", "align_t8.cu", "align_t16.cu", "align_t32.cu", "merge.cu")


def _compile(nvcc, src, obj, extra, verbose):
    cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose:
        print(r.stdout, r.stderr)
    return obj


def _link(nvcc, objs, lib_path):
    tmp = lib_path + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile every translation unit for sm_103a (in parallel) and link libhmfsr.so.
    With `checked`, also the checked test build (the alignment and merge units compiled
    with -DHMFSR_CHECKED, the rest shared) into libhmfsr_checked.so, in the same pass.
    Returns the default library's path."""
    newest = max(os.path.getmtime(f) for f in _inputs())
    need_default = force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < newest
    need_checked = checked and (force or not os.path.exists(CHECKED_LIB_PATH) or
                                os.path.getmtime(CHECKED_LIB_PATH) < newest)
    if not need_default and not need_checked:
        return LIB_PATH
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(BUILD + "_checked", exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    default_objs = {src: os.path.join(BUILD, os.path.splitext(src)[0] + ".o") for src in SOURCES}
    checked_objs = {src: os.path.join(BUILD + "_checked", os.path.splitext(src)[0] + ".o") for src in CHECKED_SOURCES}
    if need_default or not all(os.path.exists(o) for o in default_objs.values()):
        jobs += [(src, default_objs[src], []) for src in SOURCES]
    if need_checked:
        jobs += [(src, checked_objs[src], ["-DHMFSR_CHECKED"]) for src in CHECKED_SOURCES]
    with ThreadPoolExecutor(max(1, len(jobs))) as ex:
        list(ex.map(lambda j: _compile(nvcc, j[0], j[1], j[2], verbose), jobs))
    if need_default:
        _link(nvcc, [default_objs[s] for s in SOURCES], LIB_PATH)
    if need_checked:
        _link(nvcc, [checked_objs[s] if s in checked_objs else default_objs[s] for s in SOURCES], CHECKED_LIB_PATH)
    return LIB_PATH


# ---------------------------------------------------------------------------------------
# ctypes mirror of include/hmfsr.h
# ---------------------------------------------------------------------------------------
class BurstDesc(ctypes.Structure):
    _fields_ = [("n_frames", ctypes.c_int), ("height", ctypes.c_int), ("width", ctypes.c_int),
                ("pitch_elems", ctypes.c_int), ("ref", ctypes.c_int), ("cfa", ctypes.c_int),
                ("white_level", ctypes.c_int), ("black_level", ctypes.c_int)]


class AlignParamsC(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int), ("n_levels", ctypes.c_int), ("radius", ctypes.c_int * 4),
                ("lk_iters", ctypes.c_int)]


class MergeOptionsC(ctypes.Structure):
    _fields_ = [("noise_table", ctypes.c_void_p), ("hf_loss", ctypes.c_float)]


class MergeParamsC(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in ("k_detail", "k_denoise", "d_th", "d_tr", "k_stretch", "k_shrink",
                                              "t", "s1", "s2", "m_th", "noise_a", "noise_b")] + [
        ("tile", ctypes.c_int)]


OP_ALIGN, OP_MERGE, OP_MERGE_STAGES, OP_MERGE_BACKWARD, OP_ALIGN_MERGE = 0, 1, 2, 3, 4
PIPE_FP32_FMA, PIPE_MUFU_EX2 = 0, 1
NOISE_LEVELS = 129
EXPORTS = ("hmfsr_workspace_size", "hmfsr_align", "hmfsr_merge", "hmfsr_align_merge", "hmfsr_merge_chunked", "hmfsr_merge_chunked_workspace_size", "hmfsr_merge_prepare", "hmfsr_merge_accumulate",
           "hmfsr_merge_stages", "hmfsr_merge_backward", "hmfsr_merge_backward_prepared", "hmfsr_merge_static",
           "hmfsr_batch_plan_create",
           "hmfsr_batch_workspace_size", "hmfsr_batch_run", "hmfsr_batch_wait", "hmfsr_batch_vectors",
           "hmfsr_batch_set_profile", "hmfsr_batch_stage_profile", "hmfsr_batch_configure",
           "hmfsr_batch_tune", "hmfsr_batch_set_mode", "hmfsr_batch_free", "hmfsr_frame_sum", "hmfsr_snr_tuning",
           "hmfsr_noise_table", "hmfsr_merge_noise", "hmfsr_align_quadfit", "hmfsr_merge_ex",
           "hmfsr_pipe_probe", "hmfsr_check_status", "hmfsr_check_shrink", "hmfsr_status_string", "hmfsr_version")

_lib = None


def load(path: str | None = None):
    """Load libhmfsr.so (or `path`, or the file HMFSR_LIB names) once; raises if it is
    missing (there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    _lib = open_library(path or os.environ.get("HMFSR_LIB") or LIB_PATH)
    return _lib


def open_library(path: str):
    """A library file opened with every entry point's signature set (not cached)."""
    if not os.path.exists(path):
        raise RuntimeError(f"libhmfsr.so not found at {path}: run paper_1905_03277_gb300.build() first")
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, sz, ci = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
    L.hmfsr_workspace_size.argtypes = [ci, P(BurstDesc), ci, ci, ci]
    L.hmfsr_workspace_size.restype = sz
    L.hmfsr_align.argtypes = [vp, P(BurstDesc), P(AlignParamsC), vp, vp, vp, sz, vp]
    L.hmfsr_align.restype = ci
    L.hmfsr_merge.argtypes = [vp, P(BurstDesc), vp, P(MergeParamsC), ci, ci, vp, vp, vp, sz, vp]
    L.hmfsr_merge.restype = ci
    L.hmfsr_align_merge.argtypes = [vp, P(BurstDesc), P(AlignParamsC), P(MergeParamsC), ci, ci, vp, vp, vp, vp, vp, sz,
                                    vp]
    L.hmfsr_align_merge.restype = ci
    L.hmfsr_merge_chunked_workspace_size.argtypes = [P(BurstDesc), ci, ci, ci, ci]
    L.hmfsr_merge_chunked_workspace_size.restype = sz
    L.hmfsr_merge_chunked.argtypes = [vp, P(BurstDesc), vp, P(MergeParamsC), ci, ci, ci, vp, vp, vp, sz, vp]
    L.hmfsr_merge_chunked.restype = ci
    L.hmfsr_merge_prepare.argtypes = [vp, P(BurstDesc), vp, P(MergeParamsC), vp, sz, vp]
    L.hmfsr_merge_prepare.restype = ci
    L.hmfsr_merge_accumulate.argtypes = [vp, P(BurstDesc), vp, P(MergeParamsC), ci, ci, vp, vp, vp, sz, vp]
    L.hmfsr_merge_accumulate.restype = ci
    L.hmfsr_merge_stages.argtypes = [vp, P(BurstDesc), vp, P(MergeParamsC), vp, vp, vp, sz, vp]
    L.hmfsr_merge_stages.restype = ci
    L.hmfsr_merge_backward.argtypes = [vp, P(BurstDesc), vp, P(MergeParamsC), ci, ci, vp, vp, vp, vp, vp, vp, sz, vp]
    L.hmfsr_merge_backward.restype = ci
    L.hmfsr_merge_backward_prepared.argtypes = L.hmfsr_merge_backward.argtypes
    L.hmfsr_merge_backward_prepared.restype = ci
    L.hmfsr_merge_static.argtypes = [vp, P(BurstDesc), vp, P(MergeParamsC), ci, ci, vp, vp, vp]
    L.hmfsr_merge_static.restype = ci
    pp = P(vp)
    L.hmfsr_batch_plan_create.argtypes = [P(BurstDesc), ci, P(MergeParamsC), P(AlignParamsC), P(ci), P(ci), pp]
    L.hmfsr_batch_plan_create.restype = ci
    L.hmfsr_batch_workspace_size.argtypes = [vp]
    L.hmfsr_batch_workspace_size.restype = sz
    L.hmfsr_batch_run.argtypes = [vp, pp, pp, pp, vp, sz, vp]
    L.hmfsr_batch_run.restype = ci
    L.hmfsr_batch_wait.argtypes = [vp, vp, vp]
    L.hmfsr_batch_wait.restype = ci
    L.hmfsr_batch_set_profile.argtypes = [vp, ci]
    L.hmfsr_batch_set_profile.restype = ci
    L.hmfsr_batch_stage_profile.argtypes = [vp, vp, P(ctypes.c_ulonglong), ci, vp]
    L.hmfsr_batch_stage_profile.restype = ci
    L.hmfsr_batch_vectors.argtypes = [vp, vp, ci, vp, vp]
    L.hmfsr_batch_vectors.restype = ci
    L.hmfsr_batch_configure.argtypes = [vp, ci, ci, ci, ci, ci, ci]
    L.hmfsr_batch_configure.restype = ci
    L.hmfsr_batch_tune.argtypes = [vp, pp, pp, pp, vp, sz, vp, P(ctypes.c_float), P(ctypes.c_float)]
    L.hmfsr_batch_set_mode.argtypes = [vp, ci]
    L.hmfsr_batch_set_mode.restype = ci
    L.hmfsr_batch_tune.restype = ci
    L.hmfsr_batch_free.argtypes = [vp]
    L.hmfsr_batch_free.restype = None
    L.hmfsr_frame_sum.argtypes = [vp, P(BurstDesc), ci, vp, vp]
    L.hmfsr_frame_sum.restype = ci
    L.hmfsr_snr_tuning.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_float, ctypes.c_float, P(MergeParamsC),
                                   P(AlignParamsC),
                                   P(ctypes.c_double)]
    L.hmfsr_snr_tuning.restype = ci
    L.hmfsr_align_quadfit.argtypes = [vp, P(BurstDesc), P(AlignParamsC), vp, vp, vp, sz, vp]
    L.hmfsr_align_quadfit.restype = ci
    L.hmfsr_merge_ex.argtypes = [vp, P(BurstDesc), vp, P(MergeParamsC), P(MergeOptionsC), ci, ci, vp, vp, vp, sz, vp]
    L.hmfsr_merge_ex.restype = ci
    L.hmfsr_noise_table.argtypes = [ctypes.c_float, ctypes.c_float, ci, vp, vp]
    L.hmfsr_noise_table.restype = ci
    L.hmfsr_merge_noise.argtypes = [vp, P(BurstDesc), vp, P(MergeParamsC), vp, ci, ci, vp, vp, vp, sz, vp]
    L.hmfsr_merge_noise.restype = ci
    L.hmfsr_pipe_probe.argtypes = [ci, ci, ci, vp, P(ctypes.c_double), vp]
    L.hmfsr_pipe_probe.restype = ci
    L.hmfsr_status_string.argtypes = [ci]
    L.hmfsr_status_string.restype = ctypes.c_char_p
    L.hmfsr_version.argtypes = []
    L.hmfsr_version.restype = ctypes.c_char_p
    L.hmfsr_check_status.argtypes = [ci, P(ci)]
    L.hmfsr_check_status.restype = ci
    L.hmfsr_check_shrink.argtypes = [sz]
    L.hmfsr_check_shrink.restype = ci
    return L


def check(status: int, what: str):
    if status != 0:
        msg = load().hmfsr_status_string(status).decode()
        raise RuntimeError(f"{what} failed: {msg} ({status})")
