"""Build and ctypes binding of libnexel.so (the C ABI in include/nexel.h).

Argument marshalling only: every function here forwards plain pointers and
sizes to the library, which does all the work in its CUDA kernels.  There
is no fallback: if the library is missing or fails to load, calls raise.
"""
from __future__ import annotations

import concurrent.futures as cf
import ctypes as C
import glob
import os
import subprocess

_PKG = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_PKG)
_CSRC = os.path.join(_PKG, "csrc")
_INC = os.path.join(_ROOT, "include")
_BUILD = os.path.join(_PKG, "_build")
LIB_PATH = os.path.join(_PKG, "libnexel.so")

ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", _INC]

NEXEL_OK = 0
STATUS = {0: "ok", -1: "invalid argument", -2: "CUDA error", -3: "instance capacity exceeded",
          -4: "unsupported configuration", -5: "device wait timed out", -6: "numeric check failed"}
F32, F16, BF16 = 0, 1, 2
MAX_LEVELS, MAX_LAYERS = 32, 4

EXPORTS = ["nexel_workspace_size", "nexel_bwd_workspace_size", "nexel_preprocess",
           "nexel_render_fwd", "nexel_render_bwd", "nexel_instance_list", "nexel_status_string",
           "nexel_version", "nexel_launch_count", "nexel_profile_enable", "nexel_profile_read",
           "nexel_render_fwd_static", "nexel_preprocess_async", "nexel_render_batch_fwd",
           "nexel_render_batch_bwd", "nexel_read_status", "nexel_loss_workspace_size",
           "nexel_loss_image", "nexel_loss_params", "nexel_adam_step", "nexel_fps",
           "nexel_blend_error", "nexel_density_workspace_size", "nexel_densify_count",
           "nexel_densify_select",
           "nexel_densify_split", "nexel_prune", "nexel_get_tuning", "nexel_set_tuning",
           "nexel_autotune", "nexel_render_stats", "nexel_peak_l2_reductions",
           "nexel_test_tc_wait_timeout"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _sources():
    return sorted(glob.glob(os.path.join(_CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(_CSRC, "*.cuh")) + glob.glob(os.path.join(_INC, "*.h")))


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit (in parallel) and link libnexel.so."""
    os.makedirs(_BUILD, exist_ok=True)
    hdr_t = max((os.path.getmtime(h) for h in _headers()), default=0.0)
    nvcc = _nvcc()
    jobs = []
    for src in _sources():
        obj = os.path.join(_BUILD, os.path.basename(src)[:-3] + ".o")
        if force or not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(src), hdr_t):
            jobs.append((src, obj))

    def compile_one(job):
        src, obj = job
        tmp = obj + f".{os.getpid()}.tmp.o"
        cmd = [nvcc, *ARCH_FLAGS, *NVCC_FLAGS, "-c", src, "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr[-4000:]}")
        os.replace(tmp, obj)
        if verbose:
            print("compiled", os.path.basename(src))

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
            list(ex.map(compile_one, jobs))
    objs = [os.path.join(_BUILD, os.path.basename(s)[:-3] + ".o") for s in _sources()]
    if force or jobs or not os.path.exists(LIB_PATH) or \
            os.path.getmtime(LIB_PATH) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB_PATH + f".{os.getpid()}.tmp"
        cmd = [nvcc, *ARCH_FLAGS, "-shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


# ------------------------------------------------------------- C structs
class Tuning(C.Structure):
    _fields_ = [("tex_fwd_ctas_per_sm", C.c_int), ("tex_bwd_ctas_per_sm", C.c_int),
                ("f32_ctas_per_sm", C.c_int), ("hash_block", C.c_int),
                ("collect_batch", C.c_int), ("tex_fwd_stages", C.c_int)]


class LossWeights(C.Structure):
    _fields_ = [("dssim", C.c_float), ("alpha", C.c_float), ("texture", C.c_float),
                ("opacity", C.c_float), ("grid", C.c_float)]


class Camera(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("world_to_cam", C.c_float * 12),
                ("near_plane", C.c_float)]


class Settings(C.Structure):
    _fields_ = [("K", C.c_int), ("alpha_min", C.c_float), ("alpha_max", C.c_float),
                ("T_min", C.c_float), ("bg", C.c_float * 3), ("grid_dtype", C.c_int),
                ("mlp_dtype", C.c_int), ("recompute_buffers", C.c_int),
                ("cache_features", C.c_int), ("sh_degree", C.c_int)]


class Field(C.Structure):
    _fields_ = [("L", C.c_int), ("T", C.c_int), ("F", C.c_int),
                ("level_scale", C.c_float * MAX_LEVELS), ("table", C.c_void_p),
                ("n_layers", C.c_int), ("widths", C.c_int * (MAX_LAYERS + 1)),
                ("weights", C.c_void_p)]


_lib = None


def lib(auto_build: bool = False):
    """The loaded library.  Raises if it is missing (no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        if not auto_build:
            raise RuntimeError(f"libnexel.so is not built ({LIB_PATH}); run build() first")
        build()
    L = C.CDLL(LIB_PATH)
    vp, i, sz, ll = C.c_void_p, C.c_int, C.c_size_t, C.c_longlong
    L.nexel_workspace_size.argtypes = [vp, i, ll, C.POINTER(sz)]
    L.nexel_bwd_workspace_size.argtypes = [vp, vp, vp, C.POINTER(sz)]
    L.nexel_preprocess.argtypes = [vp, vp, i] + [vp] * 7 + [sz, C.POINTER(ll), vp]
    L.nexel_render_fwd.argtypes = [vp, vp, vp, i, vp, sz, vp, sz] + [vp] * 7 + [vp]
    L.nexel_render_bwd.argtypes = ([vp, vp, vp, i] + [vp] * 5 + [vp, sz, vp, sz] + [vp] * 4 +
                                   [vp] * 3 + [i] + [vp] * 8 + [vp])
    L.nexel_instance_list.argtypes = [vp, i, vp, sz, ll, vp, vp, vp, vp]
    L.nexel_render_stats.argtypes = [vp, vp, i, vp, sz, C.POINTER(ll), vp]
    L.nexel_peak_l2_reductions.argtypes = [vp, sz, ll, i, C.POINTER(C.c_float), vp]
    L.nexel_render_fwd_static.argtypes = [vp, vp, vp, i] + [vp] * 6 + [vp] * 7 + [
        C.POINTER(ll), vp]
    L.nexel_preprocess_async.argtypes = [vp, vp, i] + [vp] * 7 + [sz, vp]
    L.nexel_render_batch_fwd.argtypes = [i, vp, vp, vp, i] + [vp] * 6 + [vp] * 4 + [vp] * 7 + [vp]
    L.nexel_render_batch_bwd.argtypes = ([i, vp, vp, vp, i] + [vp] * 5 + [vp] * 4 + [vp] * 4 +
                                         [vp] * 3 + [i] + [vp] * 8 + [vp])
    L.nexel_read_status.argtypes = [vp, vp, vp, i, vp, sz, vp, sz, vp]
    L.nexel_loss_workspace_size.argtypes = [i, i, C.POINTER(sz)]
    L.nexel_loss_image.argtypes = [i, i, i, vp] + [vp] * 4 + [vp, sz, vp] + [vp] * 3 + [vp]
    L.nexel_loss_params.argtypes = [i, vp, vp, vp, vp, vp, sz, i, i, vp, vp, vp, vp]
    L.nexel_adam_step.argtypes = [i, vp, vp, vp, vp, vp, vp, C.c_float, C.c_float, C.c_float,
                                  i, vp]
    L.nexel_fps.argtypes = [i, vp, i, vp, vp, vp, vp, vp]
    L.nexel_blend_error.argtypes = [vp, vp, i, vp, sz, vp, vp, vp, vp]
    L.nexel_density_workspace_size.argtypes = [i, C.POINTER(sz)]
    L.nexel_densify_count.argtypes = [i, ll, C.POINTER(i)]
    L.nexel_densify_select.argtypes = [i, vp, vp, ll, vp, sz, vp, C.POINTER(i), vp]
    L.nexel_densify_split.argtypes = [i, i, vp, i] + [vp] * 6 + [vp]
    L.nexel_prune.argtypes = [i, C.c_float, i] + [vp] * 6 + [vp, sz] + [vp] * 7 + [vp]
    L.nexel_test_tc_wait_timeout.argtypes = [i]
    L.nexel_get_tuning.argtypes = [vp]
    L.nexel_set_tuning.argtypes = [vp]
    L.nexel_autotune.argtypes = ([vp, vp, vp, i] + [vp] * 6 + [vp, sz, vp, sz] + [vp] * 7 + [vp] +
                                 [vp] * 8 + [i, vp, sz, vp, vp, vp])
    L.nexel_launch_count.restype = C.c_longlong
    L.nexel_launch_count.argtypes = []
    L.nexel_profile_enable.argtypes = [i]
    L.nexel_profile_read.argtypes = [i, vp, vp, vp, C.POINTER(i)]
    L.nexel_status_string.restype = C.c_char_p
    L.nexel_status_string.argtypes = [i]
    L.nexel_version.restype = i
    for name in EXPORTS:
        getattr(L, name).restype = getattr(L, name).restype or i
    _lib = L
    return L


class NexelError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn} failed: {STATUS.get(code, code)} ({code})")
        self.code = code


def check(fn: str, code: int) -> int:
    if code != NEXEL_OK:
        raise NexelError(fn, code)
    return code


# Thin wrappers with the ABI's names: pointers are ints (tensor.data_ptr()),
# structs are the ctypes classes above.
def nexel_workspace_size(cam: Camera, N: int, max_instances: int) -> int:
    out = C.c_size_t(0)
    check("nexel_workspace_size", lib().nexel_workspace_size(C.byref(cam), N, max_instances,
                                                            C.byref(out)))
    return out.value


def nexel_bwd_workspace_size(cam: Camera, st: Settings, field: Field | None) -> int:
    out = C.c_size_t(0)
    check("nexel_bwd_workspace_size",
          lib().nexel_bwd_workspace_size(C.byref(cam), C.byref(st),
                                         C.byref(field) if field is not None else None,
                                         C.byref(out)))
    return out.value


def nexel_preprocess(cam, st, N, mu, quat, scale, opacity, gamma, color, ws, ws_bytes,
                     stream) -> tuple[int, int]:
    """Returns (status, n_instances); status NEXEL_ERR_CAPACITY is returned,
    not raised, so the caller can grow the workspace."""
    n = C.c_longlong(0)
    rc = lib().nexel_preprocess(C.byref(cam), C.byref(st), N, mu, quat, scale, opacity, gamma,
                                color, ws, ws_bytes, C.byref(n), stream)
    return rc, n.value


def nexel_render_fwd(cam, st, field, N, ws, ws_bytes, bws, bws_bytes, image, notex, weights,
                     ids, depths, textures, T_final, stream) -> int:
    return check("nexel_render_fwd", lib().nexel_render_fwd(
        C.byref(cam), C.byref(st), C.byref(field) if field is not None else None, N, ws, ws_bytes,
        bws, bws_bytes, image, notex, weights, ids, depths, textures, T_final, stream))


def nexel_render_bwd(cam, st, field, N, mu, quat, scale, opacity, gamma, ws, ws_bytes, bws,
                     bws_bytes, weights, ids, depths, T_final, d_image, d_weights, d_textures,
                     accumulate, d_mu, d_quat, d_scale, d_opacity, d_gamma, d_color, d_table,
                     d_mlp, stream) -> int:
    return check("nexel_render_bwd", lib().nexel_render_bwd(
        C.byref(cam), C.byref(st), C.byref(field) if field is not None else None, N, mu, quat,
        scale, opacity, gamma, ws, ws_bytes, bws, bws_bytes, weights, ids, depths, T_final,
        d_image, d_weights, d_textures, int(accumulate), d_mu, d_quat, d_scale, d_opacity,
        d_gamma, d_color, d_table, d_mlp, stream))


def nexel_instance_list(cam, N, ws, ws_bytes, n_instances, tile_out, id_out, depth_out,
                        stream) -> int:
    return check("nexel_instance_list", lib().nexel_instance_list(
        C.byref(cam), N, ws, ws_bytes, n_instances, tile_out, id_out, depth_out, stream))


RENDER_STATS = ("instances", "visible_surfels", "pairs_to_last", "pairs_full_lists",
                "longest_list", "tiles", "pairs_bwd_walk", "nonfinite_surfels")


def nexel_render_stats(cam, st, N, ws, ws_bytes, stream) -> dict:
    """Work statistics of the last forward on ws (synchronises the stream)."""
    out = (C.c_longlong * len(RENDER_STATS))()
    check("nexel_render_stats", lib().nexel_render_stats(C.byref(cam), C.byref(st), N, ws,
                                                         ws_bytes, out, stream))
    return dict(zip(RENDER_STATS, (int(v) for v in out)))


def nexel_peak_l2_reductions(buf, buf_bytes, n_ops, reps, stream) -> float:
    """Median rate of random float2 L2 reductions (1e9 per second)."""
    g = C.c_float(0.0)
    check("nexel_peak_l2_reductions", lib().nexel_peak_l2_reductions(buf, buf_bytes, n_ops, reps,
                                                                     C.byref(g), stream))
    return float(g.value)


def nexel_render_fwd_static(cam, st, field, N, mu, quat, scale, opacity, gamma, color, image,
                            notex, weights, ids, depths, textures, T_final, stream) -> tuple:
    """Allocation-free forward render; returns (status, n_instances)."""
    n = C.c_longlong(0)
    rc = lib().nexel_render_fwd_static(
        C.byref(cam), C.byref(st), C.byref(field) if field is not None else None, N, mu, quat,
        scale, opacity, gamma, color, image, notex, weights, ids, depths, textures, T_final,
        C.byref(n), stream)
    return rc, n.value


def nexel_preprocess_async(cam, st, N, mu, quat, scale, opacity, gamma, color, ws, ws_bytes,
                           stream) -> int:
    return check("nexel_preprocess_async", lib().nexel_preprocess_async(
        C.byref(cam), C.byref(st), N, mu, quat, scale, opacity, gamma, color, ws, ws_bytes,
        stream))


def _cams(cams):
    arr = (Camera * len(cams))()
    for k, c in enumerate(cams):
        arr[k] = c
    return arr


def _ptrs(xs):
    """Host array of device pointers (ints or None), or None for no array."""
    if xs is None:
        return None
    return (C.c_void_p * len(xs))(*[x if x else None for x in xs])


def _sizes(xs):
    return None if xs is None else (C.c_size_t * len(xs))(*xs)


def nexel_render_batch_fwd(cams, st, field, N, mu, quat, scale, opacity, gamma, color, ws,
                           ws_bytes, bws, bws_bytes, image, notex, weights, ids, depths,
                           textures, T_final, stream) -> int:
    """Per-view arguments are Python lists with one entry per camera."""
    n = len(cams)
    return check("nexel_render_batch_fwd", lib().nexel_render_batch_fwd(
        n, _cams(cams), C.byref(st), C.byref(field) if field is not None else None, N, mu, quat,
        scale, opacity, gamma, color, _ptrs(ws), _sizes(ws_bytes), _ptrs(bws), _sizes(bws_bytes),
        _ptrs(image), _ptrs(notex), _ptrs(weights), _ptrs(ids), _ptrs(depths), _ptrs(textures),
        _ptrs(T_final), stream))


def nexel_render_batch_bwd(cams, st, field, N, mu, quat, scale, opacity, gamma, ws, ws_bytes,
                           bws, bws_bytes, weights, ids, depths, T_final, d_image, d_weights,
                           d_textures, accumulate, d_mu, d_quat, d_scale, d_opacity, d_gamma,
                           d_color, d_table, d_mlp, stream) -> int:
    n = len(cams)
    return check("nexel_render_batch_bwd", lib().nexel_render_batch_bwd(
        n, _cams(cams), C.byref(st), C.byref(field) if field is not None else None, N, mu, quat,
        scale, opacity, gamma, _ptrs(ws), _sizes(ws_bytes), _ptrs(bws), _sizes(bws_bytes),
        _ptrs(weights), _ptrs(ids), _ptrs(depths), _ptrs(T_final), _ptrs(d_image),
        _ptrs(d_weights), _ptrs(d_textures), int(accumulate), d_mu, d_quat, d_scale, d_opacity,
        d_gamma, d_color, d_table, d_mlp, stream))


def nexel_read_status(cam, st, field, N, ws, ws_bytes, bws, bws_bytes, stream) -> int:
    """Returns the status (NEXEL_OK, NEXEL_ERR_CAPACITY, NEXEL_ERR_TIMEOUT or
    NEXEL_ERR_NUMERIC) without raising; argument errors raise."""
    rc = lib().nexel_read_status(C.byref(cam), C.byref(st),
                                 C.byref(field) if field is not None else None, N, ws, ws_bytes,
                                 bws, bws_bytes, stream)
    if rc not in (NEXEL_OK, -3, -5, -6):
        raise NexelError("nexel_read_status", rc)
    return rc


def nexel_loss_workspace_size(width: int, height: int) -> int:
    out = C.c_size_t(0)
    check("nexel_loss_workspace_size",
          lib().nexel_loss_workspace_size(width, height, C.byref(out)))
    return out.value


def nexel_loss_image(width, height, K, lw, image, target, weights, textures, ws, ws_bytes,
                     values, d_image, d_weights, d_textures, stream) -> int:
    return check("nexel_loss_image", lib().nexel_loss_image(
        width, height, K, C.byref(lw), image, target, weights, textures, ws, ws_bytes, values,
        d_image, d_weights, d_textures, stream))


def nexel_loss_params(N, opacity, field, table, lw, ws, ws_bytes, width, height, values,
                      d_opacity, d_table, stream) -> int:
    return check("nexel_loss_params", lib().nexel_loss_params(
        N, opacity, C.byref(field) if field is not None else None, table, C.byref(lw), ws,
        ws_bytes, width, height, values, d_opacity, d_table, stream))


def nexel_adam_step(params, grads, m, v, sizes, lrs, beta1, beta2, eps, step, stream) -> int:
    n = len(params)
    return check("nexel_adam_step", lib().nexel_adam_step(
        n, _ptrs(params), _ptrs(grads), _ptrs(m), _ptrs(v), (C.c_longlong * n)(*sizes),
        (C.c_float * n)(*lrs), beta1, beta2, eps, step, stream))


def nexel_fps(n, points, m, scratch, idx, d2sel, scale, stream) -> int:
    return check("nexel_fps", lib().nexel_fps(n, points, m, scratch, idx, d2sel, scale, stream))


def nexel_blend_error(cam, st, N, ws, ws_bytes, image, target, err, stream) -> int:
    return check("nexel_blend_error", lib().nexel_blend_error(
        C.byref(cam), C.byref(st), N, ws, ws_bytes, image, target, err, stream))


def nexel_density_workspace_size(N: int) -> int:
    out = C.c_size_t(0)
    check("nexel_density_workspace_size", lib().nexel_density_workspace_size(N, C.byref(out)))
    return out.value


def nexel_densify_count(N: int, budget: int) -> int:
    out = C.c_int(0)
    check("nexel_densify_count", lib().nexel_densify_count(N, budget, C.byref(out)))
    return out.value


def nexel_densify_select(N, err, expo, budget, ws, ws_bytes, sel, stream) -> int:
    """Returns the number of surfels drawn (nexel_densify_count)."""
    out = C.c_int(0)
    check("nexel_densify_select", lib().nexel_densify_select(
        N, err, expo, budget, ws, ws_bytes, sel, C.byref(out), stream))
    return out.value


def nexel_densify_split(N, n_select, sel, color_dim, mu, quat, scale, opacity, gamma, color,
                        stream) -> int:
    return check("nexel_densify_split", lib().nexel_densify_split(
        N, n_select, sel, color_dim, mu, quat, scale, opacity, gamma, color, stream))


def nexel_prune(N, threshold, color_dim, src, ws, ws_bytes, dst, n_out, stream) -> int:
    """src, dst: (mu, quat, scale, opacity, gamma, color) device pointers."""
    return check("nexel_prune", lib().nexel_prune(
        N, threshold, color_dim, *src, ws, ws_bytes, *dst, n_out, stream))


def nexel_test_tc_wait_timeout(polls: int) -> int:
    """Test hook: polls > 0 makes the tensor-core kernels issue no MMA and
    give up each completion wait after that many polls; 0 turns it off."""
    return check("nexel_test_tc_wait_timeout", lib().nexel_test_tc_wait_timeout(polls))


def nexel_get_tuning() -> Tuning:
    t = Tuning()
    check("nexel_get_tuning", lib().nexel_get_tuning(C.byref(t)))
    return t


def nexel_set_tuning(t: Tuning) -> int:
    return check("nexel_set_tuning", lib().nexel_set_tuning(C.byref(t)))


def nexel_autotune(cam, st, field, N, params, ws, ws_bytes, bws, bws_bytes, outs, d_image, grads,
                   reps, stream, flush=None, flush_bytes=0) -> tuple:
    """params: 6 device pointers (mu .. color); outs: 7 (image, notex,
    weights, ids, depths, textures, T_final); grads: 8 (d_mu .. d_mlp).
    Returns (Tuning, median ms)."""
    t = Tuning()
    ms = C.c_float(0.0)
    check("nexel_autotune", lib().nexel_autotune(
        C.byref(cam), C.byref(st), C.byref(field) if field is not None else None, N, *params, ws,
        ws_bytes, bws, bws_bytes, *outs, d_image, *grads, reps, flush, flush_bytes, C.byref(t),
        C.byref(ms), stream))
    return t, ms.value


def nexel_launch_count() -> int:
    return lib().nexel_launch_count()


def nexel_profile_enable(on: bool) -> int:
    return check("nexel_profile_enable", lib().nexel_profile_enable(1 if on else 0))


def nexel_profile_read(max_entries: int = 64) -> dict:
    """{kernel name: (total ms, launches)} of the events recorded so far."""
    names = C.create_string_buffer(32 * max_entries)
    ms = (C.c_float * max_entries)()
    cnt = (C.c_int * max_entries)()
    n = C.c_int(0)
    check("nexel_profile_read", lib().nexel_profile_read(max_entries, names, ms, cnt, C.byref(n)))
    out = {}
    for k in range(min(n.value, max_entries)):
        nm = names.raw[32 * k:32 * k + 32].split(b"\0")[0].decode()
        out[nm] = (float(ms[k]), int(cnt[k]))
    return out


def nexel_status_string(code: int) -> str:
    return lib().nexel_status_string(code).decode()


def nexel_version() -> int:
    return lib().nexel_version()
