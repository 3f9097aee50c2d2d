"""FP64 CPU oracle for the Nexels image formation.

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke``
and by the benchmark's CPU-baseline leg.  The product package never imports
it, and it imports nothing from the product package's compute path (inputs
come from the shared seeded generator, which holds no rendering arithmetic).

The compiled part (``nexel_oracle.cpp``) is the brute-force definition: every
pixel walks all surfels in centre-depth order.  This module only marshals
float64 arrays through ctypes.

Functions and the passages they follow:
  render / render_bwd   Sec. 3 (Eq. 1, centre-depth order), Sec. 4.1 (kernel,
                        Eqs. 3-4), Sec. 4.2 (collection pass, Eqs. 5-6)
  field_features        Sec. 3 (Instant-NGP hash grid), Eq. 3, supp. Sec. 7.1
  mlp, texture          Sec. 3 (G), Eq. 4, supp. Sec. 7.1 (no bias, G(0) = 0)
  map_positive, hash    supp. Sec. 7.1 (MapPositive) and the spatial hash
  depth_order           Sec. 3 (sorted by the depth of the centres)
  storage_bytes         supp. Sec. 7.1, last paragraph (2 B per Instant-NGP
                        parameter, 4 B otherwise)
  render_sh, render_bwd_sh, sh (module), 48-output MLPs (SH textures)
                        Sec. 3 (view-dependent radiance as channel-wise SH
                        coefficients) with Sec. 5's degree 3 (S = 16)
  blend_error, density (module)
                        supp. Sec. 7.2 (adaptive density control: farthest
                        point sampling initialisation, blended errors,
                        stochastic split, prune)
  objective (module)    Sec. 5, "Losses": L_1, D-SSIM, L_texture, L_alpha,
                        L_opacity, L_grid, the weighted total, and the Adam
                        step of the 3DGS scheme the paper follows (plain
                        numpy, FP64; see its header for the readings)
Parity unpinned: the shared conventions alpha_min / alpha_max / T_min, the
near plane and the level scales s_l are parameters, not facts of the paper.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nexel_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


class OCam(C.Structure):
    _fields_ = [("W", C.c_int), ("H", C.c_int), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("Rt", C.c_double * 12),
                ("near", C.c_double)]


class OSet(C.Structure):
    _fields_ = [("K", C.c_int), ("alpha_min", C.c_double), ("alpha_max", C.c_double),
                ("T_min", C.c_double), ("bg", C.c_double * 3), ("tie_tol", C.c_double),
                ("order_tol", C.c_double), ("cell_tol", C.c_double),
                ("relu_tol", C.c_double), ("edge_tol", C.c_double)]


class OField(C.Structure):
    _fields_ = [("L", C.c_int), ("T", C.c_int), ("F", C.c_int),
                ("scale", C.POINTER(C.c_double)), ("table", C.POINTER(C.c_double)),
                ("n_layers", C.c_int), ("widths", C.POINTER(C.c_int)),
                ("weights", C.POINTER(C.c_double))]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.oracle_map_positive.restype = C.c_uint64
        _lib.oracle_map_positive.argtypes = [C.c_int64]
        _lib.oracle_hash.restype = C.c_uint32
        _lib.oracle_hash.argtypes = [C.c_int64, C.c_int64, C.c_int64, C.c_uint32]
    return _lib


def _d(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _cam(cam) -> OCam:
    c = OCam()
    c.W, c.H = cam.width, cam.height
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    m = np.asarray(cam.world_to_cam, np.float64).ravel()
    for i in range(12):
        c.Rt[i] = float(m[i])
    c.near = float(cam.near)
    return c


def _set(st, tie_tol, order_tol=1e-6, cell_tol=0.0, relu_tol=0.0, edge_tol=0.0) -> OSet:
    s = OSet()
    s.K = int(st.K)
    s.alpha_min, s.alpha_max, s.T_min = float(st.alpha_min), float(st.alpha_max), float(st.T_min)
    for i in range(3):
        s.bg[i] = float(st.bg[i])
    s.tie_tol = float(tie_tol)
    s.order_tol = float(min(order_tol, tie_tol)) if tie_tol > 0 else 0.0
    s.cell_tol = float(cell_tol)
    s.relu_tol = float(relu_tol)
    s.edge_tol = float(edge_tol)
    return s


class _FieldRef:
    """Keeps the float64 copies alive while the C struct points at them."""

    def __init__(self, field, table=None, weights=None):
        self.scale = _d(field.level_scale)
        self.table = _d(field.table if table is None else table)
        self.widths = np.ascontiguousarray(np.asarray(field.widths, np.int32))
        wl = field.weights if weights is None else weights
        self.weights = _d(np.concatenate([np.asarray(w, np.float64).ravel() for w in wl]))
        self.n_mlp = self.weights.size
        self.s = OField()
        self.s.L, self.s.T, self.s.F = int(field.L), int(field.T), int(field.F)
        self.s.scale = self.scale.ctypes.data_as(C.POINTER(C.c_double))
        self.s.table = self.table.ctypes.data_as(C.POINTER(C.c_double))
        self.s.n_layers = len(field.weights)
        self.s.widths = self.widths.ctypes.data_as(C.POINTER(C.c_int))
        self.s.weights = self.weights.ctypes.data_as(C.POINTER(C.c_double))


def _surfels(scene):
    return [_d(scene.mu), _d(scene.quat), _d(scene.scale), _d(scene.opacity),
            _d(scene.gamma), _d(scene.color)]


def all_pixels(cam) -> np.ndarray:
    return np.arange(cam.width * cam.height, dtype=np.int32)


TIE_BITS = {1: "topk", 2: "alpha", 4: "T_min", 8: "near", 16: "order", 32: "cell", 64: "relu",
            128: "edge"}


def render(scene, cam, settings, field=None, pixels=None, tie_tol: float = 1e-6,
           table=None, order_tol: float = 1e-6, cell_tol: float = 0.0,
           relu_tol: float = 0.0, weights=None, edge_tol: float = 1e-6) -> dict:
    """Forward of the listed pixels.  ``table`` overrides field.table and
    ``weights`` field.weights (e.g. the FP16-rounded table and the
    BF16-rounded weights a reduced-precision path reads).  A pixel is
    flagged in ``tie`` when one of its discrete choices lies within tie_tol
    (relative) of flipping: top-K weight ties (bit 1), alpha at alpha_min or
    alpha_max (2), T(1 - alpha) at T_min (4), t* at the near plane (8), or,
    within order_tol, two consecutive composited surfels with equal centre
    depth (16); and, when cell_tol > 0, a textured intersection within
    cell_tol (world units) of a hash-cell face of some level (32), where the
    trilinear interpolation has a kink; and, when relu_tol > 0, a textured
    sample with a hidden MLP pre-activation within relu_tol (relative to the
    sum of the magnitudes of its terms) of zero (64), a ReLU kink; and a
    composited surfel whose edge-on measure |d_mu . n_c| lies within
    edge_tol of the edge-on threshold (128).  ``tie_slot`` [n, K] holds the
    kink bits (32, 64) of each slot's own sample."""
    L = lib()
    pix = all_pixels(cam) if pixels is None else np.ascontiguousarray(pixels, np.int32)
    n, K = pix.size, settings.K
    out = dict(image=np.zeros((n, 3)), notex=np.zeros((n, 3)), weights=np.zeros((n, K)),
               ids=np.zeros((n, K), np.int32), depths=np.zeros((n, K)),
               textures=np.zeros((n, K, 3)), T_final=np.zeros(n),
               n_contrib=np.zeros(n, np.int32), tie=np.zeros(n, np.int32),
               tie_slot=np.zeros((n, K), np.int32))
    fr = _FieldRef(field, table, weights) if field is not None else None
    sv = _surfels(scene)
    c, s = _cam(cam), _set(settings, tie_tol, order_tol, cell_tol, relu_tol, edge_tol)
    rc = L.oracle_render(C.byref(c), C.byref(s), C.byref(fr.s) if fr else None,
                         C.c_int(scene.n), *[_p(a) for a in sv], C.c_int(n), _p(pix),
                         *[_p(out[k]) for k in ("image", "notex", "weights", "ids", "depths",
                                                "textures", "T_final", "n_contrib", "tie",
                                                "tie_slot")])
    if rc != 0:
        raise ValueError(f"oracle_render failed ({rc})")
    out["pixels"] = pix
    return out


def render_bwd(scene, cam, settings, field, pixels, d_image, d_weights=None,
               d_textures=None, table=None, weights=None, absolute: bool = False) -> dict:
    """Analytic FP64 gradient of the listed pixels' outputs (discrete
    choices held fixed) for upstream d_image, d_weights, d_textures.  With
    ``absolute`` every entry instead holds the sum of the magnitudes of its
    contributions (per pixel and surfel, per sample and table corner, per
    sample and MLP weight)."""
    L = lib()
    pix = np.ascontiguousarray(pixels, np.int32)
    n, N = pix.size, scene.n
    fr = _FieldRef(field, table, weights) if field is not None else None
    sv = _surfels(scene)
    g = dict(mu=np.zeros((N, 3)), quat=np.zeros((N, 4)), scale=np.zeros((N, 2)),
             opacity=np.zeros(N), gamma=np.zeros((N, 2)), color=np.zeros((N, 3)))
    if fr:
        g["table"] = np.zeros((field.L, field.T, field.F))
        g["mlp"] = np.zeros(fr.n_mlp)
    dI = _d(d_image).reshape(n, 3)
    dW = None if d_weights is None else _d(d_weights).reshape(n, settings.K)
    dT = None if d_textures is None else _d(d_textures).reshape(n, settings.K, 3)
    c, s = _cam(cam), _set(settings, 0.0)
    rc = L.oracle_render_bwd(C.byref(c), C.byref(s), C.byref(fr.s) if fr else None,
                             C.c_int(N), *[_p(a) for a in sv], C.c_int(n), _p(pix),
                             _p(dI), _p(dW), _p(dT),
                             *[_p(g[k]) for k in ("mu", "quat", "scale", "opacity", "gamma",
                                                  "color")],
                             _p(g.get("table")), _p(g.get("mlp")), C.c_int(int(absolute)))
    if rc != 0:
        raise ValueError(f"oracle_render_bwd failed ({rc})")
    if fr:
        offs = np.cumsum([0] + [w.size for w in field.weights])
        g["mlp_layers"] = [g["mlp"][offs[i]:offs[i + 1]].reshape(field.weights[i].shape)
                           for i in range(len(field.weights))]
    return g


def _with_colors(scene, rgb):
    import types
    return types.SimpleNamespace(mu=scene.mu, quat=scene.quat, scale=scene.scale,
                                 opacity=scene.opacity, gamma=scene.gamma, color=rgb, n=scene.n)


def render_sh(scene, coeffs, cam, settings, field=None, pixels=None, **kw) -> dict:
    """render() with degree-3 SH per-primitive colours (coefficients
    [N, 16, 3]), evaluated per surfel as oracle/sh.py states."""
    from . import sh
    rgb = sh.primitive_colors(scene.mu, coeffs, sh.camera_center(cam))
    return render(_with_colors(scene, rgb), cam, settings, field, pixels, **kw)


def render_bwd_sh(scene, coeffs, cam, settings, field, pixels, d_image, d_weights=None,
                  d_textures=None, table=None, weights=None, absolute: bool = False) -> dict:
    """render_bwd() for SH per-primitive colours: the colour gradient is
    taken to the coefficients ([N, 16, 3]) and, through the direction, to mu.
    With ``absolute`` it returns render_bwd's magnitudes at the evaluated
    per-primitive colours (the table and MLP entries are the ones of use)."""
    from . import sh
    center = sh.camera_center(cam)
    rgb = sh.primitive_colors(scene.mu, coeffs, center)
    g = render_bwd(_with_colors(scene, rgb), cam, settings, field, pixels, d_image, d_weights,
                   d_textures, table, weights, absolute)
    if absolute:
        return g
    dc, dmu = sh.primitive_colors_bwd(scene.mu, coeffs, center, g["color"])
    g["color"] = dc
    g["mu"] = g["mu"] + dmu
    return g


def blend_error(scene, cam, settings, e_pix, pixels=None) -> np.ndarray:
    """Per-surfel blended error sum_p w_ip e_p over the listed pixels
    (supp. Sec. 7.2); e_pix [n_pix] the pixels' errors."""
    pix = all_pixels(cam) if pixels is None else np.ascontiguousarray(pixels, np.int32)
    e = _d(e_pix).reshape(pix.size)
    out = np.zeros(scene.n)
    sv = _surfels(scene)
    c, s = _cam(cam), _set(settings, 0.0)
    rc = lib().oracle_blend_error(C.byref(c), C.byref(s), C.c_int(scene.n), *[_p(a) for a in sv],
                                  C.c_int(pix.size), _p(pix), _p(e), _p(out))
    if rc != 0:
        raise ValueError(f"oracle_blend_error failed ({rc})")
    return out


def render_procedural(scene, cam, settings, freq: float, pixels=None) -> np.ndarray:
    """Eq. 1 compositing where every surfel shows the procedural world-space
    texture tau(x*) at its intersection (targets of the learned-part test)."""
    pix = all_pixels(cam) if pixels is None else np.ascontiguousarray(pixels, np.int32)
    out = np.zeros((pix.size, 3))
    sv = _surfels(scene)
    c, s = _cam(cam), _set(settings, 0.0)
    rc = lib().oracle_render_procedural(C.byref(c), C.byref(s), C.c_int(scene.n),
                                        *[_p(a) for a in sv[:5]], C.c_double(freq),
                                        C.c_int(pix.size), _p(pix), _p(out))
    if rc != 0:
        raise ValueError(f"oracle_render_procedural failed ({rc})")
    return out


def field_features(field, focal, x, t, table=None) -> np.ndarray:
    fr = _FieldRef(field, table)
    x, t = _d(x).reshape(-1, 3), _d(t).ravel()
    out = np.zeros((t.size, field.L * field.F))
    lib().oracle_field_features(C.byref(fr.s), C.c_double(focal), C.c_int(t.size), _p(x), _p(t),
                                _p(out))
    return out


def mlp(field, inp) -> np.ndarray:
    fr = _FieldRef(field)
    inp = _d(inp).reshape(-1, field.widths[0])
    out = np.zeros((inp.shape[0], field.widths[-1]))
    lib().oracle_mlp(C.byref(fr.s), C.c_int(inp.shape[0]), _p(inp), _p(out))
    return out


def texture(field, focal, x, t, table=None) -> np.ndarray:
    fr = _FieldRef(field, table)
    x, t = _d(x).reshape(-1, 3), _d(t).ravel()
    out = np.zeros((t.size, field.widths[-1]))
    lib().oracle_texture(C.byref(fr.s), C.c_double(focal), C.c_int(t.size), _p(x), _p(t), _p(out))
    return out


def map_positive(k: int) -> int:
    return int(lib().oracle_map_positive(int(k)))


def hash_index(kx: int, ky: int, kz: int, T: int) -> int:
    return int(lib().oracle_hash(int(kx), int(ky), int(kz), int(T)))


def centre_ray_cosine(cam, scene) -> np.ndarray:
    """|cos| of the angle between each surfel's normal and its centre ray
    (camera centre -> mu): 0 for a surfel seen exactly edge-on.  A pixel ray
    meets such a plane at a grazing angle, where t*, u and v are the ratios
    of nearly cancelling terms: their derivatives amplify any rounding by
    ~1 / |cos| (FP64 throughout)."""
    M = np.asarray(cam.world_to_cam, np.float64)
    R, t = M[:, :3], M[:, 3]
    o = -R.T @ t
    q = np.asarray(scene.quat, np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    n = np.stack([2 * (x * z + w * y), 2 * (y * z - w * x), 1 - 2 * (x * x + y * y)], 1)
    d = np.asarray(scene.mu, np.float64) - o
    return np.abs(np.sum(d * n, 1)) / np.linalg.norm(d, axis=1)


def depth_order(cam, mu) -> np.ndarray:
    mu = _d(mu).reshape(-1, 3)
    order = np.zeros(mu.shape[0], np.int32)
    c = _cam(cam)
    n = lib().oracle_depth_order(C.byref(c), C.c_int(mu.shape[0]), _p(mu), _p(order))
    return order[:n]


def storage_bytes(n_prims: int, floats_per_prim: int, L: int, T: int, F: int,
                  mlp_params: int) -> int:
    """Model size as the paper reports it: 2 bytes per Instant-NGP parameter
    (hash table and MLP), 4 bytes per other parameter (supp. Sec. 7.1)."""
    return 4 * n_prims * floats_per_prim + 2 * (L * T * F + mlp_params)
