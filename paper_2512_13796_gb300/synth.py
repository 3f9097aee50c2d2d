"""Seeded synthetic inputs shared by the CUDA path's tests, the benchmark and
the oracle's tests.

This module draws random numbers and lays out arrays; it holds none of the
rendering arithmetic (no intersection, compositing, hashing or network
evaluation).  Everything is float32 on the way out because that is what both
sides consume: the oracle widens the same float32 values to float64 exactly.

Scene recipe (stands in for the paper's captured scenes, which are not
available; shapes follow the paper's workloads of hundreds of thousands of
surfels seen in HD views, Sec. 5):
  * a fraction of the surfels lies on random planes (a random point in
    [-0.5, 0.5]^3 plus a random unit normal; points uniform on the plane inside
    [-1, 1]^3 by rejection), the rest is uniform in [-1, 1]^3;
  * the "room" variant uses the six faces of [-1, 1]^3 plus random vertical
    planes (normal orthogonal to the y axis);
  * scales log-uniform in [0.02, 0.2] per axis, rotations random unit
    quaternions (normalised Gaussian 4-vectors), opacity U(0.05, 0.99),
    colours U(0, 1)^3, gamma either (1, 1) or U(1, 4) per axis.
Cameras: pinhole, horizontal field of view 60 degrees, fx = fy, principal
point at the image centre, OpenCV axes (+z forward, +y down), 3 units from
the origin looking at it.
Field: hash table entries N(0, 1e-2), MLP weights Glorot-uniform, level
scales s_l = s_min * b^l from s_min = 8 to s_max = 1024 per world unit.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    world_to_cam: np.ndarray  # (3, 4) float32, x_cam = R x_world + t
    near: float = 0.2


@dataclasses.dataclass
class Scene:
    mu: np.ndarray       # (N, 3) float32
    quat: np.ndarray     # (N, 4) float32, (w, x, y, z), not necessarily unit
    scale: np.ndarray    # (N, 2) float32, sigma > 0
    opacity: np.ndarray  # (N,)   float32 in (0, 1)
    gamma: np.ndarray    # (N, 2) float32, >= 1
    color: np.ndarray    # (N, 3) float32

    @property
    def n(self) -> int:
        return int(self.mu.shape[0])


@dataclasses.dataclass
class Field:
    L: int
    T: int
    F: int
    level_scale: np.ndarray   # (L,) float32
    table: np.ndarray         # (L, T, F) float32 master copy
    widths: tuple             # e.g. (32, 64, 64, 3)
    weights: list             # per layer (out, in) float32


@dataclasses.dataclass
class Settings:
    K: int = 4
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    T_min: float = 1e-4
    bg: tuple = (0.0, 0.0, 0.0)


# ----------------------------------------------------------------- cameras
def look_at_camera(width: int, height: int, eye, target=(0.0, 0.0, 0.0),
                   fov_x_deg: float = 60.0, near: float = 0.2) -> Camera:
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    down = np.array([0.0, 1.0, 0.0])
    if abs(fwd @ down) > 0.999:
        down = np.array([0.0, 0.0, 1.0])
    right = np.cross(down, fwd)
    right /= np.linalg.norm(right)
    y = np.cross(fwd, right)
    R = np.stack([right, y, fwd])
    t = -R @ eye
    fx = (width / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)
    m = np.concatenate([R, t[:, None]], axis=1).astype(np.float32)
    return Camera(width, height, float(np.float32(fx)), float(np.float32(fx)),
                  width / 2.0, height / 2.0, m, near)


def front_camera(width: int, height: int, dist: float = 3.0) -> Camera:
    return look_at_camera(width, height, (0.0, 0.0, -dist))


def sphere_cameras(rng: np.random.Generator, sizes, radius: float = 3.0):
    cams = []
    for (w, h) in sizes:
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        cams.append(look_at_camera(w, h, radius * v))
    return cams


# ----------------------------------------------------------------- scenes
def _unit(rng, n, d):
    v = rng.normal(size=(n, d))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _points_on_plane(rng, n, p0, normal):
    a = np.cross(normal, [1.0, 0.0, 0.0])
    if np.linalg.norm(a) < 1e-3:
        a = np.cross(normal, [0.0, 1.0, 0.0])
    a /= np.linalg.norm(a)
    b = np.cross(normal, a)
    out = np.empty((0, 3))
    while out.shape[0] < n:
        m = max(64, 4 * (n - out.shape[0]))
        st = rng.uniform(-3.5, 3.5, size=(m, 2))
        p = p0 + st[:, :1] * a + st[:, 1:] * b
        ok = np.all(np.abs(p) <= 1.0, axis=1)
        out = np.concatenate([out, p[ok]])
    return out[:n]


def make_scene(n: int, n_planes: int, seed: int, *, room: bool = False,
               plane_frac: float = 0.7, gamma: str = "one") -> Scene:
    """gamma: "one" -> (1, 1); "var" -> U(1, 4) per axis."""
    rng = np.random.default_rng(seed)
    n_on = int(round(plane_frac * n))
    planes = []
    if room:
        for ax in range(3):
            for s in (-1.0, 1.0):
                nrm = np.zeros(3)
                nrm[ax] = 1.0
                planes.append((s * nrm, nrm))
        for _ in range(max(0, n_planes - 6)):
            th = rng.uniform(0, 2 * math.pi)
            nrm = np.array([math.cos(th), 0.0, math.sin(th)])
            planes.append((rng.uniform(-0.5, 0.5, 3), nrm))
    else:
        for _ in range(n_planes):
            planes.append((rng.uniform(-0.5, 0.5, 3), _unit(rng, 1, 3)[0]))
    counts = np.full(len(planes), n_on // len(planes))
    counts[: n_on - counts.sum()] += 1
    pts = [_points_on_plane(rng, int(c), p0, nrm) for c, (p0, nrm) in zip(counts, planes)]
    pts.append(rng.uniform(-1.0, 1.0, size=(n - n_on, 3)))
    mu = np.concatenate(pts)
    mu = mu[rng.permutation(n)]
    quat = _unit(rng, n, 4)
    scale = np.exp(rng.uniform(math.log(0.02), math.log(0.2), size=(n, 2)))
    opacity = rng.uniform(0.05, 0.99, size=n)
    color = rng.uniform(0.0, 1.0, size=(n, 3))
    if gamma == "one":
        g = np.ones((n, 2))
    elif gamma == "var":
        g = rng.uniform(1.0, 4.0, size=(n, 2))
    else:
        raise ValueError(gamma)
    f = np.float32
    return Scene(mu.astype(f), quat.astype(f), scale.astype(f), opacity.astype(f),
                 g.astype(f), color.astype(f))


def level_scales(L: int, s_min: float = 8.0, s_max: float = 1024.0) -> np.ndarray:
    if L == 1:
        return np.array([s_min], np.float32)
    b = math.exp((math.log(s_max) - math.log(s_min)) / (L - 1))
    return np.array([s_min * b ** l for l in range(L)], np.float64).astype(np.float32)


def make_field(L: int, log2T: int, F: int, hidden: tuple, seed: int,
               table_std: float = 1e-2, out_dim: int = 3) -> Field:
    rng = np.random.default_rng(seed + 7919)
    T = 1 << log2T
    table = rng.normal(0.0, table_std, size=(L, T, F)).astype(np.float32)
    widths = (L * F,) + tuple(hidden) + (out_dim,)
    weights = []
    for i in range(len(widths) - 1):
        fan_in, fan_out = widths[i], widths[i + 1]
        lim = math.sqrt(6.0 / (fan_in + fan_out))
        weights.append(rng.uniform(-lim, lim, size=(fan_out, fan_in)).astype(np.float32))
    return Field(L, T, F, level_scales(L), table, widths, weights)


# ------------------------------------------------- the five workloads
@dataclasses.dataclass
class Workload:
    name: str
    scene: Scene
    cameras: list
    settings: Settings
    field: Field
    grid_dtype: str   # "f32" | "f16"
    mlp_dtype: str    # "f32" | "bf16" | "f16"


def workload(idx: int, *, gamma: str | None = None, seed: int | None = None,
             precision: str | None = None) -> Workload:
    """Config 0..4 of the measurement plan.  ``precision`` overrides the
    grid/MLP storage: "f32", "bf16" (fp16 table + bf16 MLP) or "f16" (fp16
    table + fp16 MLP with loss scaling)."""
    s = idx if seed is None else seed
    if idx == 0:
        sc = make_scene(256, 3, s, gamma=gamma or "one")
        cams = [front_camera(64, 64)]
        fld = make_field(4, 12, 2, (16,), s)
        st, prec = Settings(K=2), "f32"
    elif idx == 1:
        sc = make_scene(50_000, 10, s, gamma=gamma or "one")
        cams = [front_camera(800, 800)]
        fld = make_field(8, 16, 2, (64,), s)
        st, prec = Settings(K=4), "f32"
    elif idx == 2:
        sc = make_scene(300_000, 12, s, room=True, gamma=gamma or "var")
        cams = [front_camera(1280, 720)]
        fld = make_field(16, 19, 2, (64, 64), s)
        st, prec = Settings(K=4), "bf16"
    elif idx == 3:
        sc = make_scene(600_000, 12, s, room=True, gamma=gamma or "var")
        rng = np.random.default_rng(s + 31)
        sizes = [(640, 480), (800, 600), (1024, 576), (1280, 720),
                 (1280, 960), (1440, 1080), (1600, 900), (1920, 1080)]
        cams = sphere_cameras(rng, sizes)
        fld = make_field(16, 19, 2, (64, 64), s)
        st, prec = Settings(K=4), "bf16"
    elif idx == 4:
        sc = make_scene(1_000_000, 12, s, room=True, gamma=gamma or "var")
        cams = [front_camera(1920, 1080)]
        fld = make_field(16, 20, 2, (64, 64), s)
        st, prec = Settings(K=8), "bf16"
    else:
        raise ValueError(idx)
    prec = precision or prec
    return Workload(f"config{idx}", sc, cams, st, fld,
                    "f32" if prec == "f32" else "f16",
                    prec)


def sh_coefficients(n: int, seed: int, rest_std: float = 0.2) -> np.ndarray:
    """Seeded degree-3 SH colour coefficients [n, 16, 3] (float32): the
    constant term U(-1, 1), the 15 higher ones N(0, rest_std)."""
    rng = np.random.default_rng(seed + 71)
    c = rng.normal(0.0, rest_std, size=(n, 16, 3))
    c[:, 0, :] = rng.uniform(-1.0, 1.0, size=(n, 3))
    return c.astype(np.float32)


def pixel_sample(cam: Camera, n_random: int, n_tiles: int, seed: int,
                 tile: int = 16) -> np.ndarray:
    """Fixed pixel subsample: ``n_random`` pixels by seed plus every pixel of
    ``n_tiles`` whole 16x16 tiles.  Returns sorted unique flat indices."""
    rng = np.random.default_rng(seed + 101)
    P = cam.width * cam.height
    idx = [rng.choice(P, size=min(n_random, P), replace=False)]
    tx, ty = (cam.width + tile - 1) // tile, (cam.height + tile - 1) // tile
    for t in rng.choice(tx * ty, size=min(n_tiles, tx * ty), replace=False):
        x0, y0 = (t % tx) * tile, (t // tx) * tile
        ys, xs = np.meshgrid(np.arange(y0, min(y0 + tile, cam.height)),
                             np.arange(x0, min(x0 + tile, cam.width)), indexing="ij")
        idx.append((ys * cam.width + xs).ravel())
    return np.unique(np.concatenate(idx)).astype(np.int32)
