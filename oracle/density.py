"""FP64 oracle of the adaptive density control (supp. Sec. 7.2 and Sec. 5,
"Adaptive Density Control").

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``).

  fps             farthest point sampling: I_0 = 0, then I_i = argmax over
                  unselected k of min_{j<i} d(x_k, x_{I_j}); the squared
                  distances are formed and compared in FP32 with every
                  operation rounded ((dx dx + dy dy) + dz dz), the precision
                  the kernel decides in; ties go to the lowest index
  fps_scales      the initial scale of point I_i: min_{j<i} d(x_{I_i}, x_{I_j}),
                  the distance at which it was selected; I_0 (no predecessor)
                  takes I_1's
  split_count     5 % of the primitives, rounded up, capped so that the total
                  stays within P (the paper caps the additions by P)
  select          sampling without replacement with probabilities
                  proportional to the blended errors (Efraimidis-Spirakis):
                  with exponential random numbers E_i (drawn by the caller),
                  the n smallest keys E_i / err_i (FP32 division; err_i = 0
                  never selected), ties by index.  Normalising the errors
                  (as the paper does) does not change this selection.
  split           surfel i becomes two: scales (sigma_long / 2, sigma_short)
                  and means mu -/+ (sigma_long / 2) v_long, every other
                  property copied; the paper writes it for sigma_1 >= sigma_2,
                  the reading takes the longer axis (axis 1 on a tie).  The
                  first child keeps slot i, the second is appended (in
                  selection order).
  prune_keep      the primitives with opacity >= 0.005, in order (those
                  below are pruned)
"""
from __future__ import annotations

import math

import numpy as np

PRUNE_OPACITY = 0.005
SPLIT_FRACTION = 0.05


def _d2_f32(xs, x0):
    d = xs.astype(np.float32) - x0.astype(np.float32)
    return (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]


def fps(points, m: int) -> tuple[np.ndarray, np.ndarray]:
    """(indices [m], squared FP32 distances at selection [m]; entry 0 is
    +inf)."""
    x = np.asarray(points, np.float32)
    n = x.shape[0]
    m = min(m, n)
    idx = np.zeros(m, np.int64)
    d2sel = np.full(m, np.inf, np.float32)
    mind = np.full(n, np.inf, np.float32)
    cur = 0
    for i in range(m):
        idx[i] = cur
        if i > 0:
            d2sel[i] = mind[cur]
        mind = np.minimum(mind, _d2_f32(x, x[cur]))
        mind[cur] = -1.0  # selected
        if i + 1 < m:
            cur = int(np.argmax(mind))  # first maximum: lowest index on ties
    return idx, d2sel


def fps_scales(d2sel) -> np.ndarray:
    d = np.sqrt(np.asarray(d2sel, np.float64))
    if d.size > 1:
        d[0] = d[1]
    elif d.size == 1:
        d[0] = 0.0
    return d


def split_count(n: int, cap: int) -> int:
    return max(0, min(math.ceil(SPLIT_FRACTION * n), cap - n))


def select(err, expo, n: int) -> np.ndarray:
    err = np.asarray(err, np.float32)
    e = np.asarray(expo, np.float32)
    with np.errstate(divide="ignore"):
        key = np.where(err > 0, e / np.where(err > 0, err, 1.0).astype(np.float32),
                       np.float32(np.inf)).astype(np.float32)
    order = np.argsort(key, kind="stable")
    return order[:n]


def _rot(q):
    q = np.asarray(q, np.float64)
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def split(params: dict, sel) -> dict:
    """params: mu [N,3], quat [N,4], scale [N,2], opacity [N], gamma [N,2],
    color [N,...]; returns the N + len(sel) surfels after the split."""
    out = {k: np.concatenate([np.asarray(v, np.float64),
                              np.asarray(v, np.float64)[np.asarray(sel, np.int64)]])
           for k, v in params.items()}
    N = np.asarray(params["mu"]).shape[0]
    for r, i in enumerate(np.asarray(sel, np.int64)):
        R = _rot(params["quat"][i])
        s1, s2 = float(params["scale"][i][0]), float(params["scale"][i][1])
        a = 0 if s1 >= s2 else 1
        sl = s1 if a == 0 else s2
        v = R[:, a]
        mu = np.asarray(params["mu"][i], np.float64)
        out["mu"][i] = mu - 0.5 * sl * v
        out["mu"][N + r] = mu + 0.5 * sl * v
        out["scale"][i][a] = 0.5 * sl
        out["scale"][N + r][a] = 0.5 * sl
    return out


def prune_keep(opacity) -> np.ndarray:
    return np.nonzero(np.asarray(opacity) >= np.float32(PRUNE_OPACITY))[0]
