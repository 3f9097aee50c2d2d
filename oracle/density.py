"""FP64 oracle of the adaptive density control (supp. Sec. 7.2 and Sec. 5,
"Adaptive Density Control").

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``).

  fps             farthest point sampling: I_0 = 0, then I_i = argmax over
                  unselected k of min_{j<i} d(x_k, x_{I_j}), squared
                  distances in FP64; exact ties go to the lowest index
  fps_check       validates another implementation's sampling order step by
                  step against the FP64 definition: each of its choices must
                  be the FP64 argmax, or lie within a stated relative margin
                  of it (a near-tie, counted), and the walk continues from
                  its choice; its squared distances at selection are compared
                  with the FP64 ones
  fps_scales      the initial scale of point I_i: min_{j<i} d(x_{I_i}, x_{I_j}),
                  the distance at which it was selected; I_0 (no predecessor)
                  takes I_1's
  split_count     5 % of the primitives, rounded up, capped so that the total
                  stays within P (the paper caps the additions by P)
  select          sampling without replacement with probabilities
                  proportional to the blended errors (Efraimidis-Spirakis):
                  with exponential random numbers E_i (drawn by the caller),
                  the n smallest keys E_i / err_i (FP64; err_i = 0 never
                  selected while a positive error remains), ties by index.
                  Normalising the errors (as the paper does) does not change
                  this selection.
  select_check    validates another implementation's selection: its r-th
                  key equals the FP64 r-th smallest within a stated relative
                  margin (where the indices differ, a near-tie, counted)
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


def _d2(xs, x0):
    d = np.asarray(xs, np.float64) - np.asarray(x0, np.float64)
    return (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]


def fps(points, m: int) -> tuple[np.ndarray, np.ndarray]:
    """(indices [m], squared FP64 distances at selection [m]; entry 0 is
    +inf)."""
    x = np.asarray(points, np.float64)
    n = x.shape[0]
    m = min(m, n)
    idx = np.zeros(m, np.int64)
    d2sel = np.full(m, np.inf)
    mind = np.full(n, np.inf)
    cur = 0
    for i in range(m):
        idx[i] = cur
        if i > 0:
            d2sel[i] = mind[cur]
        mind = np.minimum(mind, _d2(x, x[cur]))
        mind[cur] = -1.0  # selected
        if i + 1 < m:
            cur = int(np.argmax(mind))  # first maximum: lowest index on ties
    return idx, d2sel


def fps_check(points, idx, d2sel, rel_tol: float) -> dict:
    """Walks the order ``idx`` (with its squared distances at selection
    ``d2sel``) of another FPS implementation against the FP64 definition.
    Raises AssertionError at the first step whose choice is farther than
    rel_tol (relative) below the FP64 maximum, or repeats a point; returns
    the number of steps, of near-tie steps (a different point within
    rel_tol of the maximum), the largest relative error of d2sel and the
    FP64 squared distance at each step of the walk (``d2``)."""
    x = np.asarray(points, np.float64)
    n = x.shape[0]
    idx = np.asarray(idx, np.int64)
    m = idx.size
    assert m == 0 or idx[0] == 0, "the first sample is point 0"
    mind = np.full(n, np.inf)
    ties, d2err = 0, 0.0
    d2 = np.full(m, np.inf)
    for i in range(m):
        g = int(idx[i])
        assert 0 <= g < n and mind[g] >= 0.0, f"step {i}: point {g} invalid or already selected"
        if i > 0:
            best = int(np.argmax(mind))
            top = mind[best]
            if g != best:
                assert mind[g] >= top * (1.0 - rel_tol), \
                    f"step {i}: chose {g} at {mind[g]!r}, FP64 maximum {best} at {top!r}"
                ties += 1
            d2[i] = mind[g]
            d2err = max(d2err, abs(float(d2sel[i]) - mind[g]) / max(mind[g], 1e-300))
        mind = np.minimum(mind, _d2(x, x[g]))
        mind[g] = -1.0
    return dict(steps=m, ties=ties, d2_rel=d2err, d2=d2)


def fps_scales(d2sel) -> np.ndarray:
    d = np.sqrt(np.asarray(d2sel, np.float64))
    if d.size > 1:
        d[0] = d[1]
    elif d.size == 1:
        d[0] = 0.0
    return d


def split_count(n: int, cap: int) -> int:
    return max(0, min(math.ceil(SPLIT_FRACTION * n), cap - n))


def _keys(err, expo):
    err = np.asarray(err, np.float64)
    e = np.asarray(expo, np.float64)
    with np.errstate(divide="ignore"):
        return np.where(err > 0, e / np.where(err > 0, err, 1.0), np.inf)


def select(err, expo, n: int) -> np.ndarray:
    order = np.argsort(_keys(err, expo), kind="stable")
    return order[:n]


def select_check(err, expo, n: int, sel, rel_tol: float) -> dict:
    """Checks another implementation's selection ``sel`` (n indices, in
    increasing key order) against the FP64 one: distinct indices, and the
    r-th selected key equal to the FP64 r-th smallest key within rel_tol
    (relative; infinite keys exactly).  Returns the number of positions
    whose index differs from the FP64 selection (near-ties)."""
    k = _keys(err, expo)
    ref = select(err, expo, n)
    sel = np.asarray(sel, np.int64)
    assert sel.size == n and np.unique(sel).size == n, "indices not distinct"
    ties = 0
    for r in range(n):
        a, b = k[sel[r]], k[ref[r]]
        if sel[r] == ref[r]:
            continue
        if np.isinf(b):
            assert False, f"position {r}: {sel[r]} instead of {ref[r]} (zero errors, index order)"
        assert abs(a - b) <= rel_tol * b, f"position {r}: key {a!r} against {b!r}"
        ties += 1
    return dict(ties=ties)


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
