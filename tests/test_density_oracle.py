"""Pins of the density-control oracle (oracle/density.py, oracle.blend_error)
against facts that do not come from it: farthest point sampling by the
definition and on a lattice with a known order, the blended-error
identity sum_i err_i = sum_p e_p (1 - T_final_p), the sampling law of the
selection, the split's geometry and the prune threshold."""
import numpy as np
import pytest

import oracle
from oracle import density as D
from paper_2512_13796_gb300 import synth


def test_fps_by_definition():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(15, 3)).astype(np.float32)
    idx, _ = D.fps(x, 15)
    sel = [0]
    for _ in range(14):
        best, bd = -1, -1.0
        for k in range(15):
            if k in sel:
                continue
            d = min(float(np.sum((x[k].astype(np.float64) - x[j]) ** 2)) for j in sel)
            if d > bd:
                best, bd = k, d
        sel.append(best)
    assert list(idx) == sel


def test_fps_on_a_line_with_ties_to_the_lowest_index():
    x = np.zeros((9, 3), np.float32)
    x[:, 0] = np.arange(9)
    idx, d2 = D.fps(x, 9)
    assert list(idx) == [0, 8, 4, 2, 6, 1, 3, 5, 7]
    np.testing.assert_allclose(D.fps_scales(d2), [8, 8, 4, 2, 2, 1, 1, 1, 1])


def test_fps_check_accepts_the_definition_and_near_ties_only():
    """fps_check walks another implementation's order: the FP64 order passes
    with no tie; a swap of two well-separated choices fails; a choice within
    the stated margin of the maximum passes and is counted."""
    rng = np.random.default_rng(5)
    x = rng.normal(size=(40, 3)).astype(np.float32)
    idx, d2 = D.fps(x, 40)
    c = D.fps_check(x, idx, d2, 1e-6)
    assert c["ties"] == 0 and c["d2_rel"] == 0.0 and c["steps"] == 40
    np.testing.assert_array_equal(c["d2"][1:], d2[1:])
    bad = idx.copy()
    bad[[1, 2]] = bad[[2, 1]]
    with pytest.raises(AssertionError):
        D.fps_check(x, bad, d2, 1e-6)
    with pytest.raises(AssertionError):
        D.fps_check(x, np.r_[idx[:5], idx[4]], d2[:6], 1e-6)  # a point twice
    # two points at equal distance up to 1e-9 relative from point 0: either is valid
    y = np.array([[0, 0, 0], [4, 0, 0], [0, 4 * (1 - 1e-9), 0], [1, 1, 0]], np.float64)
    ri, rd = D.fps(y, 4)
    assert ri[1] == 1
    alt = np.array([0, 2, 1, 3])
    c = D.fps_check(y, alt, rd, 1e-6)
    assert c["ties"] == 1
    with pytest.raises(AssertionError):
        D.fps_check(y, alt, rd, 1e-10)


def test_select_check_accepts_the_definition_and_near_ties_only():
    rng = np.random.default_rng(6)
    err = rng.exponential(size=50)
    expo = rng.exponential(size=50)
    sel = D.select(err, expo, 10)
    assert D.select_check(err, expo, 10, sel, 1e-7)["ties"] == 0
    with pytest.raises(AssertionError):
        D.select_check(err, expo, 10, sel[::-1], 1e-7)
    with pytest.raises(AssertionError):
        D.select_check(err, expo, 10, np.r_[sel[:9], sel[0]], 1e-7)
    # keys 1 and 1 + 1e-9: either order passes at 1e-7, and is counted
    err2 = np.array([1.0, 1.0, 0.5, 0.0])
    expo2 = np.array([1.0 + 1e-9, 1.0, 3.0, 1.0])
    assert list(D.select(err2, expo2, 2)) == [1, 0]
    assert D.select_check(err2, expo2, 2, [0, 1], 1e-7)["ties"] == 2
    with pytest.raises(AssertionError):
        D.select_check(err2, expo2, 2, [0, 1], 1e-10)


def test_blend_error_sums_to_the_composited_weight():
    """Every pixel's weights sum to 1 - T_final (Eq. 1), so with pixel
    errors e_p: sum_i err_i = sum_p e_p (1 - T_final_p)."""
    w = synth.workload(0)
    cam, st = w.cameras[0], synth.Settings(K=0)
    ref = oracle.render(w.scene, cam, st)
    e = np.random.default_rng(1).uniform(0, 1, cam.width * cam.height)
    err = oracle.blend_error(w.scene, cam, st, e)
    assert err.shape == (w.scene.n,) and np.all(err >= 0)
    np.testing.assert_allclose(err.sum(), np.sum(e * (1 - ref["T_final"])), rtol=1e-12)
    # linear in the pixel errors
    np.testing.assert_allclose(oracle.blend_error(w.scene, cam, st, 2 * e), 2 * err, rtol=1e-12)


def test_selection_law():
    # equal exponentials: the n largest errors, ties to the lowest index
    err = np.array([0.5, 2.0, 0.0, 2.0, 1.0], np.float32)
    assert list(D.select(err, np.ones(5), 3)) == [1, 3, 4]
    # a zero error is never drawn while others remain
    assert 2 not in D.select(err, np.random.default_rng(2).exponential(size=5), 4)
    # single draws follow err / sum(err)
    rng = np.random.default_rng(3)
    w = np.array([1.0, 2.0, 3.0, 4.0], np.float32)
    counts = np.zeros(4)
    n = 20000
    for _ in range(n):
        counts[D.select(w, rng.exponential(size=4), 1)[0]] += 1
    p = w / w.sum()
    assert np.all(np.abs(counts / n - p) < 4 * np.sqrt(p * (1 - p) / n))


def test_split_geometry():
    """The children's long-axis supports [-s/2, s/2] around mu -/+ (s/2) v
    cover the parent's [-s, s] exactly; everything else is copied."""
    rng = np.random.default_rng(4)
    N = 6
    q = rng.normal(size=(N, 4))
    params = dict(mu=rng.normal(size=(N, 3)), quat=q,
                  scale=np.stack([rng.uniform(0.1, 0.3, N), rng.uniform(0.1, 0.3, N)], 1),
                  opacity=rng.uniform(0.1, 0.9, N), gamma=rng.uniform(1, 4, (N, 2)),
                  color=rng.uniform(0, 1, (N, 3)))
    sel = np.array([4, 1])
    out = D.split(params, sel)
    assert out["mu"].shape == (N + 2, 3)
    for r, i in enumerate(sel):
        a = 0 if params["scale"][i][0] >= params["scale"][i][1] else 1
        s = params["scale"][i][a]
        qq = q[i] / np.linalg.norm(q[i])
        w_, x_, y_, z_ = qq
        # the long axis, from the quaternion's rotation (column a)
        cols = [np.array([1 - 2 * (y_ * y_ + z_ * z_), 2 * (x_ * y_ + w_ * z_), 2 * (x_ * z_ - w_ * y_)]),
                np.array([2 * (x_ * y_ - w_ * z_), 1 - 2 * (x_ * x_ + z_ * z_), 2 * (y_ * z_ + w_ * x_)])]
        v = cols[a]
        A, B = out["mu"][i], out["mu"][N + r]
        np.testing.assert_allclose(B - A, s * v, atol=1e-12)
        np.testing.assert_allclose((A + B) / 2, params["mu"][i], atol=1e-12)
        for k in (i, N + r):
            assert abs(out["scale"][k][a] - s / 2) < 1e-15
            assert out["scale"][k][1 - a] == params["scale"][i][1 - a]
            for key in ("quat", "opacity", "gamma", "color"):
                np.testing.assert_array_equal(out[key][k], params[key][i])
    untouched = [k for k in range(N) if k not in sel]
    for key in params:
        np.testing.assert_array_equal(out[key][untouched], params[key][untouched])


def test_prune_threshold_and_split_count():
    o = np.array([0.005, 0.00499, 0.9, 0.0, 0.0051], np.float32)
    assert list(D.prune_keep(o)) == [0, 2, 4]
    assert D.split_count(100, 1000) == 5 and D.split_count(101, 1000) == 6
    assert D.split_count(100, 102) == 2 and D.split_count(100, 90) == 0
