"""Pins of the FP64 oracle against facts fixed by the paper and by
mathematics (closed forms, invariants, special cases, finite differences).
CPU only."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2512_13796_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def facing_camera(W=32, H=32):
    return synth.front_camera(W, H)  # R = I, eye (0, 0, -3), looks along +z


def one_surfel(mu, sigma, opacity, gamma, color, quat=(1, 0, 0, 0)):
    f = np.float32
    return synth.Scene(np.array([mu], f), np.array([quat], f), np.array([sigma], f),
                       np.array([opacity], f), np.array([gamma], f), np.array([color], f))


def pixel_hit(cam, px, py, depth):
    """World point where pixel (px, py)'s ray reaches view depth ``depth``
    for the front camera (R = I, t = (0, 0, 3))."""
    x = (px + 0.5 - cam.cx) / cam.fx * depth
    y = (py + 0.5 - cam.cy) / cam.fy * depth
    return np.array([x, y, depth - 3.0])


# --------------------------------------------------------------- closed forms
@pytest.mark.parametrize("a,b,g1,g2", [(0.0, 0.0, 1.0, 1.0), (0.5, -1.2, 1.0, 1.0),
                                        (1.3, 0.7, 2.5, 1.0), (-0.9, 1.1, 3.0, 4.0),
                                        (0.25, 2.0, 1.0, 1.7)])
def test_kernel_value_camera_facing(a, b, g1, g2):
    """Sec. 4.1: alpha = o exp(-|u|^(2 g1)/2) exp(-|v|^(2 g2)/2) at a known
    primitive-space offset; gamma = 1 is the 2D Gaussian of 2DGS (Sec. 3)."""
    cam = facing_camera()
    s1, s2, o = 0.3, 0.2, 0.8
    hit = pixel_hit(cam, 20, 9, 3.0)
    mu = hit - np.array([a * s1, b * s2, 0.0])
    sc = one_surfel(mu, (s1, s2), o, (g1, g2), (0.2, 0.5, 0.9))
    st = synth.Settings(K=0, alpha_min=1e-12, alpha_max=1.0, T_min=0.0)
    pix = np.array([9 * cam.width + 20], np.int32)
    r = oracle.render(sc, cam, st, None, pix)
    # the float32 storage of mu shifts the offset slightly: recompute a, b
    mu32 = sc.mu[0].astype(np.float64)
    a32 = (hit[0] - mu32[0]) / np.float64(np.float32(s1))
    b32 = (hit[1] - mu32[1]) / np.float64(np.float32(s2))
    g1, g2 = float(np.float32(g1)), float(np.float32(g2))
    alpha = np.float64(np.float32(o)) * math.exp(-abs(a32) ** (2 * g1) / 2) * \
        math.exp(-abs(b32) ** (2 * g2) / 2)
    np.testing.assert_allclose(r["image"][0], alpha * sc.color[0].astype(np.float64),
                               rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(r["T_final"][0], 1.0 - alpha, rtol=1e-12)
    if g1 == 1.0 and g2 == 1.0:  # 2D Gaussian
        gauss = np.float64(np.float32(o)) * math.exp(-(a32 ** 2 + b32 ** 2) / 2)
        np.testing.assert_allclose(r["image"][0] / sc.color[0].astype(np.float64), gauss,
                                   rtol=1e-12)


def test_opaque_full_screen_surfel():
    """A single opaque quad (o = 1, large gamma, alpha_max = 1) covering the
    screen returns its own colour with K = 0; with K = 1 and G = 0 (first
    layer zero, no bias) the image and N are zero (Eqs. 5-6)."""
    cam = facing_camera(16, 16)
    col = (0.3, 0.6, 0.9)
    sc = one_surfel((0.0, 0.0, 0.0), (50.0, 50.0), 1.0, (50.0, 50.0), col)
    st = synth.Settings(K=0, alpha_min=1e-12, alpha_max=1.0, T_min=0.0)
    r = oracle.render(sc, cam, st, None)
    np.testing.assert_array_equal(r["image"], np.tile(np.float64(np.float32(col)), (256, 1)))
    np.testing.assert_array_equal(r["T_final"], 0.0)
    fld = synth.make_field(2, 8, 2, (8,), 0)
    fld.weights[0][:] = 0.0
    st1 = synth.Settings(K=1, alpha_min=1e-12, alpha_max=1.0, T_min=0.0)
    r1 = oracle.render(sc, cam, st1, fld)
    np.testing.assert_array_equal(r1["image"], 0.0)
    np.testing.assert_array_equal(r1["notex"], 0.0)
    np.testing.assert_array_equal(r1["weights"], 1.0)
    np.testing.assert_array_equal(r1["ids"], 0)


def small_scene(seed, n=64, gamma="var"):
    sc = synth.make_scene(n, 2, seed, gamma=gamma)
    sc.scale *= 3.0  # larger surfels -> more overlap per pixel
    return sc


def test_transmittance_invariants():
    """Eq. 1: with unit colours, K = 0 and bg = 0 the image is sum_i w_i, and
    it telescopes to 1 - T_final <= 1.  With K > 0 the same holds for
    N + sum_j W_j (Eq. 6 with textures replaced by 1 via unit colours)."""
    cam = synth.front_camera(48, 40)
    sc = small_scene(3)
    sc.color[:] = 1.0
    st = synth.Settings(K=0, T_min=0.0)
    r = oracle.render(sc, cam, st, None)
    np.testing.assert_allclose(r["image"][:, 0] + r["T_final"], 1.0, atol=1e-13)
    assert np.all(r["T_final"] >= 0) and np.all(r["T_final"] <= 1)
    assert r["n_contrib"].max() > 4
    st2 = synth.Settings(K=3, T_min=1e-4)
    r2 = oracle.render(sc, cam, st2, None)
    tot = r2["notex"][:, 0] + r2["weights"].sum(1)
    np.testing.assert_allclose(tot + r2["T_final"], 1.0, atol=1e-13)
    # slots are in descending weight order and empty slots are (-1, 0, 0)
    w = r2["weights"]
    assert np.all(np.diff(w, axis=1) <= 0)
    empty = r2["ids"] < 0
    assert np.all(w[empty] == 0) and np.all(r2["depths"][empty] == 0)


def test_early_stop_threshold():
    """Front-to-back stop rule: a surfel whose inclusion would take T below
    T_min is not composited, so T_final stays >= T_min."""
    cam = synth.front_camera(24, 24)
    sc = small_scene(5, n=200)
    sc.opacity[:] = 0.95
    st = synth.Settings(K=2, T_min=1e-2)
    r = oracle.render(sc, cam, st, None)
    assert np.all(r["T_final"] >= 1e-2)
    st0 = synth.Settings(K=2, T_min=0.0)
    r0 = oracle.render(sc, cam, st0, None)
    assert r0["T_final"].min() < 1e-2
    assert np.all(r0["n_contrib"] >= r["n_contrib"])


def test_top_k_consistent_across_K():
    """Sec. 4.2: the K selected primitives are the K largest weights; the
    first K2 slots of a K1 > K2 buffer are the K2 buffer, and Eq. 5 moves
    exactly the weights of the extra slots back into N."""
    cam = synth.front_camera(40, 40)
    sc = small_scene(7, n=120)
    r8 = oracle.render(sc, cam, synth.Settings(K=8), None)
    r2 = oracle.render(sc, cam, synth.Settings(K=2), None)
    ok = (r8["tie"] == 0) & (r2["tie"] == 0)
    assert ok.mean() > 0.9
    np.testing.assert_array_equal(r8["ids"][ok, :2], r2["ids"][ok])
    np.testing.assert_allclose(r8["weights"][ok, :2], r2["weights"][ok], rtol=0, atol=0)
    col = sc.color.astype(np.float64)
    extra = np.zeros((r8["ids"].shape[0], 3))
    for j in range(2, 8):
        idj = r8["ids"][:, j]
        has = idj >= 0
        extra[has] += r8["weights"][has, j:j + 1] * col[idj[has]]
    np.testing.assert_allclose(r2["notex"][ok], r8["notex"][ok] + extra[ok], atol=1e-13)


def test_k_at_least_m_textures_everything():
    """Eq. 6 with K >= M: every intersected primitive is textured, N = 0 and
    C = sum_i w_i G(Delta H(x_i)); the texture is recomputed here through a
    separate call at x = o + D d."""
    cam = synth.front_camera(20, 20)
    sc = small_scene(11, n=6)
    sc.mu *= 0.3
    sc.scale[:] = 0.5
    fld = synth.make_field(3, 10, 2, (8,), 3, table_std=0.5)
    st = synth.Settings(K=8, T_min=0.0)
    r = oracle.render(sc, cam, st, fld)
    assert r["n_contrib"].max() <= 8 and r["n_contrib"].max() >= 2
    np.testing.assert_array_equal(r["notex"], 0.0)
    # world rays of the front camera: o = (0, 0, -3), d = ((x+.5-cx)/fx, (y+.5-cy)/fy, 1)
    P = cam.width * cam.height
    px, py = np.arange(P) % cam.width, np.arange(P) // cam.width
    d = np.stack([(px + 0.5 - cam.cx) / cam.fx, (py + 0.5 - cam.cy) / cam.fy, np.ones(P)], 1)
    o = np.array([0.0, 0.0, -3.0])
    C = np.zeros((P, 3))
    for j in range(8):
        has = r["ids"][:, j] >= 0
        D = r["depths"][has, j]
        x = o + D[:, None] * d[has]
        tex = oracle.texture(fld, cam.fx, x, D)
        np.testing.assert_allclose(tex, r["textures"][has, j], rtol=1e-12, atol=1e-15)
        C[has] += r["weights"][has, j:j + 1] * tex
    np.testing.assert_allclose(r["image"], C, rtol=1e-12, atol=1e-15)


def test_final_identity_eq6():
    """Eq. 6: C = N + sum_j W_j T_j + T_final bg."""
    cam = synth.front_camera(32, 24)
    sc = small_scene(13, n=80)
    fld = synth.make_field(4, 12, 2, (16,), 5, table_std=0.3)
    st = synth.Settings(K=2, bg=(0.1, 0.2, 0.3))
    r = oracle.render(sc, cam, st, fld)
    C = r["notex"] + np.einsum("pk,pkc->pc", r["weights"], r["textures"]) + \
        r["T_final"][:, None] * np.array(st.bg)
    np.testing.assert_allclose(r["image"], C, rtol=1e-13, atol=1e-15)


# ----------------------------------------------------------- neural field
def test_map_positive_is_bijection():
    """Supp. Sec. 7.1: MapPositive maps [-n, n] one-to-one onto [0, 2n]."""
    n = 1_000_000
    vals = np.fromiter((oracle.map_positive(k) for k in range(-n, n + 1)), np.int64, 2 * n + 1)
    assert np.array_equal(np.sort(vals), np.arange(2 * n + 1))
    assert oracle.map_positive(5) == 9 and oracle.map_positive(-5) == 10
    assert oracle.map_positive(0) == 0


def _golden_hash_rows():
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "spatial_hash.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                f = line.split()
                rows.append(dict(k=tuple(int(v) for v in f[0:3]), log2T=int(f[3]),
                                 m=tuple(int(v) for v in f[4:7]), h=int(f[10], 16),
                                 index=int(f[11])))
    return rows


def test_spatial_hash_golden_values():
    """The spatial hash (supp. Sec. 7.1: Instant-NGP's hash on MapPositive'd
    cell coordinates) against values worked out by hand from its definition
    (tests/golden/spatial_hash.txt): the MapPositive of every axis, the
    table index at the listed T, and 31 of the 32 bits of the hash itself
    (the index at T = 2^31).  A wrong prime, a '+' for the XOR, a swapped
    axis or a dropped MapPositive changes some row."""
    rows = _golden_hash_rows()
    assert len(rows) >= 12
    for r in rows:
        assert tuple(oracle.map_positive(k) for k in r["k"]) == r["m"], r
        assert oracle.hash_index(*r["k"], 1 << r["log2T"]) == r["index"], r
        assert oracle.hash_index(*r["k"], 1 << 31) == r["h"] & 0x7FFFFFFF, r
    # the axes are hashed with different primes: permuting a cell moves it
    assert oracle.hash_index(0, 1, 0, 1 << 31) != oracle.hash_index(0, 0, 1, 1 << 31)


def test_hash_without_collisions_is_dense_trilinear():
    """One level, T = 2^22: on a box of cells whose hashes are verified
    distinct, the hash grid equals dense trilinear interpolation, which
    reproduces any multilinear function of the lattice coordinates exactly."""
    T = 1 << 22
    lo, hi = -3, 4
    ks = [(x, y, z) for x in range(lo, hi + 1) for y in range(lo, hi + 1) for z in range(lo, hi + 1)]
    idx = [oracle.hash_index(x, y, z, T) for (x, y, z) in ks]
    assert len(set(idx)) == len(idx)
    c = np.array([0.3, -0.7, 1.1, 0.05, 0.2])

    def f(k):  # multilinear in the lattice coordinates
        x, y, z = k
        return c[0] * x + c[1] * y + c[2] * z + c[3] * x * y * z + c[4]

    s = 4.0
    fld = synth.Field(1, T, 2, np.array([s], np.float32), np.zeros((1, T, 2), np.float32),
                      (2, 3), [np.eye(3, 2, dtype=np.float32)])
    tab = np.zeros((1, T, 2))
    for k, i in zip(ks, idx):
        tab[0, i, 0] = f(k)
        tab[0, i, 1] = -2.0 * f(k) + 1.0
    rng = np.random.default_rng(0)
    g = rng.uniform(lo, hi, size=(500, 3))  # lattice coordinates inside the box
    x = g / s
    t = np.full(500, 1e-9)  # Delta = 1 to double precision (f / (s t) huge)
    feat = oracle.field_features(fld, 1000.0, x, t, table=tab)
    expect0 = np.array([f(gi) for gi in g])
    np.testing.assert_allclose(feat[:, 0], expect0, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(feat[:, 1], -2.0 * expect0 + 1.0, rtol=1e-12, atol=1e-12)


def test_downweighting_limits_and_erf_approximation():
    """Eq. 3 and its derivation (supp. Sec. 7.1): Delta -> 1 as t -> 0,
    Delta -> 0 as t -> inf, and Delta approximates erf(f / (2 sqrt2 s t))^2
    (the derivation's approximation of erf^2 by 1 - exp(-4x^2/pi))."""
    L = 3
    fld = synth.Field(L, 16, 2, np.array([8.0, 64.0, 512.0], np.float32),
                      np.ones((L, 16, 2), np.float32), (6, 3),
                      [np.zeros((3, 6), np.float32)])
    focal = 1100.0
    t = np.geomspace(1e-3, 1e4, 400)
    x = np.zeros((t.size, 3)) + 0.123
    feat = oracle.field_features(fld, focal, x, t)  # table of ones -> feature = Delta
    for l, s in enumerate([8.0, 64.0, 512.0]):
        D = feat[:, 2 * l]
        assert np.all(np.diff(D) <= 1e-15)
        assert D[0] == pytest.approx(1.0, abs=1e-12)
        assert D[-1] < 1e-3
        erf2 = np.array([math.erf(focal / (2 * math.sqrt(2) * s * ti)) ** 2 for ti in t])
        assert np.max(np.abs(D - erf2)) < 0.02


def test_mlp_no_bias_zero_and_matmul():
    """Supp. Sec. 7.1: no bias + ReLU gives G(0) = 0; otherwise G is the
    matrix chain W_n relu(... relu(W_1 h))."""
    fld = synth.make_field(16, 10, 2, (64, 64), 1)
    np.testing.assert_array_equal(oracle.mlp(fld, np.zeros((3, 32))), 0.0)
    rng = np.random.default_rng(2)
    h = rng.normal(size=(50, 32))
    W1, W2, W3 = [w.astype(np.float64) for w in fld.weights]
    ref = np.maximum(np.maximum(h @ W1.T, 0) @ W2.T, 0) @ W3.T
    np.testing.assert_allclose(oracle.mlp(fld, h), ref, rtol=1e-12, atol=1e-14)


# ----------------------------------------------------------------- sort
def test_depth_order_sorted_and_culled():
    """Sec. 3: the surfels are ordered by the view depth of their centres;
    centres at or in front of the near plane are culled."""
    sc = synth.make_scene(5000, 3, 4)
    cam = synth.front_camera(64, 64, dist=1.2)
    order = oracle.depth_order(cam, sc.mu)
    M = cam.world_to_cam.astype(np.float64)
    z = sc.mu.astype(np.float64) @ M[2, :3] + M[2, 3]
    keep = np.nonzero(z > cam.near)[0]
    assert sorted(order.tolist()) == keep.tolist()
    zs = z[order]
    assert np.all(np.diff(zs) >= 0)
    same = np.diff(zs) == 0
    assert np.all(np.diff(order)[same] > 0)  # index ascending on equal depth


def _quat_of_columns(v1, v2, n):
    """Unit quaternion (w, x, y, z) of the rotation with columns v1, v2, n."""
    R = np.stack([v1, v2, n], axis=1)
    w = math.sqrt(max(0.0, 1.0 + R[0, 0] + R[1, 1] + R[2, 2])) / 2
    x = math.copysign(math.sqrt(max(0.0, 1.0 + R[0, 0] - R[1, 1] - R[2, 2])) / 2, R[2, 1] - R[1, 2])
    y = math.copysign(math.sqrt(max(0.0, 1.0 - R[0, 0] + R[1, 1] - R[2, 2])) / 2, R[0, 2] - R[2, 0])
    z = math.copysign(math.sqrt(max(0.0, 1.0 - R[0, 0] - R[1, 1] + R[2, 2])) / 2, R[1, 0] - R[0, 1])
    return (w, x, y, z)


@pytest.mark.parametrize("tilt", [0.0, 0.1])
def test_edge_on_surfel(tilt):
    """The edge-on reading: a surfel whose plane contains its own centre ray
    (|d_mu . n_c| < 1e-7) is culled.  It would add nothing anyway: that plane
    passes through the camera centre, so every pixel ray meets it at t = 0
    (behind the near plane) or lies in it (grazing).  A surfel tilted away
    from that renders a footprint, and no pixel is flagged near the
    threshold."""
    cam = facing_camera(48, 48)
    eye = np.array([0.0, 0.0, -3.0])
    mu = np.array([0.15, -0.1, 0.0])
    ray = (mu - eye) / np.linalg.norm(mu - eye)
    n0 = np.cross(ray, [0.0, 1.0, 0.0])
    n0 /= np.linalg.norm(n0)
    n = math.cos(tilt) * n0 + math.sin(tilt) * ray
    v1 = np.cross([0.0, 1.0, 0.0], n)
    v1 /= np.linalg.norm(v1)
    v2 = np.cross(n, v1)
    q = _quat_of_columns(v1, v2, n)
    sc = one_surfel(mu, (0.5, 0.5), 0.95, (1.0, 1.0), (1.0, 1.0, 1.0), quat=q)
    st = synth.Settings(K=0)
    r = oracle.render(sc, cam, st, tie_tol=1e-5, edge_tol=1e-6)
    drawn = int(np.count_nonzero(r["n_contrib"]))
    if tilt == 0.0:
        assert drawn == 0 and np.all(r["image"] == 0.0) and np.all(r["T_final"] == 1.0)
    else:
        assert drawn > 100 and r["image"].max() > 0.5
    assert not np.any(r["tie"] & 128)


# ------------------------------------------------------- storage accounting
def test_storage_matches_paper_table():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "paper_memory.txt"))
            if l.strip() and not l.startswith("#")]
    for r in rows:
        n, fl, L, lt, F, mlp_p, mb = map(int, r[1:8])
        T = (1 << lt) if L else 0
        got = oracle.storage_bytes(n, fl, L, T, F, mlp_p) / 1e6
        assert abs(got - mb) <= 5.0, (r[0], got, mb)


# ------------------------------------------------------------ gradients
def _loss_parts(r, gi, gw, gt):
    return float((r["image"] * gi).sum() + (r["weights"] * gw).sum() + (r["textures"] * gt).sum())


def _fd_check(sc, cam, st, fld, rng, n_sample=None, h=1e-6, rtol=2e-4, atol=2e-9):
    pix = oracle.all_pixels(cam)
    base = oracle.render(sc, cam, st, fld, pix, tie_tol=1e-5)
    P, K = pix.size, st.K
    gi = rng.normal(size=(P, 3))
    gw = rng.normal(size=(P, K))
    gt = rng.normal(size=(P, K, 3))
    g = oracle.render_bwd(sc, cam, st, fld, pix, gi, gw, gt)
    params = [("mu", sc.mu, g["mu"]), ("quat", sc.quat, g["quat"]), ("scale", sc.scale, g["scale"]),
              ("opacity", sc.opacity, g["opacity"]), ("gamma", sc.gamma, g["gamma"]),
              ("color", sc.color, g["color"])]
    checked = {k: 0 for k in ("mu", "quat", "scale", "opacity", "gamma", "color", "table", "mlp")}
    skipped = 0

    def run(mod):
        return oracle.render(sc64, cam, st, fld64, pix, tie_tol=0.0)

    # float64 working copies so the perturbation is exact
    sc64 = synth.Scene(*(np.asarray(a, np.float64).copy() for a in
                         (sc.mu, sc.quat, sc.scale, sc.opacity, sc.gamma, sc.color)))
    fld64 = synth.Field(fld.L, fld.T, fld.F, fld.level_scale, fld.table.astype(np.float64),
                        fld.widths, [w.astype(np.float64) for w in fld.weights])
    targets = []
    for name, _, gr in params:
        arr = getattr(sc64, "opacity" if name == "opacity" else name)
        flat = arr.reshape(-1)
        cand = np.nonzero(np.abs(gr.reshape(-1)) > 1e-9)[0]
        if n_sample is not None and cand.size > n_sample:
            cand = rng.choice(cand, n_sample, replace=False)
        for i in cand:
            targets.append((name, flat, int(i), gr.reshape(-1)[i]))
    tflat = fld64.table.reshape(-1)
    cand = np.nonzero(np.abs(g["table"].reshape(-1)) > 1e-9)[0]
    for i in rng.choice(cand, min(cand.size, n_sample or 40), replace=False):
        targets.append(("table", tflat, int(i), g["table"].reshape(-1)[i]))
    for li, w in enumerate(fld64.weights):
        wf = w.reshape(-1)
        gl = g["mlp_layers"][li].reshape(-1)
        for i in rng.choice(wf.size, min(wf.size, 12), replace=False):
            targets.append(("mlp", wf, int(i), gl[i]))
    for name, flat, i, an in targets:
        x0 = flat[i]
        hh = h * max(1.0, abs(x0))
        flat[i] = x0 + hh
        rp = run(None)
        flat[i] = x0 - hh
        rm = run(None)
        flat[i] = x0
        if not (np.array_equal(rp["ids"], base["ids"]) and np.array_equal(rm["ids"], base["ids"])
                and np.array_equal(rp["n_contrib"], base["n_contrib"])
                and np.array_equal(rm["n_contrib"], base["n_contrib"])):
            skipped += 1
            continue
        fd = (_loss_parts(rp, gi, gw, gt) - _loss_parts(rm, gi, gw, gt)) / (2 * hh)
        if abs(fd - an) > atol + rtol * max(abs(fd), abs(an)):
            # A kink of the trilinear weights (a cell boundary of a fine
            # hash-grid level) inside [-h, h] biases the difference quotient;
            # a step ten times smaller moves past it, and must then agree.
            h2 = hh / 10
            flat[i] = x0 + h2
            rp2 = run(None)
            flat[i] = x0 - h2
            rm2 = run(None)
            flat[i] = x0
            fd2 = (_loss_parts(rp2, gi, gw, gt) - _loss_parts(rm2, gi, gw, gt)) / (2 * h2)
            assert abs(fd2 - an) <= 1e-6 + 1e-5 * max(abs(fd2), abs(an)), (name, i, fd, fd2, an)
            skipped += 1
        checked[name] += 1
    return checked, skipped


def test_gradients_finite_difference_tiny_scenes():
    """Central differences in FP64 on tiny scenes, every parameter class:
    mu, q, sigma, o, gamma, colour, hash-table entries and MLP weights."""
    rng = np.random.default_rng(0)
    for seed in range(3):
        sc = synth.make_scene(5, 1, 40 + seed, gamma="var")
        sc.scale[:] = np.random.default_rng(seed).uniform(0.3, 0.7, size=(5, 2))
        sc.opacity[:] = np.random.default_rng(seed + 9).uniform(0.2, 0.8, size=5)
        cam = synth.front_camera(16, 16)
        fld = synth.make_field(2, 8, 2, (8,), seed, table_std=0.5)
        st = synth.Settings(K=2, bg=(0.2, 0.1, 0.4))
        checked, skipped = _fd_check(sc, cam, st, fld, rng)
        for k, v in checked.items():
            assert v > 0, (k, checked)
        assert skipped < 0.2 * sum(checked.values())


def test_gradients_finite_difference_config0():
    """Config 0 (256 surfels, 64x64, K = 2, 4-level grid, 8->16->3 MLP):
    a random sample of every parameter class is checked by central FD."""
    w = synth.workload(0)
    rng = np.random.default_rng(1)
    checked, skipped = _fd_check(w.scene, w.cameras[0], w.settings, w.field, rng, n_sample=25)
    for k, v in checked.items():
        assert v > 0, (k, checked)


def test_clamped_alpha_has_no_gradient():
    """alpha above alpha_max is clamped to a constant, so its geometry gets
    no gradient through alpha."""
    cam = facing_camera(8, 8)
    sc = one_surfel((0.0, 0.0, 0.0), (5.0, 5.0), 1.0, (1.0, 1.0), (0.5, 0.5, 0.5))
    st = synth.Settings(K=0, alpha_max=0.9)
    pix = oracle.all_pixels(cam)
    g = oracle.render_bwd(sc, cam, st, None, pix, np.ones((pix.size, 3)))
    assert g["opacity"][0] == 0.0 and np.all(g["scale"] == 0.0)
    np.testing.assert_allclose(g["color"][0], 0.9 * pix.size)


def test_procedural_targets_reduce_to_constant_colour():
    """With frequency 0 the procedural texture is a constant per channel, so
    the procedural render equals the plain render (K = 0) with that colour."""
    cam = synth.front_camera(24, 20)
    sc = small_scene(17, n=90)
    st = synth.Settings(K=0)
    img = oracle.render_procedural(sc, cam, st, 0.0)
    tau = np.array([0.5 + 0.4 * math.sin(2 * c) * math.sin(c) + 0.1 * math.sin(-c)
                    for c in range(3)])
    sc2 = synth.Scene(sc.mu, sc.quat, sc.scale, sc.opacity, sc.gamma,
                      np.tile(tau, (sc.n, 1)))
    ref = oracle.render(sc2, cam, st, None)
    np.testing.assert_allclose(img, ref["image"], rtol=1e-12, atol=1e-14)


def test_absolute_mode_bounds_the_gradient():
    """render_bwd(absolute=True) sums the magnitudes of the contributions
    (the texture path evaluated on magnitudes): it bounds |gradient| entry
    by entry, equals it for the surfel parameters the texture path does not
    reach when only one pixel contributes, and is linear in |upstream|."""
    cam = synth.front_camera(24, 20)
    sc = small_scene(13, n=40)
    fld = synth.make_field(4, 10, 2, (16,), 3, table_std=0.3)
    st = synth.Settings(K=2)
    rng = np.random.default_rng(9)
    P = cam.width * cam.height
    pix = np.arange(P, dtype=np.int32)
    dI, dW = rng.normal(size=(P, 3)), rng.normal(size=(P, 2))
    g = oracle.render_bwd(sc, cam, st, fld, pix, dI, dW)
    a = oracle.render_bwd(sc, cam, st, fld, pix, dI, dW, absolute=True)
    for k in ("mu", "quat", "scale", "opacity", "gamma", "color", "table", "mlp"):
        assert np.all(a[k] >= np.abs(g[k]) - 1e-12 * (np.abs(g[k]).max() + 1)), k
        assert a[k].max() > 0, k
    a2 = oracle.render_bwd(sc, cam, st, fld, pix, 2 * dI, 2 * dW, absolute=True)
    np.testing.assert_allclose(a2["table"], 2 * a["table"], rtol=1e-12)
    one = pix[[P // 2 + cam.width // 2]]
    g1 = oracle.render_bwd(sc, cam, st, fld, one, dI[one], dW[one])
    a1 = oracle.render_bwd(sc, cam, st, fld, one, dI[one], dW[one], absolute=True)
    # one pixel: one contribution per surfel entry; the entries the texture
    # path's dt does not reach equal the magnitude of the gradient, mu and q
    # add the magnitude of what dt moves them by
    for k in ("scale", "opacity", "color"):
        np.testing.assert_allclose(a1[k], np.abs(g1[k]), rtol=1e-12, atol=1e-300)
    for k in ("mu", "quat"):
        assert np.all(a1[k] >= np.abs(g1[k]) * (1 - 1e-12)), k


def test_centre_ray_cosine():
    """|cos| between a surfel's normal and its centre ray: 1 for a surfel
    facing the camera, ~0 for one whose plane holds the camera centre."""
    cam = facing_camera(48, 48)
    face = one_surfel((0.3, -0.2, 0.5), (0.1, 0.1), 0.5, (1, 1), (1, 1, 1))
    c = oracle.centre_ray_cosine(cam, face)[0]
    d = np.array([0.3, -0.2, 3.5])
    assert abs(c - 3.5 / np.linalg.norm(d)) < 1e-6
    eye = np.array([0.0, 0.0, -3.0])
    mu = np.array([0.15, -0.1, 0.0])
    ray = (mu - eye) / np.linalg.norm(mu - eye)
    n = np.cross(ray, [0.0, 1.0, 0.0])
    n /= np.linalg.norm(n)
    v1 = np.cross([0.0, 1.0, 0.0], n)
    v1 /= np.linalg.norm(v1)
    edge = one_surfel(mu, (0.5, 0.5), 0.9, (1, 1), (1, 1, 1),
                      quat=_quat_of_columns(v1, np.cross(n, v1), n))
    assert oracle.centre_ray_cosine(cam, edge)[0] < 1e-6
