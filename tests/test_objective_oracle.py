"""Pins of the objective / optimiser oracle (oracle/objective.py) against
facts that do not come from the oracle itself: closed forms of SSIM, the
window's definition, finite differences of each term, Adam's first step in
closed form and its convergence on a quadratic."""
import numpy as np
import pytest

from oracle import objective as O


def _imgs(seed, H=14, W=12):
    rng = np.random.default_rng(seed)
    return rng.uniform(0, 1, (H, W, 3)), rng.uniform(0, 1, (H, W, 3))


def test_window_is_a_normalised_gaussian():
    w = O.gaussian_window()
    assert w.shape == (11, 11)
    assert abs(w.sum() - 1.0) < 1e-14
    np.testing.assert_allclose(w, w.T, rtol=0, atol=0)
    np.testing.assert_allclose(w, w[::-1, ::-1], rtol=0, atol=0)
    # adjacent taps along an axis through the centre: exp(-(2r+1) / (2 sigma^2))
    c = 5
    for r in range(5):
        ratio = w[c, c + r + 1] / w[c, c + r]
        assert abs(ratio - np.exp(-(2 * r + 1) / (2 * 1.5 ** 2))) < 1e-12


def test_correlation_matches_direct_sum_and_zero_padding():
    rng = np.random.default_rng(1)
    img = rng.normal(size=(9, 7))
    win = rng.normal(size=(3, 3))
    out = O.correlate_same(img, win)
    for (y, x) in [(0, 0), (4, 3), (8, 6), (0, 6)]:
        ref = 0.0
        for dy in range(3):
            for dx in range(3):
                yy, xx = y + dy - 1, x + dx - 1
                if 0 <= yy < 9 and 0 <= xx < 7:
                    ref += win[dy, dx] * img[yy, xx]
        assert abs(out[y, x] - ref) < 1e-12


def test_ssim_of_an_image_with_itself_is_one():
    x, _ = _imgs(2)
    np.testing.assert_allclose(O.ssim_map(x, x), 1.0, atol=1e-12)
    assert abs(O.dssim(x, x)) < 1e-12
    np.testing.assert_allclose(O.dssim_grad(x, x), 0.0, atol=1e-12)


def test_ssim_of_constant_images_interior_closed_form():
    """Away from the zero-padded border the local statistics of constant
    images a, b are means a, b and zero (co)variances, so
    SSIM = (2ab + C1) / (a^2 + b^2 + C1)."""
    H, W = 24, 20
    a, b = 0.3, 0.7
    s = O.ssim_map(np.full((H, W, 3), a), np.full((H, W, 3), b))
    inner = s[5:H - 5, 5:W - 5]
    np.testing.assert_allclose(inner, (2 * a * b + O.SSIM_C1) / (a * a + b * b + O.SSIM_C1),
                               rtol=1e-12)


def test_ssim_is_symmetric_and_bounded():
    x, y = _imgs(3)
    np.testing.assert_allclose(O.ssim_map(x, y), O.ssim_map(y, x), rtol=1e-12)
    assert np.all(O.ssim_map(x, y) <= 1.0 + 1e-12)


def _fd(f, x, idx, h=1e-6):
    xp, xm = x.copy(), x.copy()
    xp[idx] += h
    xm[idx] -= h
    return (f(xp) - f(xm)) / (2 * h)


def test_dssim_gradient_matches_finite_differences():
    x, y = _imgs(4)
    g = O.dssim_grad(x, y)
    rng = np.random.default_rng(5)
    for _ in range(25):
        idx = (rng.integers(x.shape[0]), rng.integers(x.shape[1]), rng.integers(3))
        fd = _fd(lambda z: O.dssim(z, y), x, idx)
        assert abs(fd - g[idx]) < 1e-7 + 1e-5 * abs(fd), (idx, fd, g[idx])
    # border pixels too
    for idx in [(0, 0, 0), (13, 11, 2), (0, 11, 1)]:
        fd = _fd(lambda z: O.dssim(z, y), x, idx)
        assert abs(fd - g[idx]) < 1e-7 + 1e-5 * abs(fd)


def test_l1_value_and_gradient():
    x, y = _imgs(6)
    assert abs(O.l1(x, y) - np.abs(x - y).sum() / x.size) < 1e-15
    g = O.l1_grad(x, y)
    for idx in [(0, 0, 0), (3, 4, 1), (13, 11, 2)]:
        assert abs(_fd(lambda z: O.l1(z, y), x, idx) - g[idx]) < 1e-8


def test_texture_loss_reduces_and_differentiates():
    rng = np.random.default_rng(7)
    H, W, K = 6, 5, 3
    tgt = rng.uniform(0, 1, (H, W, 3))
    Wt = rng.uniform(0.05, 0.5, (H, W, K))
    T = rng.normal(size=(H, W, K, 3))
    Wt[0, 0] = 0.0                      # no textured weight: no contribution
    # textures equal to the target everywhere: zero loss
    v0, _, _ = O.texture_loss(tgt, Wt, np.repeat(tgt[:, :, None, :], K, axis=2))
    assert abs(v0) < 1e-15
    # K = 1: |I - T| averaged, independent of the weight
    v1, _, _ = O.texture_loss(tgt, Wt[..., :1] + 0.1, T[:, :, :1])
    assert abs(v1 - np.abs(tgt - T[:, :, 0]).mean()) < 1e-14
    v, dW, dT = O.texture_loss(tgt, Wt, T)
    assert np.all(dW[0, 0] == 0) and np.all(dT[0, 0] == 0)
    for idx in [(1, 2, 0), (5, 4, 2), (3, 0, 1)]:
        fd = _fd(lambda z: O.texture_loss(tgt, z, T)[0], Wt, idx)
        assert abs(fd - dW[idx]) < 1e-8
    for idx in [(1, 2, 0, 0), (5, 4, 2, 2), (3, 0, 1, 1)]:
        fd = _fd(lambda z: O.texture_loss(tgt, Wt, z)[0], T, idx)
        assert abs(fd - dT[idx]) < 1e-8


def test_regularisers_value_and_gradient():
    rng = np.random.default_rng(8)
    Wt = rng.uniform(0, 0.3, (4, 5, 2))
    v, g = O.alpha_loss(Wt)
    assert abs(v - np.mean(1 - Wt.sum(axis=2))) < 1e-15
    assert abs(_fd(lambda z: O.alpha_loss(z)[0], Wt, (1, 2, 1)) - g[1, 2, 1]) < 1e-9
    o = rng.uniform(0, 1, 17)
    v, g = O.opacity_loss(o)
    assert abs(v - o.sum() / 17) < 1e-15
    assert abs(_fd(lambda z: O.opacity_loss(z)[0], o, (3,)) - g[3]) < 1e-9
    tab = rng.normal(size=(3, 8, 2))
    s = np.array([8.0, 16.0, 32.0])
    v, g = O.grid_loss(tab, s)
    assert abs(v - sum((tab[l] ** 2).sum() / s[l] ** 3 for l in range(3))) < 1e-15
    for idx in [(0, 1, 0), (2, 7, 1)]:
        assert abs(_fd(lambda z: O.grid_loss(z, s)[0], tab, idx) - g[idx]) < 1e-9


def test_objective_gradient_matches_finite_differences():
    """The total's gradient with respect to image, W and T, by central
    differences of the total."""
    rng = np.random.default_rng(9)
    H, W, K = 13, 12, 2
    img = rng.uniform(0, 1, (H, W, 3))
    tgt = rng.uniform(0, 1, (H, W, 3))
    Wt = rng.uniform(0.05, 0.4, (H, W, K))
    T = rng.uniform(0, 1, (H, W, K, 3))
    o = rng.uniform(0, 1, 5)
    tab = rng.normal(size=(2, 4, 2)) * 0.1
    s = np.array([8.0, 16.0])
    r = O.objective(img, tgt, Wt, T, o, tab, s)
    tot = lambda **kw: O.objective(kw.get("img", img), tgt, kw.get("Wt", Wt), kw.get("T", T),
                                   kw.get("o", o), kw.get("tab", tab), s)["total"]
    for idx in [(0, 0, 0), (6, 5, 1), (12, 11, 2)]:
        assert abs(_fd(lambda z: tot(img=z), img, idx) - r["d_image"][idx]) < 1e-8
    for idx in [(3, 4, 1), (12, 0, 0)]:
        assert abs(_fd(lambda z: tot(Wt=z), Wt, idx) - r["d_weights"][idx]) < 1e-8
    assert abs(_fd(lambda z: tot(T=z), T, (2, 2, 1, 2)) - r["d_textures"][2, 2, 1, 2]) < 1e-8
    assert abs(_fd(lambda z: tot(o=z), o, (4,)) - r["d_opacity"][4]) < 1e-9
    assert abs(_fd(lambda z: tot(tab=z), tab, (1, 3, 1)) - r["d_table"][1, 3, 1]) < 1e-9


def test_adam_first_step_closed_form():
    """Step 1: m_hat = g and v_hat = g^2, so the update is
    -lr g / (|g| + eps)."""
    rng = np.random.default_rng(10)
    p = rng.normal(size=50)
    g = rng.normal(size=50)
    p1, m1, v1 = O.adam_step(p, g, np.zeros(50), np.zeros(50), 0.01, 0.9, 0.999, 1e-15, 1)
    np.testing.assert_allclose(p1 - p, -0.01 * g / (np.abs(g) + 1e-15), rtol=1e-12)
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-12)
    np.testing.assert_allclose(v1, 0.001 * g * g, rtol=1e-12)


def test_adam_converges_on_a_quadratic():
    p = np.array([3.0, -2.0, 0.5])
    m = np.zeros(3)
    v = np.zeros(3)
    for t in range(1, 3001):
        p, m, v = O.adam_step(p, 2 * (p - 1.0), m, v, 0.01, 0.9, 0.999, 1e-8, t)
    np.testing.assert_allclose(p, 1.0, atol=1e-3)
