"""Pins of the spherical-harmonics oracle (oracle/sh.py) against the
mathematics of the real spherical harmonics: orthonormality on the sphere
(exact quadrature), the addition theorem (which fixes every degree's
normalisation and functional form), derivatives by finite differences, and
the colour rules' special cases."""
import numpy as np

from oracle import sh


def _unit(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def test_orthonormal_on_the_sphere():
    # Gauss-Legendre in cos(theta) x uniform phi: exact for the degree <= 6
    # products of two basis functions
    ct, wt = np.polynomial.legendre.leggauss(12)
    nphi = 24
    phi = 2 * np.pi * np.arange(nphi) / nphi
    st = np.sqrt(1 - ct * ct)
    dirs = np.stack([np.outer(st, np.cos(phi)).ravel(), np.outer(st, np.sin(phi)).ravel(),
                     np.repeat(ct, nphi)], axis=1)
    w = np.repeat(wt, nphi) * (2 * np.pi / nphi)
    Y = sh.basis(dirs)
    gram = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-12)


def test_addition_theorem():
    """sum_m Y_lm(a) Y_lm(b) = (2l + 1) / (4 pi) P_l(a . b) per degree."""
    rng = np.random.default_rng(0)
    a, b = _unit(rng, 200), _unit(rng, 200)
    Ya, Yb = sh.basis(a), sh.basis(b)
    t = np.sum(a * b, axis=1)
    P = [np.ones_like(t), t, 0.5 * (3 * t * t - 1), 0.5 * (5 * t ** 3 - 3 * t)]
    for l in range(4):
        sl = slice(l * l, (l + 1) * (l + 1))
        lhs = np.sum(Ya[:, sl] * Yb[:, sl], axis=1)
        np.testing.assert_allclose(lhs, (2 * l + 1) / (4 * np.pi) * P[l], atol=1e-13)


def test_degree_one_is_linear_in_the_direction():
    rng = np.random.default_rng(1)
    d = _unit(rng, 10)
    Y = sh.basis(d)
    k1 = np.sqrt(3 / (4 * np.pi))
    np.testing.assert_allclose(np.abs(Y[:, 1:4]), k1 * np.abs(d[:, [1, 2, 0]]), atol=1e-14)
    np.testing.assert_allclose(Y[:, 0], 1 / np.sqrt(4 * np.pi))


def test_basis_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    d = rng.normal(size=(7, 3))  # the polynomials, off the sphere too
    G = sh.basis_grad(d)
    h = 1e-6
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        fd = (sh.basis(d + e) - sh.basis(d - e)) / (2 * h)
        np.testing.assert_allclose(G[:, :, j], fd, atol=1e-8)


def test_colour_rules_special_cases():
    rng = np.random.default_rng(3)
    mu = rng.normal(size=(5, 3))
    center = np.array([0.0, 0.0, -3.0])
    np.testing.assert_allclose(sh.primitive_colors(mu, np.zeros((5, 16, 3)), center), 0.5)
    c = np.zeros((5, 16, 3))
    c[:, 0, :] = rng.normal(size=(5, 3))
    np.testing.assert_allclose(sh.primitive_colors(mu, c, center),
                               0.5 + c[:, 0, :] / np.sqrt(4 * np.pi), atol=1e-14)
    out = np.zeros((4, 48))
    np.testing.assert_allclose(sh.textured_colors(out, _unit(rng, 4)), 0.0)


def test_colour_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    mu = rng.normal(size=(6, 3))
    c = rng.normal(size=(6, 16, 3))
    center = np.array([0.2, -0.1, -3.0])
    g = rng.normal(size=(6, 3))
    dc, dmu = sh.primitive_colors_bwd(mu, c, center, g)
    f = lambda m, cc: float(np.sum(sh.primitive_colors(m, cc, center) * g))
    h = 1e-6
    for (i, k, ch) in [(0, 0, 0), (3, 9, 2), (5, 15, 1)]:
        e = np.zeros_like(c)
        e[i, k, ch] = h
        assert abs((f(mu, c + e) - f(mu, c - e)) / (2 * h) - dc[i, k, ch]) < 1e-8
    for (i, j) in [(0, 0), (2, 1), (5, 2)]:
        e = np.zeros_like(mu)
        e[i, j] = h
        assert abs((f(mu + e, c) - f(mu - e, c)) / (2 * h) - dmu[i, j]) < 1e-7


def _field48_from_field3(f3):
    """A 48-output field whose SH texture equals the RGB texture of f3: the
    constant SH band carries W3 / Y_0, every other band is zero."""
    import copy
    f = copy.deepcopy(f3)
    W3 = f3.weights[-1]
    W48 = np.zeros((48, W3.shape[1]), np.float64)
    for ch in range(3):
        W48[ch] = W3[ch] / sh.K0
    f.weights = list(f3.weights[:-1]) + [W48]
    f.widths = tuple(f3.widths[:-1]) + (48,)
    return f


def test_sh_texture_with_only_the_constant_band_equals_rgb():
    import oracle
    from paper_2512_13796_gb300 import synth
    w = synth.workload(0)
    cam, st = w.cameras[0], w.settings
    f48 = _field48_from_field3(w.field)
    a = oracle.render(w.scene, cam, st, w.field)
    b = oracle.render(w.scene, cam, st, f48)
    np.testing.assert_allclose(b["textures"], a["textures"], atol=1e-12)
    np.testing.assert_allclose(b["image"], a["image"], atol=1e-12)


def test_sh_texture_gradient_matches_finite_differences():
    """Central differences of <dI, image> against the oracle's backward for
    weights of several SH bands of a 48-output field."""
    import oracle
    from paper_2512_13796_gb300 import synth
    w = synth.workload(0)
    cam, st = w.cameras[0], w.settings
    rng = np.random.default_rng(12)
    f48 = _field48_from_field3(w.field)
    f48.weights[-1] = f48.weights[-1] + rng.normal(0, 0.3, f48.weights[-1].shape)
    pix = np.arange(0, cam.width * cam.height, 7, dtype=np.int32)
    ref = oracle.render(w.scene, cam, st, f48, pix, tie_tol=1e-5, cell_tol=1e-5, relu_tol=1e-4)
    pix = pix[ref["tie"] == 0]
    dI = rng.normal(size=(pix.size, 3))
    g = oracle.render_bwd(w.scene, cam, st, f48, pix, dI)
    f = lambda fld: float(np.sum(oracle.render(w.scene, cam, st, fld, pix)["image"] * dI))
    h = 1e-6
    n_last = f48.weights[-1].size
    offs = sum(x.size for x in f48.weights[:-1])
    import copy
    for (o, i) in [(3 * 5 + 1, 2), (3 * 12 + 2, 7), (0, 0)]:
        fp, fm = copy.deepcopy(f48), copy.deepcopy(f48)
        fp.weights[-1][o, i] += h
        fm.weights[-1][o, i] -= h
        fd = (f(fp) - f(fm)) / (2 * h)
        an = g["mlp"][offs + o * f48.weights[-1].shape[1] + i]
        assert abs(fd - an) <= 1e-6 + 1e-4 * abs(fd), (o, i, fd, an)
    assert n_last == 48 * f48.weights[-1].shape[1]
