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
