"""FP64 oracle of the degree-3 spherical-harmonics appearance.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``).

Sec. 3 gives every surfel a view-dependent radiance c (3S values,
channel-wise SH coefficients) and Sec. 5 ("Implementation") sets degree 3,
S = 16, for both appearance modes (per-primitive colour and the field's MLP
output, 48 values).  The paper does not print the basis or how the
coefficients become a colour; the readings are:
  * basis: the real spherical harmonics of degree <= 3, orthonormal on the
    unit sphere, ordered by degree l and then m = -l .. l, with the
    Condon-Shortley phase, as functions of the unit direction (x, y, z);
  * per-primitive colour: evaluated in the direction from the camera centre
    to the surfel centre, c = sum_k Y_k(dir) c_k + 1/2 (the offset makes the
    all-zero coefficients mid-grey), no clamp;
  * textured colour: the MLP's 48 outputs o[3k + ch] are the coefficients,
    evaluated in the pixel's (normalised) ray direction: T_ch = sum_k Y_k(d)
    o[3k + ch], linear, so G(0) = 0 still gives T = 0.
"""
from __future__ import annotations

import numpy as np

SQPI = np.sqrt(np.pi)
K0 = 1.0 / (2.0 * SQPI)                     # l = 0
K1 = np.sqrt(3.0) / (2.0 * SQPI)            # l = 1
K2A = np.sqrt(15.0) / (2.0 * SQPI)          # l = 2, m = -2, -1, 1
K2B = np.sqrt(5.0) / (4.0 * SQPI)           # l = 2, m = 0
K2C = np.sqrt(15.0) / (4.0 * SQPI)          # l = 2, m = 2
K3A = np.sqrt(35.0 / 2.0) / (4.0 * SQPI)    # l = 3, |m| = 3
K3B = np.sqrt(105.0) / (2.0 * SQPI)         # l = 3, m = -2
K3C = np.sqrt(21.0 / 2.0) / (4.0 * SQPI)    # l = 3, |m| = 1
K3D = np.sqrt(7.0) / (4.0 * SQPI)           # l = 3, m = 0
K3E = np.sqrt(105.0) / (4.0 * SQPI)         # l = 3, m = 2


def basis(dirs) -> np.ndarray:
    """[n, 16] real SH of degree <= 3 at unit directions [n, 3]."""
    d = np.asarray(dirs, np.float64).reshape(-1, 3)
    x, y, z = d[:, 0], d[:, 1], d[:, 2]
    xx, yy, zz = x * x, y * y, z * z
    return np.stack([
        np.full_like(x, K0),
        -K1 * y, K1 * z, -K1 * x,
        K2A * x * y, -K2A * y * z, K2B * (2 * zz - xx - yy), -K2A * x * z, K2C * (xx - yy),
        -K3A * y * (3 * xx - yy), K3B * x * y * z, -K3C * y * (4 * zz - xx - yy),
        K3D * z * (2 * zz - 3 * xx - 3 * yy), -K3C * x * (4 * zz - xx - yy),
        K3E * z * (xx - yy), -K3A * x * (xx - 3 * yy)], axis=1)


def basis_grad(dirs) -> np.ndarray:
    """[n, 16, 3]: partial derivatives of the basis polynomials above with
    respect to x, y, z (treated as independent variables)."""
    d = np.asarray(dirs, np.float64).reshape(-1, 3)
    x, y, z = d[:, 0], d[:, 1], d[:, 2]
    xx, yy, zz = x * x, y * y, z * z
    o = np.zeros_like(x)
    g = [
        (o, o, o),
        (o, -K1 + o, o), (o, o, K1 + o), (-K1 + o, o, o),
        (K2A * y, K2A * x, o), (o, -K2A * z, -K2A * y),
        (-2 * K2B * x, -2 * K2B * y, 4 * K2B * z), (-K2A * z, o, -K2A * x),
        (2 * K2C * x, -2 * K2C * y, o),
        (-6 * K3A * x * y, -K3A * (3 * xx - 3 * yy), o),
        (K3B * y * z, K3B * x * z, K3B * x * y),
        (2 * K3C * x * y, -K3C * (4 * zz - xx - 3 * yy), -8 * K3C * y * z),
        (-6 * K3D * x * z, -6 * K3D * y * z, K3D * (6 * zz - 3 * xx - 3 * yy)),
        (-K3C * (4 * zz - 3 * xx - yy), 2 * K3C * x * y, -8 * K3C * x * z),
        (2 * K3E * x * z, -2 * K3E * y * z, K3E * (xx - yy)),
        (-K3A * (3 * xx - 3 * yy), 6 * K3A * x * y, o),
    ]
    return np.stack([np.stack(t, axis=1) for t in g], axis=1)


def camera_center(cam) -> np.ndarray:
    m = np.asarray(cam.world_to_cam, np.float64).reshape(3, 4)
    return -m[:, :3].T @ m[:, 3]


def primitive_colors(mu, coeffs, center) -> np.ndarray:
    """[N, 3] colours of surfels with SH coefficients coeffs [N, 16, 3]."""
    v = np.asarray(mu, np.float64) - np.asarray(center, np.float64)
    dirs = v / np.linalg.norm(v, axis=1, keepdims=True)
    Y = basis(dirs)
    return np.einsum("nk,nkc->nc", Y, np.asarray(coeffs, np.float64).reshape(-1, 16, 3)) + 0.5


def primitive_colors_bwd(mu, coeffs, center, d_rgb):
    """Gradients of the colours with respect to the coefficients [N, 16, 3]
    and the centres [N, 3], given dL/dcolour [N, 3]."""
    v = np.asarray(mu, np.float64) - np.asarray(center, np.float64)
    r = np.linalg.norm(v, axis=1, keepdims=True)
    dirs = v / r
    Y = basis(dirs)
    G = basis_grad(dirs)
    c = np.asarray(coeffs, np.float64).reshape(-1, 16, 3)
    g = np.asarray(d_rgb, np.float64).reshape(-1, 3)
    d_coeffs = Y[:, :, None] * g[:, None, :]
    # dL/ddir (unnormalised derivative), then through dir = v / |v|
    q = np.einsum("nkc,nc,nkj->nj", c, g, G)
    d_mu = (q - dirs * np.sum(dirs * q, axis=1, keepdims=True)) / r
    return d_coeffs, d_mu


def textured_colors(out48, dirs) -> np.ndarray:
    """[n, 3] colours from MLP outputs [n, 48] and unit directions [n, 3]."""
    Y = basis(dirs)
    return np.einsum("nk,nkc->nc", Y, np.asarray(out48, np.float64).reshape(-1, 16, 3))
