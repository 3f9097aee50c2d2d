"""FP64 oracle of the training objective and the optimiser step.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): used by the tests
and the benchmark's CPU leg, never by the product package.

Definitions and the passages they follow (Sec. 5, "Losses"):
  l1              L_1 of the photometric term: mean over H x W x 3 of |I - I_GT|
  dssim           L_D-SSIM = 1 - SSIM, SSIM averaged over pixels and channels.
                  The paper takes it from 3DGS, which uses the SSIM of Wang
                  et al. (2004) with an 11 x 11 Gaussian window (sigma 1.5),
                  zero padding at the border (same-size maps), C1 = 0.01^2,
                  C2 = 0.03^2 for images in [0, 1].
  image_loss      L_image = (1 - lambda_D-SSIM) L_1 + lambda_D-SSIM L_D-SSIM
  texture_loss    L_texture: mean over pixels and channels of
                  |I_GT - sum_j W_j T_j / sum_j W_j|; a pixel with
                  sum_j W_j = 0 has no textured colour and adds nothing
                  (the paper does not say; reading)
  alpha_loss      L_alpha = mean over pixels of (1 - sum_j W_j)
  opacity_loss    L_opacity = mean of the opacities
  grid_loss       L_grid = sum_l s_l^-3 sum_{i,j} H_{l,i,j}^2: the printed
                  formula indexes s by the entry and does not square H; the
                  reading takes the level scale s_l and the square (a sum of
                  un-squared entries has no minimum, and the stated purpose is
                  zero-mean grid values)
  objective       L = L_image + lambda_alpha L_alpha + lambda_texture L_texture
                  + lambda_opacity L_opacity + lambda_grid L_grid with the
                  paper's lambdas (0.005, 0.5, 0.01, 0.01; lambda_D-SSIM 0.2)
  adam_step       Adam (Kingma and Ba, 2015), the optimiser of 3DGS, which the
                  paper follows ("we follow the scheme of 3DGS"): bias-corrected
                  first and second moments, p -= lr m_hat / (sqrt(v_hat) + eps)
Gradients are the analytic derivatives of these definitions; |.| has
derivative sign(.) with sign(0) = 0.
"""
from __future__ import annotations

import numpy as np

LAMBDAS = dict(dssim=0.2, alpha=0.005, texture=0.5, opacity=0.01, grid=0.01)
SSIM_C1 = 0.01 ** 2
SSIM_C2 = 0.03 ** 2
SSIM_WIN = 11
SSIM_SIGMA = 1.5


def gaussian_window(size: int = SSIM_WIN, sigma: float = SSIM_SIGMA) -> np.ndarray:
    """Separable Gaussian window (outer product of the normalised 1-D taps)."""
    r = np.arange(size, dtype=np.float64) - size // 2
    g = np.exp(-r * r / (2.0 * sigma * sigma))
    g /= g.sum()
    return np.outer(g, g)


def correlate_same(img: np.ndarray, win: np.ndarray) -> np.ndarray:
    """out[p] = sum_q win[q] img[p + q - c] with zeros outside the image
    (2-D, explicit shifted sums)."""
    H, W = img.shape
    k = win.shape[0]
    c = k // 2
    pad = np.zeros((H + 2 * c, W + 2 * c))
    pad[c:c + H, c:c + W] = img
    out = np.zeros((H, W))
    for dy in range(k):
        for dx in range(k):
            out += win[dy, dx] * pad[dy:dy + H, dx:dx + W]
    return out


def _stats(x, y, win):
    mx = correlate_same(x, win)
    my = correlate_same(y, win)
    exx = correlate_same(x * x, win)
    eyy = correlate_same(y * y, win)
    exy = correlate_same(x * y, win)
    return mx, my, exx - mx * mx, eyy - my * my, exy - mx * my


def ssim_map(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Per-pixel, per-channel SSIM of [H, W, 3] images."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    win = gaussian_window()
    out = np.zeros_like(x)
    for ch in range(x.shape[2]):
        mx, my, vx, vy, cxy = _stats(x[..., ch], y[..., ch], win)
        out[..., ch] = ((2 * mx * my + SSIM_C1) * (2 * cxy + SSIM_C2)) / \
                       ((mx * mx + my * my + SSIM_C1) * (vx + vy + SSIM_C2))
    return out


def dssim(x, y) -> float:
    return 1.0 - float(ssim_map(x, y).mean())


def dssim_grad(x, y) -> np.ndarray:
    """d(1 - mean SSIM)/dx.  With l1 = 2 mx my + C1, l2 = mx^2 + my^2 + C1,
    c1 = 2 cov + C2, c2 = vx + vy + C2 and S = l1 c1 / (l2 c2) at every
    pixel p, S depends on x through mx = sum w x, E[x^2] = sum w x^2 and
    E[xy] = sum w x y:
      dS/dmx     = S (2 my / l1 - 2 my / c1 - 2 mx / l2 + 2 mx / c2)
      dS/dE[x^2] = -S / c2
      dS/dE[xy]  = 2 S / c1
    and dS(p)/dx_q = w(p - q) (dS/dmx + 2 x_q dS/dE[x^2] + y_q dS/dE[xy]);
    the window is symmetric, so the sum over p is the same correlation."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    win = gaussian_window()
    M = x.size
    g = np.zeros_like(x)
    for ch in range(x.shape[2]):
        xc, yc = x[..., ch], y[..., ch]
        mx, my, vx, vy, cxy = _stats(xc, yc, win)
        l1 = 2 * mx * my + SSIM_C1
        l2 = mx * mx + my * my + SSIM_C1
        c1 = 2 * cxy + SSIM_C2
        c2 = vx + vy + SSIM_C2
        S = l1 * c1 / (l2 * c2)
        A = S * (2 * my / l1 - 2 * my / c1 - 2 * mx / l2 + 2 * mx / c2)
        B = -S / c2
        C = 2 * S / c1
        dS = correlate_same(A, win) + 2 * xc * correlate_same(B, win) + yc * correlate_same(C, win)
        g[..., ch] = -dS / M
    return g


def l1(x, y) -> float:
    return float(np.abs(np.asarray(x, np.float64) - y).mean())


def l1_grad(x, y) -> np.ndarray:
    x = np.asarray(x, np.float64)
    return np.sign(x - y) / x.size


def texture_loss(target, W, T):
    """L_texture and its gradients with respect to W [H, W, K] and
    T [H, W, K, 3]."""
    target = np.asarray(target, np.float64)
    W = np.asarray(W, np.float64)
    T = np.asarray(T, np.float64)
    H, Wd, _ = target.shape
    sw = W.sum(axis=2)
    has = sw > 0
    sws = np.where(has, sw, 1.0)
    tbar = (W[..., None] * T).sum(axis=2) / sws[..., None]
    r = np.where(has[..., None], tbar - target, 0.0)
    n = 3.0 * H * Wd
    val = float(np.abs(r).sum() / n)
    s = np.sign(r) / n                                           # dL/dtbar
    dW = ((T - tbar[:, :, None, :]) * s[:, :, None, :]).sum(axis=3) / sws[..., None]
    dT = s[:, :, None, :] * W[..., None] / sws[..., None, None]
    dW = np.where(has[..., None], dW, 0.0)
    dT = np.where(has[..., None, None], dT, 0.0)
    return val, dW, dT


def alpha_loss(W):
    W = np.asarray(W, np.float64)
    H, Wd, K = W.shape
    return float((1.0 - W.sum(axis=2)).mean()), np.full(W.shape, -1.0 / (H * Wd))


def opacity_loss(o):
    o = np.asarray(o, np.float64)
    return float(o.mean()), np.full(o.shape, 1.0 / o.size)


def grid_loss(table, level_scale):
    """table [L, T, F]; level_scale [L]."""
    t = np.asarray(table, np.float64)
    s3 = np.asarray(level_scale, np.float64)[:t.shape[0], None, None] ** -3.0
    return float((s3 * t * t).sum()), 2.0 * s3 * t


def objective(image, target, W, T, opacity, table, level_scale, lam=LAMBDAS) -> dict:
    """Every term of the training objective, the total and the gradients
    with respect to the image, W, T, the opacities and the table."""
    v_l1, g_l1 = l1(image, target), l1_grad(image, target)
    v_ds, g_ds = dssim(image, target), dssim_grad(image, target)
    v_tx, dW_tx, dT_tx = texture_loss(target, W, T)
    v_al, dW_al = alpha_loss(W)
    v_op, g_op = opacity_loss(opacity)
    v_gr, g_gr = grid_loss(table, level_scale)
    ld = lam["dssim"]
    image_loss = (1 - ld) * v_l1 + ld * v_ds
    total = (image_loss + lam["alpha"] * v_al + lam["texture"] * v_tx +
             lam["opacity"] * v_op + lam["grid"] * v_gr)
    return dict(total=total, image=image_loss, l1=v_l1, dssim=v_ds, texture=v_tx, alpha=v_al,
                opacity=v_op, grid=v_gr,
                d_image=(1 - ld) * g_l1 + ld * g_ds,
                d_weights=lam["texture"] * dW_tx + lam["alpha"] * dW_al,
                d_textures=lam["texture"] * dT_tx,
                d_opacity=lam["opacity"] * g_op,
                d_table=lam["grid"] * g_gr)


def adam_step(p, g, m, v, lr, beta1, beta2, eps, step):
    """One Adam step (step counts from 1); returns new (p, m, v)."""
    p = np.asarray(p, np.float64)
    g = np.asarray(g, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
