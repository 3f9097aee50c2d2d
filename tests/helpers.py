"""Shared test utilities: run the CUDA path through the C ABI and compare it
with the FP64 oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2512_13796_gb300 import synth

SURFEL_KEYS = ("mu", "quat", "scale", "opacity", "gamma", "color")


def gpu_params(scene, dev):
    import torch
    return {k: torch.from_numpy(np.ascontiguousarray(getattr(scene, k))).to(dev) for k in SURFEL_KEYS}


def run_gpu(scene, cam, st, field, dev, grid="f32", mlp="f32", d_image=None, d_weights=None,
            d_textures=None, ws=None, recompute=False, cache_features=False):
    """Forward (and backward when d_image is given) through the C ABI.
    Returns (fwd outputs as numpy, grads as numpy or None)."""
    import torch
    from paper_2512_13796_gb300 import render as R
    p = gpu_params(scene, dev)
    fd = R.DeviceField.from_synth(field, dev, grid, mlp) if field is not None else None
    ws = ws or R.Workspace(dev, cap_hint=1 << 16)
    cam_s = R.camera_struct(cam)
    st_s = R.settings_struct(st, grid, mlp, recompute, cache_features)
    ts = fd.storage_table() if fd is not None else None
    w = fd.weights if fd is not None else None
    out = R.forward(ws, cam_s, st_s, fd, ts, w, *[p[k] for k in SURFEL_KEYS])
    g = None
    if d_image is not None:
        t = lambda a: None if a is None else torch.from_numpy(
            np.ascontiguousarray(a, dtype=np.float32)).to(dev)
        g = R.backward(ws, cam_s, st_s, fd, ts, w, *[p[k] for k in SURFEL_KEYS[:5]], out,
                       t(d_image), t(d_weights), t(d_textures))
    torch.cuda.synchronize()
    fw = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in out.items()}
    if g is not None:
        g = {k: v.cpu().numpy() for k, v in g.items()}
    return fw, g, ws


def flat(out, K):
    """Per-pixel flat views of the GPU outputs."""
    P = out["image"].shape[0] * out["image"].shape[1]
    return dict(image=out["image"].reshape(P, 3), notex=out["notex"].reshape(P, 3),
                weights=out["weights"].reshape(P, K), ids=out["ids"].reshape(P, K),
                depths=out["depths"].reshape(P, K), textures=out["textures"].reshape(P, K, 3),
                T_final=out["T_final"].reshape(P))


# Tie bits that can change a forward output discontinuously: the top-K
# choice, the alpha_min skip, the T_min stop, the near-plane cut and the
# depth order.  Near a hash-cell face (32) or a ReLU kink (64) the texture is
# continuous -- only its derivative jumps -- so those pixels stay in the
# forward comparison and are excluded from the gradient comparisons only.
FWD_TIE_MASK = 1 | 2 | 4 | 8 | 16


def compare_forward(gpu, ref, K, tol_color, tol_rel=1e-4, check_textures=True):
    """Element-by-element comparison on the oracle's pixels that are not
    forward tie pixels.  Returns a dict of error statistics."""
    pix = ref["pixels"]
    g = {k: v[pix] for k, v in flat(gpu, K).items()}
    ok = (ref["tie"] & FWD_TIE_MASK) == 0
    stats = dict(n_pix=int(pix.size), n_tie=int((~ok).sum()))
    for bit, name in oracle.TIE_BITS.items():
        stats["tie_" + name] = int(((ref["tie"] & bit) != 0).sum())
    # ids bit-exact
    bad_ids = np.any(g["ids"][ok] != ref["ids"][ok], axis=1)
    stats["id_mismatch"] = int(bad_ids.sum())
    assert stats["id_mismatch"] == 0, f"top-K ids differ on {bad_ids.sum()} non-tie pixels"
    for k in ("image", "notex"):
        e = np.abs(g[k][ok] - ref[k][ok])
        stats[k] = float(e.max()) if e.size else 0.0
        assert stats[k] <= tol_color, (k, stats[k])
    # transmittance and blending weights are products of up to ~100 FP32
    # factors (1 - alpha_i): their rounding error is allowed twice the
    # colour tolerance
    e = np.abs(g["T_final"][ok] - ref["T_final"][ok])
    stats["T_final"] = float(e.max()) if e.size else 0.0
    assert stats["T_final"] <= 2 * tol_color, ("T_final", stats["T_final"])
    e = np.abs(g["weights"][ok] - ref["weights"][ok])
    stats["weights"] = float(e.max()) if e.size else 0.0
    assert stats["weights"] <= 2 * tol_color, ("weights", stats["weights"])
    has = ref["ids"][ok] >= 0
    d_ref = ref["depths"][ok][has]
    e = np.abs(g["depths"][ok][has] - d_ref) / np.maximum(np.abs(d_ref), 1e-12)
    stats["depths_rel"] = float(e.max()) if e.size else 0.0
    assert stats["depths_rel"] <= tol_rel, ("depths", stats["depths_rel"])
    if check_textures:
        e = np.abs(g["textures"][ok] - ref["textures"][ok])
        stats["textures"] = float(e.max()) if e.size else 0.0
        assert stats["textures"] <= tol_color, ("textures", stats["textures"])
    return stats


def rel_err(a, b, floor):
    """max |a - b| / max(|b|, floor) over elements."""
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor))) if a.size else 0.0


def compare_grads(gg, gr, rtol, keys=("mu", "quat", "scale", "opacity", "gamma", "color",
                                      "table", "mlp"), metric="max"):
    """metric "max": every entry within rtol relative, with a floor of 0.1 x
    the largest magnitude of its parameter class (so near-zero entries
    compare in absolute terms against the class's scale).  metric "l2":
    ||g - g_ref|| / ||g_ref|| per class within rtol (the max is reported)."""
    stats, bad = {}, []
    for k in keys:
        if k not in gr or k not in gg:
            continue
        a = np.asarray(gg[k], np.float64).ravel()
        b = np.asarray(gr[k], np.float64).ravel()
        scale = np.max(np.abs(b)) if b.size else 0.0
        if scale == 0.0:
            stats[k] = float(np.max(np.abs(a))) if a.size else 0.0
            if stats[k] != 0.0:
                bad.append((k, stats[k]))
            continue
        r = np.abs(a - b) / np.maximum(np.abs(b), 0.1 * scale)
        err = float(r.max())
        stats[k] = err
        if metric == "l2":
            e2 = float(np.linalg.norm(a - b) / np.linalg.norm(b))
            stats[k + "_l2"] = e2
            if e2 > rtol:
                bad.append((k, e2, err))
        elif err > rtol:
            i = int(r.argmax())
            bad.append((k, err, i, float(a[i]), float(b[i]), float(scale)))
    assert not bad, (bad, stats)
    return stats


def masked_upstream(n_pix, P, K, pixels, ok, seed, with_wt=True):
    """Random upstream gradients on the listed non-tie pixels, zero elsewhere
    (so that both sides differentiate exactly the same set of pixels)."""
    rng = np.random.default_rng(seed)
    dI = np.zeros((P, 3)); dW = np.zeros((P, K)); dT = np.zeros((P, K, 3))
    sel = pixels[ok]
    dI[sel] = rng.normal(size=(sel.size, 3))
    if with_wt:
        dW[sel] = rng.normal(size=(sel.size, K))
        dT[sel] = rng.normal(size=(sel.size, K, 3))
    return dI, dW, dT
