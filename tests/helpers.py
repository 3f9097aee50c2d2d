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
# choice, the alpha_min skip, the T_min stop, the near-plane cut, the depth
# order and the edge-on cull.  Near a hash-cell face (32) or a ReLU kink (64)
# the texture is continuous -- only its derivative jumps -- so those pixels
# stay in every comparison; the gradient comparisons cancel the texture
# gradient of the affected samples instead (kink_cancelled_upstream).
FWD_TIE_MASK = 1 | 2 | 4 | 8 | 16 | 128
KINK_BITS = 32 | 64

# Discrete-choice tolerances of the oracle's tie flags, from the FP32 path's
# arithmetic: alpha, t* and the transmittance carry ~1e-6 relative error
# (tie_tol 5e-6); the sort key is the FP32 rounding of the centre depth, so
# two depths closer than one FP32 unit in the last place (2^-23 relative)
# may share a key and fall back to the index order (order_tol 1.5e-7);
# FP32 intersection points differ from FP64 by < 1e-6 world units
# (cell_tol 2e-6); FP32 features differ from FP64 by ~5e-7, which moves a
# hidden pre-activation by ~1e-5 of the sum of its terms' magnitudes
# (relu_tol 1e-4).  Reduced-precision MLPs round every operand: the ReLU
# band is 6e-3 for BF16 (unit roundoff 2^-8) and 1e-3 for FP16 (2^-11),
# 1.5x the largest pre-activation error of an exact emulation of the
# rounding over 0.7M hidden units of the 300k-surfel 720p view.
TIE_TOL = 5e-6
ORDER_TOL = 1.5e-7
CELL_TOL = 2e-6
RELU_TOL = {"f32": 1e-4, "bf16": 6e-3, "f16": 1e-3}


def rounded_field(field, mlp):
    """The table and weights a form actually reads: the FP16 table and, for
    the tensor-core forms, the MLP weights rounded to the operand type
    (the oracle is evaluated at those parameter values)."""
    if mlp == "f32":
        return None, None
    import torch
    tab = np.asarray(field.table, np.float32).astype(np.float16).astype(np.float64)
    dt = torch.bfloat16 if mlp == "bf16" else torch.float16
    wts = [torch.from_numpy(np.asarray(w, np.float32)).to(dt).to(torch.float64).numpy()
           for w in field.weights]
    return tab, wts


def reference(scene, cam, st, field, pixels=None, mlp="f32", coeffs=None, **kw):
    """Oracle forward with the tie flags for the given form (at the
    parameters it reads); with ``coeffs`` the per-primitive colours are
    degree-3 SH."""
    tab, wts = rounded_field(field, mlp) if field is not None else (None, None)
    kw = dict(tie_tol=TIE_TOL, order_tol=ORDER_TOL, cell_tol=CELL_TOL, relu_tol=RELU_TOL[mlp],
              table=tab, weights=wts, **kw)
    if coeffs is not None:
        return oracle.render_sh(scene, coeffs, cam, st, field, pixels, **kw)
    return oracle.render(scene, cam, st, field, pixels, **kw)


UNIT_ROUNDOFF = {"f32": 0.0, "bf16": 2.0 ** -8, "f16": 2.0 ** -11}


def reference_grads(scene, cam, st, field, sel, dI, dW, dT, mlp="f32", coeffs=None):
    """The oracle's gradient for upstream (dI, dW, dT) on the pixels ``sel``
    (full-image arrays), at the parameters the form reads, and, for a
    reduced-precision form, the magnitudes of the contributions to the table
    and MLP entries (the scale of their rounding error)."""
    tab, wts = rounded_field(field, mlp) if field is not None else (None, None)
    up = (sel, dI[sel], None if dW is None else dW[sel], None if dT is None else dT[sel])
    if coeffs is not None:
        fn = lambda **kw: oracle.render_bwd_sh(scene, coeffs, cam, st, field, *up, **kw)
    else:
        fn = lambda **kw: oracle.render_bwd(scene, cam, st, field, *up, **kw)
    gr = fn(table=tab, weights=wts)
    ga = None
    if mlp != "f32":
        ga = fn(table=tab, weights=wts, absolute=True)
        ga.pop("mlp_layers", None)
        if coeffs is not None:  # the colour entries are the SH coefficients' here
            ga.pop("color", None)
    return gr, ga


def ill_conditioned(scene, cam, cos_min=0.02):
    """Surfels seen nearly edge-on (|cos| of the normal to the centre ray
    below cos_min): every pixel ray meets such a plane at a grazing angle,
    where t*, u and v are ratios of nearly cancelling terms, so the
    derivatives with respect to the centre and the rotation amplify the
    FP32 path's rounding by ~1 / |cos| (measured ~1e-5 / |cos| relative).
    Their mu and quat gradients are left out of the per-element comparison
    (counted); everything else about them is compared."""
    return np.nonzero(oracle.centre_ray_cosine(cam, scene) < cos_min)[0]


def kink_cancelled_upstream(ref, P, K, seed, with_wt=True):
    """Random upstream gradients on the oracle's pixels that are not forward
    tie pixels (zero elsewhere), arranged so that no sample at a kink of the
    texture (a hash-cell face, or a ReLU decision the other precision may
    take the other way: ``tie_slot``) gets a texture gradient: such a
    sample's d_textures is 0, and its pixel gets no d_image (which would
    reach every slot as W_j dC).  Those pixels still carry d_weights and the
    other slots' d_textures.  Every other pixel gets d_image, d_weights and
    d_textures.  Returns (dI, dW, dT, sel, stats)."""
    rng = np.random.default_rng(seed)
    pixels = ref["pixels"]
    ok = (ref["tie"] & FWD_TIE_MASK) == 0
    sel = pixels[ok]
    kink = (ref["tie_slot"][ok] & KINK_BITS) != 0  # [n_sel, K]
    kpix = kink.any(axis=1)
    dI = np.zeros((P, 3), np.float32)
    dW = np.zeros((P, K), np.float32)
    dT = np.zeros((P, K, 3), np.float32)
    dI[sel[~kpix]] = rng.normal(size=(int((~kpix).sum()), 3))
    if with_wt or kpix.any():
        dW[sel] = rng.normal(size=(sel.size, K))
    if with_wt:
        t = rng.normal(size=(sel.size, K, 3))
        t[kink] = 0.0
        dT[sel] = t
    has = ref["ids"][ok] >= 0
    stats = dict(pix=int(pixels.size), pix_compared=int(sel.size),
                 pix_with_d_image=int((~kpix).sum()), samples=int(has.sum()),
                 samples_kink=int(kink.sum()))
    return dI, dW, dT, sel, stats


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


def grad_stats(gg, gr, keys=("mu", "quat", "scale", "opacity", "gamma", "color", "table",
                               "mlp")):
    """Per class: the largest |g - g_ref| / max(|g_ref|, 0.1 x the class's
    largest |g_ref|) and the relative L2 error."""
    out = {}
    for k in keys:
        if k not in gr or k not in gg:
            continue
        a = np.asarray(gg[k], np.float64).ravel()
        b = np.asarray(gr[k], np.float64).ravel()
        scale = np.max(np.abs(b)) if b.size else 0.0
        if scale == 0.0:
            continue
        out[k] = float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 0.1 * scale)))
        out[k + "_l2"] = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    return out


def rel_err(a, b, floor):
    """max |a - b| / max(|b|, floor) over elements."""
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor))) if a.size else 0.0


def compare_grads(gg, gr, rtol, keys=("mu", "quat", "scale", "opacity", "gamma", "color",
                                      "table", "mlp"), metric="max", absolute=None, u=0.0,
                  c=4.0, skip_surfels=None):
    """metric "max": every entry within rtol relative, with a floor of 0.1 x
    the largest magnitude of its parameter class (so near-zero entries
    compare in absolute terms against the class's scale), plus, when the
    oracle's ``absolute`` gradients (the sum of the magnitudes of every
    contribution to an entry) are given, c u |contributions| for a form
    whose operands are rounded with unit roundoff u.  ``skip_surfels``:
    surfels whose mu and quat gradients are left out (ill-conditioned, see
    oracle.centre_ray_cosine).  metric "l2": ||g - g_ref|| / ||g_ref|| per
    class within rtol (the max is reported)."""
    stats, bad = {}, []
    for k in keys:
        if k not in gr or k not in gg:
            continue
        a = np.asarray(gg[k], np.float64)
        b = np.asarray(gr[k], np.float64)
        keep = None
        if skip_surfels is not None and len(skip_surfels) and k in ("mu", "quat"):
            keep = np.ones(b.shape[0], bool)
            keep[np.asarray(skip_surfels)] = False
            a, b = a[keep], b[keep]
        a, b = a.ravel(), b.ravel()
        scale = np.max(np.abs(b)) if b.size else 0.0
        if scale == 0.0:
            stats[k] = float(np.max(np.abs(a))) if a.size else 0.0
            if stats[k] != 0.0:
                bad.append((k, stats[k]))
            continue
        bound = rtol * np.maximum(np.abs(b), 0.1 * scale)
        if absolute is not None and k in absolute:
            A = np.asarray(absolute[k], np.float64)
            if keep is not None:
                A = A[keep]
            bound = bound + c * u * A.ravel()
        r = np.abs(a - b) / bound
        err = float(r.max())
        # the largest relative error (floor 0.1 x the class scale), and the
        # largest fraction of its bound an entry uses
        stats[k] = float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 0.1 * scale)))
        stats[k + "_of_bound"] = err
        if metric == "l2":
            e2 = float(np.linalg.norm(a - b) / np.linalg.norm(b))
            stats[k + "_l2"] = e2
            if e2 > rtol:
                bad.append((k, e2, err))
        elif err > 1.0:
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
