"""The training objective and the Adam step on the GPU against the FP64
oracle (oracle/objective.py), and a short training run with both.

- nexel_loss_image: every term's value and the gradients d_image, d_weights,
  d_textures, on random images with ragged sizes (not multiples of the
  256-thread blocks or of the 11-tap window) and on a real render's W and T.
- nexel_loss_params: the opacity and grid terms and their gradients (added
  to what the render backward wrote).
- nexel_adam_step: 20 tensors of ragged sizes (two launches of 16 + 4).
- Training with the full objective and the GPU Adam lowers the objective."""
import numpy as np
import pytest

from oracle import objective as O
from paper_2512_13796_gb300 import synth

from helpers import SURFEL_KEYS, gpu_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import torch
    assert torch.cuda.is_available(), "GPU test without a CUDA device"
    from paper_2512_13796_gb300 import _native
    _native.build()
    return torch.device("cuda:0")


def _t(a, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)


def _close(got, ref, rel, what):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = max(float(np.abs(ref).max()), 1e-30)
    err = float(np.abs(got - ref).max()) / scale
    assert err <= rel, (what, err)
    return err


@pytest.mark.parametrize("H,W,K", [(37, 53, 3), (64, 48, 0), (120, 161, 4)])
def test_loss_image_matches_oracle(dev, H, W, K):
    import torch
    from paper_2512_13796_gb300 import render as R
    rng = np.random.default_rng(H * W + K)
    img = rng.uniform(0, 1, (H, W, 3))
    tgt = np.clip(img + rng.normal(0, 0.1, (H, W, 3)), 0, 1)
    Wt = rng.uniform(0.0, 0.3, (H, W, max(K, 1)))[..., :K]
    T = rng.uniform(0, 1, (H, W, max(K, 1), 3))[:, :, :K]
    if K:
        Wt[0, :5] = 0.0  # pixels without textured weight
    ob = R.Objective(W, H, dev)
    # the inputs are FP32 on the GPU: the oracle evaluates the same FP32 values
    img, tgt = img.astype(np.float32), tgt.astype(np.float32)
    Wt, T = Wt.astype(np.float32), T.astype(np.float32)
    d_img, d_w, d_t = ob.image_terms(_t(img, dev), _t(tgt, dev), _t(Wt, dev) if K else None,
                                     _t(T, dev) if K else None)
    torch.cuda.synchronize()
    v = ob.read()
    lam = O.LAMBDAS
    assert abs(v["l1"] - O.l1(img, tgt)) <= 1e-5 * O.l1(img, tgt)
    assert abs(v["dssim"] - O.dssim(img, tgt)) <= 1e-5
    ref_img = (1 - lam["dssim"]) * O.l1_grad(img, tgt) + lam["dssim"] * O.dssim_grad(img, tgt)
    # d_image: the L1 part is exact; SSIM statistics in FP32
    _close(d_img.cpu().numpy(), ref_img, 1e-4, "d_image")
    if K:
        tv, tdW, tdT = O.texture_loss(tgt, Wt, T)
        av, adW = O.alpha_loss(Wt)
        assert abs(v["texture"] - tv) <= 1e-5 * max(tv, 1e-6)
        assert abs(v["alpha"] - av) <= 1e-5 * max(av, 1e-6)
        _close(d_w.cpu().numpy(), lam["texture"] * tdW + lam["alpha"] * adW, 1e-5, "d_weights")
        _close(d_t.cpu().numpy(), lam["texture"] * tdT, 1e-5, "d_textures")
        img_terms = ((1 - lam["dssim"]) * O.l1(img, tgt) + lam["dssim"] * O.dssim(img, tgt) +
                     lam["texture"] * tv + lam["alpha"] * av)
        assert abs(v["image_terms"] - img_terms) <= 1e-5 * img_terms


def test_loss_on_a_render_and_params_match_oracle(dev):
    """W and T of a real render (config 1 view at 200 x 150, K = 4), the
    parameter terms on config 1's field, and the total."""
    import torch
    from paper_2512_13796_gb300 import render as R
    w = synth.workload(1)
    cam = synth.front_camera(200, 150)
    st = w.settings
    p = gpu_params(w.scene, dev)
    fd = R.DeviceField.from_synth(w.field, dev, "f32", "f32")
    ws = R.Workspace(dev)
    out = R.forward(ws, R.camera_struct(cam), R.settings_struct(st), fd, fd.storage_table(),
                    fd.weights, *[p[k] for k in SURFEL_KEYS])
    rng = np.random.default_rng(3)
    tgt = rng.uniform(0, 1, (cam.height, cam.width, 3)).astype(np.float32)
    ob = R.Objective(cam.width, cam.height, dev)
    d_img, d_w, d_t = ob.image_terms(out["image"], _t(tgt, dev), out["weights"], out["textures"])
    # stand-ins for what the render backward wrote (small, so that taking
    # them off again is exact enough), then the regularisers add
    g_op0 = (rng.normal(size=w.scene.n) * 1e-8).astype(np.float32)
    g_tab0 = (rng.normal(size=fd.table.shape) * 1e-12).astype(np.float32)
    g_op, g_tab = _t(g_op0, dev), _t(g_tab0, dev)
    ob.param_terms(p["opacity"], fd, g_op, g_tab)
    torch.cuda.synchronize()
    v = ob.read()
    img = out["image"].cpu().numpy()
    Wt, T = out["weights"].cpu().numpy(), out["textures"].cpu().numpy()
    ref = O.objective(img, tgt, Wt, T, w.scene.opacity.astype(np.float32),
                      fd.table.cpu().numpy(), np.asarray(w.field.level_scale, np.float32))
    for k in ("l1", "dssim", "texture", "alpha", "opacity", "grid", "total"):
        assert abs(v[k] - ref[k]) <= 2e-5 * max(abs(ref[k]), 1e-6), (k, v[k], ref[k])
    _close(d_img.cpu().numpy(), ref["d_image"], 1e-4, "d_image")
    _close(d_w.cpu().numpy(), ref["d_weights"], 1e-5, "d_weights")
    _close(d_t.cpu().numpy(), ref["d_textures"], 1e-5, "d_textures")
    _close(g_op.cpu().numpy() - g_op0, ref["d_opacity"], 1e-5, "d_opacity")
    _close(g_tab.cpu().numpy() - g_tab0, ref["d_table"], 1e-4, "d_table")


def test_loss_image_full_size(dev):
    """The headline image size (1280 x 720, K = 4): every term's value, and
    d_image, d_weights, d_textures on every element, against the oracle."""
    import torch
    from paper_2512_13796_gb300 import render as R
    H, W, K = 720, 1280, 4
    rng = np.random.default_rng(41)
    img = rng.uniform(0, 1, (H, W, 3)).astype(np.float32)
    tgt = np.clip(img + rng.normal(0, 0.05, (H, W, 3)), 0, 1).astype(np.float32)
    Wt = rng.uniform(0.0, 0.25, (H, W, K)).astype(np.float32)
    T = rng.uniform(0, 1, (H, W, K, 3)).astype(np.float32)
    ob = R.Objective(W, H, dev)
    d_img, d_w, d_t = ob.image_terms(_t(img, dev), _t(tgt, dev), _t(Wt, dev), _t(T, dev))
    torch.cuda.synchronize()
    v = ob.read()
    lam = O.LAMBDAS
    assert abs(v["l1"] - O.l1(img, tgt)) <= 1e-5 * O.l1(img, tgt)
    assert abs(v["dssim"] - O.dssim(img, tgt)) <= 1e-5
    tv, tdW, tdT = O.texture_loss(tgt, Wt, T)
    av, adW = O.alpha_loss(Wt)
    assert abs(v["texture"] - tv) <= 1e-5 * tv and abs(v["alpha"] - av) <= 1e-5 * av
    ref_img = (1 - lam["dssim"]) * O.l1_grad(img, tgt) + lam["dssim"] * O.dssim_grad(img, tgt)
    _close(d_img.cpu().numpy(), ref_img, 1e-4, "d_image")
    # |.| decides the sign of the texture residual: a pixel whose residual
    # lies within FP32 rounding of zero may take the other sign (a tie);
    # the comparison skips those pixels (a handful of the 921,600)
    sw = Wt.astype(np.float64).sum(axis=2, keepdims=True)
    tb = (Wt[..., None].astype(np.float64) * T).sum(axis=2) / sw
    ok = np.all(np.abs(tb - tgt) > 1e-6, axis=2)
    assert ok.mean() > 0.999
    _close(d_w.cpu().numpy()[ok], (lam["texture"] * tdW + lam["alpha"] * adW)[ok], 1e-5,
           "d_weights")
    _close(d_t.cpu().numpy()[ok], (lam["texture"] * tdT)[ok], 1e-5, "d_textures")


def test_adam_matches_oracle(dev):
    import torch
    from paper_2512_13796_gb300 import render as R
    rng = np.random.default_rng(11)
    sizes = [1, 3, 4, 5, 255, 256, 257, 1023, 4096, 70001] + [7 + 13 * i for i in range(10)]
    ps = [rng.normal(size=n).astype(np.float32) for n in sizes]
    lrs = [10.0 ** -rng.uniform(1, 4) for _ in sizes]
    tp = [_t(x, dev) for x in ps]
    opt = R.Adam(tp, lrs, eps=1e-8)
    ref = [(x.astype(np.float64), np.zeros(x.size), np.zeros(x.size)) for x in ps]
    for step in range(1, 4):
        gs = [rng.normal(size=n).astype(np.float32) for n in sizes]
        opt.step([_t(g, dev) for g in gs])
        ref = [O.adam_step(p, g, m, v, lr, 0.9, 0.999, 1e-8, step)
               for (p, m, v), g, lr in zip(ref, gs, lrs)]
    torch.cuda.synchronize()
    for (p, _, _), t, p0 in zip(ref, tp, ps):
        got = t.cpu().numpy().astype(np.float64)
        # the parameter is stored in FP32 after every step: allow a few units
        # in its last place, plus a relative error of the update itself
        tol = 4 * np.spacing(np.abs(p0).astype(np.float32)).astype(np.float64) + \
            1e-5 * np.abs(p - p0).max()
        assert np.all(np.abs(got - p) <= tol), ("adam", float(np.max(np.abs(got - p) - tol)))


def test_training_with_full_objective_lowers_it(dev):
    """Geometry fixed, colour, table and MLP trained on 6 views of a small
    scene with the GPU objective and the GPU Adam: the objective falls."""
    import torch
    from paper_2512_13796_gb300 import render as R
    import oracle
    sc = synth.make_scene(2000, 4, 21, gamma="var")
    cams = synth.sphere_cameras(np.random.default_rng(2), [(80, 64)] * 6)
    st = synth.Settings(K=2)
    targets = [oracle.render_procedural(sc, c, synth.Settings(K=0), 30.0)
               .reshape(c.height, c.width, 3) for c in cams]
    p = gpu_params(sc, dev)
    p["color"] = p["color"].clone().fill_(0.5)
    fd = R.DeviceField.from_synth(synth.make_field(8, 14, 2, (64,), 3), dev, "f32", "f32")
    ws = R.Workspace(dev)
    ob = R.Objective(80, 64, dev)
    opt = R.Adam([p["color"], fd.table, fd.weights], [2e-2, 2e-2, 2e-3])
    tg = [_t(t, dev) for t in targets]
    first, last = [], []
    for it in range(240):
        v = it % len(cams)
        cam_s = R.camera_struct(cams[v])
        st_s = R.settings_struct(st, cache_features=True)
        ts = fd.storage_table()
        out = R.forward(ws, cam_s, st_s, fd, ts, fd.weights, *[p[k] for k in SURFEL_KEYS])
        d_img, d_w, d_t = ob.image_terms(out["image"], tg[v], out["weights"], out["textures"])
        g = R.backward(ws, cam_s, st_s, fd, ts, fd.weights, *[p[k] for k in SURFEL_KEYS[:5]],
                       out, d_img, d_w, d_t)
        ob.param_terms(p["opacity"], fd, g["opacity"], g["table"])
        opt.step([g["color"], g["table"], g["mlp"]])
        if it < 6:
            first.append(ob.read()["total"])
        elif it >= 234:
            last.append(ob.read()["total"])
    print(f"\n[objective] first views {np.mean(first):.4f} -> last {np.mean(last):.4f}")
    assert np.mean(last) < 0.8 * np.mean(first)
