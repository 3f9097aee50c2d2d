"""Adaptive density control on the GPU against the FP64 oracle
(oracle/density.py, oracle.blend_error): farthest point sampling (every
choice the FP64 argmax, or within FP32 resolution of it, counted as a
near-tie; squared distances at selection within FP32 rounding; the initial
scales), the blended-error pass on a render, the error-weighted selection
(the same keys in the same order, near-ties counted), the split and the
prune."""
import numpy as np
import pytest

import oracle
from oracle import density as D
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


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _fps_gpu(x, m, dev):
    import torch
    from paper_2512_13796_gb300 import _native as N_
    n = x.shape[0]
    xt = torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(dev)
    scratch = torch.empty(n, device=dev)
    idx = torch.empty(m, dtype=torch.int32, device=dev)
    d2 = torch.empty(m, device=dev)
    sc = torch.empty(m, device=dev)
    N_.nexel_fps(n, xt.data_ptr(), m, scratch.data_ptr(), idx.data_ptr(), d2.data_ptr(),
                 sc.data_ptr(), _stream())
    torch.cuda.synchronize()
    return idx.cpu().numpy(), d2.cpu().numpy(), sc.cpu().numpy()


# FP32 squared distances of FP32 points: each difference, square and sum is
# rounded once (relative error <= 2^-24 each), so a squared distance carries
# <= ~4 x 2^-24 = 2.4e-7 relative error and two candidates whose FP64 values
# lie within 1e-6 of each other may be ordered either way by FP32
FPS_TIE = 1e-6
FPS_D2_REL = 5e-7


@pytest.mark.parametrize("n,m", [(9, 9), (3001, 3001), (20000, 1500)])
def test_fps_against_fp64(dev, n, m):
    if n == 9:
        x = np.zeros((9, 3), np.float32)
        x[:, 0] = np.arange(9)
    else:
        x = np.random.default_rng(n).normal(size=(n, 3)).astype(np.float32)
    gi, gd, gs = _fps_gpu(x, m, dev)
    chk = D.fps_check(x, gi, gd, FPS_TIE)
    print(f"\n[fps n={n} m={m}] {chk}")
    assert chk["d2_rel"] <= FPS_D2_REL
    assert np.isinf(gd[0])
    if n == 9:  # integer lattice: every distance exact, no tie is near
        ri, rd = D.fps(x, m)
        np.testing.assert_array_equal(gi, ri)
        np.testing.assert_array_equal(gd[1:], rd[1:])
        assert chk["ties"] == 0
    else:
        assert chk["ties"] <= max(2, m // 200)
    # the initial scales: the FP64 distance at each selection, the first
    # point the second's (FP32 square root of an FP32 squared distance)
    ref_s = D.fps_scales(chk["d2"])
    np.testing.assert_allclose(gs, ref_s, rtol=5e-7, atol=0)


def test_blend_error_matches_oracle(dev):
    import torch
    from paper_2512_13796_gb300 import _native as N_
    from paper_2512_13796_gb300 import render as R
    w = synth.workload(1)
    cam = synth.front_camera(160, 120)
    st = synth.Settings(K=0)
    p = gpu_params(w.scene, dev)
    ws = R.Workspace(dev)
    cam_s, st_s = R.camera_struct(cam), R.settings_struct(st)
    out = R.forward(ws, cam_s, st_s, None, None, None, *[p[k] for k in SURFEL_KEYS])
    img = out["image"].cpu().numpy().reshape(-1, 3)
    rng = np.random.default_rng(5)
    tgt = rng.uniform(0, 1, img.shape).astype(np.float32)
    ref = oracle.render(w.scene, cam, st, tie_tol=1e-5)
    tie = ref["tie"] != 0
    tgt[tie] = img[tie]  # no error on tie pixels, on both sides
    err = torch.zeros(w.scene.n, device=dev)
    tgt_d = torch.from_numpy(tgt).to(dev)
    N_.nexel_blend_error(cam_s, st_s, w.scene.n, ws.ws.data_ptr(), ws.ws.numel(),
                         out["image"].data_ptr(), tgt_d.data_ptr(), err.data_ptr(), _stream())
    torch.cuda.synchronize()
    e_pix = np.abs(img.astype(np.float64) - tgt).mean(axis=1)
    ref_err = oracle.blend_error(w.scene, cam, st, e_pix)
    g = err.cpu().numpy()
    scale = ref_err.max()
    assert np.max(np.abs(g - ref_err)) <= 2e-5 * scale, np.max(np.abs(g - ref_err)) / scale
    assert np.count_nonzero(ref_err) > 1000


def test_select_split_prune(dev):
    import torch
    from paper_2512_13796_gb300 import _native as N_
    rng = np.random.default_rng(7)
    N = 4000
    err = rng.exponential(size=N).astype(np.float32)
    err[rng.choice(N, 300, replace=False)] = 0.0
    expo = rng.exponential(size=N).astype(np.float32)
    budget = 10 * N
    n_sel = D.split_count(N, budget)
    ws = torch.empty(N_.nexel_density_workspace_size(N + n_sel), dtype=torch.uint8, device=dev)
    sel = torch.empty(n_sel, dtype=torch.int32, device=dev)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    err_d, expo_d = t(err), t(expo)  # held: the call reads them asynchronously
    got = N_.nexel_densify_select(N, err_d.data_ptr(), expo_d.data_ptr(), budget, ws.data_ptr(),
                                  ws.numel(), sel.data_ptr(), _stream())
    torch.cuda.synchronize()
    assert got == n_sel
    # FP32 keys E / err are correctly rounded (relative error <= 2^-24)
    chk = D.select_check(err, expo, n_sel, sel.cpu().numpy(), rel_tol=2.5e-7)
    print(f"\n[select N={N} n={n_sel}] {chk}")
    # no near-tie in this draw: the selection is the FP64 one, index for index
    assert chk["ties"] == 0
    ref_sel = D.select(err, expo, n_sel)
    np.testing.assert_array_equal(sel.cpu().numpy(), ref_sel)
    for color_dim in (3, 48):
        sc = synth.make_scene(N, 3, 11, gamma="var")
        params = dict(mu=sc.mu, quat=sc.quat, scale=sc.scale, opacity=sc.opacity, gamma=sc.gamma,
                      color=(sc.color if color_dim == 3 else synth.sh_coefficients(N, 1).reshape(N, 48)))
        cap = {k: np.concatenate([v, np.zeros((n_sel,) + v.shape[1:], np.float32)])
               for k, v in params.items()}
        g = {k: t(v) for k, v in cap.items()}
        N_.nexel_densify_split(N, n_sel, sel.data_ptr(), color_dim,
                               *[g[k].data_ptr() for k in ("mu", "quat", "scale", "opacity",
                                                           "gamma", "color")], _stream())
        torch.cuda.synchronize()
        ref = D.split(params, ref_sel)
        for k in ("quat", "scale", "opacity", "gamma", "color"):
            np.testing.assert_array_equal(g[k].cpu().numpy(), ref[k].astype(np.float32), err_msg=k)
        np.testing.assert_allclose(g["mu"].cpu().numpy(), ref["mu"], atol=2e-6)
    # prune (on the split set: half-size children keep their parents' opacity)
    opac = g["opacity"].cpu().numpy()
    opac[:50] = 0.004
    opac[50:60] = np.float32(0.005)
    g["opacity"] = t(opac)
    M = N + n_sel
    dst = {k: torch.empty_like(v) for k, v in g.items()}
    n_out = torch.zeros(1, dtype=torch.int32, device=dev)
    keys = ("mu", "quat", "scale", "opacity", "gamma", "color")
    N_.nexel_prune(M, 0.005, 48, [g[k].data_ptr() for k in keys], ws.data_ptr(), ws.numel(),
                   [dst[k].data_ptr() for k in keys], n_out.data_ptr(), _stream())
    torch.cuda.synchronize()
    keep = D.prune_keep(opac)
    assert int(n_out.item()) == keep.size
    for k in keys:
        np.testing.assert_array_equal(dst[k].cpu().numpy()[:keep.size], g[k].cpu().numpy()[keep])
