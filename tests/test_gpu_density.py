"""Adaptive density control on the GPU against the oracle (oracle/density.py,
oracle.blend_error): farthest point sampling (indices and FP32 squared
distances bit-exact), the blended-error pass on a render, the error-weighted
selection (bit-exact), the split and the prune."""
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
    N_.nexel_fps(n, xt.data_ptr(), m, scratch.data_ptr(), idx.data_ptr(), d2.data_ptr(), _stream())
    torch.cuda.synchronize()
    return idx.cpu().numpy(), d2.cpu().numpy()


@pytest.mark.parametrize("n,m", [(9, 9), (3001, 3001), (20000, 1500)])
def test_fps_bit_exact(dev, n, m):
    if n == 9:
        x = np.zeros((9, 3), np.float32)
        x[:, 0] = np.arange(9)
    else:
        x = np.random.default_rng(n).normal(size=(n, 3)).astype(np.float32)
    gi, gd = _fps_gpu(x, m, dev)
    ri, rd = D.fps(x, m)
    np.testing.assert_array_equal(gi, ri)
    np.testing.assert_array_equal(gd[1:], rd[1:])
    assert np.isinf(gd[0])


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
    n_sel = D.split_count(N, 10 * N)
    ws = torch.empty(N_.nexel_density_workspace_size(N + n_sel), dtype=torch.uint8, device=dev)
    sel = torch.empty(n_sel, dtype=torch.int32, device=dev)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    err_d, expo_d = t(err), t(expo)  # held: the call reads them asynchronously
    N_.nexel_densify_select(N, err_d.data_ptr(), expo_d.data_ptr(), n_sel, ws.data_ptr(),
                            ws.numel(), sel.data_ptr(), _stream())
    torch.cuda.synchronize()
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
