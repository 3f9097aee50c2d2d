"""The training loop of the paper around the path, all on the GPU: surfels
initialised by farthest point sampling of a point cloud (scales from the
sampling distances), the objective of Sec. 5 with Adam, blended errors
accumulated across iterations, and one density step (error-weighted split
of 5 %, prune) in the middle; the objective falls and the surfel count
follows the split and prune counts."""
import math

import numpy as np
import pytest

import oracle
from paper_2512_13796_gb300 import synth

pytestmark = pytest.mark.gpu


def test_training_loop_with_density_control():
    import torch
    from paper_2512_13796_gb300 import _native
    from paper_2512_13796_gb300 import render as R
    assert torch.cuda.is_available()
    _native.build()
    dev = torch.device("cuda:0")
    ref_scene = synth.make_scene(3000, 4, 31, gamma="one")
    cams = synth.sphere_cameras(np.random.default_rng(4), [(64, 48)] * 4)
    targets = [torch.from_numpy(oracle.render_procedural(ref_scene, c, synth.Settings(K=0), 20.0)
                                .reshape(c.height, c.width, 3).astype(np.float32)).to(dev)
               for c in cams]
    # a point cloud on the scene's surfaces (the surfel centres) -> FPS
    cloud = torch.from_numpy(ref_scene.mu).to(dev)
    M = 1200
    mu, s = R.fps_init(cloud, M)
    assert torch.all(s[1:] <= s[:-1] + 1e-6)  # distances at selection never grow
    rng = np.random.default_rng(5)
    q = rng.normal(size=(M, 4)).astype(np.float32)
    p = dict(mu=mu.contiguous(), quat=torch.from_numpy(q).to(dev),
             scale=torch.stack([s, s], 1).clamp(0.01, 0.3).contiguous(),
             opacity=torch.full((M,), 0.6, device=dev), gamma=torch.ones(M, 2, device=dev),
             color=torch.full((M, 3), 0.5, device=dev))
    fd = R.DeviceField.from_synth(synth.make_field(8, 14, 2, (64,), 3), dev, "f32", "f32")
    st = synth.Settings(K=2)
    ob = R.Objective(64, 48, dev)
    dc = R.DensityControl(M, dev, budget=2000, seed=1)
    ws = R.Workspace(dev)
    lrs = dict(mu=1e-4, quat=1e-3, scale=1e-4, opacity=1e-2, gamma=0.0, color=2e-2)
    keys = ("mu", "quat", "scale", "opacity", "gamma", "color")

    def make_adam():
        return R.Adam([p[k] for k in keys] + [fd.table, fd.weights],
                      [lrs[k] for k in keys] + [2e-2, 2e-3])

    opt = make_adam()
    totals = []
    for it in range(160):
        v = it % len(cams)
        cam_s = R.camera_struct(cams[v])
        st_s = R.settings_struct(st, cache_features=True)
        ts = fd.storage_table()
        out = R.forward(ws, cam_s, st_s, fd, ts, fd.weights, *[p[k] for k in keys])
        d_img, d_w, d_t = ob.image_terms(out["image"], targets[v], out["weights"], out["textures"])
        g = R.backward(ws, cam_s, st_s, fd, ts, fd.weights, *[p[k] for k in keys[:5]], out, d_img,
                       d_w, d_t)
        ob.param_terms(p["opacity"], fd, g["opacity"], g["table"])
        dc.accumulate(ws, cam_s, st_s, p["mu"].shape[0], out["image"], targets[v])
        opt.step([g[k] for k in keys] + [g["table"], g["mlp"]])
        with torch.no_grad():
            p["opacity"].clamp_(0.0, 0.99)
            p["scale"].clamp_(min=1e-3)
        totals.append(ob.read()["total"])
        if it == 80:
            N = p["mu"].shape[0]
            n_low = int((p["opacity"] < 0.005).sum().item())
            new, n_split, n_pruned = dc.step(p)
            assert n_split == min(math.ceil(0.05 * N), 2000 - N)
            assert new["mu"].shape[0] == N + n_split - n_pruned
            assert n_pruned >= n_low  # every pruned surfel had a low opacity
            p = new
            opt = make_adam()
    assert all(np.isfinite(totals))
    first, last = np.mean(totals[:8]), np.mean(totals[-8:])
    print(f"\n[train+density] objective {first:.4f} -> {last:.4f}, surfels {M} -> "
          f"{p['mu'].shape[0]}")
    assert last < 0.8 * first
