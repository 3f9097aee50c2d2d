"""The learned part: the hash grid and MLP are trained on the GPU by this
library's own forward and backward kernels (through the autograd wrapper),
and the textured method is compared with the same training without texture
(K = 0) on held-out views.  Targets come from the FP64 oracle rendering the
same fixed geometry with a known high-frequency world-space texture."""
import math

import numpy as np
import pytest

import oracle
from paper_2512_13796_gb300 import synth

pytestmark = pytest.mark.gpu

FREQ = 40.0  # rad per world unit: a period of ~0.16, below the surfel size


def _psnr(a, b):
    mse = float(np.mean((np.clip(a, 0, 1) - b) ** 2))
    return 10.0 * math.log10(1.0 / max(mse, 1e-12))


def _train(sc, cams, targets, K, steps, dev, precision):
    import torch
    from paper_2512_13796_gb300 import render as R
    params = {k: torch.from_numpy(np.ascontiguousarray(getattr(sc, k))).to(dev)
              for k in ("mu", "quat", "scale", "opacity", "gamma", "color")}
    params["color"] = params["color"].clone().fill_(0.5).requires_grad_(True)
    grid, mlp = ("f16", "bf16") if precision == "bf16" else ("f32", "f32")
    fld = R.DeviceField.from_synth(synth.make_field(8, 16, 2, (64,), 3), dev, grid, mlp)
    fld.table.requires_grad_(True)
    fld.weights.requires_grad_(True)
    groups = [{"params": [params["color"]], "lr": 2e-2}]
    if K > 0:
        groups += [{"params": [fld.table], "lr": 2e-2}, {"params": [fld.weights], "lr": 2e-3}]
    opt = torch.optim.Adam(groups, eps=1e-15)
    st = synth.Settings(K=K)
    ws = R.Workspace(dev, cap_hint=1 << 20)
    tg = [torch.from_numpy(t.astype(np.float32)).to(dev) for t in targets]
    for it in range(steps):
        v = it % len(cams)
        img, _, _ = R.render(params, fld if K > 0 else None, cams[v], st, ws)
        loss = (img - tg[v]).abs().mean()
        opt.zero_grad(set_to_none=True)
        loss.backward()
        opt.step()
        with torch.no_grad():
            params["color"].clamp_(0.0, 1.0)
    return params, fld, st, ws


@pytest.mark.parametrize("precision", ["f32", "bf16"])
def test_neural_texture_beats_untextured_on_heldout_views(precision):
    import torch
    assert torch.cuda.is_available()
    from paper_2512_13796_gb300 import _native
    from paper_2512_13796_gb300 import render as R
    _native.build()
    dev = torch.device("cuda:0")
    sc = synth.make_scene(3000, 4, 77, gamma="var")
    sc.opacity[:] = np.random.default_rng(1).uniform(0.6, 0.99, sc.n).astype(np.float32)
    rng = np.random.default_rng(5)
    cams = synth.sphere_cameras(rng, [(96, 96)] * 10)
    st = synth.Settings(K=0)
    targets = [oracle.render_procedural(sc, c, st, FREQ).reshape(c.height, c.width, 3)
               for c in cams]
    train, held = list(range(8)), [8, 9]
    res = {}
    for K in (2, 0):
        params, fld, stK, ws = _train(sc, [cams[i] for i in train], [targets[i] for i in train],
                                      K, 600, dev, precision)
        ps = []
        with torch.no_grad():
            for i in held:
                img, _, _ = R.render(params, fld if K > 0 else None, cams[i], stK, ws)
                ps.append(_psnr(img.cpu().numpy(), targets[i]))
        res[K] = float(np.mean(ps))
    print(f"\n[learned {precision}] held-out PSNR textured(K=2)={res[2]:.2f} dB "
          f"untextured(K=0)={res[0]:.2f} dB gain={res[2] - res[0]:.2f} dB")
    assert res[2] > res[0] + 1.0
