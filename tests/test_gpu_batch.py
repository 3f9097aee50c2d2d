"""Batched multi-view step (nexel_render_batch_fwd / _bwd, the device-count
preprocess and one CUDA graph per step).

- Small scene, three views of different sizes, FP32 form: the batched step,
  eager and replayed from a captured CUDA graph, against the FP64 oracle
  (images per view; gradients summed over the views).
- Config 3 (600k surfels, 8 views 640x480 .. 1920x1080, BF16 form): the
  batched step against the single-view entry points run view after view
  (identical images and top-K buffers; gradients equal up to the summation
  order of the float atomics).
- An instance capacity that is too small is reported by nexel_read_status,
  not written past."""
import numpy as np
import pytest

import oracle
from paper_2512_13796_gb300 import synth

from helpers import (SURFEL_KEYS, UNIT_ROUNDOFF, compare_forward, compare_grads, gpu_params,
                     ill_conditioned, masked_upstream, reference, reference_grads)

pytestmark = pytest.mark.gpu

TIE, CELL, RELU = 1e-5, 2e-6, 1e-4
TOL_F32, GRAD_RTOL = 1e-5, 1e-3
ATOMIC_ORDER_L2 = 1e-5  # same arithmetic, float atomics summed in another order
MLP_ORDER_L2 = 1e-3


@pytest.fixture(scope="module")
def dev():
    import torch
    assert torch.cuda.is_available(), "GPU test without a CUDA device"
    from paper_2512_13796_gb300 import _native
    _native.build()
    return torch.device("cuda:0")


def _small_workload():
    scene = synth.make_scene(256, 3, 7, gamma="var")
    cams = synth.sphere_cameras(np.random.default_rng(11), [(48, 40), (64, 64), (80, 56)])
    field = synth.make_field(4, 12, 2, (16,), 7)
    return scene, cams, synth.Settings(K=2), field


def _numpy_out(o):
    return {k: v.cpu().numpy() for k, v in o.items()}


@pytest.mark.parametrize("graph", [False, True])
def test_batch_small_views_vs_oracle(dev, graph):
    import torch
    from paper_2512_13796_gb300 import render as R
    scene, cams, st, field = _small_workload()
    p = gpu_params(scene, dev)
    fd = R.DeviceField.from_synth(field, dev, "f32", "f32")
    step = R.BatchStep(cams, st, fd, p)
    refs, dIs, grs = [], [], None
    for v, cam in enumerate(cams):
        ref = oracle.render(scene, cam, st, field, tie_tol=TIE, cell_tol=CELL, relu_tol=RELU)
        refs.append(ref)
        pix, ok = ref["pixels"], ref["tie"] == 0
        P = cam.width * cam.height
        dI, _, _ = masked_upstream(pix.size, P, st.K, pix, ok, seed=20 + v, with_wt=False)
        dIs.append(dI)
        sel = pix[ok]
        gr = oracle.render_bwd(scene, cam, st, field, sel, dI[sel])
        grs = gr if grs is None else {k: grs[k] + gr[k] for k in gr if k != "mlp_layers"}
        step.d_image[v].copy_(torch.from_numpy(dI.astype(np.float32)).view(cam.height,
                                                                             cam.width, 3))
    if graph:
        step.capture()
        # run the graph on changed parameter storage: the result must follow
        step.params["color"].mul_(0.5)
        step.replay()
        step.params["color"].mul_(2.0)
        step.replay()
    else:
        step.step()
    torch.cuda.synchronize()
    assert step.status() == [0, 0, 0]
    for v, cam in enumerate(cams):
        fw = _numpy_out(step.out[v])
        s = compare_forward(fw, refs[v], st.K, TOL_F32)
        assert s["n_tie"] < 0.25 * s["n_pix"]
    gg = {k: x.cpu().numpy() for k, x in step.grads.items()}
    compare_grads(gg, grs, GRAD_RTOL)


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("levels,hidden", [(8, (64,)), (16, (64, 64))])
def test_batch_small_views_tensor_cores_vs_oracle(dev, graph, levels, hidden):
    """The batched step on the tensor-core path (FP16 table, BF16 MLP 16-64-3,
    or 32-64-64-3, which takes the backward with three tile groups per CTA;
    feature cache): every per-tile phase runs as one launch over the three
    views (persistent collection CTAs pulling (view, tile) items, the
    tcgen05 texturing kernels and the hash-grid backward over the views'
    concatenated tiles).  Images against the FP64 oracle at the FP32
    parameters (2e-3), gradients summed over the views per element against
    the oracle at the parameters the form reads (upstream d_image on pixels
    with no tie and no kink), with the reduced-precision bound."""
    import torch
    from paper_2512_13796_gb300 import render as R
    scene = synth.make_scene(256, 3, 7, gamma="var")
    cams = synth.sphere_cameras(np.random.default_rng(11), [(48, 40), (64, 64), (80, 56)])
    field = synth.make_field(levels, 12, 2, hidden, 7, table_std=0.3)
    st = synth.Settings(K=2)
    p = gpu_params(scene, dev)
    fd = R.DeviceField.from_synth(field, dev, "f16", "bf16")
    step = R.BatchStep(cams, st, fd, p)
    grs, gas, refs = None, None, []
    for v, cam in enumerate(cams):
        ref = reference(scene, cam, st, field)
        refs.append(ref)
        ref_b = reference(scene, cam, st, field, mlp="bf16")
        pix, ok = ref_b["pixels"], ref_b["tie"] == 0
        P = cam.width * cam.height
        dI, _, _ = masked_upstream(pix.size, P, st.K, pix, ok, seed=60 + v, with_wt=False)
        sel = pix[ok]
        gr, ga = reference_grads(scene, cam, st, field, sel, dI, None, None, "bf16")
        grs = gr if grs is None else {k: grs[k] + gr[k] for k in gr if k != "mlp_layers"}
        gas = ga if gas is None else {k: gas[k] + ga[k] for k in ga}
        step.d_image[v].copy_(torch.from_numpy(dI.astype(np.float32)).view(cam.height,
                                                                             cam.width, 3))
    if graph:
        step.capture()
        step.replay()
    else:
        step.step()
    torch.cuda.synchronize()
    assert step.status() == [0, 0, 0]
    for v, cam in enumerate(cams):
        compare_forward(_numpy_out(step.out[v]), refs[v], st.K, 2e-3)
    gg = {k: x.cpu().numpy() for k, x in step.grads.items()}
    skip = np.unique(np.concatenate([ill_conditioned(scene, c) for c in cams]))
    compare_grads(gg, grs, GRAD_RTOL, absolute=gas, u=UNIT_ROUNDOFF["bf16"], skip_surfels=skip)


def test_batch_config3_matches_single_view_calls(dev):
    import torch
    from paper_2512_13796_gb300 import render as R
    w = synth.workload(3)
    st = w.settings
    p = gpu_params(w.scene, dev)
    fd = R.DeviceField.from_synth(w.field, dev, w.grid_dtype, w.mlp_dtype)
    step = R.BatchStep(w.cameras, st, fd, p)
    rng = np.random.default_rng(5)
    for v, cam in enumerate(w.cameras):
        step.d_image[v].copy_(torch.from_numpy(
            rng.normal(size=(cam.height, cam.width, 3)).astype(np.float32) * 1e-3))
    step.capture()
    step.replay()
    torch.cuda.synchronize()
    assert step.status() == [0] * len(w.cameras)
    # the same views through nexel_preprocess / _render_fwd / _render_bwd
    ts = fd.storage_table()
    ws = R.Workspace(dev, cap_hint=1 << 24)
    grads = None
    for v, cam in enumerate(w.cameras):
        cam_s = R.camera_struct(cam)
        st_s = R.settings_struct(st, w.grid_dtype, w.mlp_dtype, cache_features=True)
        out = R.forward(ws, cam_s, st_s, fd, ts, fd.weights, *[p[k] for k in SURFEL_KEYS])
        assert out["n_instances"] == step.n_instances[v]
        for k in ("image", "notex", "weights", "ids", "depths", "textures", "T_final"):
            assert torch.equal(out[k], step.out[v][k]), (v, k)
        grads = R.backward(ws, cam_s, st_s, fd, ts, fd.weights,
                           *[p[k] for k in SURFEL_KEYS[:5]], out, step.d_image[v],
                           accumulate=grads is not None, grads=grads)
    torch.cuda.synchronize()
    for k, g in grads.items():
        a, b = step.grads[k].double(), g.double()
        err = float((a - b).norm() / b.norm())
        # the batched tcgen05 backward sums the MLP weight gradients of tiles
        # of every view in one CTA's FP32 TMEM accumulators (not view by
        # view): the same BF16 products added in another order.  The sums
        # cancel strongly (8.6M rows of random-sign terms), so the rounding
        # of a reordered FP32 sum is visible at ~1e-4 of the result.
        bound = MLP_ORDER_L2 if k == "mlp" else ATOMIC_ORDER_L2
        assert err <= bound, (k, err)


def test_batch_capacity_overflow_is_flagged(dev):
    import torch
    from paper_2512_13796_gb300 import render as R
    w = synth.workload(1)
    cams = [synth.front_camera(320, 320), synth.front_camera(160, 96)]
    p = gpu_params(w.scene, dev)
    fd = R.DeviceField.from_synth(w.field, dev, "f32", "f32")
    step = R.BatchStep(cams, w.settings, fd, p, train=False)
    assert min(step.n_instances) > 20000
    # shrink view 0's workspace to half its instances: the device-count
    # preprocess keeps the first half and flags the rest
    cs = step.cams[0]
    cap = step.n_instances[0] // 2
    nbytes = R.N_.nexel_workspace_size(cs, step.N, cap)
    step.ws[0] = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    step.ws_bytes[0] = nbytes
    step.forward()
    torch.cuda.synchronize()
    assert step.status() == [-3, 0]
    # the status words were cleared by the read
    assert step.status() == [0, 0]
    img = step.out[0]["image"]
    assert torch.isfinite(img).all()
