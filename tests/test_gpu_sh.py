"""Degree-3 spherical-harmonics per-primitive colours (settings.sh_degree =
3) against the FP64 oracle (oracle.render_sh / render_bwd_sh): images and
the gradients of every parameter, the [N, 16, 3] coefficients included, on
config 0 (every pixel, FP32 form) and on a config 1 pixel sample (FP32 and
BF16 forms)."""
import numpy as np
import pytest

import oracle
from paper_2512_13796_gb300 import synth

from helpers import (SURFEL_KEYS, UNIT_ROUNDOFF, compare_forward, compare_grads,
                     ill_conditioned, kink_cancelled_upstream, masked_upstream, reference,
                     reference_grads)

pytestmark = pytest.mark.gpu

TIE, CELL, RELU = 1e-5, 2e-6, 1e-4
GRAD_RTOL = 1e-3


def _reduced_precision_check(dev, w, cam, st, field, coeffs, pix, mlp, seed, with_wt=True):
    """Forward against the oracle at the FP32 parameters (colours 2e-3 /
    1e-3), backward per element against the oracle at the parameters the
    form reads, with the bound of test_gpu_parity.py."""
    P, K = cam.width * cam.height, st.K
    ref = reference(w.scene, cam, st, field, pix, coeffs=coeffs)
    ref_b = reference(w.scene, cam, st, field, pix, mlp=mlp, coeffs=coeffs)
    dI, dW, dT, sel, us = kink_cancelled_upstream(ref_b, P, K, seed, with_wt=with_wt)
    fw, gg = _run(w.scene, coeffs, cam, st, field, dev, "f16", mlp, dI, dW, dT)
    s = compare_forward(fw, ref, K, 2e-3 if mlp == "bf16" else 1e-3)
    gr, ga = reference_grads(w.scene, cam, st, field, sel, dI, dW, dT, mlp, coeffs=coeffs)
    st_g = compare_grads(gg, gr, GRAD_RTOL, absolute=ga, u=UNIT_ROUNDOFF[mlp],
                         skip_surfels=ill_conditioned(w.scene, cam))
    return s, st_g, us


@pytest.fixture(scope="module")
def dev():
    import torch
    assert torch.cuda.is_available(), "GPU test without a CUDA device"
    from paper_2512_13796_gb300 import _native
    _native.build()
    return torch.device("cuda:0")


def _run(scene, coeffs, cam, st, field, dev, grid, mlp, dI=None, dW=None, dT=None):
    import torch
    from paper_2512_13796_gb300 import render as R
    p = {k: torch.from_numpy(np.ascontiguousarray(getattr(scene, k))).to(dev)
         for k in SURFEL_KEYS}
    p["color"] = torch.from_numpy(coeffs).to(dev)
    fd = R.DeviceField.from_synth(field, dev, grid, mlp)
    ws = R.Workspace(dev)
    cam_s = R.camera_struct(cam)
    st_s = R.settings_struct(st, grid, mlp, sh_degree=3)
    ts = fd.storage_table()
    out = R.forward(ws, cam_s, st_s, fd, ts, fd.weights, *[p[k] for k in SURFEL_KEYS])
    g = None
    if dI is not None:
        t = lambda a: None if a is None else torch.from_numpy(a.astype(np.float32)).to(dev)
        g = R.backward(ws, cam_s, st_s, fd, ts, fd.weights, *[p[k] for k in SURFEL_KEYS[:5]],
                       out, t(dI), t(dW), t(dT))
    torch.cuda.synchronize()
    fw = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in out.items()}
    gg = None if g is None else {k: v.cpu().numpy() for k, v in g.items()}
    return fw, gg


def test_sh_config0_forward_backward(dev):
    w = synth.workload(0, gamma="var")
    cam, st = w.cameras[0], w.settings
    coeffs = synth.sh_coefficients(w.scene.n, 0)
    ref = oracle.render_sh(w.scene, coeffs, cam, st, w.field, tie_tol=TIE, cell_tol=CELL,
                           relu_tol=RELU)
    pix, ok = ref["pixels"], ref["tie"] == 0
    P, K = cam.width * cam.height, st.K
    dI, dW, dT = masked_upstream(pix.size, P, K, pix, ok, seed=31)
    fw, gg = _run(w.scene, coeffs, cam, st, w.field, dev, "f32", "f32", dI, dW, dT)
    s = compare_forward(fw, ref, K, 1e-5)
    assert s["n_tie"] < 0.25 * s["n_pix"]
    sel = pix[ok]
    gr = oracle.render_bwd_sh(w.scene, coeffs, cam, st, w.field, sel, dI[sel], dW[sel], dT[sel])
    assert gg["color"].shape == (w.scene.n, 16, 3)
    st_g = compare_grads(gg, gr, 1e-3)
    print(f"\n[sh config0] fwd image err {s['image']:.2e} grads {st_g}")


def test_sh_backward_overwrites_dirty_gradients(dev):
    """Without accumulate, the backward overwrites every gradient output,
    all 48 SH coefficients per surfel included: into buffers full of NaN
    it gives exactly what it gives into zeroed ones."""
    import torch
    from paper_2512_13796_gb300 import render as R
    w = synth.workload(0, gamma="var")
    cam, st = w.cameras[0], w.settings
    coeffs = synth.sh_coefficients(w.scene.n, 0)
    p = {k: torch.from_numpy(np.ascontiguousarray(getattr(w.scene, k))).to(dev)
         for k in SURFEL_KEYS}
    p["color"] = torch.from_numpy(coeffs).to(dev)
    fd = R.DeviceField.from_synth(w.field, dev, "f32", "f32")
    ws = R.Workspace(dev)
    cam_s = R.camera_struct(cam)
    st_s = R.settings_struct(st, "f32", "f32", sh_degree=3)
    ts = fd.storage_table()
    out = R.forward(ws, cam_s, st_s, fd, ts, fd.weights, *[p[k] for k in SURFEL_KEYS])
    dI = torch.from_numpy(np.random.default_rng(3).normal(
        size=(cam.height, cam.width, 3)).astype(np.float32)).to(dev)
    args = (ws, cam_s, st_s, fd, ts, fd.weights, *[p[k] for k in SURFEL_KEYS[:5]], out, dI)
    clean = R.backward(*args)
    shapes = {k: v.shape for k, v in clean.items()}
    dirty = {k: torch.full(sh, float("nan"), device=dev) for k, sh in shapes.items()}
    again = R.backward(*args, accumulate=False, grads=dirty)
    torch.cuda.synchronize()
    assert clean["color"].shape == (w.scene.n, 16, 3)
    for k in shapes:
        a, b = clean[k].cpu().numpy(), again[k].cpu().numpy()
        assert np.isfinite(b).all(), k
        # float atomics may sum in another order: equal up to their rounding
        assert np.allclose(a, b, rtol=1e-5, atol=1e-6 * max(1.0, float(np.abs(a).max()))), k


@pytest.mark.parametrize("form", ["f32", "bf16"])
def test_sh_config1_sampled(dev, form):
    w = synth.workload(1)
    cam, st = w.cameras[0], w.settings
    coeffs = synth.sh_coefficients(w.scene.n, 1)
    pix = synth.pixel_sample(cam, 2048, 2, seed=7)
    if form == "bf16":
        s, st_g, us = _reduced_precision_check(dev, w, cam, st, w.field, coeffs, pix, "bf16",
                                               seed=32)
        print(f"\n[sh config1 bf16] image err {s['image']:.2e} {us} grads {st_g}")
        return
    ref = oracle.render_sh(w.scene, coeffs, cam, st, w.field, pix, tie_tol=TIE, cell_tol=CELL,
                           relu_tol=RELU)
    ok = ref["tie"] == 0
    P, K = cam.width * cam.height, st.K
    dI, _, _ = masked_upstream(pix.size, P, K, pix, ok, seed=32, with_wt=False)
    fw, gg = _run(w.scene, coeffs, cam, st, w.field, dev, "f32", "f32", dI)
    s = compare_forward(fw, ref, K, 1e-5)
    assert s["n_tie"] < 0.25 * s["n_pix"]
    sel = pix[ok]
    gr = oracle.render_bwd_sh(w.scene, coeffs, cam, st, w.field, sel, dI[sel])
    compare_grads(gg, gr, 1e-3, skip_surfels=ill_conditioned(w.scene, cam))


@pytest.mark.parametrize("hidden", [(64,), (64, 64)], ids=["16-64-48", "32-64-64-48"])
def test_sh_textures_fp32_both_modes(dev, hidden):
    """Both appearance modes in SH (Sec. 5: degree 3 for both): per-primitive
    SH colours and a 48-output MLP whose outputs are the texture's SH
    coefficients, evaluated in the ray direction (FP32 form, every pixel of
    config 0)."""
    w = synth.workload(0, gamma="var")
    cam, st = w.cameras[0], w.settings
    L = 8 if len(hidden) == 1 else 16
    field = synth.make_field(L, 12, 2, hidden, 5, out_dim=48)
    coeffs = synth.sh_coefficients(w.scene.n, 3)
    ref = oracle.render_sh(w.scene, coeffs, cam, st, field, tie_tol=TIE, cell_tol=CELL,
                           relu_tol=RELU)
    pix, ok = ref["pixels"], ref["tie"] == 0
    P, K = cam.width * cam.height, st.K
    dI, dW, dT = masked_upstream(pix.size, P, K, pix, ok, seed=33)
    fw, gg = _run(w.scene, coeffs, cam, st, field, dev, "f32", "f32", dI, dW, dT)
    s = compare_forward(fw, ref, K, 1e-5)
    assert s["n_tie"] < 0.25 * s["n_pix"]
    sel = pix[ok]
    gr = oracle.render_bwd_sh(w.scene, coeffs, cam, st, field, sel, dI[sel], dW[sel], dT[sel])
    st_g = compare_grads(gg, gr, 1e-3)
    print(f"\n[sh textures {hidden}] fwd image err {s['image']:.2e} tex err "
          f"{s['textures']:.2e} grads {st_g}")


@pytest.mark.parametrize("mlp", ["bf16", "f16"])
@pytest.mark.parametrize("hidden", [(64,), (64, 64)], ids=["16-64-48", "32-64-64-48"])
def test_sh_textures_tensor_core_forms(dev, hidden, mlp):
    """The tcgen05 kernels with the 48-wide output layer (FP16 table, BF16 or
    FP16 MLP) against the FP64 oracle, both appearance modes in SH, with the
    reduced-precision tolerances of the RGB forms (colours 2e-3 / 1e-3,
    gradients per element with the rounding bound)."""
    w = synth.workload(0, gamma="var")
    cam, st = w.cameras[0], w.settings
    L = 8 if len(hidden) == 1 else 16
    field = synth.make_field(L, 12, 2, hidden, 5, out_dim=48)
    coeffs = synth.sh_coefficients(w.scene.n, 4)
    s, st_g, us = _reduced_precision_check(dev, w, cam, st, field, coeffs, None, mlp, seed=34)
    print(f"\n[sh textures tc {hidden} {mlp}] image err {s['image']:.2e} tex err "
          f"{s['textures']:.2e} {us} grads {st_g}")


def test_sh_textures_rejected_with_fp32_table_on_tensor_cores(dev):
    """The 48-output tcgen05 kernels read the FP16 table: an FP32 table with
    a tensor-core MLP and 48 outputs is refused (NEXEL_ERR_UNSUPPORTED)
    before any launch."""
    import torch
    from paper_2512_13796_gb300 import _native as N_
    from paper_2512_13796_gb300 import render as R
    w = synth.workload(0)
    field = synth.make_field(16, 12, 2, (64, 64), 5, out_dim=48)
    p = {k: torch.from_numpy(np.ascontiguousarray(getattr(w.scene, k))).to(dev)
         for k in SURFEL_KEYS}
    fd = R.DeviceField.from_synth(field, dev, "f32", "bf16")
    ws = R.Workspace(dev)
    with pytest.raises(N_.NexelError) as ei:
        R.forward(ws, R.camera_struct(w.cameras[0]), R.settings_struct(w.settings, "f32", "bf16"),
                  fd, fd.storage_table(), fd.weights, *[p[k] for k in SURFEL_KEYS])
    assert ei.value.code == -4


@pytest.mark.parametrize("mlp", ["f16", "bf16"])
def test_sh_paper_configuration_config2_sampled(dev, mlp):
    """The paper's configuration at the headline size: 300k surfels,
    1280x720, K = 4, hash 16 x 2^19 x 2 (FP16 table), degree-3 SH in both
    modes (48 colour coefficients, MLP 32-64-64-48) on the tensor cores,
    on a pixel sample (random pixels and whole tiles)."""
    w = synth.workload(2)
    cam, st = w.cameras[0], w.settings
    field = synth.make_field(16, 19, 2, (64, 64), 2, out_dim=48)
    coeffs = synth.sh_coefficients(w.scene.n, 2)
    pix = synth.pixel_sample(cam, 1024, 2, seed=22)
    s, st_g, us = _reduced_precision_check(dev, w, cam, st, field, coeffs, pix, mlp, seed=35)
    print(f"\n[sh config2 {mlp}] image err {s['image']:.2e} ties {s['n_tie']}/{s['n_pix']} "
          f"{us} grads {st_g}")
