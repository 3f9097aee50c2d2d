"""The allocation-free forward render (nexel_render_fwd_static) against the
regular entry points (nexel_preprocess + nexel_render_fwd with a
caller-allocated workspace).

nexel_render_fwd_static exists for callers that cannot allocate device
memory (a plugin inside a host application that owns all device
allocations, a frame callback on a fixed memory budget): its workspace is a
file-scope device array of the library.  This test calls it through the C
ABI twice in a row, on two different scenes, and checks both results
against the regular path within the FP32 tolerance used by the other GPU
tests (1e-5), so a stale workspace from the first call would show up in the
second.  It lives in a file of its own that pytest collects last."""
import numpy as np
import pytest

from paper_2512_13796_gb300 import synth

from helpers import run_gpu

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _static_forward(scene, cam, st, field, dev):
    import torch
    from paper_2512_13796_gb300 import _native as N_
    from paper_2512_13796_gb300 import render as R
    H, W, K = cam.height, cam.width, st.K
    p = {k: torch.from_numpy(np.ascontiguousarray(getattr(scene, k))).to(dev)
         for k in ("mu", "quat", "scale", "opacity", "gamma", "color")}
    fd = R.DeviceField.from_synth(field, dev)
    ts = fd.storage_table()
    out = dict(image=torch.empty(H, W, 3, device=dev), notex=torch.empty(H, W, 3, device=dev),
               weights=torch.empty(H, W, K, device=dev),
               ids=torch.empty(H, W, K, dtype=torch.int32, device=dev),
               depths=torch.empty(H, W, K, device=dev),
               textures=torch.empty(H, W, K, 3, device=dev),
               T_final=torch.empty(H, W, device=dev))
    rc, n_inst = N_.nexel_render_fwd_static(
        R.camera_struct(cam), R.settings_struct(st), fd.struct(ts, fd.weights), scene.n,
        *[p[k].data_ptr() for k in ("mu", "quat", "scale", "opacity", "gamma", "color")],
        *[out[k].data_ptr() for k in ("image", "notex", "weights", "ids", "depths", "textures",
                                      "T_final")],
        torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert rc == 0, N_.nexel_status_string(rc)
    return {k: v.cpu().numpy() for k, v in out.items()}, n_inst


def test_static_workspace_forward_matches_regular_path():
    import torch
    assert torch.cuda.is_available(), "GPU test without a CUDA device"
    from paper_2512_13796_gb300 import _native as N_
    N_.build()
    dev = torch.device("cuda:0")
    cam = synth.front_camera(160, 120)
    st = synth.Settings(K=4)
    for seed in (11, 12):  # two calls in a row, different scenes
        sc = synth.make_scene(3000 + 500 * (seed - 11), 3, seed, gamma="var")
        fld = synth.make_field(8, 14, 2, (64,), seed, table_std=0.3)
        got, n_inst = _static_forward(sc, cam, st, fld, dev)
        ref, _, _ = run_gpu(sc, cam, st, fld, dev)
        assert n_inst == ref["n_instances"] and n_inst > 0
        np.testing.assert_array_equal(got["ids"], ref["ids"])
        for k in ("image", "notex", "weights", "depths", "textures", "T_final"):
            np.testing.assert_allclose(got[k], ref[k], rtol=0, atol=TOL, err_msg=k)


def test_static_workspace_rejects_oversize():
    import ctypes as C

    import torch
    assert torch.cuda.is_available(), "GPU test without a CUDA device"
    from paper_2512_13796_gb300 import _native as N_
    from paper_2512_13796_gb300 import render as R
    N_.build()
    n = C.c_longlong(0)
    big = R.camera_struct(synth.front_camera(512, 512))
    st = R.settings_struct(synth.Settings(K=0))
    rc = N_.lib().nexel_render_fwd_static(C.byref(big), C.byref(st), None, 0, *([None] * 13),
                                          C.byref(n), None)
    assert rc == -1  # NEXEL_ERR_INVALID_ARG: more pixels than the static workspace serves
    cam = R.camera_struct(synth.front_camera(64, 64))
    rc = N_.lib().nexel_render_fwd_static(C.byref(cam), C.byref(st), None, 16385,
                                          *([None] * 13), C.byref(n), None)
    assert rc == -1
    # a feature cache needs the backward scratch, which this call does not take
    st_cache = R.settings_struct(synth.Settings(K=4), cache_features=True)
    rc = N_.lib().nexel_render_fwd_static(C.byref(cam), C.byref(st_cache), None, 10,
                                          *([None] * 13), C.byref(n), None)
    assert rc == -1
