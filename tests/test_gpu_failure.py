"""Failure paths of the library on the GPU, made on the host: surfels with
NaN or infinite parameters (culled, counted, reported as NEXEL_ERR_NUMERIC,
and the rest of the scene renders as if they were absent), and a bounded
tensor-core wait made to run out by the test hook (NEXEL_ERR_TIMEOUT, TMEM
freed, the next call correct).  Nothing here faults, traps or hangs the
GPU: every wait involved is bounded."""
import numpy as np
import pytest

import oracle
from paper_2512_13796_gb300 import synth

from helpers import SURFEL_KEYS, compare_forward, gpu_params, reference, run_gpu

pytestmark = pytest.mark.gpu

NEXEL_OK, NEXEL_ERR_TIMEOUT, NEXEL_ERR_NUMERIC = 0, -5, -6


@pytest.fixture(scope="module")
def dev():
    import torch
    assert torch.cuda.is_available(), "GPU test without a CUDA device"
    from paper_2512_13796_gb300 import _native
    _native.build()
    _native.lib()
    return torch.device("cuda:0")


def _status(ws, cam, st, field_s, N, bws=None):
    import torch
    from paper_2512_13796_gb300 import _native as N_
    return N_.nexel_read_status(cam, st, field_s, N, ws.ws.data_ptr(), ws.ws.numel(),
                                bws.data_ptr() if bws is not None else None,
                                bws.numel() if bws is not None else 0,
                                torch.cuda.current_stream().cuda_stream)


def test_nonfinite_surfels_are_culled_and_counted(dev):
    """NaN / infinite parameters and a zero quaternion, injected on the host
    into 7 surfels: the render equals the oracle's render of the scene
    without them, nexel_render_stats counts 7, nexel_read_status reports
    NEXEL_ERR_NUMERIC once (it clears the word), and their gradients are
    zero while every gradient stays finite."""
    import torch
    from paper_2512_13796_gb300 import _native as N_
    from paper_2512_13796_gb300 import render as R
    w = synth.workload(0)
    cam, st = w.cameras[0], w.settings
    sc = synth.Scene(*(getattr(w.scene, k).copy() for k in SURFEL_KEYS))
    bad = np.array([3, 17, 40, 41, 99, 150, 200])
    sc.mu[bad[0], 1] = np.nan
    sc.mu[bad[1], 2] = np.inf
    sc.scale[bad[2], 0] = np.inf
    sc.opacity[bad[3]] = np.nan
    sc.quat[bad[4]] = 0.0
    sc.gamma[bad[5], 1] = -np.inf
    sc.color[bad[6], 0] = np.nan
    keep = np.setdiff1d(np.arange(sc.n), bad)
    P, K = cam.width * cam.height, st.K
    rng = np.random.default_rng(2)
    dI = rng.normal(size=(P, 3)).astype(np.float32)
    fw, g, ws = run_gpu(sc, cam, st, w.field, dev, d_image=dI)
    cam_s, st_s = R.camera_struct(cam), R.settings_struct(st)
    stats = N_.nexel_render_stats(cam_s, st_s, sc.n, ws.ws.data_ptr(), ws.ws.numel(),
                                  torch.cuda.current_stream().cuda_stream)
    assert stats["nonfinite_surfels"] == bad.size
    assert _status(ws, cam_s, st_s, None, sc.n) == NEXEL_ERR_NUMERIC
    assert _status(ws, cam_s, st_s, None, sc.n) == NEXEL_OK  # read and cleared
    clean = synth.Scene(*(getattr(sc, k)[keep] for k in SURFEL_KEYS))
    ref = reference(clean, cam, st, w.field)
    fw_ids = fw["ids"].copy()
    has = fw_ids >= 0
    assert not np.isin(fw_ids[has], bad).any()
    fw["ids"][has] = np.searchsorted(keep, fw_ids[has])  # ids of the scene without them
    s = compare_forward(fw, ref, K, 1e-5)
    print(f"\n[non-finite surfels] {stats['nonfinite_surfels']} culled; fwd {s}")
    for k, v in g.items():
        assert np.all(np.isfinite(v)), k
    for k in SURFEL_KEYS:
        assert np.all(g[k][bad] == 0.0), k


@pytest.mark.parametrize("mlp", ["bf16", "f16"])
@pytest.mark.parametrize("levels,hidden", [(8, (64,)), (16, (64, 64))])
def test_tc_wait_timeout_reported_and_recovered(dev, mlp, levels, hidden):
    """The test hook makes every tensor-core kernel wait, with a short
    bound, for MMAs it never issued: the forward and the backward return,
    nexel_read_status reports NEXEL_ERR_TIMEOUT, and with the hook off the
    same calls run normally again (each CTA freed its TMEM) and match a
    fresh run.  Two hidden layers with 32 inputs take the backward with
    three tile groups per CTA and a dedicated MMA thread."""
    import torch
    from paper_2512_13796_gb300 import _native as N_
    from paper_2512_13796_gb300 import render as R
    w = synth.workload(0)
    sc, cam, st = w.scene, synth.front_camera(96, 80), w.settings
    fld = synth.make_field(levels, 12, 2, hidden, 0)
    P, K = cam.width * cam.height, st.K
    dI = np.random.default_rng(3).normal(size=(P, 3)).astype(np.float32)
    good, g_good, _ = run_gpu(sc, cam, st, fld, dev, grid="f16", mlp=mlp, d_image=dI,
                              cache_features=True)
    N_.nexel_test_tc_wait_timeout(64)
    try:
        _, _, ws = run_gpu(sc, cam, st, fld, dev, grid="f16", mlp=mlp, d_image=dI,
                           cache_features=True)
        cam_s = R.camera_struct(cam)
        st_s = R.settings_struct(st, "f16", mlp, False, True)
        fs = R.DeviceField.from_synth(fld, dev, "f16", mlp)
        fstruct = fs.struct(fs.storage_table(), fs.weights)
        rc = _status(ws, cam_s, st_s, fstruct, sc.n, ws.bws)
    finally:
        N_.nexel_test_tc_wait_timeout(0)
    assert rc == NEXEL_ERR_TIMEOUT
    again, g_again, ws2 = run_gpu(sc, cam, st, fld, dev, grid="f16", mlp=mlp, d_image=dI,
                                  cache_features=True)
    assert _status(ws2, cam_s, st_s, fstruct, sc.n, ws2.bws) == NEXEL_OK
    for k in ("image", "textures", "ids", "weights"):
        np.testing.assert_array_equal(again[k], good[k], err_msg=k)
    for k in g_good:
        np.testing.assert_allclose(g_again[k], g_good[k], rtol=1e-4,
                                   atol=1e-6 * float(np.abs(g_good[k]).max() + 1e-30),
                                   err_msg=k)


@pytest.mark.parametrize("mlp", ["f32", "bf16"])
def test_status_clean_after_backward_on_dirty_scratch(dev, mlp):
    """The backward scratch is the caller's memory, uninitialised: filled
    with 0xFF bytes before the call, a normal forward + backward still
    reads back NEXEL_OK (the backward clears its status word on entry in
    every form)."""
    import torch
    from paper_2512_13796_gb300 import render as R
    w = synth.workload(0)
    sc, cam, st = w.scene, synth.front_camera(96, 80), w.settings
    grid = "f32" if mlp == "f32" else "f16"
    fld = synth.make_field(8, 12, 2, (64,), 0)
    P = cam.width * cam.height
    dI = np.random.default_rng(5).normal(size=(P, 3)).astype(np.float32)
    ws = R.Workspace(dev, cap_hint=1 << 16)
    cam_s = R.camera_struct(cam)
    st_s = R.settings_struct(st, grid, mlp)
    fs = R.DeviceField.from_synth(fld, dev, grid, mlp)
    fstruct = fs.struct(fs.storage_table(), fs.weights)
    ws.bwd(cam_s, st_s, fstruct).fill_(255)
    run_gpu(sc, cam, st, fld, dev, grid=grid, mlp=mlp, d_image=dI, ws=ws)
    assert _status(ws, cam_s, st_s, fstruct, sc.n, ws.bws) == NEXEL_OK
