"""The C-ABI library builds, loads and exports every entry point declared in
include/*.h; host-side argument checks answer without touching a GPU."""
import ctypes as C
import glob
import os
import re

import pytest

from paper_2512_13796_gb300 import _native as N_
from paper_2512_13796_gb300 import render as R
from paper_2512_13796_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"^[A-Za-z_][\w \t\*]*?\b(nexel_\w+)\s*\(", src, flags=re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    N_.build()
    return N_.lib()


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert {"nexel_preprocess", "nexel_render_fwd", "nexel_render_bwd"} <= names
    for n in names:
        assert hasattr(lib, n), n
    assert set(N_.EXPORTS) <= names


def test_status_strings(lib):
    assert N_.nexel_status_string(0) == "ok"
    assert N_.nexel_status_string(-3) == "instance capacity exceeded"
    assert N_.nexel_version() >= 100


def test_workspace_sizes_are_host_only(lib):
    cam = R.camera_struct(synth.front_camera(1280, 720))
    a = N_.nexel_workspace_size(cam, 300_000, 10_000_000)
    b = N_.nexel_workspace_size(cam, 300_000, 20_000_000)
    assert b > a > 300_000 * 80
    # 1920 x 1080 (13 tile bits) and 600k surfels (20 rank bits): the
    # instances are placed by tile with 32-bit keys holding the rank alone,
    # two 4-byte key buffers per instance (64-bit keys would take 16 B)
    big = R.camera_struct(synth.front_camera(1920, 1080))
    per_inst = (N_.nexel_workspace_size(big, 600_000, 20_000_000) -
                N_.nexel_workspace_size(big, 600_000, 10_000_000)) / 10_000_000
    assert 8 <= per_inst < 9, per_inst
    st = R.settings_struct(synth.Settings(K=4))
    f = N_.Field()
    f.L, f.T, f.F = 16, 1 << 19, 2
    assert N_.nexel_bwd_workspace_size(cam, st, f) >= 1280 * 720 * 4 * (8 + 32 * 4 + 16)


def test_invalid_arguments_rejected_before_launch(lib):
    cam = R.camera_struct(synth.front_camera(64, 64))
    bad = R.camera_struct(synth.front_camera(64, 64))
    bad.width = 0
    st = R.settings_struct(synth.Settings(K=2))
    n = C.c_longlong(0)
    assert lib.nexel_preprocess(C.byref(bad), C.byref(st), 1, *([None] * 7), 0, C.byref(n), None) == -1
    assert lib.nexel_preprocess(C.byref(cam), C.byref(st), 5, *([None] * 7), 0, C.byref(n), None) == -1
    st9 = R.settings_struct(synth.Settings(K=9))
    assert lib.nexel_preprocess(C.byref(cam), C.byref(st9), 0, *([None] * 7), 0, C.byref(n), None) == -1
    out = C.c_size_t(0)
    assert lib.nexel_workspace_size(C.byref(bad), 10, 10, C.byref(out)) == -1
    assert lib.nexel_workspace_size(C.byref(cam), -1, 10, C.byref(out)) == -1


def test_batched_calls_check_every_view_before_launch(lib):
    """The batched entry points validate all views' arguments first; a bad
    view anywhere in the batch returns NEXEL_ERR_INVALID_ARG with nothing
    launched (the fake device pointers below are never dereferenced)."""
    cams = [R.camera_struct(synth.front_camera(64, 48)), R.camera_struct(synth.front_camera(32, 32))]
    st = R.settings_struct(synth.Settings(K=0))
    N = 16
    fake = 1 << 20
    sizes = [N_.nexel_workspace_size(c, N, 1000) for c in cams]
    arr = (N_.Camera * 2)(*cams)
    P = lambda xs: (C.c_void_p * len(xs))(*xs)
    S = lambda xs: (C.c_size_t * len(xs))(*xs)
    params = [fake] * 6

    def fwd(n, cam_arr, ws_ptrs, ws_sizes):
        return lib.nexel_render_batch_fwd(n, cam_arr, C.byref(st), None, N, *params, ws_ptrs,
                                          ws_sizes, None, None, P([fake] * 2), P([fake] * 2),
                                          None, None, None, None, P([fake] * 2), None)

    assert fwd(0, arr, P([fake] * 2), S(sizes)) == -1
    assert fwd(2, None, P([fake] * 2), S(sizes)) == -1
    assert fwd(2, arr, P([fake, 0]), S(sizes)) == -1            # view 1 has no workspace
    assert fwd(2, arr, P([fake] * 2), S([sizes[0], 64])) == -1  # view 1's is too small
    bad = (N_.Camera * 2)(cams[0], cams[1])
    bad[1].width = 0
    assert fwd(2, bad, P([fake] * 2), S(sizes)) == -1
    assert lib.nexel_render_batch_bwd(2, arr, C.byref(st), None, N, *params[:5], P([fake] * 2),
                                      S(sizes), None, None, None, None, None, P([fake] * 2),
                                      None, None, None, 0, *([None] * 8), None) == -1  # no d_image
    assert lib.nexel_preprocess_async(C.byref(cams[0]), C.byref(st), N, *([None] * 6), fake,
                                      sizes[0], None) == -1
    assert lib.nexel_read_status(C.byref(cams[0]), C.byref(st), None, N, None, 0, None, 0,
                                 None) == -1


def test_densify_count_is_the_split_fraction_within_the_budget(lib):
    """nexel_densify_count (host only): 5 % of the surfels rounded up,
    capped by the budget (supp. Sec. 7.2), as the oracle's split_count."""
    from oracle import density as D
    out = C.c_int(-1)
    for N, budget in [(0, 10), (1, 10), (19, 100), (20, 100), (21, 100), (100, 1000),
                      (101, 1000), (100, 102), (100, 90), (300_000, 10**6),
                      (300_000, 300_001), (2_000_000_000 // 21, 1 << 40)]:
        assert lib.nexel_densify_count(N, C.c_longlong(budget), C.byref(out)) == 0
        assert out.value == D.split_count(N, budget), (N, budget, out.value)
    assert lib.nexel_densify_count(-1, C.c_longlong(10), C.byref(out)) == -1
    assert lib.nexel_densify_count(10, C.c_longlong(10), None) == -1


def test_objective_and_density_calls_check_arguments_before_launch(lib):
    """Argument errors of the objective, Adam and density entry points come
    back before any launch."""
    out = C.c_size_t(0)
    assert lib.nexel_loss_workspace_size(0, 10, C.byref(out)) == -1
    assert lib.nexel_density_workspace_size(-1, C.byref(out)) == -1
    assert lib.nexel_density_workspace_size(100, C.byref(out)) == 0 and out.value > 800
    fake = 1 << 20
    assert lib.nexel_fps(10, None, 5, None, None, None, None, None) == -1
    assert lib.nexel_fps(10, fake, 11, fake, fake, fake, None, None) == -1    # m > n
    n_sel = C.c_int(-7)
    assert lib.nexel_densify_select(-1, fake, fake, C.c_longlong(100), fake, 1 << 20, fake,
                                    C.byref(n_sel), None) == -1
    assert lib.nexel_densify_select(100, fake, fake, C.c_longlong(1000), fake, 16, fake,
                                    C.byref(n_sel), None) == -1  # small ws
    assert lib.nexel_densify_select(100, fake, fake, C.c_longlong(1000), fake, 1 << 20, fake,
                                    None, None) == -1  # no count output
    assert lib.nexel_densify_split(10, 2, fake, 5, *([fake] * 6), None) == -1      # color_dim
    assert lib.nexel_adam_step(1, None, None, None, None, None, None, C.c_float(0.9),
                               C.c_float(0.999), C.c_float(1e-8), 1, None) == -1
    sz = (C.c_longlong * 1)(10)
    lr = (C.c_float * 1)(0.1)
    ptrs = (C.c_void_p * 1)(fake)
    assert lib.nexel_adam_step(1, ptrs, ptrs, ptrs, ptrs, sz, lr, C.c_float(0.9),
                               C.c_float(0.999), C.c_float(1e-8), 0, None) == -1  # step 0


def test_tuning_round_trip_and_checks(lib):
    fields = ("tex_fwd_ctas_per_sm", "tex_bwd_ctas_per_sm", "f32_ctas_per_sm", "hash_block",
              "collect_batch", "tex_fwd_stages")
    t0 = N_.nexel_get_tuning()
    assert tuple(getattr(t0, f) for f in fields) == (2, 3, 2, 256, 256, 4)
    t = N_.Tuning(1, 1, 1, 128, 512, 2)
    N_.nexel_set_tuning(t)
    g = N_.nexel_get_tuning()
    assert tuple(getattr(g, f) for f in fields) == (1, 1, 1, 128, 512, 2)
    for bad in (N_.Tuning(0, 1, 1, 128, 256, 4), N_.Tuning(3, 1, 1, 128, 256, 4),
                N_.Tuning(1, 4, 1, 128, 256, 4), N_.Tuning(1, 1, 1, 64, 256, 4),
                N_.Tuning(1, 1, 1, 128, 64, 4), N_.Tuning(1, 1, 1, 128, 256, 1),
                N_.Tuning(1, 1, 1, 128, 256, 5)):
        assert lib.nexel_set_tuning(C.byref(bad)) == -1
    N_.nexel_set_tuning(t0)
    best = N_.Tuning()
    assert lib.nexel_autotune(None, None, None, 0, *([None] * 6), None, 0, None, 0, *([None] * 7),
                              None, *([None] * 8), 0, None, 0, C.byref(best), None, None) == -1


def test_stats_and_reduction_probe_check_arguments(lib):
    """nexel_render_stats and nexel_peak_l2_reductions reject bad arguments
    before any CUDA call (the fake device pointers are never used)."""
    cam = R.camera_struct(synth.front_camera(64, 64))
    st = R.settings_struct(synth.Settings(K=2))
    out = (C.c_longlong * 7)()
    assert lib.nexel_render_stats(C.byref(cam), C.byref(st), 10, None, 1 << 20, out, None) == -1
    assert lib.nexel_render_stats(C.byref(cam), C.byref(st), 10, 4096, 1 << 20, None, None) == -1
    assert lib.nexel_render_stats(C.byref(cam), C.byref(st), -1, 4096, 1 << 20, out, None) == -1
    g = C.c_float(0.0)
    assert lib.nexel_peak_l2_reductions(None, 1 << 20, 1000, 1, C.byref(g), None) == -1
    assert lib.nexel_peak_l2_reductions(4096, 1 << 20, 1000, 0, C.byref(g), None) == -1  # reps
    assert lib.nexel_peak_l2_reductions(4096, 1 << 20, 0, 1, C.byref(g), None) == -1  # no ops
    assert lib.nexel_peak_l2_reductions(4100, 1 << 20, 1000, 1, C.byref(g), None) == -1  # alignment
    assert lib.nexel_peak_l2_reductions(4096, 4, 1000, 1, C.byref(g), None) == -1  # < one entry
    assert lib.nexel_peak_l2_reductions(4096, 1 << 20, 1000, 1, None, None) == -1
