"""CUDA path (through the C ABI) against the FP64 oracle, element by element
on the same seeded inputs.  FP32 form: colours within 1e-5 absolute,
gradients within 1e-3 relative (per element, against 0.1 x the class's
largest magnitude at least), top-K ids and sort keys bit-exact.  Pixels
whose discrete choices lie within the FP32 path's resolution of a threshold
or a tie are excluded and counted (at most 5 % of the sampled pixels);
samples at a kink of the texture (a hash-cell face, a ReLU decision) keep
their pixel in the comparison with their texture gradient cancelled
(helpers.kink_cancelled_upstream).  Reduced-precision forms: colours within
2e-3 (BF16) / 1e-3 (FP16) of the oracle at the FP32 parameters; gradients
per element against the oracle evaluated at the parameters those forms read
(FP16 table, MLP weights rounded to the operand type), with the bound
derived from their rounding (see the constants below)."""
import functools

import numpy as np
import pytest

import oracle
from paper_2512_13796_gb300 import synth

from helpers import (UNIT_ROUNDOFF, compare_forward, compare_grads, grad_stats,
                     ill_conditioned, kink_cancelled_upstream, reference, reference_grads,
                     rounded_field, run_gpu)

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-5
GRAD_RTOL = 1e-3
MAX_TIE_FRAC = 0.05


@pytest.fixture(scope="module")
def dev():
    import torch
    assert torch.cuda.is_available(), "GPU test without a CUDA device"
    from paper_2512_13796_gb300 import _native
    _native.build()
    _native.lib()
    return torch.device("cuda:0")


def _report(name, stats):
    print(f"\n[{name}] " + " ".join(f"{k}={v:.3g}" if isinstance(v, float) else f"{k}={v}"
                                    for k, v in stats.items()))


def _backward_check(dev, w, cam, pix, ref, mlp, seed, cache=False, name=""):
    """Forward + backward on the GPU with kink-cancelled upstream gradients
    on the oracle's non-tie pixels, against the oracle's backward at the
    parameters the form reads; per-element comparison."""
    st = w.settings
    P, K = cam.width * cam.height, st.K
    dI, dW, dT, sel, us = kink_cancelled_upstream(ref, P, K, seed)
    grid = "f32" if mlp == "f32" else "f16"
    _, gg, _ = run_gpu(w.scene, cam, st, w.field, dev, grid=grid, mlp=mlp, d_image=dI,
                       d_weights=dW, d_textures=dT, cache_features=cache)
    gr, ga = reference_grads(w.scene, cam, st, w.field, sel, dI, dW, dT, mlp)
    skip = ill_conditioned(w.scene, cam)
    us["surfels_ill_conditioned"] = int(skip.size)
    _report(f"{name} upstream", us)
    _report(f"{name} grads", grad_stats(gg, gr))
    assert us["pix_compared"] >= (1 - MAX_TIE_FRAC) * us["pix"]
    return compare_grads(gg, gr, GRAD_RTOL, absolute=ga, u=UNIT_ROUNDOFF[mlp],
                         skip_surfels=skip)


@pytest.mark.parametrize("gamma", ["one", "var"])
def test_config0_forward(dev, gamma):
    w = synth.workload(0, gamma=gamma)
    cam, st = w.cameras[0], w.settings
    fw, _, _ = run_gpu(w.scene, cam, st, w.field, dev)
    ref = reference(w.scene, cam, st, w.field)
    s = compare_forward(fw, ref, st.K, TOL_F32)
    _report(f"config0 fwd gamma={gamma}", s)
    assert s["n_tie"] <= MAX_TIE_FRAC * s["n_pix"]


@pytest.mark.parametrize("gamma", ["one", "var"])
def test_config0_backward(dev, gamma):
    w = synth.workload(0, gamma=gamma)
    cam = w.cameras[0]
    ref = reference(w.scene, cam, w.settings, w.field)
    _backward_check(dev, w, cam, ref["pixels"], ref, "f32", seed=5,
                    name=f"config0 bwd gamma={gamma}")


@functools.lru_cache(maxsize=None)
def _sampled(idx, mlp="f32"):
    """Config 1 (800x800, 50k surfels) or 2 (1280x720, 300k surfels) with a
    fixed pixel sample (random pixels plus whole 16x16 tiles) and the
    oracle's forward on it for the given form."""
    w = synth.workload(idx, precision="f32")
    cam = w.cameras[0]
    pix = synth.pixel_sample(cam, 4096 if idx == 1 else 2048, 4 if idx == 1 else 3, seed=idx)
    return w, pix, reference(w.scene, cam, w.settings, w.field, pix, mlp=mlp)


@pytest.mark.parametrize("idx", [1, 2])
def test_fp32_forward_sampled(dev, idx):
    w, pix, ref = _sampled(idx)
    fw, _, _ = run_gpu(w.scene, w.cameras[0], w.settings, w.field, dev)
    s = compare_forward(fw, ref, w.settings.K, TOL_F32)
    _report(f"config{idx} fp32 fwd", s)
    assert s["n_tie"] <= MAX_TIE_FRAC * s["n_pix"]


@pytest.mark.parametrize("idx", [1, 2])
def test_fp32_backward_sampled(dev, idx):
    w, pix, ref = _sampled(idx)
    _backward_check(dev, w, w.cameras[0], pix, ref, "f32", seed=5 + idx,
                    name=f"config{idx} fp32 bwd")


# Reduced-precision forms: FP16 table, BF16 (or FP16) MLP on the tensor cores
# with FP32 accumulation.  Colours within 2e-3 per channel (BF16) of the FP64
# oracle at the FP32 parameters.
TOL_BF16 = 2e-3
TOL_F16 = 1e-3
# Gradients, per element, against the oracle at the parameters these forms
# read (FP16 table, weights rounded to the operand type), with the ReLU
# decisions the rounding may flip cancelled (RELU_TOL in helpers).  What
# remains is the rounding of the backward's operands: the texture gradient,
# the hidden-layer deltas, the features and the activations are each
# rounded to the operand type (unit roundoff u = 2^-8 for BF16, 2^-11 for
# FP16) before FP32-accumulated products, so every contribution to a
# gradient entry carries a relative error of at most ~3u (three roundings on
# its chain).  An entry's bound is therefore the FP32 one plus 4u times the
# sum of the magnitudes of its contributions (the oracle's absolute mode):
# |g - g_ref| <= 1e-3 max(|g_ref|, 0.1 scale) + 4 u sum|contributions|.
# A surfel seen nearly edge-on: its mu and quat gradients are left out of the
# 1e-3 comparison when |cos| of its normal to its centre ray is below 0.02
# (helpers.ill_conditioned; counted, everything else about it compared).


@pytest.mark.parametrize("mlp", ["bf16", "f16"])
@pytest.mark.parametrize("idx", [1, 2])
def test_reduced_precision_forward_sampled(dev, idx, mlp):
    w, pix, ref = _sampled(idx)
    fw, _, _ = run_gpu(w.scene, w.cameras[0], w.settings, w.field, dev, grid="f16", mlp=mlp)
    s = compare_forward(fw, ref, w.settings.K, TOL_BF16 if mlp == "bf16" else TOL_F16)
    _report(f"config{idx} {mlp} fwd", s)


@pytest.mark.parametrize("cache", [False, True], ids=["gather", "cached"])
@pytest.mark.parametrize("mlp", ["bf16", "f16"])
@pytest.mark.parametrize("idx", [1, 2])
def test_reduced_precision_backward_sampled(dev, idx, mlp, cache):
    """BF16 / FP16 backward, per element, with the features cached by the
    forward or gathered again by the backward (both then run the MLP
    backward and the weight gradients on tcgen05)."""
    w, pix, ref = _sampled(idx, mlp)
    _backward_check(dev, w, w.cameras[0], pix, ref, mlp, seed=8 + idx, cache=cache,
                    name=f"config{idx} {mlp} bwd {'cached' if cache else 'gather'}")


@pytest.mark.parametrize("idx", [1, 2])
def test_binning_order_bit_exact(dev, idx):
    """The per-tile lists are a stable sort of (tile, centre depth, index):
    bit-exact against a CPU sort of the same float32 keys; depths match the
    FP64 centre depth, and near-equal depths (key ties) are counted."""
    import torch
    from paper_2512_13796_gb300 import _native as N_
    from paper_2512_13796_gb300 import render as R
    w = synth.workload(idx, precision="f32")
    cam = w.cameras[0]
    fw, _, ws = run_gpu(w.scene, cam, w.settings, w.field, dev)
    n = fw["n_instances"]
    tiles = torch.empty(n, dtype=torch.int32, device=dev)
    ids = torch.empty(n, dtype=torch.int32, device=dev)
    dep = torch.empty(n, dtype=torch.float32, device=dev)
    N_.nexel_instance_list(R.camera_struct(cam), w.scene.n, ws.ws.data_ptr(), ws.ws.numel(), n,
                           tiles.data_ptr(), ids.data_ptr(), dep.data_ptr(),
                           torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    t, i, d = tiles.cpu().numpy(), ids.cpu().numpy(), dep.cpu().numpy()
    order = np.lexsort((i, d.view(np.uint32), t))
    assert np.array_equal(order, np.arange(n)), "instance list is not (tile, depth, id) sorted"
    M = cam.world_to_cam.astype(np.float64)
    z = w.scene.mu.astype(np.float64) @ M[2, :3] + M[2, 3]
    rel = np.abs(d - z[i]) / z[i]
    assert rel.max() < 1e-6
    zs = np.sort(z[z > cam.near])
    ties = int(np.sum(np.diff(zs) < 1e-6 * zs[1:]))
    print(f"\n[binning config{idx}] n_instances={n} mean tiles/surfel={n / w.scene.n:.2f} "
          f"max depth rel err={rel.max():.2e} key ties(1e-6)={ties}")
    # every surfel appears at most once per tile
    key = t.astype(np.int64) * (w.scene.n + 1) + i
    assert np.unique(key).size == n


def test_ragged_image_all_K(dev):
    """Image sizes that are not multiples of the 16x16 tile, every K."""
    sc = synth.make_scene(400, 3, 21, gamma="var")
    sc.scale *= 2.0
    fld = synth.make_field(4, 12, 2, (16,), 21, table_std=0.3)
    cam = synth.front_camera(37, 29)
    for K in range(0, 9):
        st = synth.Settings(K=K)
        fw, _, _ = run_gpu(sc, cam, st, fld if K else None, dev)
        ref = reference(sc, cam, st, fld if K else None)
        if K == 0:
            ok = ref["tie"] == 0
            e = np.abs(fw["image"].reshape(-1, 3)[ok] - ref["image"][ok]).max()
            assert e <= TOL_F32
        else:
            compare_forward(fw, ref, K, TOL_F32)


@pytest.mark.parametrize("mlp", ["f32", "bf16", "f16"])
def test_ragged_image_all_K_64_wide(dev, mlp):
    """The 16-64-3 MLP (chunked FP32 kernels, tcgen05 kernels) on an image
    that is not a multiple of the tile, every K from 1 to 8 (so every padded
    row count KP, and chunks of K floor(64 / K) samples): forward and
    backward against the oracle."""
    sc = synth.make_scene(400, 3, 22, gamma="var")
    sc.scale *= 2.0
    fld = synth.make_field(8, 12, 2, (64,), 22, table_std=0.3)
    cam = synth.front_camera(37, 29)
    grid = "f32" if mlp == "f32" else "f16"
    tol = {"f32": TOL_F32, "bf16": TOL_BF16, "f16": TOL_F16}[mlp]
    skip = ill_conditioned(sc, cam)
    P = cam.width * cam.height
    for K in range(1, 9):
        st = synth.Settings(K=K)
        ref = reference(sc, cam, st, fld)
        ref_b = ref if mlp == "f32" else reference(sc, cam, st, fld, mlp=mlp)
        dI, dW, dT, sel, _ = kink_cancelled_upstream(ref_b, P, K, seed=40 + K)
        fw, gg, _ = run_gpu(sc, cam, st, fld, dev, grid=grid, mlp=mlp, d_image=dI, d_weights=dW,
                            d_textures=dT, cache_features=(K % 2 == 0))
        compare_forward(fw, ref, K, tol)
        gr, ga = reference_grads(sc, cam, st, fld, sel, dI, dW, dT, mlp)
        compare_grads(gg, gr, GRAD_RTOL, absolute=ga, u=UNIT_ROUNDOFF[mlp], skip_surfels=skip)


def test_empty_and_culled_scenes(dev):
    """N = 0, and surfels all behind the camera: image = T_final bg = bg."""
    cam = synth.front_camera(40, 24)
    st = synth.Settings(K=2, bg=(0.25, 0.5, 0.75))
    fld = synth.make_field(4, 12, 2, (16,), 0)
    empty = synth.make_scene(1, 1, 0)
    empty = synth.Scene(*(getattr(empty, k)[:0] for k in ("mu", "quat", "scale", "opacity",
                                                          "gamma", "color")))
    fw, _, _ = run_gpu(empty, cam, st, fld, dev)
    np.testing.assert_array_equal(fw["image"], np.broadcast_to(np.float32(st.bg), fw["image"].shape))
    assert np.all(fw["ids"] == -1) and np.all(fw["T_final"] == 1.0)
    behind = synth.make_scene(50, 1, 3)
    behind.mu[:, 2] = -5.0  # camera at z = -3 looking along +z
    fw, _, _ = run_gpu(behind, cam, st, fld, dev)
    assert fw["n_instances"] == 0
    np.testing.assert_array_equal(fw["image"], np.broadcast_to(np.float32(st.bg), fw["image"].shape))


def test_capacity_growth(dev):
    """A workspace sized for too few instances returns the capacity error,
    the wrapper grows it and the result matches a large workspace."""
    from paper_2512_13796_gb300 import render as R
    w = synth.workload(0)
    ws = R.Workspace(dev, cap_hint=16)
    fw, _, _ = run_gpu(w.scene, w.cameras[0], w.settings, w.field, dev, ws=ws)
    assert ws.cap >= fw["n_instances"]
    fw2, _, _ = run_gpu(w.scene, w.cameras[0], w.settings, w.field, dev)
    for k in ("image", "ids", "weights"):
        np.testing.assert_array_equal(fw[k], fw2[k])


def test_deterministic_forward(dev):
    w = synth.workload(1)
    a, _, _ = run_gpu(w.scene, w.cameras[0], w.settings, w.field, dev)
    b, _, _ = run_gpu(w.scene, w.cameras[0], w.settings, w.field, dev)
    for k in ("image", "ids", "weights", "depths", "textures", "T_final"):
        np.testing.assert_array_equal(a[k], b[k])


@pytest.mark.parametrize("mlp", ["f32", "bf16"])
def test_recomputed_buffers_match_stored(dev, mlp):
    """Backward with I, W, D, T_final recomputed inside the backward (the
    memory-saving variant) gives the same gradients as the backward that
    reads the forward's saved buffers (up to the summation order of the
    float atomics)."""
    w = synth.workload(1)
    cam, st = w.cameras[0], w.settings
    P, K = cam.width * cam.height, st.K
    rng = np.random.default_rng(3)
    dI = rng.normal(size=(P, 3))
    dW = rng.normal(size=(P, K))
    grid = "f16" if mlp == "bf16" else "f32"
    _, g1, _ = run_gpu(w.scene, cam, st, w.field, dev, grid=grid, mlp=mlp, d_image=dI, d_weights=dW)
    _, g2, _ = run_gpu(w.scene, cam, st, w.field, dev, grid=grid, mlp=mlp, d_image=dI, d_weights=dW,
                       recompute=True)
    compare_grads(g2, g1, 1e-4)


@pytest.mark.parametrize("mlp", ["f32", "bf16"])
@pytest.mark.parametrize("recompute", [False, True])
def test_cached_features_match_gathered(dev, mlp, recompute):
    """A training step whose forward leaves the field features for the
    backward (cache_features) gives the same outputs and gradients as one
    whose backward gathers them again: the cached features are the very
    values the gather produces, so only the summation order of the float
    atomics differs (FP32 form: 1e-4 in the max metric; BF16 form, whose
    backward runs the same tcgen05 kernel either way: 1e-2 in relative L2,
    leaving room for the atomics' order through BF16-rounded operands)."""
    w = synth.workload(1)
    cam, st = w.cameras[0], w.settings
    P, K = cam.width * cam.height, st.K
    rng = np.random.default_rng(5)
    dI = rng.normal(size=(P, 3))
    dW = rng.normal(size=(P, K))
    dT = rng.normal(size=(P, K, 3))
    grid = "f16" if mlp == "bf16" else "f32"
    f1, g1, _ = run_gpu(w.scene, cam, st, w.field, dev, grid=grid, mlp=mlp, d_image=dI,
                        d_weights=dW, d_textures=dT, recompute=recompute)
    f2, g2, _ = run_gpu(w.scene, cam, st, w.field, dev, grid=grid, mlp=mlp, d_image=dI,
                        d_weights=dW, d_textures=dT, recompute=recompute, cache_features=True)
    for k in ("image", "weights", "ids", "textures", "T_final"):
        assert np.array_equal(f1[k], f2[k]), k
    if mlp == "f32":
        compare_grads(g2, g1, 1e-4)
    else:
        s = compare_grads(g2, g1, 1e-2, metric="l2")
        _report(f"cached vs gathered bf16 recompute={recompute}", s)


@pytest.mark.parametrize("idx", [0, 1])
def test_render_stats(dev, idx):
    """nexel_render_stats against the instance list (instances, visible
    surfels, per-tile list lengths) and, on the 64x64 view, against the
    oracle's composited counts: every pixel's last list position lies between
    the number of surfels it composited and its tile's list length."""
    import torch
    from paper_2512_13796_gb300 import _native as N_
    from paper_2512_13796_gb300 import render as R
    w = synth.workload(idx, precision="f32")
    cam = w.cameras[0]
    fw, _, ws = run_gpu(w.scene, cam, w.settings, w.field, dev)
    cam_s = R.camera_struct(cam)
    st_s = R.settings_struct(w.settings)
    stream = torch.cuda.current_stream().cuda_stream
    s = N_.nexel_render_stats(cam_s, st_s, w.scene.n, ws.ws.data_ptr(), ws.ws.numel(), stream)
    n = fw["n_instances"]
    assert s["instances"] == n
    tiles = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    ids = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    N_.nexel_instance_list(cam_s, w.scene.n, ws.ws.data_ptr(), ws.ws.numel(), n,
                           tiles.data_ptr(), ids.data_ptr(), None, stream)
    torch.cuda.synchronize()
    t, i = tiles.cpu().numpy()[:n], ids.cpu().numpy()[:n]
    tx, ty = (cam.width + 15) // 16, (cam.height + 15) // 16
    assert s["tiles"] == tx * ty
    assert s["visible_surfels"] == np.unique(i).size
    lens = np.bincount(t, minlength=tx * ty).astype(np.int64)
    pw = np.minimum(16, cam.width - 16 * (np.arange(tx * ty) % tx))
    ph = np.minimum(16, cam.height - 16 * (np.arange(tx * ty) // tx))
    assert s["pairs_full_lists"] == int(np.sum(lens * pw * ph))
    assert s["longest_list"] == int(lens.max())
    assert 0 < s["pairs_to_last"] <= s["pairs_bwd_walk"] <= s["pairs_full_lists"]
    if idx == 0:
        ref = oracle.render(w.scene, cam, w.settings, w.field)
        assert s["pairs_to_last"] >= int(ref["n_contrib"].sum())
    print(f"\n[stats config{idx}] {s}")


def _instance_order_checked(dev, scene, cam, st, field):
    """Forward through the C ABI, then the binned (tile, id, depth) sequence:
    a stable (tile, centre depth, id) order with every surfel at most once
    per tile.  Returns the forward outputs."""
    import torch
    from paper_2512_13796_gb300 import _native as N_
    from paper_2512_13796_gb300 import render as R
    fw, _, ws = run_gpu(scene, cam, st, field, dev)
    n = fw["n_instances"]
    assert n > 0
    tiles = torch.empty(n, dtype=torch.int32, device=dev)
    ids = torch.empty(n, dtype=torch.int32, device=dev)
    dep = torch.empty(n, dtype=torch.float32, device=dev)
    N_.nexel_instance_list(R.camera_struct(cam), scene.n, ws.ws.data_ptr(), ws.ws.numel(), n,
                           tiles.data_ptr(), ids.data_ptr(), dep.data_ptr(),
                           torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    t, i, d = tiles.cpu().numpy(), ids.cpu().numpy(), dep.cpu().numpy()
    order = np.lexsort((i, d.view(np.uint32), t))
    assert np.array_equal(order, np.arange(n)), "instance list is not (tile, depth, id) sorted"
    key = t.astype(np.int64) * (scene.n + 1) + i
    assert np.unique(key).size == n
    return fw


def test_tile_sort_path_beyond_placement_tiles(dev):
    """An image of more than 8192 16x16 tiles (1600 x 1400: 8800 tiles) with
    32-bit keys bins through the emit-and-sort path (the LSD tile sort): the
    order is the stable one and the forward matches the oracle."""
    scene = synth.make_scene(2000, 3, 41, gamma="var")
    cam = synth.front_camera(1600, 1400)
    st = synth.Settings(K=2)
    field = synth.make_field(4, 12, 2, (16,), 3)
    fw = _instance_order_checked(dev, scene, cam, st, field)
    pix = synth.pixel_sample(cam, 2048, 2, seed=3)
    ref = reference(scene, cam, st, field, pix)
    _report("tile-sort path fwd", compare_forward(fw, ref, st.K, TOL_F32))


def test_placement_with_rank_only_keys(dev):
    """530k surfels on a 1920 x 1080 view (8160 tiles: 13 tile bits and 20
    rank bits, more than 32): the instances are still placed by tile, with
    keys that hold the depth rank alone (the slot gives the tile); the
    binned order is the stable (tile, depth, id) one, every surfel appears
    once per tile, and the forward matches the oracle."""
    scene = synth.make_scene(530_000, 12, 47, room=True, gamma="var")
    cam = synth.front_camera(1920, 1080)
    st = synth.Settings(K=2)
    field = synth.make_field(4, 12, 2, (16,), 7)
    fw = _instance_order_checked(dev, scene, cam, st, field)
    pix = synth.pixel_sample(cam, 384, 1, seed=8)
    ref = reference(scene, cam, st, field, pix)
    _report("rank-only placed keys fwd", compare_forward(fw, ref, st.K, TOL_F32))


def test_tile_sort_with_64_bit_keys(dev):
    """More than 8192 tiles (1600 x 1400: 8800 tiles, 14 bits) and 270k
    surfels (19 rank bits): the emit-and-sort path with 64-bit (tile, rank)
    keys; the order is the stable one and the forward matches the oracle."""
    scene = synth.make_scene(270_000, 12, 49, room=True, gamma="var")
    cam = synth.front_camera(1600, 1400)
    st = synth.Settings(K=2)
    field = synth.make_field(4, 12, 2, (16,), 9)
    fw = _instance_order_checked(dev, scene, cam, st, field)
    pix = synth.pixel_sample(cam, 384, 1, seed=10)
    ref = reference(scene, cam, st, field, pix)
    _report("64-bit tile sort fwd", compare_forward(fw, ref, st.K, TOL_F32))


def test_placement_with_tile_decisions_tested_again(dev):
    """Surfels so large on screen that their stored tile decisions overflow
    the room of 8 words per surfel (up to 113 words each on a 1280 x 720
    view): the later ones are tested again during the direct placement, and
    the order and the forward still match."""
    import dataclasses
    base = synth.make_scene(300, 2, 43, gamma="one")
    scene = dataclasses.replace(base, scale=(base.scale * 8.0).astype(np.float32))
    cam = synth.front_camera(1280, 720)
    st = synth.Settings(K=2)
    field = synth.make_field(4, 12, 2, (16,), 3)
    fw = _instance_order_checked(dev, scene, cam, st, field)
    # far more decision words than the room holds: ~3600 tiles per surfel
    assert fw["n_instances"] > 300 * 8 * 32
    pix = synth.pixel_sample(cam, 2048, 2, seed=4)
    ref = reference(scene, cam, st, field, pix)
    _report("placement with re-tested tiles fwd", compare_forward(fw, ref, st.K, TOL_F32))


def test_placement_retested_across_rank_blocks(dev):
    """Large surfels in several 1024-rank blocks of the direct placement
    (2600 of them: three blocks), enough that their stored tile decisions
    overflow the room and are tested again during the placement, where each
    block's instances start at its per-block prefix from the column scan:
    the order is the stable (tile, depth, id) one, every surfel appears once
    per tile, and the forward matches the oracle."""
    import dataclasses
    base = synth.make_scene(2600, 4, 45, gamma="one")
    scene = dataclasses.replace(base, scale=(base.scale * 6.0).astype(np.float32))
    cam = synth.front_camera(1280, 720)
    st = synth.Settings(K=2)
    field = synth.make_field(4, 12, 2, (16,), 5)
    fw = _instance_order_checked(dev, scene, cam, st, field)
    assert fw["n_instances"] > 2600 * 8 * 32
    pix = synth.pixel_sample(cam, 2048, 2, seed=6)
    ref = reference(scene, cam, st, field, pix)
    _report("placement across rank blocks fwd", compare_forward(fw, ref, st.K, TOL_F32))
