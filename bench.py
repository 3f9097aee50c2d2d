"""Benchmark of the Nexels hot path on one GB300 (and N replicas).

A step is one pass of the whole differentiable image formation over one
view: preprocess + binning + sort, collection pass, texturing pass (hash
gather + MLP + composite), and the full backward (MLP and hash-grid
backward, collection backward, preprocess backward), with the inputs
resident in HBM.  The loss and the optimizer are outside the step.

Workload: 300k surfels (box room + facades), 1280x720, K = 4, hash grid
16 levels x 2^19 x 2, MLP 32 -> 64 -> 64 -> 3; the BF16 form (FP16 table,
BF16 tensor-core MLP, FP32 accumulation) is the headline and the FP32 form
is reported beside it, together with render FPS (forward only) for both.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "train-step Mpix/s and render FPS, 300k surfels 720p K=4, BF16 vs FP32 path"
WORKLOAD = "config2: 300k surfels (box room + facades), 1280x720, K=4, hash 16x2^19x2, MLP 32-64-64-3"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed
    region (read only)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            # raw samples: NEXEL_CLOCKS_DIR when set, else the temp directory
            out_dir = os.environ.get("NEXEL_CLOCKS_DIR") or tempfile.gettempdir()
            os.makedirs(out_dir, exist_ok=True)
            self.path = os.path.join(out_dir, f"nexel_clocks_rank{self.idx}_{os.getpid()}.csv")
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        # nvidia-smi takes a moment to start: wait (at most 5 s) for its
        # first sample so that the samples cover the timed region
        t0 = time.time()
        while time.time() - t0 < 5.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# --------------------------------------------------------------- workload
class Job:
    """Device-resident inputs and workspaces of one form (bf16 or f32)."""

    def __init__(self, w, dev, precision: str, sh: bool = False):
        import torch
        from paper_2512_13796_gb300 import render as R
        from paper_2512_13796_gb300 import synth
        self.R = R
        self.precision = precision
        grid, mlp = {"bf16": ("f16", "bf16"), "f16": ("f16", "f16"),
                     "f32": ("f32", "f32")}[precision]
        self.cam, self.st = w.cameras[0], w.settings
        self.cam_s = R.camera_struct(self.cam)
        shd = 3 if sh else 0
        self.st_s = R.settings_struct(self.st, grid, mlp, sh_degree=shd)
        # a training step: the forward leaves the field features for the backward
        self.st_train = R.settings_struct(self.st, grid, mlp, cache_features=True, sh_degree=shd)
        self.p = {k: torch.from_numpy(np.ascontiguousarray(getattr(w.scene, k))).to(dev)
                  for k in ("mu", "quat", "scale", "opacity", "gamma", "color")}
        field = w.field
        if sh:
            # the paper's configuration: degree-3 SH for both appearance modes
            # (48 colour coefficients per surfel, 48 MLP outputs)
            self.p["color"] = torch.from_numpy(synth.sh_coefficients(w.scene.n, 2)).to(dev)
            field = synth.make_field(w.field.L, int(np.log2(w.field.T)), w.field.F,
                                     tuple(w.field.widths[1:-1]), 2, out_dim=48)
        self.field = R.DeviceField.from_synth(field, dev, grid, mlp)
        self.ts = self.field.storage_table()
        self.wts = self.field.weights
        self.ws = R.Workspace(dev, cap_hint=32 << 20)
        H, W = self.cam.height, self.cam.width
        g = torch.Generator(device="cpu").manual_seed(123)
        self.d_image = (torch.randn(H, W, 3, generator=g) * 1e-3).to(dev)
        self.N = w.scene.n
        self.grads = None
        self.fwd_out = None

    def forward(self, st_s=None):
        p = self.p
        self.fwd_out = self.R.forward(self.ws, self.cam_s, st_s or self.st_s, self.field, self.ts,
                                      self.wts, p["mu"], p["quat"], p["scale"], p["opacity"],
                                      p["gamma"], p["color"])
        return self.fwd_out

    def full_step(self):
        """A whole training iteration: forward, the paper's objective
        (nexel_loss_image / _params) against a fixed target, backward, and
        the Adam step over every parameter (learning rates 0, so the timed
        workload stays the same from step to step; the arithmetic is the
        same), plus the FP16 refresh of the table's storage copy."""
        R, p = self.R, self.p
        if not hasattr(self, "objective"):
            import torch
            H, W = self.cam.height, self.cam.width
            g = torch.Generator(device="cpu").manual_seed(321)
            self.target = torch.rand(H, W, 3, generator=g).to(self.d_image.device)
            self.objective = R.Objective(W, H, self.d_image.device)
            ts = [p[k] for k in ("mu", "quat", "scale", "opacity", "gamma", "color")]
            self.adam = R.Adam(ts + [self.field.table, self.field.weights], [0.0] * 8)
        out = self.forward(self.st_train)
        d_img, d_w, d_t = self.objective.image_terms(out["image"], self.target, out["weights"],
                                                     out["textures"])
        g = self.R.backward(self.ws, self.cam_s, self.st_train, self.field, self.ts, self.wts,
                            p["mu"], p["quat"], p["scale"], p["opacity"], p["gamma"], out,
                            d_img, d_w, d_t, grads=self.grads)
        self.grads = g
        self.objective.param_terms(p["opacity"], self.field, g["opacity"], g["table"])
        self.adam.step([g[k] for k in ("mu", "quat", "scale", "opacity", "gamma", "color",
                                       "table", "mlp")])
        self.ts.copy_(self.field.table)
        return out

    def autotune(self, flush_buf) -> dict:
        """nexel_autotune on this form's training step, every timed step
        after an L2 flush as in the timed regions; the choice stays set for
        the rest of the run (all forms)."""
        import torch
        R, p = self.R, self.p
        out = self.forward(self.st_train)
        N_ = R.N_
        fs = self.field.struct(self.ts, self.wts)
        bws = self.ws.bwd(self.cam_s, self.st_train, fs)
        g = self.R.backward(self.ws, self.cam_s, self.st_train, self.field, self.ts, self.wts,
                            p["mu"], p["quat"], p["scale"], p["opacity"], p["gamma"], out,
                            self.d_image)
        best, ms = N_.nexel_autotune(
            self.cam_s, self.st_train, fs, self.N,
            [p[k].data_ptr() for k in ("mu", "quat", "scale", "opacity", "gamma", "color")],
            self.ws.ws.data_ptr(), self.ws.ws.numel(), bws.data_ptr(), bws.numel(),
            [out[k].data_ptr() for k in ("image", "notex", "weights", "ids", "depths",
                                         "textures", "T_final")], self.d_image.data_ptr(),
            [g[k].data_ptr() for k in ("mu", "quat", "scale", "opacity", "gamma", "color",
                                       "table", "mlp")], 5, torch.cuda.current_stream().cuda_stream,
            flush_buf.data_ptr(), flush_buf.numel())
        return {"tex_fwd_ctas_per_sm": best.tex_fwd_ctas_per_sm,
                "tex_bwd_ctas_per_sm": best.tex_bwd_ctas_per_sm,
                "f32_ctas_per_sm": best.f32_ctas_per_sm, "hash_block": best.hash_block,
                "collect_batch": best.collect_batch, "tex_fwd_stages": best.tex_fwd_stages,
                "tuned_step_ms": ms}

    def step(self, st_s=None):
        st_s = st_s or self.st_train
        out = self.forward(st_s)
        p = self.p
        self.grads = self.R.backward(self.ws, self.cam_s, st_s, self.field, self.ts,
                                     self.wts,
                                     p["mu"], p["quat"], p["scale"], p["opacity"], p["gamma"], out,
                                     self.d_image, grads=self.grads)
        return out


class BatchJob:
    """The batched form: one training step over 8 views of uneven resolution
    of a 600k-surfel scene (BF16 form), captured in one CUDA graph, beside
    the same views through the single-view calls one after another."""
    WORKLOAD = ("config3: 600k surfels, 8 views 640x480..1920x1080 (8.6 Mpix), K=4, "
                "hash 16x2^19x2 FP16, MLP 32-64-64-3 BF16")

    def __init__(self, dev):
        import torch
        from paper_2512_13796_gb300 import render as R
        from paper_2512_13796_gb300 import synth
        self.R = R
        w = synth.workload(3)
        self.w = w
        self.p = {k: torch.from_numpy(np.ascontiguousarray(getattr(w.scene, k))).to(dev)
                  for k in ("mu", "quat", "scale", "opacity", "gamma", "color")}
        self.field = R.DeviceField.from_synth(w.field, dev, "f16", "bf16")
        self.step = R.BatchStep(w.cameras, w.settings, self.field, self.p)
        g = torch.Generator(device="cpu").manual_seed(7)
        for d in self.step.d_image:
            d.copy_(torch.randn(d.shape, generator=g) * 1e-3)
        self.step.capture()
        self.pixels = self.step.pixels
        # the single-view path
        self.ts = self.field.storage_table()
        self.ws = [R.Workspace(dev, cap_hint=n + 4096) for n in self.step.n_instances]
        self.cam_s = [R.camera_struct(c) for c in w.cameras]
        self.st_s = R.settings_struct(w.settings, "f16", "bf16", cache_features=True)
        self.grads = None

    def replay(self):
        self.step.replay()

    def sequential(self):
        R, p = self.R, self.p
        for v, cs in enumerate(self.cam_s):
            out = R.forward(self.ws[v], cs, self.st_s, self.field, self.ts, self.field.weights,
                            p["mu"], p["quat"], p["scale"], p["opacity"], p["gamma"], p["color"])
            self.grads = R.backward(self.ws[v], cs, self.st_s, self.field, self.ts,
                                    self.field.weights, p["mu"], p["quat"], p["scale"],
                                    p["opacity"], p["gamma"], out, self.step.d_image[v],
                                    accumulate=v > 0, grads=self.grads)


def max_over_ranks(x: float, device, world: int) -> float:
    """The slowest rank's value (the job's time): an all-reduce MAX over the
    process group when there is more than one rank."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mpix(pixels_per_rank: int, ms_max: float, world: int) -> float:
    """Replicas (weak scaling): every rank renders its own view in the
    slowest rank's time, so the job's throughput is world x pixels / time."""
    return world * pixels_per_rank / (ms_max * 1e-3) / 1e6


def timed(fn, steps, flush, stream):
    """Per-step CUDA-event times (ms) with an L2 flush before each step."""
    import torch
    times = []
    for _ in range(steps):
        flush()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        times.append((a, b))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in times]


def measured_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` on `workload` from the ncu capture
    recorded in profiles/dram_traffic.txt, or None when there is none or the
    kernel's source file has changed since (its SHA-1 no longer matches)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        f = line.split()
        if len(f) < 5 or line.startswith("#") or f[0] != kernel or f[1] != workload:
            continue
        src = os.path.join(ROOT, f[3])
        if not os.path.exists(src):
            return None
        if hashlib.sha1(open(src, "rb").read()).hexdigest() != f[4]:
            return None
        return int(f[2])
    return None


def roofline(prof: dict, job: Job, peaks: dict, peak_kind: str, n_steps: int, workload: str,
             kernel: str | None = None, as_name: str | None = None):
    """Roofline entry of the dominant kernel (or of `kernel`) from live
    per-kernel events; `as_name` selects the accounting (e.g. the tcgen05
    backward counted in MMA FLOPs)."""
    if kernel is None:
        name, (ms_tot, launches) = max(prof.items(), key=lambda kv: kv[1][0])
    else:
        name, (ms_tot, launches) = kernel, prof[kernel]
    label = name
    name = as_name or name
    ms = ms_tot / max(launches, 1)
    w = job
    P = w.cam.width * w.cam.height
    K = w.st.K
    L, F = w.field.L, w.field.F
    b_entry = 2 if w.precision == "bf16" else 4
    out = {"kernel": label, "ms_per_launch": ms, "launches": launches}
    samples = int((w.fwd_out["ids"] >= 0).sum().item()) if w.fwd_out is not None else P * K
    if name == "texture_bwd_tc_flops":
        # the tcgen05 MLP backward in algorithmic MMA FLOPs per sample row:
        # forward recompute, input-side deltas and weight gradients
        widths = w.field.widths
        macs = sum(widths[i] * widths[i + 1] for i in range(len(widths) - 1))
        rows = ((P * (1 << (K - 1).bit_length()) + 15) // 16) * 16
        A = rows * 2 * macs * 3 / (ms * 1e-3) / 1e12
        pk = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
        out.update(bound="tensor", achieved=A, peak=pk, unit="TFLOP/s",
                   peak_source=f"bf16_tflops_sustained ({peak_kind})", units_per_launch=rows,
                   flop_per_unit=2 * macs * 3)
        out["frac"] = A / pk
    elif name.startswith("texture_fwd") or name.startswith("texture_bwd"):
        # algorithmic bytes: the table entries the gather reads (8 corners x
        # L levels x F features), plus, in the backward, an FP32 read-modify-
        # write of the same entries in the table gradient
        per = L * 8 * F * b_entry + (L * 8 * F * 4 * 2 if "bwd" in name else 0)
        A = samples * per / (ms * 1e-3) / 1e9
        out.update(bound="hbm", achieved=A, peak=peaks["hbm_gbs"], unit="GB/s",
                   peak_source=f"hbm_gbs ({peak_kind})", units_per_launch=samples,
                   bytes_per_unit=per)
        out["frac"] = A / out["peak"]
    elif name.startswith("hash_bwd"):
        # algorithmic bytes per textured sample, as for the gather: the table
        # entries read for dL/dD (L levels x 8 corners x F in the storage
        # type) plus the same entries of the FP32 table gradient added to
        per = L * 8 * F * (b_entry + 4)
        A = samples * per / (ms * 1e-3) / 1e9
        out.update(bound="hbm", achieved=A, peak=peaks["hbm_gbs"], unit="GB/s",
                   peak_source=f"hbm_gbs ({peak_kind})", units_per_launch=samples,
                   bytes_per_unit=per)
        out["frac"] = A / out["peak"]
    elif name.startswith("mlp_wgrad"):
        widths = w.field.widths
        macs = sum(widths[i] * widths[i + 1] for i in range(len(widths) - 1))
        rows = ((P * (1 << (K - 1).bit_length()) + 15) // 16) * 16
        flop = rows * 2 * macs * 3  # forward recompute, input-side deltas, weight gradient
        A = flop / (ms * 1e-3) / 1e12
        pk = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
        out.update(bound="tensor", achieved=A, peak=pk, unit="TFLOP/s",
                   peak_source=f"bf16_tflops_sustained ({peak_kind})", units_per_launch=rows,
                   flop_per_unit=2 * macs * 3)
        out["frac"] = A / pk
    else:
        # sort / scan / collection kernels: report bytes moved per launch
        # against the HBM peak (algorithmic bytes set by the caller)
        out.update(bound="hbm", achieved=None, peak=peaks["hbm_gbs"], unit="GB/s", frac=None)
    out["traffic"] = measured_traffic(label, workload)
    return out


def key_layout(N: int, width: int, height: int) -> dict:
    """The binning's key layout for N surfels on a width x height view (as
    the library derives it): 16 x 16 tiles; direct placement for at most
    8192 tiles, with 32-bit (tile, depth rank) keys when tile and rank bits
    fit and keys holding the rank alone otherwise; beyond 8192 tiles the LSD
    tile sort, with 64-bit keys when the bits do not fit."""
    tiles = ((width + 15) // 16) * ((height + 15) // 16)
    tile_bits = max(1, (tiles - 1).bit_length())
    rank_bits = max(1, (N - 1).bit_length())
    placement = tiles <= 8192
    fits32 = tile_bits + rank_bits <= 32
    return {"tiles": tiles, "tile_bits": tile_bits, "key64": (not placement) and not fits32,
            "rank_only": placement and not fits32, "placement": placement,
            "tile_passes": (tile_bits + 7) // 8}


def sort_rooflines(prof: dict, steps: int, N: int, n_inst: int, layout: dict, peaks: dict,
                   peak_kind: str) -> dict:
    """HBM roofline of the binning's sorts, from live per-kernel events.
    The depth sort: N (key, value) pairs, 4 passes of 8 bits; per pair and
    pass the histogram reads the 4 B key and the scatter reads and writes
    key and value: 20 B.  The LSD tile sort (64-bit keys or more than 8192
    tiles): n_inst keys, ceil(tile_bits / 8) passes, 3 key widths per key
    and pass.  The direct placement's writer: 4 B key written per instance
    and 16 B of rank data read per surfel (its stored tile decisions are
    the library's own cache and not counted)."""
    out = {}
    hb = peaks["hbm_gbs"]
    t_sort = sum(prof[k][0] for k in ("radix_hist", "radix_scatter") if k in prof) / steps
    if t_sort > 0:
        kb = 8 if layout["key64"] else 4
        tile_b = 0 if layout["placement"] else n_inst * layout["tile_passes"] * 3 * kb
        by = N * 4 * 20 + tile_b
        A = by / (t_sort * 1e-3) / 1e9
        out["radix_sort"] = {
            "kernel": "radix_hist + radix_scatter", "ms_per_step": t_sort, "bound": "hbm",
            "achieved": A, "peak": hb, "unit": "GB/s", "frac": A / hb,
            "peak_source": f"hbm_gbs ({peak_kind})", "bytes_per_step": by,
            "keys": {"depth_sort": N, "tile_sort": 0 if layout["placement"] else n_inst},
            "passes": {"depth_sort": 4, "tile_sort": 0 if layout["placement"]
                       else layout["tile_passes"]},
            "mean_tiles_per_surfel": n_inst / max(N, 1)}
    if "place_write" in prof:
        t = prof["place_write"][0] / steps
        by = n_inst * 4 + N * 16
        A = by / (t * 1e-3) / 1e9
        out["place_write"] = {
            "kernel": "place_write", "ms_per_step": t, "bound": "hbm", "achieved": A,
            "peak": hb, "unit": "GB/s", "frac": A / hb, "peak_source": f"hbm_gbs ({peak_kind})",
            "bytes_per_step": by, "instances": n_inst,
            "note": "the writer is bound by its shared-memory rank masks, not by HBM"}
    return out


def config1_leg(dev, steps, flush, stream, agg) -> dict:
    """Config 1 (50k surfels, 800x800, K = 4, hash 8 x 2^16 x 2, MLP 16-64-3):
    the BF16 and FP32 train steps and render FPS."""
    from paper_2512_13796_gb300 import synth
    w = synth.workload(1)
    P = w.cameras[0].width * w.cameras[0].height
    out = {"workload": "config1: 50k surfels (10 planes), 800x800, K=4, hash 8x2^16x2, "
                       "MLP 16-64-3"}
    for prec in ("bf16", "f32"):
        j = Job(w, dev, prec)
        for _ in range(3):
            j.step()
        t = agg(timed(j.step, steps, flush, stream))
        f = agg(timed(j.forward, steps, flush, stream))
        out[prec] = {"train_mpix_s": P / (t * 1e-3) / 1e6, "train_ms": t,
                     "render_fps": 1e3 / f, "render_ms": f}
        del j
    return out


def config4_leg(dev, steps, flush, stream, agg, peaks, peak_kind) -> dict:
    """Config 4 (1M surfels, 1920x1080, K = 8, hash 16 x 2^20 x 2 FP16, BF16
    MLP): the train step with the per-pixel buffers I, W, D, T_final stored
    between forward and backward against the one that recomputes them in
    the backward (time, and the memory each holds), and the inference-only
    render FPS."""
    import torch
    from paper_2512_13796_gb300 import render as R
    from paper_2512_13796_gb300 import synth
    w = synth.workload(4)
    cam = w.cameras[0]
    P, K = cam.width * cam.height, w.settings.K
    j = Job(w, dev, "bf16")
    st_rc = R.settings_struct(w.settings, "f16", "bf16", recompute=True, cache_features=True)
    res = {"workload": "config4: 1M surfels (box room + facades), 1920x1080, K=8, "
                       "hash 16x2^20x2 FP16, MLP 32-64-64-3 BF16"}
    fs = j.field.struct(j.ts, j.wts)
    from paper_2512_13796_gb300 import _native as N_
    bws_stored = N_.nexel_bwd_workspace_size(j.cam_s, j.st_train, fs)
    bws_rc = N_.nexel_bwd_workspace_size(j.cam_s, st_rc, fs)
    for name, st_s in (("stored", j.st_train), ("recompute", st_rc)):
        for _ in range(3):
            j.step(st_s)
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats(dev)
        base = torch.cuda.memory_allocated(dev)
        t = agg(timed(lambda: j.step(st_s), steps, flush, stream))
        peak = torch.cuda.max_memory_allocated(dev)
        res[name] = {"train_ms": t, "train_mpix_s": P / (t * 1e-3) / 1e6,
                     "peak_allocated_bytes": int(peak), "resident_before_step_bytes": int(base)}
    res["stored"]["held_between_fwd_and_bwd_bytes"] = P * K * (4 + 4 + 4) + P * 4
    res["recompute"]["held_between_fwd_and_bwd_bytes"] = 0
    res["stored"]["bwd_scratch_bytes"] = bws_stored
    res["recompute"]["bwd_scratch_bytes"] = bws_rc
    res["memory_note"] = ("held_between_fwd_and_bwd: the weights W, ids I, depths D [H][W][K] "
                          "and T_final the stored variant's backward reads; the recompute "
                          "variant's backward rebuilds them in its own scratch (bwd_scratch "
                          "grows by that much), so a caller may drop or reuse the forward's "
                          "copies once the loss has read them")
    for _ in range(3):
        j.forward()
    f = agg(timed(j.forward, steps, flush, stream))
    res["render"] = {"fps": 1e3 / f, "ms": f, "mpix_s": P / (f * 1e-3) / 1e6,
                     "note": "inference forward only (preprocess, binning, collection, texturing, "
                             "composite), no feature cache"}
    N_.nexel_profile_enable(True)
    timed(lambda: j.step(j.st_train), 3, flush, stream)
    prof = N_.nexel_profile_read()
    N_.nexel_profile_enable(False)
    n_inst = j.fwd_out["n_instances"]
    lay = key_layout(w.scene.n, cam.width, cam.height)
    res["binning"] = {"instances": int(n_inst), "key64": lay["key64"],
                      "path": "direct placement" if lay["placement"] else "LSD tile sort"}
    res["rooflines"] = sort_rooflines(prof, 3, w.scene.n, n_inst, lay, peaks, peak_kind)
    del j
    torch.cuda.empty_cache()
    return res


def cpu_baseline(w, seconds_target: float = 15.0) -> dict:
    """The FP64 oracle as it stands, forward + backward on a pixel sample of
    the same view, on this host's cores."""
    import oracle
    from paper_2512_13796_gb300 import synth
    cam, st = w.cameras[0], w.settings
    n = 256
    t_used = 0.0
    done = 0
    rng_seed = 0
    while t_used < seconds_target and n <= 65536:
        pix = synth.pixel_sample(cam, n, 0, seed=rng_seed)
        t0 = time.perf_counter()
        oracle.render(w.scene, cam, st, w.field, pix)
        dI = np.ones((pix.size, 3)) * 1e-3
        oracle.render_bwd(w.scene, cam, st, w.field, pix, dI)
        dt = time.perf_counter() - t0
        t_used += dt
        done += pix.size
        rng_seed += 1
        if dt < seconds_target / 4:
            n *= 2
    return {"value": done / t_used / 1e6, "unit": "Mpix/s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"{done} random pixels of the 1280x720 view, forward + backward, FP64 "
                      f"brute force over all 300k surfels ({t_used:.1f} s)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="nexels", choices=["nexels", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-json", default=None, help="write per-kernel times here")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes instead of nexel_autotune's choice")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched 8-view form (600k surfels)")
    ap.add_argument("--config", type=int, default=2, choices=[1, 2],
                    help="2: the headline workload; 1: the 50k-surfel 800x800 case (profiling)")
    ap.add_argument("--no-config1", action="store_true",
                    help="skip the 50k-surfel 800x800 (config 1) train-step line")
    ap.add_argument("--no-config4", action="store_true",
                    help="skip the 1M-surfel 1080p K=8 (config 4) leg")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    from paper_2512_13796_gb300 import synth

    if args.impl == "reference":
        # the oracle, timed on the host: rank 0 only
        if rank != 0:
            return
        w = synth.workload(2)
        import oracle
        cam, st = w.cameras[0], w.settings
        per_step = 512
        for k in range(args.warmup):
            pix = synth.pixel_sample(cam, 64, 0, seed=1000 + k)
            oracle.render(w.scene, cam, st, w.field, pix)
        t = []
        for k in range(args.steps):
            pix = synth.pixel_sample(cam, per_step, 0, seed=k)
            t0 = time.perf_counter()
            oracle.render(w.scene, cam, st, w.field, pix)
            oracle.render_bwd(w.scene, cam, st, w.field, pix, np.ones((pix.size, 3)) * 1e-3)
            t.append(time.perf_counter() - t0)
        v = per_step * args.steps / sum(t) / 1e6
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mpix/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * sum(t) / len(t), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "sample": f"{per_step} pixels per step"},
                "cpu_baseline": {"value": v, "unit": "Mpix/s", "cores": os.cpu_count(),
                                 "kind": "oracle",
                                 "sample": f"{per_step} random pixels per step, forward + "
                                           "backward, FP64 brute force"},
                "e2e": {"value": v, "unit": "Mpix/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2512_13796_gb300 import _native
    _native.build()
    _native.lib()
    stream = torch.cuda.current_stream()
    peaks, peak_kind = load_peaks()
    w = synth.workload(args.config)
    jobs = {"bf16": Job(w, dev, "bf16"), "f32": Job(w, dev, "f32"), "f16": Job(w, dev, "f16"),
            "sh_f16": Job(w, dev, "f16", sh=True)}
    P = w.cameras[0].width * w.cameras[0].height
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def flush():
        flush_buf.zero_()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for j in jobs.values():
        for _ in range(max(args.warmup, 3)):
            j.step()
    barrier()
    tuning = None
    if not args.no_autotune:
        tuning = jobs["bf16"].autotune(flush_buf)

    results = {}
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = _native.nexel_launch_count()
    t_train = timed(jobs["bf16"].step, args.steps, flush, stream)
    launches = (_native.nexel_launch_count() - launches0) // args.steps
    barrier()
    results["bf16_train"] = t_train
    results["f32_train"] = timed(jobs["f32"].step, args.steps, flush, stream)
    results["bf16_fwd"] = timed(jobs["bf16"].forward, args.steps, flush, stream)
    results["f32_fwd"] = timed(jobs["f32"].forward, args.steps, flush, stream)
    results["f16_train"] = timed(jobs["f16"].step, args.steps, flush, stream)
    results["f16_fwd"] = timed(jobs["f16"].forward, args.steps, flush, stream)
    results["sh_f16_train"] = timed(jobs["sh_f16"].step, args.steps, flush, stream)
    results["sh_f16_fwd"] = timed(jobs["sh_f16"].forward, args.steps, flush, stream)
    for _ in range(3):
        jobs["bf16"].full_step()
    results["bf16_full"] = timed(jobs["bf16"].full_step, args.steps, flush, stream)
    barrier()
    clk = clocks.stop()  # samples over all four timed regions
    # per-kernel CUDA events on the launch stream, same steps again
    _native.nexel_profile_enable(True)
    results["bf16_train_profiled"] = timed(jobs["bf16"].step, args.steps, flush, stream)
    prof = _native.nexel_profile_read()
    _native.nexel_profile_enable(True)
    results["f32_train_profiled"] = timed(jobs["f32"].step, args.steps, flush, stream)
    prof_f32 = _native.nexel_profile_read()
    _native.nexel_profile_enable(False)

    def agg(ts):
        # the median of the timed steps (the measurement plan's statistic),
        # the slowest rank's
        return max_over_ranks(float(np.median(ts)), dev, world)

    ms = {k: agg(v) for k, v in results.items()}

    # end to end through the public API: target image H2D from pinned memory,
    # autograd render, L1 loss, backward, loss D2H
    from paper_2512_13796_gb300 import render as R
    jb = jobs["bf16"]
    params = {k: v.clone().requires_grad_(True) for k, v in jb.p.items()}
    fld = R.DeviceField.from_synth(w.field, dev, "f16", "bf16")
    fld.table.requires_grad_(True)
    fld.weights.requires_grad_(True)
    H, W = w.cameras[0].height, w.cameras[0].width
    target_host = torch.rand(H, W, 3).pin_memory()
    loss_host = torch.empty(1).pin_memory()
    ws_e2e = R.Workspace(dev, cap_hint=32 << 20)

    grad_leaves = list(params.values()) + [fld.table, fld.weights]

    def e2e_step():
        for t in grad_leaves:  # a training step starts with no gradients
            t.grad = None
        tgt = target_host.to(dev, non_blocking=True)
        img, _, _ = R.render(params, fld, w.cameras[0], w.settings, ws_e2e)
        loss = (img - tgt).abs().mean()
        loss.backward()
        loss_host.copy_(loss.detach().reshape(1), non_blocking=True)

    for _ in range(3):
        e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    e2e_ms = agg([e2e_ms])

    # the same step through the graph API (render.BatchStep with one view):
    # target H2D, one CUDA graph (forward, L1 loss and its gradient in torch,
    # backward), loss D2H
    gstep = R.BatchStep([w.cameras[0]], w.settings, fld,
                        {k: v.detach() for k, v in params.items()})
    tgt_dev = torch.empty(H, W, 3, device=dev)
    loss_dev = torch.zeros(1, device=dev)

    def l1_and_grad():
        diff = gstep.out[0]["image"] - tgt_dev
        loss_dev.copy_(diff.abs().mean().reshape(1))
        gstep.d_image[0].copy_(torch.sign(diff) / diff.numel())

    tgt_dev.copy_(target_host.to(dev))
    gstep.capture(l1_and_grad)

    def e2e_graph_step():
        tgt_dev.copy_(target_host, non_blocking=True)
        gstep.replay()
        loss_host.copy_(loss_dev, non_blocking=True)

    for _ in range(3):
        e2e_graph_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_graph_step()
    torch.cuda.synchronize()
    e2e_graph_ms = agg([(time.perf_counter() - t0) * 1e3 / args.steps])

    # the batched 8-view form, last (its 600k-surfel scene and 8 views'
    # buffers are allocated only now), with its own clock samples
    batch, clk_batch = None, None
    if not args.no_batch:
        batch = BatchJob(dev)
        for _ in range(max(args.warmup, 3)):
            batch.replay()
            batch.sequential()
        barrier()
        cs = ClockSampler(local)
        cs.start()
        nb = max(3, min(args.steps, 10))
        ms["batch_graph"] = agg(timed(batch.replay, nb, flush, stream))
        ms["batch_sequential"] = agg(timed(batch.sequential, nb, flush, stream))
        barrier()
        clk_batch = cs.stop()

    # the other configurations the measurement plan names, after the
    # headline ones (each allocates its own scene and buffers)
    legs = {}
    if not args.no_config1 and args.config == 2:
        legs["config1"] = config1_leg(dev, max(5, min(args.steps, 20)), flush, stream, agg)
        torch.cuda.empty_cache()
    if not args.no_config4:
        cs4 = ClockSampler(local)
        cs4.start()
        legs["config4"] = config4_leg(dev, max(5, min(args.steps, 10)), flush, stream, agg,
                                      peaks, peak_kind)
        legs["config4"]["clocks"] = cs4.stop()
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w)

    if args.profile_json and rank == 0:
        with open(args.profile_json, "w") as f:
            json.dump({"bf16_train": prof, "f32_train": prof_f32, "steps": args.steps}, f, indent=1)

    rl = roofline(prof, jobs["bf16"], peaks, peak_kind, args.steps, f"config{args.config}")
    # the other two kernels the measurement plan names: the hash gather (HBM
    # bytes of the table reads, in the fused texturing forward) and the MLP
    # backward on the tensor cores (MMA FLOPs against the sustained peak)
    more = {}
    for kname, acct in (("texture_fwd_tc", None), ("texture_bwd_tc", "texture_bwd_tc_flops")):
        if kname in prof:
            more[kname] = roofline(prof, jobs["bf16"], peaks, peak_kind, args.steps,
                                   f"config{args.config}", kname, acct)
    n_inst = jobs["bf16"].fwd_out["n_instances"]
    more.update(sort_rooflines(prof, args.steps, w.scene.n, n_inst,
                               key_layout(w.scene.n, w.cameras[0].width, w.cameras[0].height),
                               peaks, peak_kind))
    mpix = lambda m: whole_job_mpix(P, m, world)
    # the hash backward's real ceiling: L2 vector reductions.  Their rate is
    # measured here (random float2 reductions into a 64 MiB table, the size
    # of the FP32 gradient table, inside the flush buffer) and set against
    # the reduction sectors ncu counted for one launch of the kernel.
    red_peak = _native.nexel_peak_l2_reductions(flush_buf.data_ptr(), 64 << 20, 200_000_000, 3,
                                                torch.cuda.current_stream().cuda_stream)
    red_sectors = measured_traffic("hash_bwd_red_sectors", f"config{args.config}")
    if "hash_bwd" in prof:
        t_hb = prof["hash_bwd"][0] / prof["hash_bwd"][1]
        ach = red_sectors / (t_hb * 1e-3) / 1e9 if red_sectors else None
        more["hash_bwd_l2_reductions"] = {
            "kernel": "hash_bwd", "ms_per_launch": t_hb, "bound": "l2_reductions",
            "achieved": ach, "peak": red_peak, "unit": "G reduction sectors/s",
            "frac": ach / red_peak if ach else None, "red_sectors_per_launch": red_sectors,
            "peak_source": "nexel_peak_l2_reductions in this run: random float2 reductions "
                           "into a 64 MiB L2-resident table (median of 3 x 2e8)",
            "note": "red_sectors_per_launch = lts__t_sectors_srcunit_tex_op_red.sum of one ncu "
                    "capture (profiles/hash_bwd_config2.md); null when hash_bwd.cu changed since"}
    # work counts of the collection pass (device reduction over the BF16
    # job's last forward, outside the timed regions)
    jb = jobs["bf16"]
    stats = _native.nexel_render_stats(jb.cam_s, jb.st_train, jb.N, jb.ws.ws.data_ptr(),
                                       jb.ws.ws.numel(), torch.cuda.current_stream().cuda_stream)
    t_cf = prof["collect_fwd"][0] / args.steps if "collect_fwd" in prof else None
    t_cb = prof["collect_bwd"][0] / args.steps if "collect_bwd" in prof else None
    collection = {
        "visible_surfels": stats["visible_surfels"],
        "mean_tiles_per_visible_surfel": n_inst / max(stats["visible_surfels"], 1),
        "longest_tile_list": stats["longest_list"], "tiles": stats["tiles"],
        "pairs_to_last": stats["pairs_to_last"], "pairs_full_lists": stats["pairs_full_lists"],
        "fwd_gpairs_per_s": stats["pairs_to_last"] / (t_cf * 1e-3) / 1e9 if t_cf else None,
        "pairs_bwd_walk": stats["pairs_bwd_walk"],
        "bwd_gpairs_per_s": stats["pairs_bwd_walk"] / (t_cb * 1e-3) / 1e9 if t_cb else None,
        "note": "pairs_to_last = sum over pixels of the last list position composited (a "
                "lower bound of the (pixel, surfel) pairs the forward evaluates); "
                "pairs_bwd_walk = sum over tiles of the largest last position x tile pixels "
                "(the pair evaluations the collection backward runs); pairs_full_lists = sum "
                "over tiles of list length x tile pixels (no early termination)"}
    line = {
        "metric": METRIC, "value": mpix(ms["bf16_train"]), "unit": "Mpix/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms["bf16_train"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.config == 2 else "config1: 50k surfels, 800x800, K=4, hash 8x2^16x2, MLP 16-64-3", "surfels": w.scene.n, "width": W, "height": H,
                   "K": w.settings.K, "n_instances": int(n_inst),
                   "l2": "flushed (256 MB write) before every timed step",
                   "launch_tuning": tuning,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "full_training_iteration": {
            "train_mpix_s": mpix(ms["bf16_full"]), "train_ms": ms["bf16_full"],
            "note": "BF16 form: forward + the paper's objective (L1, D-SSIM, texture, alpha, "
                    "opacity, grid) + backward + Adam over all parameters + FP16 table "
                    "refresh, all on the GPU"},
        "batched": None if batch is None else {
            "workload": BatchJob.WORKLOAD, "pixels_per_step": batch.pixels,
            "graph_train_mpix_s": world * batch.pixels / (ms["batch_graph"] * 1e-3) / 1e6,
            "graph_train_ms": ms["batch_graph"],
            "sequential_train_mpix_s": world * batch.pixels / (ms["batch_sequential"] * 1e-3) / 1e6,
            "sequential_train_ms": ms["batch_sequential"],
            "note": "graph: one CUDA graph per step (device-count preprocess, views as parallel "
                    "branches, gradients summed); sequential: the single-view calls view after "
                    "view, each preprocess reading its instance count back to the host",
            "clocks": clk_batch},
        "kernels_ms_per_step": {k: v[0] / args.steps for k, v in sorted(prof.items(),
                                                                        key=lambda kv: -kv[1][0])},
        "kernels_ms_per_step_f32": {k: v[0] / args.steps for k, v in
                                    sorted(prof_f32.items(), key=lambda kv: -kv[1][0])},
        "profiled_ms_per_step": {"bf16": ms["bf16_train_profiled"], "f32": ms["f32_train_profiled"]},
        "roofline": rl,
        "rooflines_other": more,
        "collection": collection,
        "cpu_baseline": cpu,
        "e2e": {"value": mpix(e2e_ms), "unit": "Mpix/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": H * W * 3 * 4, "d2h_bytes_per_step": 4,
                "path": "render() autograd API: gradients set to None, H2D target, forward, L1 loss, backward, D2H loss; "
                        "no L2 flush between steps; the surfel parameters, hash table and MLP "
                        "stay resident on the device across steps, as in training (only the "
                        "target image and the loss cross the bus)"},
        "e2e_graph": {"value": mpix(e2e_graph_ms), "unit": "Mpix/s", "ms_per_step": e2e_graph_ms,
                      "h2d_bytes_per_step": H * W * 3 * 4, "d2h_bytes_per_step": 4,
                      "path": "render.BatchStep graph API (one view): H2D target, one CUDA graph "
                              "replay (forward, L1 loss, backward), D2H loss; no L2 flush between "
                              "steps"},
        "gpu_launches": int(launches),
        "gpu_launches_note": "kernels of libnexel per timed step (library launch counter)",
        "clocks": clk,
        "statistic": "median of the timed steps (CUDA events), max over ranks",
        "configs": legs,
        "forms": {
            "bf16": {"train_mpix_s": mpix(ms["bf16_train"]), "train_ms": ms["bf16_train"],
                     "render_fps": 1e3 / ms["bf16_fwd"], "render_ms": ms["bf16_fwd"]},
            "f32": {"train_mpix_s": mpix(ms["f32_train"]), "train_ms": ms["f32_train"],
                    "render_fps": 1e3 / ms["f32_fwd"], "render_ms": ms["f32_fwd"]},
            "f16_mlp_loss_scaled": {"train_mpix_s": mpix(ms["f16_train"]),
                                    "train_ms": ms["f16_train"],
                                    "render_fps": 1e3 / ms["f16_fwd"],
                                    "render_ms": ms["f16_fwd"]},
            "paper_sh3_f16": {"train_mpix_s": mpix(ms["sh_f16_train"]),
                              "train_ms": ms["sh_f16_train"],
                              "render_fps": 1e3 / ms["sh_f16_fwd"],
                              "render_ms": ms["sh_f16_fwd"],
                              "note": "the paper's configuration: degree-3 SH for both "
                                      "appearance modes (48 coefficients per surfel, MLP "
                                      "32-64-64-48), FP16 table, FP16 MLP with loss scale 128"},
        },
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
