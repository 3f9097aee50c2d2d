"""PyTorch-facing API: device buffers, streams and autograd around libnexel.

Everything here is argument marshalling.  PyTorch provides device memory and
the current CUDA stream; the three library calls (preprocess, forward,
backward) do all of the rendering arithmetic in CUDA kernels.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import _native as N_


def camera_struct(cam) -> N_.Camera:
    c = N_.Camera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    m = np.asarray(cam.world_to_cam, np.float32).ravel()
    for i in range(12):
        c.world_to_cam[i] = float(m[i])
    c.near_plane = float(cam.near)
    return c


def settings_struct(st, grid_dtype: str = "f32", mlp_dtype: str = "f32",
                    recompute: bool = False, cache_features: bool = False,
                    sh_degree: int = 0) -> N_.Settings:
    s = N_.Settings()
    s.K = int(st.K)
    s.alpha_min, s.alpha_max, s.T_min = float(st.alpha_min), float(st.alpha_max), float(st.T_min)
    for i in range(3):
        s.bg[i] = float(st.bg[i])
    s.grid_dtype = {"f32": N_.F32, "f16": N_.F16}[grid_dtype]
    s.mlp_dtype = {"f32": N_.F32, "bf16": N_.BF16, "f16": N_.F16}[mlp_dtype]
    s.recompute_buffers = 1 if recompute else 0
    s.cache_features = 1 if cache_features else 0
    s.sh_degree = int(sh_degree)
    return s


@dataclasses.dataclass
class DeviceField:
    """Neural field on the device: FP32 master table and weights, plus the
    storage copy of the table the kernels read (FP16 in the precision form)."""
    L: int
    T: int
    F: int
    level_scale: tuple
    widths: tuple
    table: torch.Tensor        # (L, T, F) float32 master
    weights: torch.Tensor      # flat float32, layer after layer, (out, in) row-major
    grid_dtype: str = "f32"
    mlp_dtype: str = "f32"

    @staticmethod
    def from_synth(f, device, grid_dtype="f32", mlp_dtype="f32") -> "DeviceField":
        w = torch.from_numpy(np.concatenate([x.ravel() for x in f.weights]).astype(np.float32))
        return DeviceField(f.L, f.T, f.F, tuple(float(s) for s in f.level_scale), tuple(f.widths),
                           torch.from_numpy(f.table).to(device).contiguous(),
                           w.to(device).contiguous(), grid_dtype, mlp_dtype)

    def storage_table(self, table: torch.Tensor | None = None) -> torch.Tensor:
        t = self.table if table is None else table
        return t.detach().to(torch.float16).contiguous() if self.grid_dtype == "f16" else \
            t.detach().contiguous()

    def struct(self, table_store: torch.Tensor, weights: torch.Tensor) -> N_.Field:
        f = N_.Field()
        f.L, f.T, f.F = self.L, self.T, self.F
        for l in range(self.L):
            f.level_scale[l] = float(self.level_scale[l])
        f.table = table_store.data_ptr()
        f.n_layers = len(self.widths) - 1
        for i, w in enumerate(self.widths):
            f.widths[i] = int(w)
        f.weights = weights.data_ptr()
        return f


def _ptr(t):
    return None if t is None else t.data_ptr()


class Workspace:
    """Device scratch for one camera and surfel count; grows on demand."""

    def __init__(self, device, cap_hint: int = 1 << 20):
        self.device = torch.device(device)
        self.cap = int(cap_hint)
        self.ws = None
        self.ws_key = None
        self.bws = None
        self.bws_key = None

    def main(self, cam_s: N_.Camera, N: int):
        key = (cam_s.width, cam_s.height, N, self.cap)
        if self.ws_key != key:
            nbytes = N_.nexel_workspace_size(cam_s, N, self.cap)
            self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self.ws_key = key
        return self.ws

    def bwd(self, cam_s, st_s, field_s):
        nbytes = N_.nexel_bwd_workspace_size(cam_s, st_s, field_s)
        if self.bws is None or self.bws.numel() < nbytes:
            self.bws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        return self.bws


def _stream():
    return torch.cuda.current_stream().cuda_stream


def preprocess(ws: Workspace, cam_s, st_s, mu, quat, scale, opacity, gamma, color) -> int:
    N = mu.shape[0]
    while True:
        buf = ws.main(cam_s, N)
        rc, n_inst = N_.nexel_preprocess(cam_s, st_s, N, mu.data_ptr(), quat.data_ptr(),
                                         scale.data_ptr(), opacity.data_ptr(), gamma.data_ptr(),
                                         color.data_ptr(), buf.data_ptr(), buf.numel(), _stream())
        if rc == -3:  # capacity: grow and redo
            ws.cap = int(n_inst * 1.25) + 1024
            continue
        N_.check("nexel_preprocess", rc)
        return n_inst


def forward(ws: Workspace, cam_s, st_s, field: DeviceField | None, table_store, weights, mu,
            quat, scale, opacity, gamma, color) -> dict:
    """Preprocess + forward render; returns the output tensors."""
    dev = mu.device
    H, W, K = cam_s.height, cam_s.width, st_s.K
    n_inst = preprocess(ws, cam_s, st_s, mu, quat, scale, opacity, gamma, color)
    out = dict(image=torch.empty(H, W, 3, device=dev), notex=torch.empty(H, W, 3, device=dev),
               weights=torch.empty(H, W, K, device=dev),
               ids=torch.empty(H, W, K, dtype=torch.int32, device=dev),
               depths=torch.empty(H, W, K, device=dev),
               textures=torch.empty(H, W, K, 3, device=dev), T_final=torch.empty(H, W, device=dev))
    fs = field.struct(table_store, weights) if (field is not None and K > 0) else None
    buf = ws.ws
    # a training step leaves the field features in the backward scratch
    bws = ws.bwd(cam_s, st_s, fs) if (st_s.cache_features and K > 0) else None
    N_.nexel_render_fwd(cam_s, st_s, fs, mu.shape[0], buf.data_ptr(), buf.numel(),
                        _ptr(bws), bws.numel() if bws is not None else 0,
                        out["image"].data_ptr(), out["notex"].data_ptr(),
                        _ptr(out["weights"]) if K else None, _ptr(out["ids"]) if K else None,
                        _ptr(out["depths"]) if K else None, _ptr(out["textures"]) if K else None,
                        out["T_final"].data_ptr(), _stream())
    out["n_instances"] = n_inst
    return out


def backward(ws: Workspace, cam_s, st_s, field, table_store, weights, mu, quat, scale, opacity,
             gamma, fwd: dict, d_image, d_weights=None, d_textures=None, accumulate=False,
             grads: dict | None = None) -> dict:
    dev = mu.device
    N = mu.shape[0]
    K = st_s.K
    g = grads if grads is not None else {}
    # new gradient buffers: without accumulate the library overwrites them
    # (it zeroes every gradient output itself), so they need no fill here
    new = torch.zeros if accumulate else torch.empty
    cshape = (N, 16, 3) if st_s.sh_degree == 3 else (N, 3)
    for k, shape in (("mu", (N, 3)), ("quat", (N, 4)), ("scale", (N, 2)), ("opacity", (N,)),
                     ("gamma", (N, 2)), ("color", cshape)):
        if k not in g:
            g[k] = new(shape, device=dev)
    fs = None
    if field is not None and K > 0:
        fs = field.struct(table_store, weights)
        if "table" not in g:
            g["table"] = new(field.table.shape, device=dev)
        if "mlp" not in g:
            g["mlp"] = new(field.weights.shape, device=dev)
    bws = ws.bwd(cam_s, st_s, fs)
    buf = ws.ws
    N_.nexel_render_bwd(cam_s, st_s, fs, N, mu.data_ptr(), quat.data_ptr(), scale.data_ptr(),
                        opacity.data_ptr(), gamma.data_ptr(), buf.data_ptr(), buf.numel(),
                        bws.data_ptr(), bws.numel(),
                        *((None, None, None, None) if st_s.recompute_buffers else
                          (_ptr(fwd["weights"]) if K else None, _ptr(fwd["ids"]) if K else None,
                           _ptr(fwd["depths"]) if K else None, fwd["T_final"].data_ptr())),
                        d_image.contiguous().data_ptr(),
                        _ptr(d_weights.contiguous()) if d_weights is not None else None,
                        _ptr(d_textures.contiguous()) if d_textures is not None else None,
                        accumulate, g["mu"].data_ptr(), g["quat"].data_ptr(),
                        g["scale"].data_ptr(), g["opacity"].data_ptr(), g["gamma"].data_ptr(),
                        g["color"].data_ptr(), _ptr(g.get("table")), _ptr(g.get("mlp")),
                        _stream())
    return g


class NexelRender(torch.autograd.Function):
    """Differentiable render: inputs are the activated surfel parameters and
    the field's FP32 master table and weights; outputs image, W and T."""

    @staticmethod
    def forward(ctx, mu, quat, scale, opacity, gamma, color, table, weights, cfg):
        ws, cam_s, st_s, field = cfg["ws"], cfg["cam"], cfg["settings"], cfg["field"]
        args = [t.detach().contiguous() for t in (mu, quat, scale, opacity, gamma, color)]
        ts = field.storage_table(table) if field is not None else None
        w = weights.detach().contiguous() if weights is not None else None
        out = forward(ws, cam_s, st_s, field, ts, w, *args)
        ctx.cfg = cfg
        ctx.args, ctx.ts, ctx.w = args, ts, w
        ctx.out = out
        return out["image"], out["weights"], out["textures"]

    @staticmethod
    def backward(ctx, d_image, d_weights, d_textures):
        cfg = ctx.cfg
        mu, quat, scale, opacity, gamma, color = ctx.args
        g = backward(cfg["ws"], cfg["cam"], cfg["settings"], cfg["field"], ctx.ts, ctx.w, mu, quat,
                     scale, opacity, gamma, ctx.out, d_image, d_weights, d_textures)
        return (g["mu"], g["quat"], g["scale"], g["opacity"], g["gamma"], g["color"],
                g.get("table"), g.get("mlp"), None)


def render(params: dict, field: DeviceField | None, cam, settings, ws: Workspace | None = None):
    """Differentiable render of one view.  ``params`` holds activated
    surfel tensors mu, quat, scale, opacity, gamma, color (float32, cuda).
    Returns (image [H,W,3], weights [H,W,K], textures [H,W,K,3])."""
    dev = params["mu"].device
    ws = ws or Workspace(dev)
    # when a backward will follow, the forward leaves the field features for it
    train = torch.is_grad_enabled() and (
        any(t.requires_grad for t in params.values()) or
        (field is not None and (field.table.requires_grad or field.weights.requires_grad)))
    cfg = dict(ws=ws, cam=camera_struct(cam),
               settings=settings_struct(settings, field.grid_dtype if field else "f32",
                                        field.mlp_dtype if field else "f32",
                                        cache_features=train),
               field=field)
    tab = field.table if field is not None else None
    w = field.weights if field is not None else None
    return NexelRender.apply(params["mu"], params["quat"], params["scale"], params["opacity"],
                             params["gamma"], params["color"], tab, w, cfg)


class BatchStep:
    """Multi-view training step of one scene (views of uneven resolutions)
    through the batched entry points, with no host synchronisation inside
    the step, so that the whole step can be captured in one CUDA graph.

    Construction runs the synchronising preprocess once per view to size
    each view's workspace (instance count x ``margin``); later steps use
    the device-count preprocess, whose overflow (a scene that moved far)
    ``status()`` reports.  ``d_image[v]`` are static upstream-gradient
    buffers the caller fills (or computes inside the captured graph);
    ``grads`` receives the gradients summed over the views.  Parameter,
    table and weight tensors are read through their storage, so a captured
    graph sees in-place updates of them; ``refresh_table()`` copies the FP32
    master table into the storage copy in place."""

    def __init__(self, cams, settings, field: DeviceField | None, params: dict,
                 margin: float = 1.25, train: bool = True):
        self.params = {k: params[k].detach().contiguous() for k in
                       ("mu", "quat", "scale", "opacity", "gamma", "color")}
        dev = self.params["mu"].device
        self.dev = dev
        self.N = int(self.params["mu"].shape[0])
        self.field = field
        self.cams = [camera_struct(c) for c in cams]
        K = int(settings.K)
        self.K = K
        self.train = train
        self.st = settings_struct(settings, field.grid_dtype if field else "f32",
                                  field.mlp_dtype if field else "f32",
                                  cache_features=train and K > 0)
        self.ts = field.storage_table() if field is not None else None
        self.w = field.weights if field is not None else None
        self.fs = field.struct(self.ts, self.w) if (field is not None and K > 0) else None
        p = [self.params[k] for k in ("mu", "quat", "scale", "opacity", "gamma", "color")]
        self.ws, self.ws_bytes, self.bws, self.bws_bytes, self.out = [], [], [], [], []
        self.n_instances = []
        for cs in self.cams:
            probe = Workspace(dev, cap_hint=1 << 20)
            n = preprocess(probe, cs, self.st, *p)
            self.n_instances.append(n)
            cap = int(n * margin) + 4096
            nbytes = N_.nexel_workspace_size(cs, self.N, cap)
            self.ws.append(torch.empty(nbytes, dtype=torch.uint8, device=dev))
            self.ws_bytes.append(nbytes)
            bn = N_.nexel_bwd_workspace_size(cs, self.st, self.fs) if train else 0
            self.bws.append(torch.empty(bn, dtype=torch.uint8, device=dev) if bn else None)
            self.bws_bytes.append(bn)
            H, W = cs.height, cs.width
            self.out.append(dict(
                image=torch.empty(H, W, 3, device=dev), notex=torch.empty(H, W, 3, device=dev),
                weights=torch.empty(H, W, K, device=dev),
                ids=torch.empty(H, W, K, dtype=torch.int32, device=dev),
                depths=torch.empty(H, W, K, device=dev),
                textures=torch.empty(H, W, K, 3, device=dev),
                T_final=torch.empty(H, W, device=dev)))
            del probe
        self.d_image = [torch.zeros(cs.height, cs.width, 3, device=dev) for cs in self.cams]
        N = self.N
        self.grads = dict(mu=torch.zeros(N, 3, device=dev), quat=torch.zeros(N, 4, device=dev),
                          scale=torch.zeros(N, 2, device=dev), opacity=torch.zeros(N, device=dev),
                          gamma=torch.zeros(N, 2, device=dev),
                          color=torch.zeros_like(self.params["color"]))
        if self.fs is not None:
            self.grads["table"] = torch.zeros_like(field.table)
            self.grads["mlp"] = torch.zeros_like(field.weights)
        self.graph = None

    @property
    def pixels(self) -> int:
        return sum(c.width * c.height for c in self.cams)

    def refresh_table(self):
        if self.field is not None:
            self.ts.copy_(self.field.table.detach().to(self.ts.dtype))

    def _outs(self, key):
        return [o[key].data_ptr() for o in self.out] if (self.K > 0 or key in
                                                          ("image", "notex", "T_final")) else None

    def forward(self):
        p = self.params
        N_.nexel_render_batch_fwd(
            self.cams, self.st, self.fs, self.N, p["mu"].data_ptr(), p["quat"].data_ptr(),
            p["scale"].data_ptr(), p["opacity"].data_ptr(), p["gamma"].data_ptr(),
            p["color"].data_ptr(), [b.data_ptr() for b in self.ws], self.ws_bytes,
            [_ptr(b) for b in self.bws], self.bws_bytes, self._outs("image"), self._outs("notex"),
            self._outs("weights"), self._outs("ids"), self._outs("depths"),
            self._outs("textures"), self._outs("T_final"), _stream())

    def backward(self, accumulate: bool = False):
        p, g = self.params, self.grads
        N_.nexel_render_batch_bwd(
            self.cams, self.st, self.fs, self.N, p["mu"].data_ptr(), p["quat"].data_ptr(),
            p["scale"].data_ptr(), p["opacity"].data_ptr(), p["gamma"].data_ptr(),
            [b.data_ptr() for b in self.ws], self.ws_bytes, [_ptr(b) for b in self.bws],
            self.bws_bytes, self._outs("weights"), self._outs("ids"), self._outs("depths"),
            self._outs("T_final"), [d.data_ptr() for d in self.d_image], None, None, accumulate,
            g["mu"].data_ptr(), g["quat"].data_ptr(), g["scale"].data_ptr(),
            g["opacity"].data_ptr(), g["gamma"].data_ptr(), g["color"].data_ptr(),
            _ptr(g.get("table")), _ptr(g.get("mlp")), _stream())

    def step(self):
        self.forward()
        if self.train:
            self.backward()

    def capture(self, extra=None):
        """Captures forward (+ ``extra()``, e.g. a loss that writes d_image)
        + backward into one CUDA graph, after one eager warm-up step on a
        side stream (which also creates the library's branch streams)."""
        s = torch.cuda.Stream(device=self.dev)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.forward()
            if extra is not None:
                extra()
            if self.train:
                self.backward()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize(self.dev)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.forward()
            if extra is not None:
                extra()
            if self.train:
                self.backward()
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def status(self) -> list[int]:
        """Per-view device status (synchronises): 0, or the NEXEL_ERR_*
        code of an instance-capacity overflow or a device timeout."""
        return [N_.nexel_read_status(cs, self.st, self.fs, self.N, self.ws[v].data_ptr(),
                                     self.ws_bytes[v], _ptr(self.bws[v]), self.bws_bytes[v],
                                     _stream()) for v, cs in enumerate(self.cams)]


PAPER_LOSS_WEIGHTS = dict(dssim=0.2, alpha=0.005, texture=0.5, opacity=0.01, grid=0.01)


class Objective:
    """The training objective of the paper's Sec. 5 on the GPU
    (nexel_loss_image / nexel_loss_params) for one image size.  ``values``
    (device, 8 floats) holds L_1, L_D-SSIM, L_texture, L_alpha, their
    weighted sum, L_opacity, L_grid and the total after both calls."""

    NAMES = ("l1", "dssim", "texture", "alpha", "image_terms", "opacity", "grid", "total")

    def __init__(self, width: int, height: int, device, weights: dict | None = None):
        self.W, self.H = int(width), int(height)
        w = dict(PAPER_LOSS_WEIGHTS, **(weights or {}))
        self.lw = N_.LossWeights(**{k: float(w[k]) for k in ("dssim", "alpha", "texture",
                                                               "opacity", "grid")})
        nbytes = N_.nexel_loss_workspace_size(self.W, self.H)
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.values = torch.zeros(8, device=device)

    def image_terms(self, image, target, weights=None, textures=None):
        """Returns (d_image, d_weights, d_textures) for nexel_render_bwd."""
        K = 0 if weights is None else int(weights.shape[-1])
        d_image = torch.empty_like(image)
        d_w = torch.empty_like(weights) if K else None
        d_t = torch.empty_like(textures) if K else None
        N_.nexel_loss_image(self.W, self.H, K, self.lw, image.data_ptr(), target.data_ptr(),
                            _ptr(weights) if K else None, _ptr(textures) if K else None,
                            self.ws.data_ptr(), self.ws.numel(), self.values.data_ptr(),
                            d_image.data_ptr(), _ptr(d_w), _ptr(d_t), _stream())
        return d_image, d_w, d_t

    def param_terms(self, opacity, field: DeviceField | None, d_opacity=None, d_table=None):
        """Adds the opacity and grid regularisers' gradients (after the
        render backward) and completes ``values``."""
        fs = None
        if field is not None:
            fs = N_.Field()
            fs.L, fs.T, fs.F = field.L, field.T, field.F
            for l in range(field.L):
                fs.level_scale[l] = float(field.level_scale[l])
        N_.nexel_loss_params(int(opacity.shape[0]), opacity.data_ptr(), fs,
                             field.table.data_ptr() if field is not None else None, self.lw,
                             self.ws.data_ptr(), self.ws.numel(), self.W, self.H,
                             self.values.data_ptr(), _ptr(d_opacity), _ptr(d_table), _stream())

    def read(self) -> dict:
        v = self.values.cpu().tolist()
        return dict(zip(self.NAMES, v))


class Adam:
    """Adam over a list of FP32 tensors, one launch (nexel_adam_step) per
    step for up to 16 tensors."""

    def __init__(self, tensors: list, lrs: list, betas=(0.9, 0.999), eps: float = 1e-15):
        self.p = list(tensors)
        self.lrs = [float(x) for x in lrs]
        self.m = [torch.zeros_like(t) for t in self.p]
        self.v = [torch.zeros_like(t) for t in self.p]
        self.b1, self.b2 = float(betas[0]), float(betas[1])
        self.eps = float(eps)
        self.t = 0

    def step(self, grads: list):
        self.t += 1
        N_.nexel_adam_step([t.data_ptr() for t in self.p], [g.data_ptr() for g in grads],
                           [t.data_ptr() for t in self.m], [t.data_ptr() for t in self.v],
                           [t.numel() for t in self.p], self.lrs, self.b1, self.b2, self.eps,
                           self.t, _stream())


class DensityControl:
    """Adaptive density control of supp. Sec. 7.2 around the library calls:
    blended errors accumulated across iterations (nexel_blend_error), then a
    density step that draws 5 % of the surfels (capped by the budget) in
    proportion to their errors (nexel_densify_select, with exponential
    random numbers drawn here from a seeded generator), splits them along
    their long axis (nexel_densify_split) and prunes those with opacity
    below 0.005 (nexel_prune).  Parameters are the activated surfel tensors
    (mu, quat, scale, opacity, gamma, color); a density step returns new
    tensors (the surfel count changes)."""

    PRUNE_OPACITY = 0.005

    def __init__(self, n: int, device, budget: int, seed: int = 0):
        self.device = torch.device(device)
        self.budget = int(budget)
        self.err = torch.zeros(n, device=self.device)
        self.gen = torch.Generator(device="cpu").manual_seed(seed)

    def accumulate(self, ws: Workspace, cam_s, st_s, n: int, image, target):
        """Adds this view's blended errors (after its forward on ws)."""
        N_.nexel_blend_error(cam_s, st_s, n, ws.ws.data_ptr(), ws.ws.numel(), image.data_ptr(),
                             target.data_ptr(), self.err.data_ptr(), _stream())

    def step(self, params: dict) -> tuple[dict, int, int]:
        """(new params, surfels split, surfels pruned); resets the errors."""
        keys = ("mu", "quat", "scale", "opacity", "gamma", "color")
        N = int(params["mu"].shape[0])
        n_sel = N_.nexel_densify_count(N, self.budget)
        color_dim = int(params["color"][0].numel())
        ws = torch.empty(N_.nexel_density_workspace_size(N + n_sel), dtype=torch.uint8,
                         device=self.device)
        # room for the second children, then the split in place
        grown = {k: torch.cat([params[k].detach(),
                               torch.zeros((n_sel,) + tuple(params[k].shape[1:]),
                                           device=self.device)]).contiguous() for k in keys}
        if n_sel > 0:
            expo = torch.empty(N).exponential_(generator=self.gen).to(self.device)
            sel = torch.empty(n_sel, dtype=torch.int32, device=self.device)
            N_.nexel_densify_select(N, self.err.data_ptr(), expo.data_ptr(), self.budget,
                                    ws.data_ptr(), ws.numel(), sel.data_ptr(), _stream())
            N_.nexel_densify_split(N, n_sel, sel.data_ptr(), color_dim,
                                   *[grown[k].data_ptr() for k in keys], _stream())
        M = N + n_sel
        out = {k: torch.empty_like(v) for k, v in grown.items()}
        n_out = torch.zeros(1, dtype=torch.int32, device=self.device)
        N_.nexel_prune(M, self.PRUNE_OPACITY, color_dim, [grown[k].data_ptr() for k in keys],
                       ws.data_ptr(), ws.numel(), [out[k].data_ptr() for k in keys],
                       n_out.data_ptr(), _stream())
        kept = int(n_out.item())
        new = {k: v[:kept].clone() for k, v in out.items()}
        self.err = torch.zeros(kept, device=self.device)
        return new, n_sel, M - kept


def fps_init(points, m: int) -> tuple:
    """Farthest point sampling of a point cloud [n, 3] (device float32) to m
    centres, and their initial scales: the distance at which each was
    selected (supp. Sec. 7.2; the first takes the second's)."""
    n = int(points.shape[0])
    scratch = torch.empty(n, device=points.device)
    idx = torch.empty(m, dtype=torch.int32, device=points.device)
    d2 = torch.empty(m, device=points.device)
    s = torch.empty(m, device=points.device)
    N_.nexel_fps(n, points.contiguous().data_ptr(), m, scratch.data_ptr(), idx.data_ptr(),
                 d2.data_ptr(), s.data_ptr(), _stream())
    return points[idx.long()], s
