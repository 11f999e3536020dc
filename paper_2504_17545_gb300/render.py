"""PyTorch-facing layer over the C ABI: device tensors in, device tensors out.

PyTorch supplies device memory and the current stream; every step of the
render and of its backward runs in the library's CUDA kernels.  Nothing here
computes any part of the method.
"""
from __future__ import annotations

import math
from typing import Dict, Optional, Sequence

import torch

from . import native as N

_DTYPES = {torch.float32: N.GES_F32, torch.float16: N.GES_F16, torch.bfloat16: N.GES_BF16}
_SCENE_KEYS = ("s_pos", "s_rot", "s_scale", "s_sh", "g_pos", "g_rot", "g_scale", "g_opac", "g_sh")
_GRAD_KEYS = ("g_pos", "g_rot", "g_scale", "g_opac", "g_sh", "s_sh")


def camera_struct(cam) -> N.ges_camera:
    """ges_camera from any object (or dict) with width, height, fx, fy, cx, cy,
    world_to_cam (3x4), znear, bg."""
    get = (lambda k: cam[k]) if isinstance(cam, dict) else (lambda k: getattr(cam, k))
    c = N.ges_camera()
    c.width, c.height = int(get("width")), int(get("height"))
    c.fx, c.fy, c.cx, c.cy = (float(get(k)) for k in ("fx", "fy", "cx", "cy"))
    w2c = [float(x) for row in get("world_to_cam") for x in row]
    if len(w2c) != 12:
        raise ValueError("world_to_cam must be 3x4")
    c.world_to_cam[:] = w2c
    c.znear = float(get("znear"))
    c.bg[:] = [float(x) for x in get("bg")]
    return c


def _arg(t, name: str, dtype, numel: int, dev) -> torch.Tensor:
    """A caller's tensor that a kernel will read or write: it must sit on the
    scene's device, have the dtype and exactly the element count the kernel
    addresses, and be contiguous (the ABI takes a bare pointer).  Raises
    ValueError before anything is launched."""
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name}: expected a tensor, got {type(t).__name__}")
    if t.device != dev:
        raise ValueError(f"{name}: on {t.device}, the scene is on {dev}")
    if t.dtype != dtype:
        raise ValueError(f"{name}: dtype {t.dtype}, expected {dtype}")
    if t.numel() != numel:
        raise ValueError(f"{name}: {t.numel()} elements (shape {tuple(t.shape)}), expected {numel}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: not contiguous")
    return t


def opts_struct(opts: Optional[dict]) -> N.ges_render_opts:
    o = N.ges_default_opts()
    for k, v in (opts or {}).items():
        if k.startswith("tol_"):
            continue  # ambiguity bands of the parity tests, not render options
        if not hasattr(o, k):
            raise KeyError(f"unknown render option {k!r}")
        setattr(o, k, v)
    return o


def _scene_layout(t: Dict[str, torch.Tensor], sh_degree: int) -> int:
    """Check the scene tensors against the ABI's layout (N surfels and M
    Gaussians taken from the positions, K = (sh_degree + 1)^2): one device,
    positions float32 [N,3] / [M,3], rotations [.,4], surfel scales [N,2],
    Gaussian scales [M,3] (or [M,2]: 2D Gaussians), opacities [M], SH [.,K,3],
    one dtype for rotations, scales and opacities and one for both SH arrays.
    Returns the Gaussian kind (3 or 2); raises ValueError / TypeError before the
    library sees a pointer whose array is shorter than its kernels read."""
    if not 0 <= int(sh_degree) <= 3:
        raise ValueError(f"sh_degree {sh_degree} outside 0..3")
    K = (int(sh_degree) + 1) ** 2
    dev = t["s_pos"].device
    for k in _SCENE_KEYS:
        if t[k].device != dev:
            raise ValueError(f"{k} is on {t[k].device}, s_pos on {dev}")
    if t["s_pos"].dtype != torch.float32 or t["g_pos"].dtype != torch.float32:
        raise TypeError("positions are float32")
    attr = t["s_rot"].dtype
    for k in ("s_scale", "g_rot", "g_scale", "g_opac"):
        if t[k].dtype != attr:
            raise TypeError("rotations, scales and opacities must share one dtype")
    if attr not in _DTYPES or t["s_sh"].dtype not in _DTYPES:
        raise TypeError("attributes are float32, float16 or bfloat16")
    if t["s_sh"].dtype != t["g_sh"].dtype:
        raise TypeError("surfel and Gaussian SH must share one dtype")
    for k in ("s_pos", "g_pos"):
        if t[k].dim() != 2 or t[k].shape[1] != 3:
            raise ValueError(f"{k} must be [n,3], got {tuple(t[k].shape)}")
    n, m = t["s_pos"].shape[0], t["g_pos"].shape[0]
    gs = t["g_scale"]
    gdim = 2 if gs.dim() == 2 and gs.shape[1] == 2 else 3
    want = {"s_rot": (n, 4), "s_scale": (n, 2), "s_sh": (n, K, 3), "g_rot": (m, 4), "g_scale": (m, gdim),
            "g_opac": (m,), "g_sh": (m, K, 3)}
    for k, shape in want.items():
        if tuple(t[k].shape) != shape:
            raise ValueError(f"{k} must be {list(shape)}, got {list(t[k].shape)}")
    return gdim


class GESScene:
    """A GES scene resident in device memory (tensors owned here) and the
    library's handle that views them."""

    def __init__(self, sh_degree: int, g_filter3d: Optional[torch.Tensor] = None, **tensors: torch.Tensor):
        missing = [k for k in _SCENE_KEYS if k not in tensors]
        if missing:
            raise KeyError(f"missing scene tensors {missing}")
        self.sh_degree = int(sh_degree)
        self.t: Dict[str, torch.Tensor] = {}
        for k in _SCENE_KEYS:
            v = tensors[k]
            if not v.is_cuda:
                raise ValueError(f"{k} must be a CUDA tensor")
            self.t[k] = v.contiguous()
        self.gauss_dim = _scene_layout(self.t, self.sh_degree)
        self.g_filter3d = self._check_filter(g_filter3d)
        self.attr_dtype = _DTYPES[self.t["s_rot"].dtype]
        self.sh_dtype = _DTYPES[self.t["s_sh"].dtype]
        self._desc = self._make_desc()
        self.handle = N.ges_create_scene(self._desc)

    def _check_filter(self, f: Optional[torch.Tensor]) -> Optional[torch.Tensor]:
        if f is None:
            return None
        if f.device != self.t["g_pos"].device or f.dtype != torch.float32 or tuple(f.shape) != (self.n_gaussians,):
            raise ValueError("g_filter3d must be a float32 tensor of shape [M] on the scene's device")
        return f.contiguous()

    @classmethod
    def from_arrays(cls, scene, device="cuda", attr_dtype=torch.float32, sh_dtype=torch.float32) -> "GESScene":
        """From a host scene (``scenegen.Scene`` or anything with the same array
        attributes; an optional ``g_filter3d`` array is carried over)."""
        t = {}
        for k in _SCENE_KEYS:
            a = torch.as_tensor(getattr(scene, k))
            dt = torch.float32
            if k in ("s_rot", "s_scale", "g_rot", "g_scale", "g_opac"):
                dt = attr_dtype
            elif k in ("s_sh", "g_sh"):
                dt = sh_dtype
            t[k] = a.to(device=device, dtype=dt).contiguous()
        f3 = getattr(scene, "g_filter3d", None)
        f3 = None if f3 is None else torch.as_tensor(f3).to(device=device, dtype=torch.float32).contiguous()
        return cls(scene.sh_degree, g_filter3d=f3, **t)

    @property
    def n_surfels(self) -> int:
        return int(self.t["s_pos"].shape[0])

    @property
    def n_gaussians(self) -> int:
        return int(self.t["g_pos"].shape[0])

    def _make_desc(self) -> N.ges_scene_desc:
        d = N.ges_scene_desc()
        d.n_surfels, d.n_gaussians = self.n_surfels, self.n_gaussians
        d.sh_degree, d.attr_dtype, d.sh_dtype = self.sh_degree, self.attr_dtype, self.sh_dtype
        d.gauss_dim = self.gauss_dim
        for k in _SCENE_KEYS:
            setattr(d, k, self.t[k].data_ptr() if self.t[k].numel() else None)
        f3 = getattr(self, "g_filter3d", None)
        d.g_filter3d = f3.data_ptr() if f3 is not None and f3.numel() else None
        return d

    def update(self, **tensors: torch.Tensor):
        """Swap some attribute tensors (same dtypes) and re-point the handle.
        ``g_filter3d=None`` removes the Mip-GES 3D filter."""
        t = dict(self.t)
        for k, v in tensors.items():
            if k == "g_filter3d":
                continue
            if k not in _SCENE_KEYS:
                raise KeyError(k)
            t[k] = v.contiguous()
        # checked before anything changes: a rejected update leaves the scene as it was
        if self.t["s_rot"].dtype != t["s_rot"].dtype or self.t["s_sh"].dtype != t["s_sh"].dtype:
            raise TypeError("an update keeps the scene's attribute and SH dtypes")
        gdim = _scene_layout(t, self.sh_degree)
        old = (self.t, self.gauss_dim, self.g_filter3d)
        self.t, self.gauss_dim = t, gdim
        try:
            if "g_filter3d" in tensors:
                self.g_filter3d = self._check_filter(tensors["g_filter3d"])
            elif self.g_filter3d is not None:
                self._check_filter(self.g_filter3d)     # the kept filter must still fit M
        except ValueError:
            self.t, self.gauss_dim, self.g_filter3d = old
            raise
        self._desc = self._make_desc()
        N.ges_scene_update(self.handle, self._desc)

    def compute_filter3d(self, cams, s3d: float = 0.2) -> torch.Tensor:
        """Mip-GES 3D filter variance per Gaussian from training cameras
        (ges_compute_filter3d); pass it to ``update(g_filter3d=...)``."""
        out = torch.empty((self.n_gaussians,), device=self.t["g_pos"].device, dtype=torch.float32)
        self.bind_stream()
        N.ges_compute_filter3d(self.handle, [camera_struct(c) for c in cams], s3d,
                               out.data_ptr() if out.numel() else None)
        return out

    def bind_stream(self):
        N.ges_set_stream(self.handle, torch.cuda.current_stream(self.t["s_pos"].device).cuda_stream)

    def stats(self) -> N.ges_stats:
        return N.ges_get_stats(self.handle)

    def close(self):
        if getattr(self, "handle", None) is not None:
            N.ges_destroy_scene(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def render(scene: GESScene, cam, opts: Optional[dict] = None, with_aux: bool = True):
    """Forward render.  Returns dict(rgb [3,H,W], depth [H,W], id [H,W] int32
    ([4,H,W] with ``samples=4``), aux [H,W] (W_G)); id and aux only when
    ``with_aux``."""
    c = camera_struct(cam)
    o = opts_struct(opts)
    dev = scene.t["s_pos"].device
    H, W = c.height, c.width
    rgb = torch.empty((3, H, W), device=dev, dtype=torch.float32)
    depth = torch.empty((H, W), device=dev, dtype=torch.float32)
    out = dict(rgb=rgb, depth=depth)
    sid = aux = None
    if with_aux:
        sid = torch.empty((H, W) if o.samples == 1 else (o.samples, H, W), device=dev, dtype=torch.int32)
        aux = torch.empty((H, W), device=dev, dtype=torch.float32)
        out.update(id=sid, aux=aux)
    scene.bind_stream()
    N.ges_render_ex(scene.handle, c, o, rgb.data_ptr(), depth.data_ptr(),
                    sid.data_ptr() if sid is not None else 0, aux.data_ptr() if aux is not None else 0)
    return out


def render_geom(scene: GESScene, cam, opts: Optional[dict] = None):
    """Render plus the geometry maps of Sec. 6.4 (Eq. 10-12), camera space:
    dict(rgb, depth, ns [3,H,W], dsmooth [H,W], nsmooth [3,H,W], dg [H,W],
    ng [3,H,W])."""
    c = camera_struct(cam)
    dev = scene.t["s_pos"].device
    H, W = c.height, c.width
    e = lambda *shape: torch.empty(shape, device=dev, dtype=torch.float32)
    out = dict(rgb=e(3, H, W), depth=e(H, W), ns=e(3, H, W), dsmooth=e(H, W), nsmooth=e(3, H, W),
               dg=e(H, W), ng=e(3, H, W))
    scene.bind_stream()
    N.ges_render_geom(scene.handle, c, opts_struct(opts),
                      *[out[k].data_ptr() for k in ("rgb", "depth", "ns", "dsmooth", "nsmooth", "dg", "ng")])
    return out


def render_translucent(scene: GESScene, cam, w: torch.Tensor, front_first: bool = True, opts: Optional[dict] = None,
                       cover: bool = False):
    """Translucent-surfel render of the coarse stage (Sec. 4.1, Eq. 6-7) with
    the opacity modulating parameters w [N] (float32 CUDA tensor): dict(rgb
    [3,H,W], T, front, last, Tlast [H,W]; cover [N] int32 when ``cover``)."""
    c = camera_struct(cam)
    dev = scene.t["s_pos"].device
    H, W = c.height, c.width
    wt = _arg(w.contiguous().float(), "w", torch.float32, scene.n_surfels, dev)
    out = dict(rgb=torch.empty((3, H, W), device=dev), T=torch.empty((H, W), device=dev),
               front=torch.empty((H, W), device=dev, dtype=torch.int32),
               last=torch.empty((H, W), device=dev, dtype=torch.int32), Tlast=torch.empty((H, W), device=dev))
    if cover:
        out["cover"] = torch.empty((scene.n_surfels,), device=dev, dtype=torch.int32)
    scene.bind_stream()
    N.ges_render_translucent(scene.handle, c, opts_struct(opts), wt.data_ptr() if wt.numel() else 0, front_first,
                             *[out[k].data_ptr() for k in ("rgb", "T", "front", "last", "Tlast")],
                             out["cover"].data_ptr() if cover and scene.n_surfels else 0)
    out["w"] = wt
    return out


def render_translucent_backward(scene: GESScene, cam, w: torch.Tensor, fwd: dict, dL_drgb: torch.Tensor,
                                front_first: bool = True, opts: Optional[dict] = None):
    """Gradients of sum(dL_drgb * C) of the translucent render: s_pos, s_rot,
    s_scale, s_w, s_sh (float32)."""
    c = camera_struct(cam)
    dev = scene.t["s_pos"].device
    n, K = scene.n_surfels, (scene.sh_degree + 1) ** 2
    g = {"s_pos": torch.empty((n, 3), device=dev), "s_rot": torch.empty((n, 4), device=dev),
         "s_scale": torch.empty((n, 2), device=dev), "s_w": torch.empty((n,), device=dev),
         "s_sh": torch.empty((n, K, 3), device=dev)}
    gr = N.ges_tgrads()
    for k in ("s_pos", "s_rot", "s_scale", "s_w", "s_sh"):
        setattr(gr, k, g[k].data_ptr() if g[k].numel() else None)
    H, W = c.height, c.width
    wt = _arg(w.contiguous().float(), "w", torch.float32, n, dev)
    dl = _arg(dL_drgb.contiguous().float(), "dL_drgb", torch.float32, 3 * H * W, dev)
    for k, dt in (("T", torch.float32), ("front", torch.int32), ("last", torch.int32), ("Tlast", torch.float32)):
        _arg(fwd[k], f"fwd[{k!r}]", dt, H * W, dev)
    scene.bind_stream()
    N.ges_render_translucent_backward(scene.handle, c, opts_struct(opts), wt.data_ptr() if wt.numel() else 0,
                                      front_first, dl.data_ptr(), fwd["T"].data_ptr(), fwd["front"].data_ptr(),
                                      fwd["last"].data_ptr(), fwd["Tlast"].data_ptr(), gr)
    return g


def contribution_scores(scene: GESScene, cam, fwd: dict, opts: Optional[dict] = None) -> torch.Tensor:
    """Contribution score of each Gaussian (Sec. 4.2, Eq. 9) from a render's
    depth and aux outputs."""
    c = camera_struct(cam)
    dev = scene.t["g_pos"].device
    for k in ("depth", "aux"):
        _arg(fwd[k], f"fwd[{k!r}]", torch.float32, c.height * c.width, dev)
    out = torch.empty((scene.n_gaussians,), device=dev)
    scene.bind_stream()
    N.ges_contribution_scores(scene.handle, c, opts_struct(opts), fwd["depth"].data_ptr(), fwd["aux"].data_ptr(),
                              out.data_ptr() if out.numel() else 0)
    return out


def render_backward(scene: GESScene, cam, fwd: dict, dL_drgb: torch.Tensor, opts: Optional[dict] = None):
    """Gradients of sum(dL_drgb * C) (Sec. 4.2); returns a dict of float32
    tensors (g_scale [M,2] for the 2D Gaussians of 2D-GES)."""
    c = camera_struct(cam)
    dev = scene.t["s_pos"].device
    g = {
        "g_pos": torch.empty((scene.n_gaussians, 3), device=dev),
        "g_rot": torch.empty((scene.n_gaussians, 4), device=dev),
        "g_scale": torch.empty((scene.n_gaussians, scene.gauss_dim), device=dev),
        "g_opac": torch.empty((scene.n_gaussians,), device=dev),
        "g_sh": torch.empty(tuple(scene.t["g_sh"].shape), device=dev),
        "s_sh": torch.empty(tuple(scene.t["s_sh"].shape), device=dev),
    }
    gr = N.ges_grads()
    for k in _GRAD_KEYS:
        setattr(gr, k, g[k].data_ptr() if g[k].numel() else None)
    H, W, o = c.height, c.width, opts_struct(opts)
    dl = _arg(dL_drgb.contiguous().float(), "dL_drgb", torch.float32, 3 * H * W, dev)
    for k, dt, n in (("rgb", torch.float32, 3 * H * W), ("depth", torch.float32, H * W),
                     ("id", torch.int32, o.samples * H * W), ("aux", torch.float32, H * W)):
        _arg(fwd[k], f"fwd[{k!r}]", dt, n, dev)
    scene.bind_stream()
    N.ges_render_backward(scene.handle, c, o, dl.data_ptr(), fwd["rgb"].data_ptr(),
                          fwd["depth"].data_ptr(), fwd["id"].data_ptr(), fwd["aux"].data_ptr(), gr)
    return g


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, scene, cam, opts, g_pos, g_rot, g_scale, g_opac, g_sh, s_sh):
        out = render(scene, cam, opts, with_aux=True)
        ctx.scene, ctx.cam, ctx.opts = scene, cam, opts
        ctx.save_for_backward(out["rgb"], out["depth"], out["id"], out["aux"])
        ctx.mark_non_differentiable(out["depth"], out["id"], out["aux"])
        return out["rgb"], out["depth"], out["id"], out["aux"]

    @staticmethod
    def backward(ctx, grad_rgb, _gd, _gi, _ga):
        rgb, depth, sid, aux = ctx.saved_tensors
        g = render_backward(ctx.scene, ctx.cam, dict(rgb=rgb, depth=depth, id=sid, aux=aux), grad_rgb, ctx.opts)
        return (None, None, None, g["g_pos"], g["g_rot"], g["g_scale"], g["g_opac"], g["g_sh"], g["s_sh"])


def render_differentiable(scene: GESScene, cam, opts: Optional[dict] = None):
    """Differentiable render: gradients flow to the scene's Gaussian tensors and
    surfel SH (set requires_grad on them).  Returns (rgb, depth, id, aux)."""
    t = scene.t
    return _RenderFn.apply(scene, cam, opts, t["g_pos"], t["g_rot"], t["g_scale"], t["g_opac"], t["g_sh"],
                           t["s_sh"])


def render_batch(scenes: Sequence[GESScene], cams: Sequence, scene_of_view: Optional[Sequence[int]] = None,
                 opts: Optional[dict] = None, outputs=None):
    """Render many views in one batch (one host synchronisation).  Returns a
    list of (rgb, depth) tensor pairs (or fills ``outputs``)."""
    n = len(cams)
    if scene_of_view is None:
        scene_of_view = [0] * n
    cstructs = [camera_struct(c) for c in cams]
    dev = scenes[0].t["s_pos"].device
    if outputs is None:
        outputs = [(torch.empty((3, c.height, c.width), device=dev), torch.empty((c.height, c.width), device=dev))
                   for c in cstructs]
    if len(outputs) != n:
        raise ValueError(f"outputs: {len(outputs)} pairs for {n} views")
    for v, (c, (rgb, depth)) in enumerate(zip(cstructs, outputs)):
        _arg(rgb, f"outputs[{v}][0]", torch.float32, 3 * c.height * c.width, dev)
        if depth is not None:
            _arg(depth, f"outputs[{v}][1]", torch.float32, c.height * c.width, dev)
    scenes[0].bind_stream()
    N.ges_render_batch([s.handle for s in scenes], cstructs, list(scene_of_view), opts_struct(opts),
                       [o[0].data_ptr() for o in outputs], [o[1].data_ptr() if o[1] is not None else 0
                                                            for o in outputs])
    return outputs


class GESBatch:
    """A fixed set of views rendered by one captured CUDA graph (every phase one
    launch over all views, persistent raster, autotuned launch shape).  Output
    tensors are allocated here and overwritten by every launch."""

    def __init__(self, scenes: Sequence[GESScene], cams: Sequence, scene_of_view: Optional[Sequence[int]] = None,
                 opts: Optional[dict] = None, with_depth: bool = True):
        n = len(cams)
        self.scenes = list(scenes)
        self.scene_of_view = list(scene_of_view) if scene_of_view is not None else [0] * n
        cs = [camera_struct(c) for c in cams]
        self._sizes = [(c.height, c.width) for c in cs]
        self._samples = opts_struct(opts).samples
        dev = self.scenes[0].t["s_pos"].device
        self.rgb = [torch.empty((3, c.height, c.width), device=dev) for c in cs]
        self.depth = [torch.empty((c.height, c.width), device=dev) for c in cs] if with_depth else None
        self.scenes[0].bind_stream()
        self.handle = N.ges_batch_create([s.handle for s in self.scenes], cs, self.scene_of_view,
                                         opts_struct(opts), [t.data_ptr() for t in self.rgb],
                                         [t.data_ptr() for t in self.depth] if with_depth else None)

    def launch(self):
        N.ges_batch_launch(self.handle, torch.cuda.current_stream(self.rgb[0].device).cuda_stream)

    def sync(self):
        N.ges_batch_sync(self.handle)

    def set_camera(self, view: int, cam):
        N.ges_batch_set_camera(self.handle, view, camera_struct(cam))

    def set_id_output(self, view: int, out_id: Optional[torch.Tensor], aux: Optional[torch.Tensor] = None):
        """Also write view ``view``'s surfel id map (int32 [samples,H,W]) and
        W_G (float32 [H,W]) in the following launches (None: not written).
        The tensors must stay alive while they are set."""
        if not 0 <= view < len(self._sizes):
            raise ValueError(f"view {view} out of range (0..{len(self._sizes) - 1})")
        H, W = self._sizes[view]
        dev = self.rgb[0].device
        if out_id is not None:
            _arg(out_id, "out_id", torch.int32, self._samples * H * W, dev)
        if aux is not None:
            _arg(aux, "aux", torch.float32, H * W, dev)
        self._id_keep = getattr(self, "_id_keep", {})
        self._id_keep[view] = (out_id, aux)
        N.ges_batch_set_id_output(self.handle, view, out_id.data_ptr() if out_id is not None else 0,
                                  aux.data_ptr() if aux is not None else 0)

    def info(self):
        return N.ges_batch_get_info(self.handle)

    def profile(self, reset: bool = False):
        return N.ges_batch_get_profile(self.handle, reset)

    def view_times(self):
        """Per-view completion times (ms from the batch's start) of the last
        synchronised launch."""
        return N.ges_batch_get_view_times(self.handle, len(self.rgb))

    def close(self):
        if getattr(self, "handle", None) is not None:
            N.ges_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
