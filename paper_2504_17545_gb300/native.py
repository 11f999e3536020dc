"""ctypes binding of ``libges.so`` (the C ABI of ``include/ges.h``).

Argument marshalling only: every function here forwards to the C entry point
of the same name and raises :class:`GesError` on a non-zero status.  The
library must exist (``build.build()`` makes it); there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

GES_OK, GES_ERR_INVALID_ARG, GES_ERR_CUDA, GES_ERR_OOM, GES_ERR_TIMEOUT, GES_ERR_INTERNAL, \
    GES_ERR_UNSUPPORTED, GES_ERR_CAPACITY = range(8)
GES_F32, GES_F16, GES_BF16 = 0, 1, 2
GES_MODE_FULL, GES_MODE_SURFELS_ONLY, GES_MODE_GAUSSIANS_ONLY = 0, 1, 2
GES_FILTER_EWA, GES_FILTER_MIP = 0, 1
GES_EPS_ADAPTIVE, GES_EPS_ZERO, GES_EPS_CONST = 0, 1, 2
GES_PROFILE_SLOTS = 8

STATUS_NAMES = {0: "GES_OK", 1: "GES_ERR_INVALID_ARG", 2: "GES_ERR_CUDA", 3: "GES_ERR_OOM",
                4: "GES_ERR_TIMEOUT", 5: "GES_ERR_INTERNAL", 6: "GES_ERR_UNSUPPORTED", 7: "GES_ERR_CAPACITY"}


class GesError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class ges_scene_desc(C.Structure):
    _fields_ = [("n_surfels", C.c_int64), ("n_gaussians", C.c_int64), ("sh_degree", C.c_int32),
                ("attr_dtype", C.c_int32), ("sh_dtype", C.c_int32),
                ("s_pos", C.c_void_p), ("s_rot", C.c_void_p), ("s_scale", C.c_void_p), ("s_sh", C.c_void_p),
                ("g_pos", C.c_void_p), ("g_rot", C.c_void_p), ("g_scale", C.c_void_p), ("g_opac", C.c_void_p),
                ("g_sh", C.c_void_p), ("g_filter3d", C.c_void_p), ("gauss_dim", C.c_int32)]


class ges_camera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("world_to_cam", C.c_float * 12), ("znear", C.c_float),
                ("bg", C.c_float * 3)]


class ges_render_opts(C.Structure):
    _fields_ = [("eps_mode", C.c_int32), ("eps_value", C.c_float), ("eps_factor", C.c_float),
                ("lowpass", C.c_float), ("alpha_min", C.c_float), ("surfel_r2", C.c_float), ("mode", C.c_int32),
                ("samples", C.c_int32), ("filter", C.c_int32)]


class ges_grads(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("g_pos", "g_rot", "g_scale", "g_opac", "g_sh", "s_sh")]


class ges_tgrads(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("s_pos", "s_rot", "s_scale", "s_w", "s_sh")]


class ges_stats(C.Structure):
    _fields_ = [("visible_surfels", C.c_int64), ("visible_gaussians", C.c_int64),
                ("surfel_tile_pairs", C.c_int64), ("gauss_tile_pairs", C.c_int64),
                ("tiles_x", C.c_int32), ("tiles_y", C.c_int32)]


class ges_batch_info(C.Structure):
    _fields_ = [("n_views", C.c_int32), ("prims_per_cta", C.c_int32), ("raster_ctas_per_sm", C.c_int32),
                ("candidates", C.c_int32), ("tuned_ms", C.c_double), ("h2d_bytes", C.c_int64),
                ("d2h_bytes", C.c_int64), ("tile_w", C.c_int32), ("tile_h", C.c_int32)]


class ges_profile(C.Structure):
    _fields_ = [("n", C.c_int32), ("names", (C.c_char * 24) * GES_PROFILE_SLOTS),
                ("ms", C.c_double * GES_PROFILE_SLOTS), ("launches", C.c_int64 * GES_PROFILE_SLOTS)]


# every symbol the header declares, with its C signature
_P = C.POINTER
_SIGS = {
    "ges_default_opts": (C.c_int, [_P(ges_render_opts)]),
    "ges_create_scene": (C.c_int, [_P(ges_scene_desc), _P(C.c_void_p)]),
    "ges_scene_update": (C.c_int, [C.c_void_p, _P(ges_scene_desc)]),
    "ges_destroy_scene": (C.c_int, [C.c_void_p]),
    "ges_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ges_render": (C.c_int, [C.c_void_p, _P(ges_camera), C.c_void_p, C.c_void_p]),
    "ges_render_ex": (C.c_int, [C.c_void_p, _P(ges_camera), _P(ges_render_opts), C.c_void_p, C.c_void_p,
                                C.c_void_p, C.c_void_p]),
    "ges_render_geom": (C.c_int, [C.c_void_p, _P(ges_camera), _P(ges_render_opts)] + [C.c_void_p] * 7),
    "ges_render_translucent": (C.c_int, [C.c_void_p, _P(ges_camera), _P(ges_render_opts), C.c_void_p, C.c_int32]
                               + [C.c_void_p] * 6),
    "ges_render_translucent_backward": (C.c_int, [C.c_void_p, _P(ges_camera), _P(ges_render_opts), C.c_void_p,
                                                  C.c_int32] + [C.c_void_p] * 5 + [_P(ges_tgrads)]),
    "ges_contribution_scores": (C.c_int, [C.c_void_p, _P(ges_camera), _P(ges_render_opts)] + [C.c_void_p] * 3),
    "ges_render_backward": (C.c_int, [C.c_void_p, _P(ges_camera), _P(ges_render_opts), C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p, _P(ges_grads)]),
    "ges_render_batch": (C.c_int, [_P(C.c_void_p), _P(ges_camera), _P(C.c_int32), C.c_int32,
                                   _P(ges_render_opts), _P(C.c_void_p), _P(C.c_void_p)]),
    "ges_render_noalloc": (C.c_int, [_P(ges_scene_desc), _P(ges_camera), _P(ges_render_opts), C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ges_compute_filter3d": (C.c_int, [C.c_void_p, _P(ges_camera), C.c_int32, C.c_float, C.c_void_p]),
    "ges_count_fragments": (C.c_int, [C.c_void_p, _P(ges_camera), _P(ges_render_opts), _P(C.c_int64),
                                      _P(C.c_int64)]),
    "ges_batch_create": (C.c_int, [_P(C.c_void_p), _P(ges_camera), _P(C.c_int32), C.c_int32,
                                   _P(ges_render_opts), _P(C.c_void_p), _P(C.c_void_p), _P(C.c_void_p)]),
    "ges_batch_set_camera": (C.c_int, [C.c_void_p, C.c_int32, _P(ges_camera)]),
    "ges_batch_set_id_output": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "ges_batch_launch": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ges_batch_sync": (C.c_int, [C.c_void_p]),
    "ges_batch_get_info": (C.c_int, [C.c_void_p, _P(ges_batch_info)]),
    "ges_batch_get_profile": (C.c_int, [C.c_void_p, _P(ges_profile), C.c_int32]),
    "ges_batch_get_view_times": (C.c_int, [C.c_void_p, _P(C.c_double)]),
    "ges_batch_destroy": (C.c_int, [C.c_void_p]),
    "ges_get_stats": (C.c_int, [C.c_void_p, _P(ges_stats)]),
    "ges_set_profiling": (C.c_int, [C.c_void_p, C.c_int32]),
    "ges_get_profile": (C.c_int, [C.c_void_p, _P(ges_profile)]),
    "ges_last_error_message": (C.c_char_p, []),
    "ges_version": (C.c_int32, []),
}

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    """The in-tree build, or the library named by GES_LIBRARY (another build
    of the same sources, e.g. with different compile options)."""
    return os.environ.get("GES_LIBRARY") or _build.LIB


def load(build_if_missing: bool = True):
    """Load libges.so (building it first if it is missing or stale).
    Raises if it cannot be built or loaded: there is no other path."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if build_if_missing and path == _build.LIB:
                _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library {path} is missing; run paper_2504_17545_gb300.build.build()")
            lib = C.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(status: int):
    if status != GES_OK:
        raise GesError(status, load().ges_last_error_message().decode(errors="replace"))


def ges_default_opts() -> ges_render_opts:
    o = ges_render_opts()
    _check(load().ges_default_opts(C.byref(o)))
    return o


def ges_create_scene(desc: ges_scene_desc) -> C.c_void_p:
    h = C.c_void_p()
    _check(load().ges_create_scene(C.byref(desc), C.byref(h)))
    return h


def ges_scene_update(scene, desc: ges_scene_desc):
    _check(load().ges_scene_update(scene, C.byref(desc)))


def ges_destroy_scene(scene):
    _check(load().ges_destroy_scene(scene))


def ges_set_stream(scene, stream: int):
    _check(load().ges_set_stream(scene, C.c_void_p(stream)))


def ges_render(scene, cam: ges_camera, out_rgb: int, out_depth: int):
    _check(load().ges_render(scene, C.byref(cam), C.c_void_p(out_rgb), C.c_void_p(out_depth)))


def ges_render_ex(scene, cam: ges_camera, opts, out_rgb: int, out_depth: int, out_id: int, aux: int):
    _check(load().ges_render_ex(scene, C.byref(cam), C.byref(opts) if opts is not None else None,
                                C.c_void_p(out_rgb), C.c_void_p(out_depth), C.c_void_p(out_id), C.c_void_p(aux)))


def ges_render_geom(scene, cam: ges_camera, opts, out_rgb: int, out_depth: int, out_ns: int, out_dsm: int,
                    out_nsm: int, out_dg: int, out_ng: int):
    _check(load().ges_render_geom(scene, C.byref(cam), C.byref(opts) if opts is not None else None,
                                  *[C.c_void_p(p) for p in (out_rgb, out_depth, out_ns, out_dsm, out_nsm,
                                                             out_dg, out_ng)]))


def ges_render_translucent(scene, cam: ges_camera, opts, w: int, front_first: bool, out_rgb: int, out_T: int,
                           out_front: int, out_last: int, out_Tlast: int, out_cover: int):
    _check(load().ges_render_translucent(scene, C.byref(cam), C.byref(opts) if opts is not None else None,
                                         C.c_void_p(w), int(bool(front_first)),
                                         *[C.c_void_p(p) for p in (out_rgb, out_T, out_front, out_last, out_Tlast,
                                                                    out_cover)]))


def ges_render_translucent_backward(scene, cam: ges_camera, opts, w: int, front_first: bool, dL: int, T: int,
                                    front: int, last: int, Tlast: int, grads: "ges_tgrads"):
    _check(load().ges_render_translucent_backward(scene, C.byref(cam), C.byref(opts) if opts is not None else None,
                                                  C.c_void_p(w), int(bool(front_first)),
                                                  *[C.c_void_p(p) for p in (dL, T, front, last, Tlast)],
                                                  C.byref(grads)))


def ges_contribution_scores(scene, cam: ges_camera, opts, depth: int, aux: int, out: int):
    _check(load().ges_contribution_scores(scene, C.byref(cam), C.byref(opts) if opts is not None else None,
                                          C.c_void_p(depth), C.c_void_p(aux), C.c_void_p(out)))


def ges_render_backward(scene, cam: ges_camera, opts, dL_drgb: int, out_rgb: int, out_depth: int,
                        surfel_id: int, aux: int, grads: ges_grads):
    _check(load().ges_render_backward(scene, C.byref(cam), C.byref(opts) if opts is not None else None,
                                      C.c_void_p(dL_drgb), C.c_void_p(out_rgb), C.c_void_p(out_depth),
                                      C.c_void_p(surfel_id), C.c_void_p(aux), C.byref(grads)))


def ges_render_batch(scenes, cams, scene_of_view, opts, out_rgb, out_depth):
    n = len(cams)
    sc = (C.c_void_p * len(scenes))(*[s.value if isinstance(s, C.c_void_p) else s for s in scenes])
    cm = (ges_camera * n)(*cams)
    sv = (C.c_int32 * n)(*scene_of_view)
    rg = (C.c_void_p * n)(*out_rgb)
    dp = (C.c_void_p * n)(*out_depth) if out_depth is not None else None
    _check(load().ges_render_batch(sc, cm, sv, n, C.byref(opts) if opts is not None else None, rg, dp))


def ges_get_stats(scene) -> ges_stats:
    s = ges_stats()
    _check(load().ges_get_stats(scene, C.byref(s)))
    return s


def ges_set_profiling(scene, enable: bool):
    _check(load().ges_set_profiling(scene, int(bool(enable))))


def ges_get_profile(scene) -> dict:
    p = ges_profile()
    _check(load().ges_get_profile(scene, C.byref(p)))
    return {bytes(p.names[i]).split(b"\0")[0].decode(): (p.ms[i], p.launches[i]) for i in range(p.n)}


def ges_last_error_message() -> str:
    return load().ges_last_error_message().decode(errors="replace")


def ges_version() -> int:
    return int(load().ges_version())


def ges_count_fragments(scene, cam: ges_camera, opts):
    a, b = C.c_int64(), C.c_int64()
    _check(load().ges_count_fragments(scene, C.byref(cam), C.byref(opts) if opts is not None else None,
                                      C.byref(a), C.byref(b)))
    return a.value, b.value


def ges_compute_filter3d(scene, cams, s3d: float, out_var) -> None:
    n = len(cams)
    cm = (ges_camera * n)(*cams)
    _check(load().ges_compute_filter3d(scene, cm, n, float(s3d), out_var))


def ges_batch_create(scenes, cams, scene_of_view, opts, out_rgb, out_depth):
    n = len(cams)
    sc = (C.c_void_p * len(scenes))(*[x.value if isinstance(x, C.c_void_p) else x for x in scenes])
    cm = (ges_camera * n)(*cams)
    sv = (C.c_int32 * n)(*scene_of_view)
    rg = (C.c_void_p * n)(*out_rgb)
    dp = (C.c_void_p * n)(*out_depth) if out_depth is not None else None
    h = C.c_void_p()
    _check(load().ges_batch_create(sc, cm, sv, n, C.byref(opts) if opts is not None else None, rg, dp, C.byref(h)))
    return h


def ges_batch_set_camera(batch, view: int, cam: ges_camera):
    _check(load().ges_batch_set_camera(batch, int(view), C.byref(cam)))


def ges_batch_set_id_output(batch, view: int, out_surfel_id: int, aux: int):
    _check(load().ges_batch_set_id_output(batch, int(view), out_surfel_id or None, aux or None))


def ges_batch_launch(batch, stream: int):
    _check(load().ges_batch_launch(batch, C.c_void_p(stream)))


def ges_batch_sync(batch):
    _check(load().ges_batch_sync(batch))


def ges_batch_get_info(batch) -> ges_batch_info:
    i = ges_batch_info()
    _check(load().ges_batch_get_info(batch, C.byref(i)))
    return i


def ges_batch_destroy(batch):
    _check(load().ges_batch_destroy(batch))


def ges_batch_get_view_times(batch, n_views: int):
    out = (C.c_double * n_views)()
    _check(load().ges_batch_get_view_times(batch, out))
    return list(out)


def ges_batch_get_profile(batch, reset: bool = False) -> dict:
    p = ges_profile()
    _check(load().ges_batch_get_profile(batch, C.byref(p), int(bool(reset))))
    return {bytes(p.names[i]).split(b"\0")[0].decode(): (p.ms[i], p.launches[i]) for i in range(p.n)}
