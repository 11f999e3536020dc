"""ctypes binding of the FP64 oracle (``ges_oracle.c``).

TEST INFRASTRUCTURE: used by the tests, the smoke check and the benchmark's
CPU-baseline leg only.  Every array handed to the C code is float64; FP32 (or
dequantised FP16/BF16) scene attributes are widened exactly.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ges_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "libges_oracle.so")
_lock = threading.Lock()
_lib = None

# Paper defaults: eps_i = 5 * mean axis length (Sec. 5), 1/255 clamp (Sec. 3),
# opaque extent 2 ln 255 (Sec. 4.1), 3DGS's fixed screen low-pass 0.3.
# The tol_* entries are the ambiguity bands of the parity tests, each the
# float32 error bound of the quantity it guards (u = 2^-24):
#   tol_disc_rel, tol_disc_graze  a fragment's a^2 + b^2 against r^2: the
#       disc forms' coefficients (6u each, three terms of at most 3 times the
#       rim's 1/z) and evaluation, 2 (20u + 20u + 20u) = 120u, plus the frame's
#       rounding eps_f = 20u in the plane, 2 eps_f = 40u: 160u <= 1e-5; the
#       frame's tilt moves the fragment in the plane by 2 eps_f / |cos| =
#       2.4e-6 / |cos| = 1e-5 x 0.24 / |cos| (0.25 taken)
#   tol_depth_rel  two fragments ordered by depth: each 1/z within 26u (its
#       coefficients and evaluation), 52u = 3.1e-6 (3.5e-6 taken)
#   tol_gdepth_rel  a Gaussian's key d - eps against D_s: 2u and 28u, 30u = 1.8e-6
#   tol_alpha  alpha at the 1/255 cut: q = y0^2 + y1^2 within 26u relative,
#       alpha within 9e-6 relative, 3.4e-8 absolute at the cut (1e-5 taken)
#   tol_graze  |cos| below which a fragment is grazing outright
#   tol_centre_rel  the translucent render's blend order: a centre's camera
#       depth is the double-float transform rounded once (within u of the
#       exact value), and rounding keeps order, so two centres can only swap
#       into a tie when they lie within 2u = 1.2e-7 of each other
DEFAULT_OPTS = dict(eps_mode=0, eps_value=0.1, eps_factor=5.0, lowpass=0.3,
                    alpha_min=1.0 / 255.0, surfel_r2=2.0 * math.log(255.0), mode=0,
                    tol_depth_rel=3.5e-6, tol_disc_rel=1e-5, tol_graze=1e-3, tol_alpha=1e-5,
                    tol_gdepth_rel=2e-6, samples=1, filter=0, tol_disc_graze=0.25, tol_centre_rel=1.2e-7)


class _Scene(C.Structure):
    _fields_ = [("n_surfels", C.c_int64), ("n_gaussians", C.c_int64), ("sh_degree", C.c_int32)] + \
               [(n, C.c_void_p) for n in ("s_pos", "s_rot", "s_scale", "s_sh",
                                          "g_pos", "g_rot", "g_scale", "g_opac", "g_sh", "g_filt3")] + \
               [("gauss_dim", C.c_int32)]


class _Camera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("w2c", C.c_double * 12),
                ("znear", C.c_double), ("bg", C.c_double * 3)]


class _Opts(C.Structure):
    _fields_ = [("eps_mode", C.c_int32), ("eps_value", C.c_double), ("eps_factor", C.c_double),
                ("lowpass", C.c_double), ("alpha_min", C.c_double), ("surfel_r2", C.c_double),
                ("mode", C.c_int32), ("tol_depth_rel", C.c_double), ("tol_disc_rel", C.c_double),
                ("tol_graze", C.c_double), ("tol_alpha", C.c_double), ("tol_gdepth_rel", C.c_double),
                ("samples", C.c_int32), ("filter", C.c_int32), ("tol_disc_graze", C.c_double),
                ("tol_centre_rel", C.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no fast-math, no FMA contraction)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        P = C.POINTER
        lib.ora_render.argtypes = [P(_Scene), P(_Camera), P(_Opts), C.c_int, C.c_int] + [C.c_void_p] * 6
        lib.ora_backward.argtypes = [P(_Scene), P(_Camera), P(_Opts), C.c_int] + [C.c_void_p] * 7
        lib.ora_sh_basis.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
        lib.ora_surfel_eval.argtypes = [P(_Scene), P(_Camera), P(_Opts), C.c_int64] + [C.c_void_p] * 7
        lib.ora_surfel_info.argtypes = [P(_Scene), P(_Camera), P(_Opts), C.c_int64, C.c_void_p]
        lib.ora_gauss_info.argtypes = [P(_Scene), P(_Camera), P(_Opts), C.c_int64, C.c_void_p]
        lib.ora_touching.argtypes = [P(_Scene), P(_Camera), P(_Opts), C.c_void_p, C.c_void_p, C.c_void_p]
        lib.ora_check_ids.argtypes = [P(_Scene), P(_Camera), P(_Opts), C.c_void_p, C.c_void_p]
        lib.ora_count_fragments.argtypes = [P(_Scene), P(_Camera), P(_Opts), C.c_void_p, C.c_void_p]
        lib.ora_filter3d.argtypes = [P(_Scene), C.c_void_p, C.c_int, C.c_double, C.c_void_p]
        lib.ora_render_geom.argtypes = [P(_Scene), P(_Camera), P(_Opts), C.c_int, C.c_int] + [C.c_void_p] * 6
        lib.ora_render_translucent.argtypes = [P(_Scene), P(_Camera), P(_Opts), C.c_void_p, C.c_int, C.c_int,
                                               C.c_int] + [C.c_void_p] * 5
        lib.ora_backward_translucent.argtypes = [P(_Scene), P(_Camera), P(_Opts), C.c_void_p, C.c_int, C.c_int,
                                                 C.c_void_p] + [C.c_void_p] * 5
        lib.ora_covering_counts.argtypes = [P(_Scene), P(_Camera), P(_Opts), C.c_void_p, C.c_void_p]
        lib.ora_contribution.argtypes = [P(_Scene), P(_Camera), P(_Opts), C.c_void_p]
        _lib = lib
    return _lib


def _d(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class _Pinned:
    """Keeps the float64 copies alive while the C structure points at them."""

    def __init__(self, scene, cam, opts):
        self.arrs = {k: _d(v) for k, v in scene.arrays().items()}
        f3 = getattr(scene, "g_filter3d", None)
        if f3 is not None:
            self.arrs["g_filt3"] = _d(f3)
            assert self.arrs["g_filt3"].shape == (scene.n_gaussians,)
        self.s = _Scene(scene.n_surfels, scene.n_gaussians, scene.sh_degree,
                        *[self.arrs[k].ctypes.data for k in ("s_pos", "s_rot", "s_scale", "s_sh",
                                                              "g_pos", "g_rot", "g_scale", "g_opac", "g_sh")],
                        self.arrs["g_filt3"].ctypes.data if f3 is not None else None,
                        int(np.asarray(scene.g_scale).reshape(scene.n_gaussians, -1).shape[1])
                        if scene.n_gaussians else 3)
        w2c = np.asarray(cam.world_to_cam, np.float64).reshape(12)
        self.c = _Camera(cam.width, cam.height, float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy),
                         (C.c_double * 12)(*w2c), float(cam.znear), (C.c_double * 3)(*map(float, cam.bg)))
        o = dict(DEFAULT_OPTS)
        o.update(opts or {})
        self.o = _Opts(**o)


def _check(st, what):
    if st != 0:
        raise RuntimeError(f"oracle {what} failed with status {st}")


def render(scene, cam, opts=None, culled: bool = True, nthreads: int = 0):
    """FP64 render: rgb [3,H,W], depth [H,W] (+inf where no surfel), id [H,W]
    (-1; [4,H,W], one plane per sample, with ``samples=4``), wg [H,W] (W_G),
    amb [H,W] (bit 1: id/depth ambiguous at some sample, bit 2: colour
    ambiguous) and ncontrib [H,W] (Gaussians that contributed)."""
    lib = load()
    pin = _Pinned(scene, cam, opts)
    H, W = cam.height, cam.width
    ns = int(pin.o.samples)
    if ns not in (1, 4):
        raise ValueError("samples must be 1 or 4")
    out = dict(rgb=np.empty((3, H, W)), depth=np.empty((H, W)),
               id=np.empty((H, W) if ns == 1 else (4, H, W), np.int32),
               wg=np.empty((H, W)), amb=np.empty((H, W), np.uint8), ncontrib=np.empty((H, W), np.int32))
    st = lib.ora_render(C.byref(pin.s), C.byref(pin.c), C.byref(pin.o), int(culled), int(nthreads),
                        *[out[k].ctypes.data for k in ("rgb", "depth", "id", "wg", "amb", "ncontrib")])
    _check(st, "render")
    return out


def render_geom(scene, cam, opts=None, culled: bool = True, nthreads: int = 0):
    """FP64 geometry maps (Sec. 6.4, Eq. 10-12), camera space: ns [3,H,W]
    (surfel normal), dg [H,W] (D_G), ng [3,H,W] (N_G), dsmooth [H,W],
    nsmooth [3,H,W], amb [H,W]."""
    lib = load()
    pin = _Pinned(scene, cam, opts)
    H, W = cam.height, cam.width
    out = dict(ns=np.empty((3, H, W)), dg=np.empty((H, W)), ng=np.empty((3, H, W)),
               dsmooth=np.empty((H, W)), nsmooth=np.empty((3, H, W)), amb=np.empty((H, W), np.uint8))
    st = lib.ora_render_geom(C.byref(pin.s), C.byref(pin.c), C.byref(pin.o), int(culled), int(nthreads),
                             *[out[k].ctypes.data for k in ("ns", "dg", "ng", "dsmooth", "nsmooth", "amb")])
    _check(st, "render_geom")
    return out


def render_translucent(scene, cam, w, front_first: bool = True, opts=None, culled: bool = True, nthreads: int = 0):
    """FP64 translucent-surfel render (Sec. 4.1, Eq. 6-7) with the opacity
    modulating parameters w [N]: rgb [3,H,W], T [H,W] (final transmittance),
    front [H,W] (frontmost contributing surfel, -1), nblend [H,W] (surfels
    blended), amb [H,W] (bit 2: a decision within the bands)."""
    lib = load()
    pin = _Pinned(scene, cam, opts)
    ww = _d(w)
    assert ww.shape == (scene.n_surfels,)
    H, W = cam.height, cam.width
    out = dict(rgb=np.empty((3, H, W)), T=np.empty((H, W)), front=np.empty((H, W), np.int32),
               nblend=np.empty((H, W), np.int32), amb=np.empty((H, W), np.uint8))
    st = lib.ora_render_translucent(C.byref(pin.s), C.byref(pin.c), C.byref(pin.o), ww.ctypes.data, int(front_first),
                                    int(culled), int(nthreads),
                                    *[out[k].ctypes.data for k in ("rgb", "T", "front", "nblend", "amb")])
    _check(st, "render_translucent")
    return out


def backward_translucent(scene, cam, w, dL_drgb, front_first: bool = True, opts=None, nthreads: int = 0):
    """Analytic FP64 gradients of sum(dL_drgb * C) of the translucent render:
    s_pos [N,3], s_rot [N,4], s_scale [N,2], s_w [N], s_sh [N,K,3]."""
    lib = load()
    pin = _Pinned(scene, cam, opts)
    ww = _d(w)
    g = _d(dL_drgb)
    N, K = scene.n_surfels, (scene.sh_degree + 1) ** 2
    out = dict(s_pos=np.empty((N, 3)), s_rot=np.empty((N, 4)), s_scale=np.empty((N, 2)), s_w=np.empty((N,)),
               s_sh=np.empty((N, K, 3)))
    st = lib.ora_backward_translucent(C.byref(pin.s), C.byref(pin.c), C.byref(pin.o), ww.ctypes.data,
                                      int(front_first), int(nthreads), g.ctypes.data,
                                      *[out[k].ctypes.data for k in ("s_pos", "s_rot", "s_scale", "s_w", "s_sh")])
    _check(st, "backward_translucent")
    return out


def covering_counts(scene, cam, w, opts=None):
    """Pixels at which each surfel is the frontmost contributor (Sec. 4.1)."""
    lib = load()
    pin = _Pinned(scene, cam, opts)
    ww = _d(w)
    out = np.empty(scene.n_surfels, np.int64)
    _check(lib.ora_covering_counts(C.byref(pin.s), C.byref(pin.c), C.byref(pin.o), ww.ctypes.data, out.ctypes.data),
           "covering_counts")
    return out


def contribution(scene, cam, opts=None):
    """Contribution score of each Gaussian (Sec. 4.2, Eq. 9)."""
    lib = load()
    pin = _Pinned(scene, cam, opts)
    out = np.empty(scene.n_gaussians)
    _check(lib.ora_contribution(C.byref(pin.s), C.byref(pin.c), C.byref(pin.o), out.ctypes.data), "contribution")
    return out


def backward(scene, cam, dL_drgb, opts=None, nthreads: int = 0):
    """Analytic FP64 gradients of sum(dL_drgb * C); g_scale is [M, 3] for 3D
    Gaussians and [M, 2] for the 2D Gaussians of 2D-GES (Sec. 6.4)."""
    lib = load()
    pin = _Pinned(scene, cam, opts)
    K = (scene.sh_degree + 1) ** 2
    M, N = scene.n_gaussians, scene.n_surfels
    g = _d(dL_drgb)
    assert g.shape == (3, cam.height, cam.width)
    out = dict(g_pos=np.empty((M, 3)), g_rot=np.empty((M, 4)), g_scale=np.empty((M, pin.s.gauss_dim)),
               g_opac=np.empty((M,)), g_sh=np.empty((M, K, 3)), s_sh=np.empty((N, K, 3)))
    st = lib.ora_backward(C.byref(pin.s), C.byref(pin.c), C.byref(pin.o), int(nthreads), g.ctypes.data,
                          *[out[k].ctypes.data for k in ("g_pos", "g_rot", "g_scale", "g_opac", "g_sh", "s_sh")])
    _check(st, "backward")
    return out


def sh_basis(deg: int, d):
    """Real SH basis values Y[K] and gradients dY[K,3] at the unit vector d."""
    lib = load()
    K = (deg + 1) ** 2
    dd = _d(d)
    Y, dY = np.empty(K), np.empty((K, 3))
    lib.ora_sh_basis(int(deg), dd.ctypes.data, Y.ctypes.data, dY.ctypes.data)
    return Y, dY


def surfel_eval(scene, cam, px, py, sid, opts=None):
    """Evaluate surfel sid[k] at pixel (px[k], py[k]): depth, rho=a^2+b^2, cos(n, ray), hit flag."""
    lib = load()
    pin = _Pinned(scene, cam, opts)
    px = np.ascontiguousarray(px, np.int32)
    py = np.ascontiguousarray(py, np.int32)
    sid = np.ascontiguousarray(sid, np.int32)
    n = px.size
    z, rho, nd = np.empty(n), np.empty(n), np.empty(n)
    ok = np.empty(n, np.int32)
    st = lib.ora_surfel_eval(C.byref(pin.s), C.byref(pin.c), C.byref(pin.o), n, px.ctypes.data,
                             py.ctypes.data, sid.ctypes.data, z.ctypes.data, rho.ctypes.data,
                             nd.ctypes.data, ok.ctypes.data)
    _check(st, "surfel_eval")
    return z, rho, nd, ok


def surfel_info(scene, cam, i, opts=None):
    lib = load()
    pin = _Pinned(scene, cam, opts)
    out = np.empty(14)
    _check(lib.ora_surfel_info(C.byref(pin.s), C.byref(pin.c), C.byref(pin.o), int(i), out.ctypes.data),
           "surfel_info")
    return dict(valid=bool(out[0]), rgb=out[1:4], pc=out[4:7], n=out[7:10], bbox=out[10:14].astype(int))


def gauss_info(scene, cam, i, opts=None):
    lib = load()
    pin = _Pinned(scene, cam, opts)
    out = np.empty(26)
    _check(lib.ora_gauss_info(C.byref(pin.s), C.byref(pin.c), C.byref(pin.o), int(i), out.ctypes.data),
           "gauss_info")
    return dict(valid=bool(out[0]), px=out[1], py=out[2], conic=out[3:6], sigma2=out[6:9],
                sigma=out[9], d=out[10], eps=out[11], rgb=out[12:15], bbox=out[15:19].astype(int),
                nrm=out[19:22], S=out[22:24], scale_filtered=out[24:26])


def id_validity(scene, cam, ref, ids, opts=None):
    """Which surfel ids are acceptable z-buffer answers at each pixel (bool
    [H,W]).  Where ``ids`` equals the oracle's winner it is valid by
    definition; elsewhere the oracle checks that the candidate's fragment is
    inside its disc (up to the rim band) and that no surfel clearly in front of
    it is clearly inside its own disc (``ora_check_ids``)."""
    lib = load()
    ids = np.ascontiguousarray(ids, np.int32)
    pin = _Pinned(scene, cam, opts)
    v = np.empty(ids.shape, np.uint8)
    _check(lib.ora_check_ids(C.byref(pin.s), C.byref(pin.c), C.byref(pin.o), ids.ctypes.data, v.ctypes.data),
           "check_ids")
    return (ids == ref["id"]) | (v != 0)


def touching(scene, cam, flag, opts=None):
    """(surfel_mask, gaussian_mask): primitives that touch a pixel where ``flag`` is set."""
    lib = load()
    pin = _Pinned(scene, cam, opts)
    f = np.ascontiguousarray(flag, np.uint8)
    assert f.shape == (cam.height, cam.width)
    st_ = np.empty(scene.n_surfels, np.uint8)
    gt_ = np.empty(scene.n_gaussians, np.uint8)
    _check(lib.ora_touching(C.byref(pin.s), C.byref(pin.c), C.byref(pin.o), f.ctypes.data, st_.ctypes.data,
                            gt_.ctypes.data), "touching")
    return st_.astype(bool), gt_.astype(bool)


def filter3d(scene, cams, s3d: float = 0.2):
    """Mip-GES 3D filter variance per Gaussian from the cameras ``cams``
    (``ora_filter3d``); s3d = 0.2 is Mip-Splatting's filter size."""
    lib = load()
    pins = [_Pinned(scene, c, None) for c in cams]
    arr = (_Camera * len(cams))(*[p.c for p in pins])
    out = np.empty(scene.n_gaussians)
    _check(lib.ora_filter3d(C.byref(pins[0].s), C.cast(arr, C.c_void_p), len(cams), float(s3d), out.ctypes.data),
           "filter3d")
    return out


def count_fragments(scene, cam, opts=None):
    """(surfel fragments inside their discs, Gaussian terms with alpha >= alpha_min)."""
    lib = load()
    pin = _Pinned(scene, cam, opts)
    a, b = C.c_int64(), C.c_int64()
    _check(lib.ora_count_fragments(C.byref(pin.s), C.byref(pin.c), C.byref(pin.o), C.addressof(a), C.addressof(b)),
           "count_fragments")
    return a.value, b.value
