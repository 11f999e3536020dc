"""Seeded synthetic inputs for the GES renderer and its FP64 oracle.

This module only *places* primitives and cameras; it holds none of the
rendering arithmetic (no projection, no SH evaluation, no compositing).  Both
the CUDA path's tests/bench and the oracle consume its arrays.

Representation (Sec. 3): a surfel is ``{p, r, s, SH}`` with ``s`` in R^2, a 3D
Gaussian is ``{p, sigma, r, s, SH}`` with ``s`` in R^3.  Arrays are SoA,
C-contiguous, float32:

    s_pos [N,3]  s_rot [N,4] (w,x,y,z)  s_scale [N,2]  s_sh [N,K,3]
    g_pos [M,3]  g_rot [M,4] (w,x,y,z)  g_scale [M,3]  g_opac [M]  g_sh [M,K,3]

with K = (deg+1)^2 SH coefficients per colour channel, coefficient-major.
Scales are linear axis lengths, opacities are activated values in [0,1].

Cameras follow the OpenCV convention (x right, y down, z forward), a row-major
world-to-camera ``[R|t]`` and a pinhole ``fx, fy, cx, cy``; the vertical field
of view fixes ``fx = fy = (H/2)/tan(fov/2)`` and ``cx = W/2, cy = H/2``.

Workload recipe (stand-in for the paper's datasets, which are not used):
surfel centres uniform on object surfaces (area weighted), tangent frame from
the surface normal with a uniform in-plane angle, axis scales U(0.01, 0.05),
SH DC ~ U(0,1) and higher bands ~ N(0, 0.05); Gaussian means are random surfel
centres plus N(0, 0.02^2) offsets, log-scales ~ N(-5, 0.5), uniformly random
unit quaternions, opacity ~ U(0.05, 0.9).  Surfels on planar objects get an
offset N(0, plane_jitter^2) along the plane normal (default 2 mm): optimised
surfels are never exactly coplanar, and exactly coplanar discs would make the
z-buffer winner depend only on float rounding of the inputs.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "Scene", "Camera", "look_at", "orbit_cameras", "random_scene",
    "config_scene", "crop_scene", "perturbed_scene", "CONFIG_NAMES",
]


@dataclasses.dataclass
class Scene:
    sh_degree: int
    s_pos: np.ndarray
    s_rot: np.ndarray
    s_scale: np.ndarray
    s_sh: np.ndarray
    g_pos: np.ndarray
    g_rot: np.ndarray
    g_scale: np.ndarray
    g_opac: np.ndarray
    g_sh: np.ndarray
    g_filter3d: Optional[np.ndarray] = None   # per-Gaussian 3D filter variance (Mip-GES), or none

    @property
    def n_surfels(self) -> int:
        return int(self.s_pos.shape[0])

    @property
    def n_gaussians(self) -> int:
        return int(self.g_pos.shape[0])

    def subset(self, s_idx=None, g_idx=None) -> "Scene":
        s_idx = slice(None) if s_idx is None else s_idx
        g_idx = slice(None) if g_idx is None else g_idx
        c = np.ascontiguousarray
        return Scene(self.sh_degree,
                     c(self.s_pos[s_idx]), c(self.s_rot[s_idx]), c(self.s_scale[s_idx]), c(self.s_sh[s_idx]),
                     c(self.g_pos[g_idx]), c(self.g_rot[g_idx]), c(self.g_scale[g_idx]),
                     c(self.g_opac[g_idx]), c(self.g_sh[g_idx]),
                     None if self.g_filter3d is None else c(self.g_filter3d[g_idx]))

    def arrays(self):
        return dict(s_pos=self.s_pos, s_rot=self.s_rot, s_scale=self.s_scale, s_sh=self.s_sh,
                    g_pos=self.g_pos, g_rot=self.g_rot, g_scale=self.g_scale,
                    g_opac=self.g_opac, g_sh=self.g_sh)


@dataclasses.dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    world_to_cam: np.ndarray  # (3,4) float32, row-major [R|t]
    znear: float = 0.01
    bg: Tuple[float, float, float] = (0.0, 0.0, 0.0)

    def crop(self, x0: int, y0: int, w: int, h: int) -> "Camera":
        """The same camera restricted to the pixel window [x0,x0+w) x [y0,y0+h)."""
        return Camera(w, h, self.fx, self.fy, float(np.float32(self.cx - x0)),
                      float(np.float32(self.cy - y0)), self.world_to_cam.copy(), self.znear, self.bg)


def _f32(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float32))


def look_at(eye, target, up, width: int, height: int, fov_deg: float = 60.0,
            znear: float = 0.01, bg=(0.0, 0.0, 0.0)) -> Camera:
    """Pinhole camera at ``eye`` looking at ``target``; ``up`` fixes the roll.

    Camera axes: z = forward, x = forward x up (normalised), y = z x x, which
    is right-handed with y pointing away from ``up`` (image rows grow down).
    """
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    x = np.cross(f, np.asarray(up, np.float64))
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    R = np.stack([x, y, f])
    t = -R @ eye
    focal = (height / 2.0) / math.tan(math.radians(fov_deg) / 2.0)
    w2c = np.concatenate([R, t[:, None]], axis=1)
    return Camera(int(width), int(height), float(np.float32(focal)), float(np.float32(focal)),
                  float(np.float32(width / 2.0)), float(np.float32(height / 2.0)),
                  _f32(w2c), float(np.float32(znear)), tuple(float(np.float32(b)) for b in bg))


def orbit_cameras(n: int, width: int, height: int, radius: float = 15.0, elevation: float = 5.0,
                  fov_deg: float = 60.0, target=(0.0, 0.0, 0.0)) -> List[Camera]:
    """``n`` cameras evenly spaced on a horizontal circle (world up = +z)."""
    cams = []
    for k in range(n):
        th = 2.0 * math.pi * k / n
        eye = (radius * math.cos(th), radius * math.sin(th), elevation)
        cams.append(look_at(eye, target, (0.0, 0.0, 1.0), width, height, fov_deg))
    return cams


# ---------------------------------------------------------------------------
# primitive placement

def _unit(rng, n):
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _tangent_basis(nrm):
    """Two unit vectors spanning the plane orthogonal to each row of ``nrm``."""
    a = np.where(np.abs(nrm[:, :1]) < 0.9, np.array([[1.0, 0.0, 0.0]]), np.array([[0.0, 1.0, 0.0]]))
    b1 = np.cross(nrm, a)
    b1 /= np.linalg.norm(b1, axis=1, keepdims=True)
    b2 = np.cross(nrm, b1)
    return b1, b2


def _frame_to_quat(tu, tv, nrm):
    """Unit quaternion (w,x,y,z) of the rotation whose columns are tu, tv, n."""
    m00, m10, m20 = tu[:, 0], tu[:, 1], tu[:, 2]
    m01, m11, m21 = tv[:, 0], tv[:, 1], tv[:, 2]
    m02, m12, m22 = nrm[:, 0], nrm[:, 1], nrm[:, 2]
    tr = m00 + m11 + m22
    q = np.empty((tu.shape[0], 4))
    c0 = tr > 0
    s = np.sqrt(np.maximum(tr + 1.0, 1e-300)) * 2.0
    q[c0] = np.stack([0.25 * s, (m21 - m12) / s, (m02 - m20) / s, (m10 - m01) / s], 1)[c0]
    c1 = (~c0) & (m00 > m11) & (m00 > m22)
    s = np.sqrt(np.maximum(1.0 + m00 - m11 - m22, 1e-300)) * 2.0
    q[c1] = np.stack([(m21 - m12) / s, 0.25 * s, (m01 + m10) / s, (m02 + m20) / s], 1)[c1]
    c2 = (~c0) & (~c1) & (m11 > m22)
    s = np.sqrt(np.maximum(1.0 + m11 - m00 - m22, 1e-300)) * 2.0
    q[c2] = np.stack([(m02 - m20) / s, (m01 + m10) / s, 0.25 * s, (m12 + m21) / s], 1)[c2]
    c3 = (~c0) & (~c1) & (~c2)
    s = np.sqrt(np.maximum(1.0 + m22 - m00 - m11, 1e-300)) * 2.0
    q[c3] = np.stack([(m10 - m01) / s, (m02 + m20) / s, (m12 + m21) / s, 0.25 * s], 1)[c3]
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _sh_coeffs(rng, n, degree):
    K = (degree + 1) ** 2
    sh = np.empty((n, K, 3))
    sh[:, 0, :] = rng.uniform(0.0, 1.0, (n, 3))
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.05, (n, K - 1, 3))
    return sh


def _objects(rng, n_obj, box, sphere_r, plane_side, sphere_frac, centre_box=None):
    cb = box if centre_box is None else centre_box
    is_sphere = rng.random(n_obj) < sphere_frac
    centres = rng.uniform(-cb, cb, (n_obj, 3))
    radii = rng.uniform(sphere_r[0], sphere_r[1], n_obj)
    sides = rng.uniform(plane_side[0], plane_side[1], n_obj)
    normals = _unit(rng, n_obj)
    area = np.where(is_sphere, 4.0 * np.pi * radii ** 2, sides ** 2)
    return dict(is_sphere=is_sphere, centres=centres, radii=radii, sides=sides,
                normals=normals, area=area)


def random_scene(seed, n_surfels: int, n_gaussians: int, *, n_objects: int = 200,
                 box: float = 10.0, sphere_r=(0.5, 1.0), plane_side=(1.0, 4.0),
                 sphere_frac: float = 0.5, centre_box=None, sh_degree: int = 3,
                 surfel_scale=(0.01, 0.05), gauss_offset: float = 0.02,
                 gauss_logscale=(-5.0, 0.5), opacity=(0.05, 0.9),
                 plane_jitter: float = 0.002) -> Scene:
    """Surfels on seeded spheres and squares; Gaussians scattered around them."""
    rng = np.random.Generator(np.random.PCG64(seed))
    obj = _objects(rng, n_objects, box, sphere_r, plane_side, sphere_frac, centre_box)
    N, M = int(n_surfels), int(n_gaussians)
    which = rng.choice(n_objects, size=N, p=obj["area"] / obj["area"].sum())
    sph = obj["is_sphere"][which]
    # surface points and normals
    dirs = _unit(rng, N)
    pos_s = obj["centres"][which] + obj["radii"][which, None] * dirs
    pn = obj["normals"][which]
    b1, b2 = _tangent_basis(pn)
    uv = rng.uniform(-0.5, 0.5, (N, 2)) * obj["sides"][which, None]
    jit = rng.normal(0.0, plane_jitter, N) if plane_jitter > 0 else np.zeros(N)
    pos_p = obj["centres"][which] + uv[:, :1] * b1 + uv[:, 1:] * b2 + jit[:, None] * pn
    pos = np.where(sph[:, None], pos_s, pos_p)
    nrm = np.where(sph[:, None], dirs, pn)
    # tangent frame with a uniform in-plane angle
    t1, t2 = _tangent_basis(nrm)
    phi = rng.uniform(0.0, 2.0 * np.pi, N)
    tu = np.cos(phi)[:, None] * t1 + np.sin(phi)[:, None] * t2
    tv = np.cross(nrm, tu)
    s_rot = _frame_to_quat(tu, tv, nrm)
    s_scale = rng.uniform(surfel_scale[0], surfel_scale[1], (N, 2))
    s_sh = _sh_coeffs(rng, N, sh_degree)
    # Gaussians around random surfel centres
    if N > 0:
        anchor = pos[rng.integers(0, N, M)]
    else:
        anchor = rng.uniform(-box, box, (M, 3))
    g_pos = anchor + rng.normal(0.0, gauss_offset, (M, 3))
    g_scale = np.exp(rng.normal(gauss_logscale[0], gauss_logscale[1], (M, 3)))
    q = rng.standard_normal((M, 4))
    g_rot = q / np.linalg.norm(q, axis=1, keepdims=True)
    g_opac = rng.uniform(opacity[0], opacity[1], M)
    g_sh = _sh_coeffs(rng, M, sh_degree)
    return Scene(sh_degree, _f32(pos), _f32(s_rot), _f32(s_scale), _f32(s_sh),
                 _f32(g_pos), _f32(g_rot), _f32(g_scale), _f32(g_opac), _f32(g_sh))


def perturbed_scene(scene: Scene, seed, pos_sigma: float = 0.01, sh_sigma: float = 0.05) -> Scene:
    """Target scene for the training-step workload: means and SH jittered."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = dataclasses.replace(scene)
    out.g_pos = _f32(scene.g_pos + rng.normal(0.0, pos_sigma, scene.g_pos.shape))
    out.g_sh = _f32(scene.g_sh + rng.normal(0.0, sh_sigma, scene.g_sh.shape))
    out.s_sh = _f32(scene.s_sh + rng.normal(0.0, sh_sigma, scene.s_sh.shape))
    return out


def crop_scene(seed, width: int = 64, height: int = 64, n_surfels: int = 20,
               n_gaussians: int = 50, sh_degree: int = 3) -> Tuple[Scene, Camera]:
    """A small scene filling a ``width x height`` view: surfels on a tilted
    backdrop and Gaussians in front of and around them (finite-difference size)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cam = look_at((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), width, height, 60.0)
    N, M = n_surfels, n_gaussians
    pos = np.stack([rng.uniform(-0.9, 0.9, N), rng.uniform(-0.9, 0.9, N),
                    rng.uniform(0.0, 0.6, N)], 1)
    nrm = _unit(rng, N) * 0.35 + np.array([0.0, 0.0, -1.0])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    t1, t2 = _tangent_basis(nrm)
    phi = rng.uniform(0.0, 2.0 * np.pi, N)
    tu = np.cos(phi)[:, None] * t1 + np.sin(phi)[:, None] * t2
    tv = np.cross(nrm, tu)
    s_rot = _frame_to_quat(tu, tv, nrm)
    s_scale = rng.uniform(0.08, 0.2, (N, 2))
    g_pos = np.stack([rng.uniform(-0.8, 0.8, M), rng.uniform(-0.8, 0.8, M),
                      rng.uniform(-0.3, 0.3, M)], 1)
    g_scale = np.exp(rng.normal(-3.2, 0.3, (M, 3)))
    q = rng.standard_normal((M, 4))
    g_rot = q / np.linalg.norm(q, axis=1, keepdims=True)
    g_opac = rng.uniform(0.1, 0.9, M)
    scene = Scene(sh_degree, _f32(pos), _f32(s_rot), _f32(s_scale), _f32(_sh_coeffs(rng, N, sh_degree)),
                  _f32(g_pos), _f32(g_rot), _f32(g_scale), _f32(g_opac), _f32(_sh_coeffs(rng, M, sh_degree)))
    return scene, cam


# ---------------------------------------------------------------------------
# the five workloads

CONFIG_NAMES = {
    0: "parity-128x128-1k-surfels-4k-gaussians",
    1: "1080p-1M-surfels-300k-gaussians-fp32-orbit64",
    2: "batched-16x1264x832-2M-surfels-500k-gaussians",
    3: "train-step-1600x1060-500k-surfels-500k-gaussians",
    4: "uneven-8-scenes-100k-to-3M-fp16",
}

_UNEVEN_TOTALS = (100_000, 250_000, 500_000, 750_000, 1_000_000, 1_500_000, 2_000_000, 3_000_000)
_UNEVEN_RES = ((640, 480), (800, 600), (1280, 720), (1600, 900), (1920, 1080),
               (2560, 1440), (3200, 1800), (3840, 2160))


def config_scene(k: int, part: int = 0) -> Tuple[Scene, List[Camera]]:
    """Scene and cameras of workload ``k`` (``part`` selects the scene of the
    uneven batch, k=4).  Seed of workload k is k; the uneven batch uses (4, part)."""
    if k == 0:
        scene = random_scene(0, 1000, 4000, n_objects=3, sphere_frac=1.0, centre_box=0.7)
        cam = look_at((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 128, 128, 60.0)
        return scene, [cam]
    if k == 1:
        return random_scene(1, 1_000_000, 300_000), orbit_cameras(64, 1920, 1080)
    if k == 2:
        return random_scene(2, 2_000_000, 500_000), orbit_cameras(16, 1264, 832)
    if k == 3:
        return random_scene(3, 500_000, 500_000), orbit_cameras(1, 1600, 1060)
    if k == 4:
        tot = _UNEVEN_TOTALS[part]
        ns = tot * 3 // 4
        w, h = _UNEVEN_RES[part]
        scene = random_scene([4, part], ns, tot - ns)
        th = 2.0 * math.pi * part / len(_UNEVEN_TOTALS)
        cam = look_at((15.0 * math.cos(th), 15.0 * math.sin(th), 5.0), (0, 0, 0), (0, 0, 1), w, h, 60.0)
        return scene, [cam]
    if k == 100:  # paper-shaped context: Garden-like counts (Table 6)
        return random_scene(100, 200_000, 2_500_000), orbit_cameras(8, 1920, 1080)
    raise ValueError(f"unknown workload {k}")


def uneven_parts() -> Sequence[int]:
    return range(len(_UNEVEN_TOTALS))
