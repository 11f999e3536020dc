"""Hand-placed discs at and behind the camera (test inputs, no method
arithmetic): each drives a branch of the surfel set-up that random scenes
rarely reach.  The camera is the identity (camera space = world space), and a
small random scene sits 2-4 units in front of it as background."""
import math

import numpy as np

import scenegen as sg


def camera():
    return sg.Camera(96, 64, 45.7, 45.7, 48.0, 32.0,
                     np.concatenate([np.eye(3), np.zeros((3, 1))], 1).astype(np.float32))


def background():
    scene = sg.random_scene(36, 300, 600, n_objects=5, box=1.0, sphere_r=(0.3, 0.6), plane_side=(0.6, 1.2),
                            surfel_scale=(0.03, 0.1), gauss_logscale=(-3.8, 0.4))
    scene.s_pos = np.ascontiguousarray(scene.s_pos + np.float32([0, 0, 3]))
    scene.g_pos = np.ascontiguousarray(scene.g_pos + np.float32([0, 0, 3]))
    return scene


def with_discs(scene, discs, seed):
    """scene plus surfels discs = [(centre, tu, tv, (s1, s2))], appended
    after the scene's own (their ids start at scene.n_surfels)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    tu = np.array([d[1] for d in discs], np.float64)
    tv = np.array([d[2] for d in discs], np.float64)
    q = sg._frame_to_quat(tu, tv, np.cross(tu, tv))
    sh = np.zeros((len(discs),) + scene.s_sh.shape[1:], np.float32)
    sh[:, 0, :] = rng.uniform(0.2, 1.0, (len(discs), 3))
    f32 = lambda a: np.ascontiguousarray(np.asarray(a, np.float32))
    out = scene.subset()
    out.s_pos = f32(np.concatenate([scene.s_pos, [d[0] for d in discs]]))
    out.s_rot = f32(np.concatenate([scene.s_rot, q]))
    out.s_scale = f32(np.concatenate([scene.s_scale, [d[3] for d in discs]]))
    out.s_sh = f32(np.concatenate([scene.s_sh, sh]))
    return out


def walls():
    """Ids n0..n0+3 after the background's n0 surfels: (0) a wall whose
    centre is behind the camera and whose far point at 0.9 r is behind the
    near plane too, (1) a wall whose centre is behind the camera but whose
    far point is in front, both reaching through the near plane; (2) a disc
    wholly behind the camera; (3) a disc seen edge-on."""
    P = np.array([0.3, 0.2, 2.0])
    etu = P / np.linalg.norm(P)
    etv = np.cross(etu, [1.0, 0.0, 0.0])
    etv /= np.linalg.norm(etv)
    return [((0.05, 0.0, -3.1), (0, 0, 1), (0, 1, 0), (1.0, 0.5)),
            ((-0.05, 0.0, -0.5), (0, 0, 1), (0, -1, 0), (0.5, 0.3)),
            ((0.0, 0.0, -1.0), (1, 0, 0), (0, 1, 0), (0.3, 0.3)),
            (tuple(P), tuple(etu), tuple(etv), (0.1, 0.1))]


def tilted():
    """A small disc crossing the near plane, tilted 60 degrees, close to the
    image centre."""
    return [((0.03, 0.02, 0.03), (1, 0, 0), (0, 0.5, math.sqrt(0.75)), (0.02, 0.02))]


def depth_extent(d, r=math.sqrt(2.0 * math.log(255.0))):
    """Half the camera-depth extent of disc d: r |(s1 tu_z, s2 tv_z)|."""
    return r * math.hypot(d[3][0] * d[1][2], d[3][1] * d[2][2])


def flat(scene):
    """The same scene with 2D Gaussians (the first two axes of each)."""
    sc = scene.subset()
    sc.g_scale = np.ascontiguousarray(sc.g_scale[:, :2])
    return sc


def with_splats(scene, splats, seed):
    """2D-Gaussian scene plus splats = [(centre, tu, tv, (s1, s2), opacity)],
    appended after the scene's own."""
    rng = np.random.Generator(np.random.PCG64(seed))
    tu = np.array([d[1] for d in splats], np.float64)
    tv = np.array([d[2] for d in splats], np.float64)
    q = sg._frame_to_quat(tu, tv, np.cross(tu, tv))
    sh = np.zeros((len(splats),) + scene.g_sh.shape[1:], np.float32)
    sh[:, 0, :] = rng.uniform(0.2, 1.0, (len(splats), 3))
    f32 = lambda a: np.ascontiguousarray(np.asarray(a, np.float32))
    out = scene.subset()
    out.g_pos = f32(np.concatenate([scene.g_pos, [d[0] for d in splats]]))
    out.g_rot = f32(np.concatenate([scene.g_rot, q]))
    out.g_scale = f32(np.concatenate([scene.g_scale, [d[3] for d in splats]]))
    out.g_opac = f32(np.concatenate([scene.g_opac, [d[4] for d in splats]]))
    out.g_sh = f32(np.concatenate([scene.g_sh, sh]))
    return out


def splats():
    """2D Gaussians with the centre in front of the camera that reach back
    through the near plane: (0) a wall in the plane x = -0.05 whose centre
    is 0.3 in front (reference pixel at the far point at 0.9 r), (1) a small
    splat crossing the near plane at 60 degrees."""
    return [((-0.05, 0.0, 0.3), (0, 0, 1), (0, -1, 0), (0.5, 0.3), 0.9),
            ((0.03, 0.02, 0.03), (1, 0, 0), (0, 0.5, math.sqrt(0.75)), (0.02, 0.02), 0.8)]
