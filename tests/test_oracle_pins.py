"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test ties one part of the oracle to a closed form, a library routine, an
invariant the paper states, brute force, the paper's printed constants, or
finite differences, chosen so that a dropped term, a wrong sign or index, or
a transposed operand fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import scenegen as sg

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "paper_constants.json")))


def ident_cam(W, H, f, cx=None, cy=None, bg=(0.0, 0.0, 0.0)):
    w2c = np.zeros((3, 4))
    w2c[:, :3] = np.eye(3)
    return sg.Camera(W, H, f, f, W / 2 if cx is None else cx, H / 2 if cy is None else cy, w2c, 0.01, bg)


def mk_scene(deg=3, s_pos=None, s_rot=None, s_scale=None, s_sh=None,
             g_pos=None, g_rot=None, g_scale=None, g_opac=None, g_sh=None):
    K = (deg + 1) ** 2
    z = lambda *shape: np.zeros(shape)
    return sg.Scene(deg,
                    z(0, 3) if s_pos is None else np.asarray(s_pos, float),
                    z(0, 4) if s_rot is None else np.asarray(s_rot, float),
                    z(0, 2) if s_scale is None else np.asarray(s_scale, float),
                    z(0, K, 3) if s_sh is None else np.asarray(s_sh, float),
                    z(0, 3) if g_pos is None else np.asarray(g_pos, float),
                    z(0, 4) if g_rot is None else np.asarray(g_rot, float),
                    z(0, 3) if g_scale is None else np.asarray(g_scale, float),
                    z(0) if g_opac is None else np.asarray(g_opac, float),
                    z(0, K, 3) if g_sh is None else np.asarray(g_sh, float))


def f64(scene):
    """Same scene with float64 arrays (for transforms that must not re-round)."""
    return sg.Scene(scene.sh_degree, *[np.asarray(v, np.float64) for v in scene.arrays().values()])


def pixel_dirs(cam):
    u = np.arange(cam.width) + 0.5
    v = np.arange(cam.height) + 0.5
    U, V = np.meshgrid(u, v)
    return (U - cam.cx) / cam.fx, (V - cam.cy) / cam.fy


# ---------------------------------------------------------------- SH (Eq. 1)

def _rand_dirs(n, seed=0):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def test_sh_low_order_closed_forms(oracle_lib):
    c0 = 1.0 / (2.0 * math.sqrt(math.pi))
    c1 = math.sqrt(3.0 / (4.0 * math.pi))
    for d in _rand_dirs(20):
        Y, _ = oracle_lib.sh_basis(3, d)
        x, y, z = d
        assert Y[0] == pytest.approx(c0, abs=1e-15)
        np.testing.assert_allclose(Y[1:4], [-c1 * y, c1 * z, -c1 * x], atol=1e-15)


def test_sh_matches_scipy_complex_harmonics(oracle_lib):
    """Real SH = sqrt2 Re/Im of scipy's complex SH (which carries the
    Condon-Shortley phase), m = 0 unchanged."""
    from scipy.special import sph_harm_y
    for d in _rand_dirs(25, seed=1):
        th = math.acos(np.clip(d[2], -1, 1))
        ph = math.atan2(d[1], d[0])
        Y, _ = oracle_lib.sh_basis(3, d)
        for l in range(4):
            for m in range(-l, l + 1):
                Yc = sph_harm_y(l, abs(m), th, ph)
                ref = Yc.real if m == 0 else math.sqrt(2) * (Yc.real if m > 0 else Yc.imag)
                assert Y[l * l + l + m] == pytest.approx(ref, abs=1e-12), (l, m)


def test_sh_orthonormal_by_quadrature(oracle_lib):
    zn, zw = np.polynomial.legendre.leggauss(16)
    nphi = 32
    G = np.zeros((16, 16))
    for z, w in zip(zn, zw):
        s = math.sqrt(1 - z * z)
        for k in range(nphi):
            ph = 2 * math.pi * k / nphi
            Y, _ = oracle_lib.sh_basis(3, [s * math.cos(ph), s * math.sin(ph), z])
            G += np.outer(Y, Y) * w * (2 * math.pi / nphi)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_gradient_matches_tangential_fd(oracle_lib):
    h = 1e-6
    for d in _rand_dirs(10, seed=2):
        Y, dY = oracle_lib.sh_basis(3, d)
        P = np.eye(3) - np.outer(d, d)
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            Yp, _ = oracle_lib.sh_basis(3, (d + e) / np.linalg.norm(d + e))
            Ym, _ = oracle_lib.sh_basis(3, (d - e) / np.linalg.norm(d - e))
            fd = (Yp - Ym) / (2 * h)
            np.testing.assert_allclose(fd, (dY @ P)[:, a], atol=1e-8)


# ------------------------------------------------------ surfel pass (Sec. 3)

def _disc_scene(z0, s, deg=0, dc=(0.4, 0.6, 0.8)):
    K = (deg + 1) ** 2
    sh = np.zeros((1, K, 3))
    sh[0, 0] = dc
    return mk_scene(deg, s_pos=[[0.0, 0.0, z0]], s_rot=[[1.0, 0, 0, 0]], s_scale=[[s, s]], s_sh=sh)


def test_fronto_parallel_disc_closed_form(oracle_lib):
    cam = ident_cam(64, 64, 50.0)
    z0, s = 2.0, 0.1
    r2 = oracle_lib.DEFAULT_OPTS["surfel_r2"]
    out = oracle_lib.render(_disc_scene(z0, s), cam)
    dx, dy = pixel_dirs(cam)
    lhs = (dx ** 2 + dy ** 2) * (z0 / s) ** 2
    assert np.min(np.abs(lhs - r2)) > 1e-6  # no pixel centre sits on the rim
    np.testing.assert_array_equal(out["id"] == 0, lhs <= r2)
    cov = out["id"] == 0
    np.testing.assert_allclose(out["depth"][cov], z0, rtol=1e-14)
    assert np.all(np.isinf(out["depth"][~cov]))
    # colour of a degree-0 surfel: 0.5 + Y00 * DC (Eq. 1)
    want = 0.5 + np.array([0.4, 0.6, 0.8]) / (2 * math.sqrt(math.pi))
    np.testing.assert_allclose(out["rgb"][:, cov].T, np.broadcast_to(want, (cov.sum(), 3)), rtol=1e-14)


def test_opaque_radius_is_papers_value(oracle_lib):
    r = math.sqrt(oracle_lib.DEFAULT_OPTS["surfel_r2"])
    g = GOLD["opaque_radius"]
    assert abs(r - g["value"]) <= g["abs_tol"]
    # and the rendered disc has that radius in local units: largest covered and
    # smallest uncovered local radius bracket it
    cam = ident_cam(96, 96, 80.0)
    z0, s = 3.0, 0.12
    out = oracle_lib.render(_disc_scene(z0, s), cam)
    dx, dy = pixel_dirs(cam)
    rl = np.sqrt(dx ** 2 + dy ** 2) * z0 / s
    assert rl[out["id"] == 0].max() <= r < rl[out["id"] < 0].min()


def _homography_rho_depth(scene, cam, i):
    """(a, b) of every pixel by inverting the 2DGS-style homography
    K [s1 tu, s2 tv, p] (an independent route to the ray-plane hit)."""
    q = scene.s_rot[i] / np.linalg.norm(scene.s_rot[i])
    w, x, y, z = q
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    Rc, tc = cam.world_to_cam[:, :3], cam.world_to_cam[:, 3]
    M = Rc @ np.stack([R[:, 0] * scene.s_scale[i, 0], R[:, 1] * scene.s_scale[i, 1],
                       scene.s_pos[i]], 1)
    M[:, 2] += tc
    Kmat = np.array([[cam.fx, 0, cam.cx], [0, cam.fy, cam.cy], [0, 0, 1.0]])
    Hinv = np.linalg.inv(Kmat @ M)
    u = np.arange(cam.width) + 0.5
    v = np.arange(cam.height) + 0.5
    U, V = np.meshgrid(u, v)
    P = np.stack([U, V, np.ones_like(U)], 0).reshape(3, -1)
    ab = Hinv @ P
    a, b = ab[0] / ab[2], ab[1] / ab[2]
    X = M @ np.stack([a, b, np.ones_like(a)])
    return (a * a + b * b).reshape(U.shape), X[2].reshape(U.shape), U, V


def test_tilted_surfel_ray_plane_equals_homography(oracle_lib):
    rng = np.random.default_rng(5)
    cam = sg.look_at((0.3, -0.2, -2.5), (0, 0, 0), (0, 1, 0), 48, 40, 50.0)
    # an exactly orthonormal rotation (float64), so that camera-space dot
    # products and the homography describe the same world-space disc
    U_, _, Vt_ = np.linalg.svd(cam.world_to_cam[:, :3].astype(np.float64))
    cam.world_to_cam = np.concatenate([U_ @ Vt_, cam.world_to_cam[:, 3:].astype(np.float64)], 1)
    for _ in range(4):
        q = rng.standard_normal(4)
        scene = f64(mk_scene(0, s_pos=[rng.uniform(-0.3, 0.3, 3)], s_rot=[q / np.linalg.norm(q)],
                             s_scale=[rng.uniform(0.05, 0.15, 2)], s_sh=[[[0.5, 0.5, 0.5]]]))
        rho_h, z_h, U, V = _homography_rho_depth(scene, cam, 0)
        px = np.floor(U).astype(np.int32).ravel()
        py = np.floor(V).astype(np.int32).ravel()
        z, rho, nd, ok = oracle_lib.surfel_eval(scene, cam, px, py, np.zeros_like(px))
        assert ok.all()
        np.testing.assert_allclose(rho, rho_h.ravel(), rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(z, z_h.ravel(), rtol=1e-10)


def test_zbuffer_is_min_depth_with_index_tiebreak(oracle_lib):
    """Two identical coplanar discs: the lower index wins (z-buffer with a
    strict less-than test, in draw order)."""
    cam = ident_cam(32, 32, 30.0)
    sc = mk_scene(0, s_pos=[[0, 0, 2.0], [0, 0, 2.0], [0, 0, 2.5]], s_rot=[[1.0, 0, 0, 0]] * 3,
                  s_scale=[[0.1, 0.1]] * 3, s_sh=[[[0.1, 0.1, 0.1]], [[0.9, 0.9, 0.9]], [[0.5, 0.5, 0.5]]])
    out = oracle_lib.render(sc, cam)
    assert set(np.unique(out["id"])) <= {-1, 0, 2}
    assert (out["id"] == 0).sum() > 0
    assert np.all(out["amb"][out["id"] == 0] & 1)  # exact tie is flagged as ambiguous


def _random_small(seed, n_s=60, n_g=200):
    sc = sg.random_scene(seed, n_s, n_g, n_objects=4, box=1.0, sphere_r=(0.3, 0.6),
                         plane_side=(0.6, 1.2), surfel_scale=(0.05, 0.15), gauss_logscale=(-3.5, 0.4))
    return sc


@pytest.mark.parametrize("seed", [11, 12])
def test_culled_equals_brute_force_bitwise(oracle_lib, seed):
    sc = _random_small(seed)
    # a camera inside the scene's extent: discs straddle the near plane
    cams = [sg.look_at((0.0, 0.0, -2.6), (0, 0, 0), (0, 1, 0), 53, 37, 60.0),
            sg.look_at((0.2, 0.1, -0.5), (0, 0.1, 1), (0, 1, 0), 40, 29, 90.0)]
    for cam in cams:
        for mode in (0, 1, 2):
            a = oracle_lib.render(sc, cam, dict(mode=mode), culled=True)
            b = oracle_lib.render(sc, cam, dict(mode=mode), culled=False)
            for k in a:
                np.testing.assert_array_equal(a[k], b[k], err_msg=f"{k} mode={mode}")


def test_discs_at_and_behind_the_camera_brute_force_and_closed_form(oracle_lib):
    """Discs reaching through the near plane from behind the camera, one
    wholly behind it and one edge-on, and 2D-Gaussian splats reaching back
    through it: the culled render equals brute force bitwise, and where the wall in the plane x = 0.05 wins, its depth is the
    ray-plane hit z = 0.05 fx / (u + 1/2 - cx) (a pixel ray (du, dv, 1)
    meets x = 0.05 at t = 0.05 / du)."""
    import camera_discs as cd
    cam, base = cd.camera(), cd.background()
    n0 = base.n_surfels
    scenes = [cd.with_discs(base, cd.walls(), 37), cd.with_discs(base, cd.tilted(), 38)]
    scenes += [cd.with_splats(cd.flat(base), [sp], 40 + k) for k, sp in enumerate(cd.splats())]
    for sc in scenes:
        a = oracle_lib.render(sc, cam, culled=True)
        b = oracle_lib.render(sc, cam, culled=False)
        for k in a:
            np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    sc = cd.with_discs(base, cd.walls(), 37)
    a = oracle_lib.render(sc, cam)
    jj, ii = np.nonzero(a["id"] == n0)
    assert jj.size > 1000
    z = 0.05 * cam.fx / (ii + 0.5 - cam.cx)
    # the scene is float32: the plane sits at float32(0.05), the frame at float32 rounding
    np.testing.assert_allclose(a["depth"][jj, ii], z, rtol=1e-6)
    assert not (a["id"] == n0 + 2).any()           # wholly behind the camera
    assert not (a["id"] == n0 + 3).any()           # edge-on: no area on screen


def test_frame_tilt_moves_depth_by_the_ratio_bound(oracle_lib):
    """The depth tolerance's frame term: tilting a disc's frame by eps about
    an axis through its centre P moves the hit X = z d by at most
    eps |X - P| / (|X| |cos|) relative (first order: t = n.P / n.d, so
    dz/z = delta.(P - X) / n.P and |n.P| = |X| |cos|).  Checked in FP64 on the
    wall whose centre is 3.1 behind the camera (|X - P| / |X| about 45), where
    the bound must also be nearly reached."""
    import camera_discs as cd
    cam = cd.camera()
    sc = f64(cd.with_discs(cd.background().subset(s_idx=np.zeros(0, int)), cd.walls()[:1], 37))
    eps = 1e-7
    tilted = f64(sc)
    tilted.s_rot = _quat_mul(sc.s_rot[0], np.array([[math.cos(eps / 2), 0.0, math.sin(eps / 2), 0.0]]))
    jj, ii = np.nonzero(oracle_lib.render(sc, cam)["id"] == 0)
    assert jj.size > 1000
    z0, _, nd, ok = oracle_lib.surfel_eval(sc, cam, ii, jj, np.zeros(ii.size, int))
    z1, _, _, ok1 = oracle_lib.surfel_eval(tilted, cam, ii, jj, np.zeros(ii.size, int))
    keep = (ok != 0) & (ok1 != 0)
    d = np.stack([(ii + 0.5 - cam.cx) / cam.fx, (jj + 0.5 - cam.cy) / cam.fy, np.ones(ii.size)], 1)[keep]
    X = z0[keep, None] * d
    ratio = np.linalg.norm(X - sc.s_pos[0], axis=1) / np.linalg.norm(X, axis=1)
    rel = np.abs(z1[keep] - z0[keep]) / z0[keep]
    bound = eps * ratio / np.abs(nd[keep])
    assert ratio.min() > 10.0                          # far outside the 0.3 of small discs
    assert np.all(rel <= bound * (1 + 1e-6))
    assert (rel / bound).max() > 0.5                   # the ratio term is needed, not just safe


def test_culled_equals_brute_force_parity_workload(oracle_lib):
    sc, cams = sg.config_scene(0)
    a = oracle_lib.render(sc, cams[0], culled=True)
    b = oracle_lib.render(sc, cams[0], culled=False)
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])


def _quat_mul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b.T
    return np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], 1)


def _rot_of(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _move(scene, cam, q, t):
    """Apply the rigid motion x -> R x + t to scene and camera together."""
    R = _rot_of(q)
    s = f64(scene)
    s.s_pos = s.s_pos @ R.T + t
    s.g_pos = s.g_pos @ R.T + t
    s.s_rot = _quat_mul(q, s.s_rot / np.linalg.norm(s.s_rot, axis=1, keepdims=True))
    s.g_rot = _quat_mul(q, s.g_rot / np.linalg.norm(s.g_rot, axis=1, keepdims=True))
    Rc, tc = cam.world_to_cam[:, :3].astype(float), cam.world_to_cam[:, 3].astype(float)
    w2c = np.concatenate([Rc @ R.T, (tc - Rc @ R.T @ t)[:, None]], 1)
    c2 = sg.Camera(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, w2c, cam.znear, cam.bg)
    return s, c2


def test_rigid_motion_invariance(oracle_lib):
    sc = f64(_random_small(21))
    cam = sg.look_at((0.0, 0.3, -2.6), (0, 0, 0), (0, 1, 0), 48, 36, 60.0)
    cam.world_to_cam = cam.world_to_cam.astype(np.float64)
    ref = oracle_lib.render(sc, cam)
    # translation: directions unchanged, so even SH colour is invariant
    s2, c2 = _move(sc, cam, np.array([1.0, 0, 0, 0]), np.array([0.7, -1.3, 2.1]))
    out = oracle_lib.render(s2, c2)
    np.testing.assert_array_equal(out["id"], ref["id"])
    np.testing.assert_allclose(out["depth"], ref["depth"], rtol=1e-10)
    np.testing.assert_allclose(out["rgb"], ref["rgb"], atol=1e-10)
    # rotation: geometry invariant; with SH degree 0 so is the colour
    sc0 = mk_scene(0, sc.s_pos, sc.s_rot, sc.s_scale, sc.s_sh[:, :1], sc.g_pos, sc.g_rot, sc.g_scale,
                   sc.g_opac, sc.g_sh[:, :1])
    ref0 = oracle_lib.render(sc0, cam)
    q = np.array([0.8, 0.3, -0.4, 0.33])
    q /= np.linalg.norm(q)
    s3, c3 = _move(sc0, cam, q, np.array([0.2, 0.5, -0.4]))
    out = oracle_lib.render(s3, c3)
    ok = (ref0["amb"] == 0)
    np.testing.assert_array_equal(out["id"][ok], ref0["id"][ok])
    np.testing.assert_allclose(out["depth"], ref0["depth"], rtol=1e-10)
    np.testing.assert_allclose(out["wg"], ref0["wg"], atol=1e-10)
    np.testing.assert_allclose(out["rgb"], ref0["rgb"], atol=1e-10)


def test_gaussian_order_does_not_matter(oracle_lib):
    """Sorting-free accumulation (Sec. 3, after Eq. 5)."""
    sc, cams = sg.config_scene(0)
    ref = oracle_lib.render(sc, cams[0])
    perm = np.random.default_rng(3).permutation(sc.n_gaussians)
    out = oracle_lib.render(sc.subset(g_idx=perm), cams[0])
    np.testing.assert_array_equal(out["id"], ref["id"])
    np.testing.assert_allclose(out["rgb"], ref["rgb"], atol=1e-12)
    np.testing.assert_allclose(out["wg"], ref["wg"], atol=1e-12)


def test_surfel_order_only_relabels_ids(oracle_lib):
    sc, cams = sg.config_scene(0)
    ref = oracle_lib.render(sc, cams[0])
    perm = np.random.default_rng(4).permutation(sc.n_surfels)
    out = oracle_lib.render(sc.subset(s_idx=perm), cams[0])
    lab = np.where(out["id"] >= 0, perm[np.maximum(out["id"], 0)], -1)
    ok = (ref["amb"] & 1) == 0
    np.testing.assert_array_equal(lab[ok], ref["id"][ok])
    np.testing.assert_array_equal(out["depth"][ok], ref["depth"][ok])
    np.testing.assert_array_equal(out["rgb"][:, ok], ref["rgb"][:, ok])


# ---------------------------------------------------- Gaussian pass (Eq. 2-4)

def _one_gaussian(z0, s, sigma, dc=(0.3, 0.5, 0.7), offset=(0.0, 0.0)):
    sh = np.zeros((1, 1, 3))
    sh[0, 0] = dc
    return mk_scene(0, g_pos=[[offset[0], offset[1], z0]], g_rot=[[1.0, 0, 0, 0]], g_scale=[[s, s, s]],
                    g_opac=[sigma], g_sh=sh)


def test_single_gaussian_closed_form(oracle_lib):
    """Isotropic Gaussian on the optical axis: Sigma2 = ((f s/z)^2 + 0.3) I,
    alpha at the centre pixel = sigma, C = sigma c/(1 + sigma) over bg 0."""
    f, z0, s, sig = 40.0, 2.0, 0.05, 0.7
    cam = ident_cam(65, 65, f, cx=32.5, cy=32.5)
    sc = _one_gaussian(z0, s, sig)
    info = oracle_lib.gauss_info(sc, cam, 0)
    var = (f * s / z0) ** 2 + 0.3
    np.testing.assert_allclose(info["sigma2"], [var, 0.0, var], atol=1e-14)
    np.testing.assert_allclose([info["px"], info["py"]], [32.5, 32.5], atol=1e-14)
    out = oracle_lib.render(sc, cam)
    c = 0.5 + np.array([0.3, 0.5, 0.7]) / (2 * math.sqrt(math.pi))
    np.testing.assert_allclose(out["rgb"][:, 32, 32], sig * c / (1 + sig), rtol=1e-14)
    # footprint: alpha >= 1/255 exactly where r^2/var <= 2 ln(255 sigma)
    dx, dy = np.meshgrid(np.arange(65) + 0.5 - 32.5, np.arange(65) + 0.5 - 32.5)
    alpha = sig * np.exp(-0.5 * (dx ** 2 + dy ** 2) / var)
    cut = GOLD["alpha_cutoff"]["value"]
    assert np.min(np.abs(alpha - cut)) > 1e-9
    np.testing.assert_array_equal(out["ncontrib"] == 1, alpha >= cut)
    np.testing.assert_allclose(out["wg"], np.where(alpha >= cut, alpha, 0.0), rtol=1e-13, atol=0)


def test_eps_is_five_times_mean_axis(oracle_lib):
    g = GOLD["eps_factor"]
    sc = mk_scene(0, g_pos=[[0.1, 0.0, 2.0]], g_rot=[[0.9, 0.1, 0.2, 0.3]], g_scale=[[0.01, 0.02, 0.04]],
                  g_opac=[0.5], g_sh=np.zeros((1, 1, 3)))
    info = oracle_lib.gauss_info(sc, ident_cam(32, 32, 30.0), 0)
    assert info["eps"] == pytest.approx(g["value"] / g["dim"] * 0.07, rel=1e-14)
    info = oracle_lib.gauss_info(sc, ident_cam(32, 32, 30.0), 0, dict(eps_mode=2, eps_value=GOLD["eps_const_ablation"]["value"]))
    assert info["eps"] == 0.1


def _wall_scene(n_g, g_z, deg=0, seed=0, extra_g=None):
    """A large fronto-parallel surfel wall at z=1 and Gaussians at depth g_z."""
    rng = np.random.default_rng(seed)
    K = (deg + 1) ** 2
    s_sh = np.zeros((1, K, 3))
    s_sh[0, 0] = (0.2, 0.4, 0.6)
    g_pos = np.stack([rng.uniform(-0.3, 0.3, n_g), rng.uniform(-0.3, 0.3, n_g), np.full(n_g, g_z)], 1)
    g_sh = np.zeros((n_g, K, 3))
    g_sh[:, 0] = rng.uniform(0, 1, (n_g, 3))
    return mk_scene(deg, s_pos=[[0, 0, 1.0]], s_rot=[[1.0, 0, 0, 0]], s_scale=[[1.0, 1.0]], s_sh=s_sh,
                    g_pos=g_pos, g_rot=np.tile([1.0, 0, 0, 0], (n_g, 1)), g_scale=np.full((n_g, 3), 0.02),
                    g_opac=rng.uniform(0.3, 0.9, n_g), g_sh=g_sh)


def test_gaussians_behind_wall_are_hidden(oracle_lib):
    cam = ident_cam(40, 40, 40.0)
    sc = _wall_scene(30, 1.5)  # 0.5 behind the wall, eps = 5*0.02 = 0.1
    out = oracle_lib.render(sc, cam)
    assert np.all(out["id"] == 0)
    assert np.all(out["wg"] == 0)
    only_s = oracle_lib.render(sc, cam, dict(mode=1))
    np.testing.assert_array_equal(out["rgb"], only_s["rgb"])


def test_gaussian_on_surface_passes_depth_test(oracle_lib):
    """d_i = D_s < D_s + eps_i: a Gaussian centred on the surfel is kept;
    with eps = 0 (Table 5 ablation) the strict test drops it."""
    cam = ident_cam(40, 40, 40.0)
    sc = _wall_scene(10, 1.0)
    out = oracle_lib.render(sc, cam)
    assert out["wg"].max() > 0.1
    out0 = oracle_lib.render(sc, cam, dict(eps_mode=1))
    assert out0["wg"].max() == 0.0


def test_zero_gaussians_reproduces_surfel_map(oracle_lib):
    sc, cams = sg.config_scene(0)
    empty = sc.subset(g_idx=np.zeros(0, int))
    full = oracle_lib.render(empty, cams[0])
    only = oracle_lib.render(sc, cams[0], dict(mode=1))
    np.testing.assert_array_equal(full["rgb"], only["rgb"])
    np.testing.assert_array_equal(full["id"], only["id"])
    assert np.all(full["wg"] == 0)


def test_composite_decomposition(oracle_lib):
    """Surfel part C_s/(1+W_G) plus Gaussian part C_G/(1+W_G) is the image
    (Sec. 7, ablation).  Gaussians in front of the wall so that the
    Gaussians-only render (no depth test) has the same C_G, W_G."""
    cam = ident_cam(40, 40, 40.0)
    sc = _wall_scene(40, 0.8, seed=2)
    full = oracle_lib.render(sc, cam)
    s_only = oracle_lib.render(sc, cam, dict(mode=1))
    g_only = oracle_lib.render(sc, cam, dict(mode=2))
    np.testing.assert_allclose(g_only["wg"], full["wg"], rtol=0, atol=0)
    W = full["wg"]
    CG = np.where(W > 0, g_only["rgb"] * W, 0.0)
    np.testing.assert_allclose(s_only["rgb"] / (1 + W) + CG / (1 + W), full["rgb"], atol=1e-14)
    assert np.all(np.isinf(g_only["depth"])) and np.all(g_only["id"] == -1)


def test_background_where_nothing_covers(oracle_lib):
    cam = ident_cam(16, 12, 20.0, bg=(0.25, 0.5, 1.0))
    out = oracle_lib.render(mk_scene(3), cam)
    np.testing.assert_array_equal(out["rgb"], np.broadcast_to(np.array([0.25, 0.5, 1.0])[:, None, None], (3, 12, 16)))
    assert np.all(out["id"] == -1) and np.all(np.isinf(out["depth"]))
    g_only = oracle_lib.render(mk_scene(3), cam, dict(mode=2))
    np.testing.assert_array_equal(g_only["rgb"], out["rgb"])


# ------------------------------------------------- backward (Sec. 4.2, FD)

def _loss(oracle_lib, sc, cam, g):
    out = oracle_lib.render(sc, cam, nthreads=1)
    return float(np.sum(out["rgb"] * g)), out


@pytest.mark.parametrize("mode", [0, 2])
def test_backward_matches_central_differences(oracle_lib, mode):
    sc, cam = sg.crop_scene(7)
    sc = f64(sc)
    rng = np.random.default_rng(8)
    g = rng.standard_normal((3, cam.height, cam.width))
    opts = dict(mode=mode)
    grads = oracle_lib.backward(sc, cam, g, opts)
    base = oracle_lib.render(sc, cam, opts)
    assert base["ncontrib"].sum() > 200  # Gaussians do contribute
    checks = [("g_pos", "g_pos"), ("g_rot", "g_rot"), ("g_scale", "g_scale"), ("g_opac", "g_opac"),
              ("g_sh", "g_sh")]
    if mode == 0:
        checks.append(("s_sh", "s_sh"))
    n_checked = 0
    for arr_name, grad_name in checks:
        arr = getattr(sc, arr_name)
        flat = arr.reshape(-1)
        idx = range(flat.size) if flat.size <= 200 else rng.choice(flat.size, 200, replace=False)
        gmax = np.abs(grads[grad_name]).max()
        for k in idx:
            h = 1e-6 * max(1.0, abs(flat[k]))
            if arr_name == "g_scale":
                h = 1e-6 * abs(flat[k])
            old = flat[k]
            flat[k] = old + h
            lp, op = _loss_mode(oracle_lib, sc, cam, g, opts)
            flat[k] = old - h
            lm, om = _loss_mode(oracle_lib, sc, cam, g, opts)
            flat[k] = old
            if not (np.array_equal(op["ncontrib"], om["ncontrib"]) and np.array_equal(op["id"], om["id"])
                    and np.array_equal(op["ncontrib"], base["ncontrib"])):
                continue  # a cutoff or depth-test flips inside [-h, h]: not differentiable here
            fd = (lp - lm) / (2 * h)
            an = grads[grad_name].reshape(-1)[k]
            assert abs(fd - an) <= 2e-5 * abs(an) + 1e-6 * gmax + 1e-9, (arr_name, k, fd, an)
            n_checked += 1
    assert n_checked > 300


def _loss_mode(oracle_lib, sc, cam, g, opts):
    out = oracle_lib.render(sc, cam, opts, nthreads=1)
    return float(np.sum(out["rgb"] * g)), out


def test_backward_surfel_geometry_gets_no_gradient_and_hidden_gaussians_none(oracle_lib):
    cam = ident_cam(40, 40, 40.0)
    sc = _wall_scene(20, 1.5)
    g = np.ones((3, 40, 40))
    gr = oracle_lib.backward(sc, cam, g)
    assert np.all(gr["g_pos"] == 0) and np.all(gr["g_opac"] == 0) and np.all(gr["g_sh"] == 0)
    # the wall wins every pixel with k = 1/(1+0) = 1: dL/dc_s = #pixels, dL/dSH_0 = Y00 * that
    np.testing.assert_allclose(gr["s_sh"][0, 0], 1600 / (2 * math.sqrt(math.pi)), rtol=1e-13)


def test_sh_direction_points_from_primitive_to_camera(oracle_lib):
    """Eq. 1 evaluates SH at the direction from the surfel centre to the
    camera position (Sec. 3).  A surfel/Gaussian carrying only the l=1, m=0
    coefficient (Y = sqrt(3/4pi) z) seen from -z gets 0.5 - sqrt(3/4pi) * c."""
    c1 = math.sqrt(3.0 / (4.0 * math.pi))
    cam = ident_cam(33, 33, 30.0, cx=16.5, cy=16.5)   # camera at the origin, looking along +z
    sh = np.zeros((1, 4, 3))
    sh[0, 2] = (0.4, 0.2, -0.1)
    sc = mk_scene(1, s_pos=[[0, 0, 2.0]], s_rot=[[1.0, 0, 0, 0]], s_scale=[[0.2, 0.2]], s_sh=sh)
    out = oracle_lib.render(sc, cam)
    np.testing.assert_allclose(out["rgb"][:, 16, 16], 0.5 - c1 * np.array([0.4, 0.2, -0.1]), rtol=1e-14)
    sg_ = mk_scene(1, g_pos=[[0, 0, 2.0]], g_rot=[[1.0, 0, 0, 0]], g_scale=[[0.01] * 3], g_opac=[0.5], g_sh=sh)
    info = oracle_lib.gauss_info(sg_, cam, 0)
    np.testing.assert_allclose(info["rgb"], 0.5 - c1 * np.array([0.4, 0.2, -0.1]), rtol=1e-14)


def test_touching_marks_exactly_the_primitives_at_flagged_pixels(oracle_lib):
    f, z0, s, sig = 40.0, 2.0, 0.05, 0.7
    cam = ident_cam(65, 65, f, cx=32.5, cy=32.5)
    sc = _one_gaussian(z0, s, sig)
    sc = mk_scene(0, s_pos=[[0.0, 0.0, 3.0], [5.0, 5.0, 3.0]], s_rot=[[1.0, 0, 0, 0]] * 2,
                  s_scale=[[0.1, 0.1]] * 2, s_sh=np.zeros((2, 1, 3)), g_pos=sc.g_pos, g_rot=sc.g_rot,
                  g_scale=sc.g_scale, g_opac=sc.g_opac, g_sh=sc.g_sh)
    flag = np.zeros((65, 65), np.uint8)
    st, gt = oracle_lib.touching(sc, cam, flag)
    assert not st.any() and not gt.any()
    flag[32, 32] = 1   # the Gaussian's centre pixel, inside surfel 0's disc
    st, gt = oracle_lib.touching(sc, cam, flag)
    assert st.tolist() == [True, False] and gt.tolist() == [True]
    flag[:] = 0
    flag[0, 0] = 1     # far from everything
    st, gt = oracle_lib.touching(sc, cam, flag)
    assert not st.any() and not gt.any()


def _raw_check(oracle_lib, sc, cam, ids):
    import ctypes
    lib = oracle_lib.load()
    pin = oracle_lib.oracle._Pinned(sc, cam, None)
    ids = np.ascontiguousarray(ids, np.int32)
    v = np.empty(ids.shape, np.uint8)
    assert lib.ora_check_ids(ctypes.byref(pin.s), ctypes.byref(pin.c), ctypes.byref(pin.o),
                             ids.ctypes.data, v.ctypes.data) == 0
    return v.astype(bool)


def test_id_check_accepts_exactly_the_correct_answers(oracle_lib):
    sc, cams = sg.config_scene(0)
    cam = cams[0]
    ref = oracle_lib.render(sc, cam)
    # the oracle's own answer is acceptable everywhere
    assert _raw_check(oracle_lib, sc, cam, ref["id"]).all()
    amb = (ref["amb"] & 1) != 0
    cov = ref["id"] >= 0
    # "nothing here" where a surfel clearly covers the pixel is wrong
    v = _raw_check(oracle_lib, sc, cam, np.where(cov, -1, ref["id"]))
    assert not v[cov & ~amb].any()
    # a surfel that does not cover the pixel at all is wrong
    far = np.where(cov, (ref["id"] + 500) % sc.n_surfels, ref["id"])
    z, rho, nd, ok = oracle_lib.surfel_eval(sc, cam, *np.nonzero(cov)[::-1], far[cov])
    outside = (ok == 0) | (rho > oracle_lib.DEFAULT_OPTS["surfel_r2"] * 1.01)
    v = _raw_check(oracle_lib, sc, cam, far)
    assert not v[cov][outside].any()


def test_id_check_tie_and_runner_up(oracle_lib):
    """Two identical coplanar discs: both ids are correct.  A disc clearly
    behind another one is not."""
    cam = ident_cam(32, 32, 30.0)
    sc = mk_scene(0, s_pos=[[0, 0, 2.0], [0, 0, 2.0], [0, 0, 2.5]], s_rot=[[1.0, 0, 0, 0]] * 3,
                  s_scale=[[0.1, 0.1], [0.1, 0.1], [0.2, 0.2]], s_sh=np.zeros((3, 1, 3)))
    ref = oracle_lib.render(sc, cam)
    both = ref["id"] == 0
    assert _raw_check(oracle_lib, sc, cam, np.where(both, 1, ref["id"]))[both].all()
    assert not _raw_check(oracle_lib, sc, cam, np.where(both, 2, ref["id"]))[both].any()


def test_fragment_counts_closed_form(oracle_lib):
    """A lone fronto-parallel disc covers exactly the closed-form pixel set; a
    lone on-axis Gaussian has exactly its closed-form 1/255 footprint."""
    cam = ident_cam(64, 64, 50.0)
    z0, s = 2.0, 0.1
    ns, ng = oracle_lib.count_fragments(_disc_scene(z0, s), cam)
    dx, dy = pixel_dirs(cam)
    assert ns == int(((dx ** 2 + dy ** 2) * (z0 / s) ** 2 <= oracle_lib.DEFAULT_OPTS["surfel_r2"]).sum()) and ng == 0
    cam = ident_cam(65, 65, 40.0, cx=32.5, cy=32.5)
    ns, ng = oracle_lib.count_fragments(_one_gaussian(2.0, 0.05, 0.7), cam)
    var = (40.0 * 0.05 / 2.0) ** 2 + 0.3
    dx, dy = np.meshgrid(np.arange(65) + 0.5 - 32.5, np.arange(65) + 0.5 - 32.5)
    assert ns == 0 and ng == int((0.7 * np.exp(-0.5 * (dx ** 2 + dy ** 2) / var) >= 1 / 255).sum())
