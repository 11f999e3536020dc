"""Pins of the oracle's 2D-GES pass 2 (Sec. 6.4, Eq. 17-18: 2D Gaussians with
planar depth and the object-space EWA filter) and of the geometry maps
(Eq. 10-12) on the CPU.

The 2D Gaussian is tied to things computed another way: to the 3D Gaussian
with the screen filter where the object-space filter is exact (an on-axis,
fronto-parallel splat), to the homography inverse of the splat with a Jacobian
taken by finite differences, and to depth maps read back as 3D points.
"""
import numpy as np
import pytest

import scenegen as sg
from test_oracle_mip_pins import _rot
from test_oracle_pins import _wall_scene, f64, ident_cam, mk_scene


def _splat_scene(pos, q, s, sigma, dc=(0.3, 0.5, 0.7), surfels=None):
    sh = np.zeros((1, 1, 3))
    sh[0, 0] = dc
    kw = {}
    if surfels is not None:
        kw = dict(s_pos=surfels["pos"], s_rot=surfels["rot"], s_scale=surfels["scale"], s_sh=surfels["sh"])
    return mk_scene(0, g_pos=[pos], g_rot=[q], g_scale=[s], g_opac=[sigma], g_sh=sh, **kw)


def _ortho_cam(cam):
    U_, _, Vt_ = np.linalg.svd(cam.world_to_cam[:, :3].astype(np.float64))
    cam.world_to_cam = np.concatenate([U_ @ Vt_, cam.world_to_cam[:, 3:].astype(np.float64)], 1)
    return cam


def _splat_homography(pos, q, s, cam):
    """(a, b, z) of every pixel centre on the plane of the splat (local units
    of the scales s), by inverting the homography K [s1 tu, s2 tv, p]."""
    R = _rot(q)
    Rc, tc = cam.world_to_cam[:, :3], cam.world_to_cam[:, 3]
    M = Rc @ np.stack([R[:, 0] * s[0], R[:, 1] * s[1], np.asarray(pos, float)], 1)
    M[:, 2] += tc
    Kmat = np.array([[cam.fx, 0, cam.cx], [0, cam.fy, cam.cy], [0, 0, 1.0]])
    U, V = np.meshgrid(np.arange(cam.width) + 0.5, np.arange(cam.height) + 0.5)
    ab = np.linalg.inv(Kmat @ M) @ np.stack([U, V, np.ones_like(U)], 0).reshape(3, -1)
    a, b = ab[0] / ab[2], ab[1] / ab[2]
    X = M @ np.stack([a, b, np.ones_like(a)])
    return a.reshape(U.shape), b.reshape(U.shape), X[2].reshape(U.shape)


def _filter_factors_fd(pos, q, s, cam, r, h=1e-7):
    """S_k = sqrt(1 + r ((J^T J)^-1)_kk) with J, local unit coordinates ->
    pixels at the centre, by central differences of the projection."""
    R = _rot(q)
    Rc, tc = cam.world_to_cam[:, :3], cam.world_to_cam[:, 3]

    def proj(a, b):
        X = Rc @ (np.asarray(pos, float) + a * s[0] * R[:, 0] + b * s[1] * R[:, 1]) + tc
        return np.array([cam.fx * X[0] / X[2] + cam.cx, cam.fy * X[1] / X[2] + cam.cy])

    J = np.stack([(proj(h, 0) - proj(-h, 0)) / (2 * h), (proj(0, h) - proj(0, -h)) / (2 * h)], 1)
    Minv = np.linalg.inv(J.T @ J)
    return np.sqrt(1 + r * Minv[0, 0]), np.sqrt(1 + r * Minv[1, 1])


@pytest.mark.parametrize("angle", [0.0, 0.7])
def test_onaxis_splat_equals_3d_gaussian_with_screen_filter(oracle_lib, angle):
    """A fronto-parallel splat on the optical axis: J is diagonal up to an
    in-plane rotation, the object-space filter is exact, and the splat must
    render exactly like a flat 3D Gaussian under the Mip screen filter of the
    same size (Eq. 17 = Eq. 18)."""
    cam = ident_cam(65, 65, 45.0, cx=32.5, cy=32.5)
    q = [np.cos(angle / 2), 0.0, 0.0, np.sin(angle / 2)]
    s2 = _splat_scene([0.0, 0.0, 2.0], q, [0.15, 0.055], 0.7)
    s3 = _splat_scene([0.0, 0.0, 2.0], q, [0.15, 0.055, 1e-9], 0.7)
    opts = dict(eps_mode=2, eps_value=0.1)
    for lp in (0.3, 1.0):
        a = oracle_lib.render(s2, cam, dict(opts, lowpass=lp))
        b = oracle_lib.render(s3, cam, dict(opts, lowpass=lp, filter=1))
        assert (a["wg"] > 0).sum() > 50
        np.testing.assert_allclose(a["wg"], b["wg"], rtol=1e-10, atol=1e-15)
        np.testing.assert_allclose(a["rgb"], b["rgb"], rtol=1e-10, atol=1e-15)


def test_tilted_splat_equals_homography(oracle_lib):
    """alpha = sigma/(S1 S2) exp(-(a'^2 + b'^2)/2) at the ray-splat hit, with
    (a', b') from the homography of the filtered splat and S from a
    finite-difference Jacobian."""
    rng = np.random.default_rng(7)
    cam = _ortho_cam(sg.look_at((0.3, -0.2, -2.5), (0, 0, 0), (0, 1, 0), 56, 44, 50.0))
    n_checked = 0
    for _ in range(5):
        q = rng.standard_normal(4)
        q /= np.linalg.norm(q)
        pos, s, sig = rng.uniform(-0.2, 0.2, 3), rng.uniform(0.03, 0.12, 2), 0.8
        sc = f64(_splat_scene(pos, q, s, sig))
        out = oracle_lib.render(sc, cam, dict(mode=2))
        S1, S2 = _filter_factors_fd(pos, q, s, cam, 0.3)
        info = oracle_lib.gauss_info(sc, cam, 0)
        np.testing.assert_allclose(info["S"], [S1, S2], rtol=1e-6)
        a, b, z = _splat_homography(pos, q, s * np.array([S1, S2]), cam)
        alpha = sig / (S1 * S2) * np.exp(-0.5 * (a * a + b * b))
        keep = (alpha >= 1 / 255 * (1 + 1e-5)) & (z > 0.01)
        drop = alpha < 1 / 255 * (1 - 1e-5)
        W = out["wg"]
        np.testing.assert_allclose(W[keep], alpha[keep], rtol=1e-5)
        assert np.all(W[drop] == 0)
        n_checked += keep.sum()
    assert n_checked > 300


def test_planar_depth_decides_the_depth_test(oracle_lib):
    """A splat tilted through an opaque wall (eps = 0): it contributes exactly
    where its planar depth is in front of the wall."""
    cam = _ortho_cam(ident_cam(60, 60, 50.0))
    q = np.array([np.cos(0.5), np.sin(0.5), 0.0, 0.0])     # tilted about x
    wall = _wall_scene(0, 1.0)
    sc = f64(_splat_scene([0.0, 0.0, 1.0], q, [0.2, 0.2], 0.9,
                          surfels=dict(pos=wall.s_pos, rot=wall.s_rot, scale=wall.s_scale, sh=wall.s_sh)))
    out = oracle_lib.render(sc, cam, dict(eps_mode=1))
    S1, S2 = _filter_factors_fd([0, 0, 1.0], q, [0.2, 0.2], cam, 0.3)
    a, b, z = _splat_homography([0, 0, 1.0], q, np.array([0.2 * S1, 0.2 * S2]), cam)
    alpha = 0.9 / (S1 * S2) * np.exp(-0.5 * (a * a + b * b))
    inside = alpha >= 1 / 255 * (1 + 1e-5)
    front = inside & (z < 1.0 - 1e-9)
    behind = inside & (z > 1.0 + 1e-9)
    assert front.sum() > 100 and behind.sum() > 100
    assert np.all(out["wg"][front] > 0) and np.all(out["wg"][behind] == 0)


def test_geometry_maps_of_a_tilted_surfel(oracle_lib):
    """N_s is the unit plane normal facing the camera: it equals the normal of
    the plane through the depth map's 3D points; with no Gaussians the smoothed
    maps are D_s and N_s, and +inf / 0 where nothing covers."""
    cam = _ortho_cam(sg.look_at((0.3, -0.2, -2.5), (0, 0, 0), (0, 1, 0), 48, 40, 50.0))
    q = np.array([0.8, 0.3, -0.4, 0.2])
    sc = f64(mk_scene(0, s_pos=[[0.05, 0.0, 0.1]], s_rot=[q / np.linalg.norm(q)], s_scale=[[0.25, 0.15]],
                      s_sh=[[[0.5, 0.5, 0.5]]]))
    geo = oracle_lib.render_geom(sc, cam)
    out = oracle_lib.render(sc, cam)
    cov = out["id"] >= 0
    assert cov.sum() > 150
    U, V = np.meshgrid(np.arange(cam.width) + 0.5, np.arange(cam.height) + 0.5)
    X = np.stack([(U - cam.cx) / cam.fx, (V - cam.cy) / cam.fy, np.ones_like(U)]) * out["depth"]
    j, i = np.argwhere(cov[1:-1, 1:-1] & cov[2:, 1:-1] & cov[1:-1, 2:])[0] + 1
    n = np.cross(X[:, j, i + 1] - X[:, j, i], X[:, j + 1, i] - X[:, j, i])
    n /= np.linalg.norm(n)
    n = -n if n @ X[:, j, i] > 0 else n
    Ns = geo["ns"][:, cov]
    np.testing.assert_allclose(Ns, np.broadcast_to(n[:, None], Ns.shape), atol=1e-9)
    np.testing.assert_allclose(np.linalg.norm(Ns, axis=0), 1.0, rtol=1e-12)
    np.testing.assert_array_equal(geo["dsmooth"][cov], out["depth"][cov])
    np.testing.assert_array_equal(geo["nsmooth"][:, cov], Ns)
    assert np.all(np.isinf(geo["dsmooth"][~cov])) and np.all(geo["nsmooth"][:, ~cov] == 0)


def test_geometry_of_gaussians_alone(oracle_lib):
    """No surfels: D_smooth = D_G / W_G is the centre depth for a 3D Gaussian
    and the planar depth for a 2D one; N_smooth their normal (smallest axis /
    splat normal, camera space, facing the camera)."""
    cam = _ortho_cam(sg.look_at((0.3, -0.2, -2.5), (0, 0, 0), (0, 1, 0), 48, 40, 50.0))
    q = np.array([0.8, 0.3, -0.4, 0.2])
    q /= np.linalg.norm(q)
    R, Rc, tc = _rot(q), cam.world_to_cam[:, :3], cam.world_to_cam[:, 3]
    pos = np.array([0.05, 0.0, 0.1])
    t = Rc @ pos + tc
    # 3D: scales with the smallest along the second axis
    s3 = f64(_splat_scene(pos, q, [0.25, 0.04, 0.16], 0.8))
    g3 = oracle_lib.render_geom(s3, cam)
    w3 = oracle_lib.render(s3, cam)["wg"] > 0
    assert w3.sum() > 100
    n3 = Rc @ R[:, 1]
    n3 = -n3 if n3 @ t > 0 else n3
    np.testing.assert_allclose(g3["dsmooth"][w3], t[2], rtol=1e-12)
    np.testing.assert_allclose(g3["nsmooth"][:, w3], np.broadcast_to(n3[:, None], (3, w3.sum())), atol=1e-12)
    # 2D splat
    s2 = f64(_splat_scene(pos, q, [0.25, 0.16], 0.8))
    g2 = oracle_lib.render_geom(s2, cam)
    w2 = oracle_lib.render(s2, cam)["wg"] > 0
    assert w2.sum() > 100
    n2 = Rc @ R[:, 2]
    n2 = -n2 if n2 @ t > 0 else n2
    _, _, z = _splat_homography(pos, q, [0.25, 0.16], cam)
    np.testing.assert_allclose(g2["dsmooth"][w2], z[w2], rtol=1e-10)
    np.testing.assert_allclose(g2["nsmooth"][:, w2], np.broadcast_to(n2[:, None], (3, w2.sum())), atol=1e-12)


@pytest.mark.parametrize("dim", [3, 2])
def test_geometry_eq12_decomposition(oracle_lib, dim):
    """(W_s + W_G) D_smooth - D_G = D_s and (W_s + W_G) N_smooth - N_G = N_s
    where a surfel covers (W_s = 1)."""
    cam = ident_cam(40, 40, 40.0)
    sc = _wall_scene(40, 0.9, seed=3)
    if dim == 2:
        sc.g_scale = sc.g_scale[:, :2].copy()
        rng = np.random.default_rng(4)
        q = rng.standard_normal((sc.n_gaussians, 4))
        sc.g_rot = q / np.linalg.norm(q, axis=1, keepdims=True)
    out = oracle_lib.render(sc, cam)
    geo = oracle_lib.render_geom(sc, cam)
    W = out["wg"]
    assert (W > 0).mean() > 0.3 and np.all(out["id"] == 0)
    np.testing.assert_allclose((1 + W) * geo["dsmooth"] - geo["dg"], out["depth"], rtol=1e-12)
    np.testing.assert_allclose((1 + W)[None] * geo["nsmooth"] - geo["ng"], geo["ns"], atol=1e-12)
    np.testing.assert_allclose(geo["ns"][2], -1.0)


def _random_2d(seed, n_s=60, n_g=200):
    sc = sg.random_scene(seed, n_s, n_g, n_objects=4, box=1.0, sphere_r=(0.3, 0.6), plane_side=(0.6, 1.2),
                         surfel_scale=(0.05, 0.15), gauss_logscale=(-3.0, 0.4))
    sc.g_scale = np.ascontiguousarray(sc.g_scale[:, :2])
    return sc


def test_2d_culled_equals_brute_force_bitwise(oracle_lib):
    sc = _random_2d(71)
    cams = [sg.look_at((0.0, 0.0, -2.6), (0, 0, 0), (0, 1, 0), 53, 37, 60.0),
            sg.look_at((0.2, 0.1, -0.5), (0, 0.1, 1), (0, 1, 0), 40, 29, 90.0)]
    for cam in cams:
        for mode in (0, 2):
            a = oracle_lib.render(sc, cam, dict(mode=mode), culled=True)
            b = oracle_lib.render(sc, cam, dict(mode=mode), culled=False)
            for k in a:
                np.testing.assert_array_equal(a[k], b[k], err_msg=f"{k} mode={mode}")
        ga = oracle_lib.render_geom(sc, cam, culled=True)
        gb = oracle_lib.render_geom(sc, cam, culled=False)
        for k in ga:
            np.testing.assert_array_equal(ga[k], gb[k], err_msg=k)
    assert (oracle_lib.render(sc, cams[0])["wg"] > 0).mean() > 0.2


@pytest.mark.parametrize("dim", [3, 2])
def test_geometry_gaussian_order_independent(oracle_lib, dim):
    sc = _random_2d(72) if dim == 2 else sg.random_scene(72, 60, 200, n_objects=4, box=1.0, sphere_r=(0.3, 0.6),
                                                         plane_side=(0.6, 1.2), surfel_scale=(0.05, 0.15),
                                                         gauss_logscale=(-3.0, 0.4))
    cam = sg.look_at((0.0, 0.2, -2.6), (0, 0, 0), (0, 1, 0), 53, 37, 60.0)
    perm = np.random.default_rng(1).permutation(sc.n_gaussians)
    a = oracle_lib.render_geom(sc, cam)
    b = oracle_lib.render_geom(sc.subset(g_idx=perm), cam)
    for k in ("ns", "dg", "ng", "nsmooth"):
        np.testing.assert_allclose(a[k], b[k], rtol=1e-12, atol=1e-12, err_msg=k)
    fin = np.isfinite(a["dsmooth"])
    np.testing.assert_array_equal(fin, np.isfinite(b["dsmooth"]))
    np.testing.assert_allclose(a["dsmooth"][fin], b["dsmooth"][fin], rtol=1e-12)


def test_2d_eps_uses_two_axes(oracle_lib):
    """eps_i = (5/D) sum_j s_ij with D = 2 for a 2D Gaussian (Sec. 5)."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_constants.json")))
    cam = ident_cam(32, 32, 30.0)
    sc = _splat_scene([0.0, 0.0, 2.0], [1.0, 0, 0, 0], [0.03, 0.05], 0.5)
    info = oracle_lib.gauss_info(sc, cam, 0)
    np.testing.assert_allclose(info["eps"], gold["eps_factor"]["value"] / 2.0 * 0.08, rtol=1e-15)


# ---------------------------------------------- backward (Sec. 6.4, FD)

def _flat_crop(seed, **kw):
    sc, cam = sg.crop_scene(seed, **kw)
    sc = f64(sc)
    sc.g_scale = np.ascontiguousarray(sc.g_scale[:, :2])
    return sc, cam


@pytest.mark.parametrize("opts", [dict(mode=0), dict(mode=2), dict(mode=0, lowpass=1.0, samples=4)])
def test_2d_backward_matches_central_differences(opts):
    """Every gradient of the 2D-GES backward (through the ray-splat hit, the
    object-space filter factors S_k of Eq. 17-18 and the view direction of the
    SH colour) against central differences of the FP64 render, wherever no
    alpha cut or depth test flips inside the step."""
    import oracle as O
    sc, cam = _flat_crop(11)
    rng = np.random.default_rng(12)
    g = rng.standard_normal((3, cam.height, cam.width))
    grads = O.backward(sc, cam, g, opts)
    base = O.render(sc, cam, opts, nthreads=1)
    assert grads["g_scale"].shape == (sc.n_gaussians, 2)
    assert base["ncontrib"].sum() > 200

    def loss(o):
        out = O.render(sc, cam, opts, nthreads=1)
        return float(np.sum(out["rgb"] * g)), out

    n_checked = {}
    for arr_name in ("g_pos", "g_rot", "g_scale", "g_opac", "g_sh", "s_sh"):
        arr = getattr(sc, arr_name)
        flat = arr.reshape(-1)
        idx = range(flat.size) if flat.size <= 160 else rng.choice(flat.size, 160, replace=False)
        gmax = np.abs(grads[arr_name]).max()
        for k in idx:
            h = 1e-6 * (abs(flat[k]) if arr_name == "g_scale" else max(1.0, abs(flat[k])))
            old = flat[k]
            flat[k] = old + h
            lp, op = loss(opts)
            flat[k] = old - h
            lm, om = loss(opts)
            flat[k] = old
            if not (np.array_equal(op["ncontrib"], om["ncontrib"]) and np.array_equal(op["id"], om["id"])
                    and np.array_equal(op["ncontrib"], base["ncontrib"])):
                continue
            fd = (lp - lm) / (2 * h)
            an = grads[arr_name].reshape(-1)[k]
            assert abs(fd - an) <= 2e-5 * abs(an) + 1e-6 * gmax + 1e-9, (arr_name, k, fd, an)
            n_checked[arr_name] = n_checked.get(arr_name, 0) + (abs(an) > 1e-3 * gmax)
    # each kind of gradient is checked where it is not negligible
    assert all(n_checked.get(k, 0) >= 10 for k in ("g_pos", "g_rot", "g_scale", "g_opac", "g_sh")), n_checked


def test_2d_backward_filter_factor_chain_on_a_sub_pixel_splat():
    """A splat far below a pixel is almost all filter: f_k = s_k S_k tends to
    sqrt(r) times the pixel footprint, so dL/ds_k is small while the opacity
    gradient carries the 1/(S1 S2) factor.  Checked by central differences on
    one tilted, off-axis splat where S1, S2 differ from 1 by a factor of
    several, so a dropped S-term or a swapped M00/M11 shows at once."""
    import oracle as O
    cam = sg.look_at((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 48, 40, 60.0)
    q = np.array([0.9, 0.3, -0.25, 0.2])
    q /= np.linalg.norm(q)
    sc = f64(_splat_scene([0.35, -0.2, 0.1], q, [0.012, 0.004], 0.8))
    g = np.random.default_rng(3).standard_normal((3, cam.height, cam.width))
    opts = dict(lowpass=0.5)
    info = O.gauss_info(sc, cam, 0, opts)
    gr = O.backward(sc, cam, g, opts)
    for name, k in (("g_scale", 0), ("g_scale", 1), ("g_opac", 0), ("g_pos", 0), ("g_pos", 2), ("g_rot", 1)):
        flat = getattr(sc, name).reshape(-1)
        h = 1e-7 if name != "g_scale" else 1e-5 * flat[k]
        old = flat[k]
        flat[k] = old + h
        lp = float(np.sum(O.render(sc, cam, opts)["rgb"] * g))
        flat[k] = old - h
        lm = float(np.sum(O.render(sc, cam, opts)["rgb"] * g))
        flat[k] = old
        fd = (lp - lm) / (2 * h)
        np.testing.assert_allclose(gr[name].reshape(-1)[k], fd, rtol=2e-6, atol=1e-10, err_msg=f"{name}[{k}]")
    assert info["valid"] and min(info["S"]) > 2.0 and info["S"][1] > 1.5 * info["S"][0], info["S"]
