"""Pins of the oracle's Mip-GES filters (Sec. 6.1: Mip-Splatting's 3D world
filter and screen-space filter applied to the Gaussians) on the CPU.

Both filters are convolutions with a normalised Gaussian kernel: the filtered
Gaussian's peak must equal the convolution integral (computed here by
Gauss-Hermite quadrature, independently of the oracle's determinant ratios),
and the screen filter must keep the footprint's integral (a Riemann sum over
pixels) whatever its variance.
"""
import math

import numpy as np
import pytest

import scenegen as sg
from test_oracle_pins import _loss_mode, _one_gaussian, f64, ident_cam, mk_scene

MIP = dict(filter=1, lowpass=0.1)


def _rot(q):
    w, x, y, z = np.asarray(q, float) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _gauss(z0, scale, q, sigma, offset=(0.0, 0.0), filt=None):
    sh = np.zeros((1, 1, 3))
    sh[0, 0] = (0.3, 0.5, 0.7)
    sc = mk_scene(0, g_pos=[[offset[0], offset[1], z0]], g_rot=[q], g_scale=[scale], g_opac=[sigma], g_sh=sh)
    if filt is not None:
        sc.g_filter3d = np.array([filt], float)
    return sc


def _gh_peak(cov, var, n=200):
    """Value at 0 of exp(-y^T cov^-1 y / 2) convolved with the normalised
    isotropic Gaussian N(0, var I).  The kernel is isotropic, so in the
    eigenbasis of cov the integral of their product splits into 1D integrals
    int exp(-y^2 / (2 l)) N(y; 0, var) dy, each done by Gauss-Hermite
    quadrature against the narrower of its two factors."""
    x, w = np.polynomial.hermite_e.hermegauss(n)     # weight exp(-x^2/2)
    w = w / math.sqrt(2 * math.pi)                   # E over N(0, 1)
    out = 1.0
    for lam in np.linalg.eigvalsh(cov):
        if lam < var:      # y = sqrt(lam) x: exp(-x^2/2) sqrt(2 pi lam) N(y; 0, var)
            y = math.sqrt(lam) * x
            f = np.exp(-0.5 * y * y / var) / math.sqrt(2 * math.pi * var) * math.sqrt(2 * math.pi * lam)
        else:              # y = sqrt(var) x: N(y; 0, var) is the weight
            y = math.sqrt(var) * x
            f = np.exp(-0.5 * y * y / lam)
        out *= float(np.sum(w * f))
    return out


def test_screen_filter_peak_is_the_convolution(oracle_lib):
    """filter = 1: alpha at the centre = sigma times the 2D convolution of the
    projected Gaussian with N(0, lowpass I), evaluated at the centre."""
    f = 40.0
    cam = ident_cam(65, 65, f, cx=32.5, cy=32.5)
    sc = _gauss(2.0, [0.02, 0.005, 0.01], [0.9, 0.2, -0.3, 0.25], 0.8)
    for lp in (0.1, 0.3, 1.0):
        info = oracle_lib.gauss_info(sc, cam, 0, dict(filter=1, lowpass=lp))
        R2 = np.array([[info["sigma2"][0] - lp, info["sigma2"][1]], [info["sigma2"][1], info["sigma2"][2] - lp]])
        want = 0.8 * _gh_peak(R2, lp)
        assert abs(info["sigma"] - want) < 1e-12, (lp, info["sigma"], want)
        out = oracle_lib.render(sc, cam, dict(filter=1, lowpass=lp))
        assert abs(out["wg"][32, 32] - info["sigma"]) < 1e-14
    # filter = 0 keeps the opacity (3DGS's fixed dilation)
    assert oracle_lib.gauss_info(sc, cam, 0, dict(filter=0, lowpass=0.1))["sigma"] == 0.8


def test_screen_filter_keeps_the_footprint_integral(oracle_lib):
    """The pixel sum of alpha (a Gaussian several pixels wide, no cut-off in
    effect) does not depend on the screen filter's variance with filter = 1,
    and grows with it with filter = 0."""
    cam = ident_cam(96, 96, 60.0, cx=47.3, cy=48.1)
    sc = _gauss(2.0, [0.35, 0.12, 0.2], [0.8, -0.1, 0.4, 0.3], 0.6)
    opts = lambda flt, lp: dict(filter=flt, lowpass=lp, alpha_min=1e-300, tol_alpha=0.0)
    s1 = [oracle_lib.render(sc, cam, opts(1, lp))["wg"].sum() for lp in (0.1, 0.5, 2.0)]
    s0 = [oracle_lib.render(sc, cam, opts(0, lp))["wg"].sum() for lp in (0.1, 0.5, 2.0)]
    np.testing.assert_allclose(s1, s1[0], rtol=1e-9)
    assert s0[2] > s0[1] * 1.01 > s0[0] * 1.02


def test_world_filter_peak_is_the_convolution(oracle_lib):
    """The 3D filter: the effective opacity is sigma times the 3D convolution
    of the Gaussian with N(0, v I) at its centre; the image equals that of the
    Gaussian with axes sqrt(s^2 + v) and that opacity (Sigma3 + v I)."""
    f = 40.0
    cam = ident_cam(65, 65, f, cx=32.5, cy=32.5)
    s, q, v = np.array([0.02, 0.004, 0.011]), [0.9, 0.2, -0.3, 0.25], 3e-5
    sc = _gauss(2.0, s, q, 0.8, filt=v)
    R = _rot(q)
    want = 0.8 * _gh_peak(R @ np.diag(s ** 2) @ R.T, v)
    info = oracle_lib.gauss_info(sc, cam, 0)
    assert abs(info["sigma"] - want) < 1e-12, (info["sigma"], want)
    twin = _gauss(2.0, np.sqrt(s ** 2 + v), q, want)
    a = oracle_lib.render(sc, cam)
    b = oracle_lib.render(twin, cam)
    np.testing.assert_allclose(a["rgb"], b["rgb"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(a["wg"], b["wg"], rtol=1e-11, atol=1e-15)
    # eps_i uses the stored axis lengths, not the filtered ones
    np.testing.assert_allclose(info["eps"], 5.0 / 3.0 * s.sum(), rtol=1e-15)


def test_filters_compose(oracle_lib):
    """3D filter, then projection, then the screen filter: the opacity is the
    product of the two convolution peaks."""
    cam = ident_cam(65, 65, 40.0, cx=32.5, cy=32.5)
    s, q, v = np.array([0.02, 0.004, 0.011]), [0.9, 0.2, -0.3, 0.25], 3e-5
    sc = _gauss(2.0, s, q, 0.8, filt=v)
    i3 = oracle_lib.gauss_info(sc, cam, 0)
    i32 = oracle_lib.gauss_info(sc, cam, 0, MIP)
    lp = MIP["lowpass"]
    R2 = np.array([[i32["sigma2"][0] - lp, i32["sigma2"][1]], [i32["sigma2"][1], i32["sigma2"][2] - lp]])
    assert abs(i32["sigma"] - i3["sigma"] * _gh_peak(R2, lp)) < 1e-12


def test_mip_culled_equals_brute_force_bitwise(oracle_lib):
    sc = sg.random_scene(51, 60, 200, n_objects=4, box=1.0, sphere_r=(0.3, 0.6), plane_side=(0.6, 1.2),
                         surfel_scale=(0.05, 0.15), gauss_logscale=(-3.5, 0.4))
    sc.g_filter3d = np.random.default_rng(5).uniform(0, 4e-4, sc.n_gaussians)
    cam = sg.look_at((0.0, 0.0, -2.6), (0, 0, 0), (0, 1, 0), 53, 37, 60.0)
    for mode in (0, 2):
        a = oracle_lib.render(sc, cam, dict(MIP, mode=mode), culled=True)
        b = oracle_lib.render(sc, cam, dict(MIP, mode=mode), culled=False)
        for k in a:
            np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def test_filter3d_closed_forms(oracle_lib):
    """v = s3d (z/f)^2 at the camera that sees the centre at the highest rate
    (max(fx, fy)/z); outside every image: the largest v of the others."""
    sc = mk_scene(0, g_pos=[[0.1, 0.0, 2.0], [0.0, 0.05, 5.0], [30.0, 0.0, 2.0]], g_rot=[[1.0, 0, 0, 0]] * 3,
                  g_scale=[[0.01] * 3] * 3, g_opac=[0.5] * 3, g_sh=np.zeros((3, 1, 3)))
    c1 = ident_cam(64, 48, 50.0)
    c1.fy = 55.0
    c2 = ident_cam(64, 48, 40.0)
    c2.world_to_cam = c2.world_to_cam.copy()
    c2.world_to_cam[2, 3] = -1.0        # 1 m closer to the scene
    v = oracle_lib.filter3d(sc, [c1], 0.2)
    np.testing.assert_allclose(v[:2], [0.2 * (2.0 / 55.0) ** 2, 0.2 * (5.0 / 55.0) ** 2], rtol=1e-14)
    assert v[2] == v[1]
    v2 = oracle_lib.filter3d(sc, [c1, c2], 0.2)
    # point 0: 55/2 = 27.5 (c1) vs 40/1 = 40 (c2): c2 wins; point 1: 55/5 = 11 vs 40/4 = 10: c1
    np.testing.assert_allclose(v2[:2], [0.2 / 40.0 ** 2, 0.2 * (5.0 / 55.0) ** 2], rtol=1e-14)
    assert v2[2] == max(v2[:2])
    # behind every camera
    assert np.all(oracle_lib.filter3d(mk_scene(0, g_pos=[[0, 0, -3.0]], g_rot=[[1.0, 0, 0, 0]],
                                               g_scale=[[0.01] * 3], g_opac=[0.5], g_sh=np.zeros((1, 1, 3))),
                                      [c1], 0.2) == 0.0)


def test_filter3d_brute_force(oracle_lib):
    sc = sg.random_scene(52, 10, 300, n_objects=3, box=1.0, sphere_r=(0.3, 0.6), plane_side=(0.6, 1.2),
                         surfel_scale=(0.05, 0.15), gauss_logscale=(-3.5, 0.4))
    sc.g_pos = sc.g_pos.copy()
    sc.g_pos[:7] += np.array([0.0, 40.0, 0.0], np.float32)    # above every camera's view
    cams = [sg.look_at((2.5 * math.cos(a), 0.4, 2.5 * math.sin(a)), (0, 0, 0), (0, 1, 0), 80, 60, 50.0)
            for a in np.linspace(0, 2 * math.pi, 5, endpoint=False)]
    v = oracle_lib.filter3d(sc, cams, 0.2)
    want = np.full(sc.n_gaussians, -1.0)
    for i in range(sc.n_gaussians):
        best = 0.0
        for c in cams:
            W = np.asarray(c.world_to_cam, float)
            t = W[:, :3] @ np.asarray(sc.g_pos[i], float) + W[:, 3]
            if t[2] <= c.znear:
                continue
            u, w = c.fx * t[0] / t[2] + c.cx, c.fy * t[1] / t[2] + c.cy
            if 0 <= u <= c.width and 0 <= w <= c.height:
                best = max(best, max(c.fx, c.fy) / t[2])
        if best > 0:
            want[i] = 0.2 / best ** 2
    assert (want > 0).sum() > 200 and (want < 0).any()
    want[want < 0] = want.max()
    np.testing.assert_allclose(v, want, rtol=1e-12)


@pytest.mark.parametrize("mode", [0, 2])
def test_mip_backward_matches_central_differences(oracle_lib, mode):
    sc, cam = sg.crop_scene(7)
    sc = f64(sc)
    rng = np.random.default_rng(17)
    sc.g_filter3d = rng.uniform(0.0, 2e-4, sc.n_gaussians)
    g = rng.standard_normal((3, cam.height, cam.width))
    opts = dict(MIP, mode=mode)
    grads = oracle_lib.backward(sc, cam, g, opts)
    base = oracle_lib.render(sc, cam, opts)
    assert base["ncontrib"].sum() > 200
    n_checked = 0
    for name in ("g_pos", "g_rot", "g_scale", "g_opac", "g_sh"):
        flat = getattr(sc, name).reshape(-1)
        gmax = np.abs(grads[name]).max()
        idx = range(flat.size) if flat.size <= 200 else rng.choice(flat.size, 200, replace=False)
        for k in idx:
            h = 1e-6 * abs(flat[k]) if name == "g_scale" else 1e-6 * max(1.0, abs(flat[k]))
            old = flat[k]
            flat[k] = old + h
            lp, op = _loss_mode(oracle_lib, sc, cam, g, opts)
            flat[k] = old - h
            lm, om = _loss_mode(oracle_lib, sc, cam, g, opts)
            flat[k] = old
            if not (np.array_equal(op["ncontrib"], om["ncontrib"]) and np.array_equal(op["ncontrib"], base["ncontrib"])):
                continue
            fd = (lp - lm) / (2 * h)
            an = grads[name].reshape(-1)[k]
            assert abs(fd - an) <= 2e-5 * abs(an) + 1e-6 * gmax + 1e-9, (name, k, fd, an)
            n_checked += 1
    assert n_checked > 300
