"""Pins of the oracle's EWA projection of 3D Gaussians away from the optical
axis (Sec. 3, Eq. 4, with the projected covariance of 3DGS that the paper
builds on).

The projected covariance is the first-order (affine) image of the 3D
covariance under the pinhole map: Sigma2 = J W Sigma3 W^T J^T + lowpass I,
J the Jacobian of (x, y, z) -> (fx x/z + cx, fy y/z + cy) at the camera-space
centre, W the world-to-camera rotation.  None of these tests writes J down:

- the complex-step derivative of the pinhole map gives J to machine precision
  (an analytic map, so Im f(t + i h e_k)/h is exact up to rounding), and the
  rotation comes from scipy's quaternion conversion;
- a Gauss-Hermite cubature of the exact projection of a tiny Gaussian gives
  its projected second moment, which the linearisation must reproduce up to
  O((s/z)^2);
- a brute-force image of a lone off-axis Gaussian against numpy.

Centres reach |x/z|, |y/z| of about 1, where a sign or form error in J's third
column (the -f x/z^2, -f y/z^2 terms) changes Sigma2 by O(1).
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import scenegen as sg


def _camera(W=320, H=240, fov=100.0):
    return sg.look_at((1.3, -0.7, -4.0), (0.2, 0.1, 0.0), (0.1, 1.0, 0.05), W, H, fov)


def _w2c(cam):
    m = np.asarray(cam.world_to_cam, np.float64).reshape(3, 4)
    return m[:, :3], m[:, 3]


def _gaussians(cam, n=24, seed=5):
    """n Gaussians whose camera-space centres have |x/z|, |y/z| up to ~1.05
    at depths 1.5 .. 9, anisotropic scales and random rotations."""
    rng = np.random.default_rng(seed)
    Rc, tc = _w2c(cam)
    z = rng.uniform(1.5, 9.0, n)
    xz = rng.uniform(-1.05, 1.05, n)
    yz = rng.uniform(-1.05, 1.05, n)
    xz[:4] = [1.0, -1.0, 0.9, -0.95]
    yz[:4] = [0.95, 1.0, -1.0, -0.9]
    t = np.stack([xz * z, yz * z, z], 1)
    p = (t - tc) @ Rc                       # world = R^T (t - tc)
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    s = np.exp(rng.uniform(-3.5, -1.2, (n, 3)))
    s[:, 0] *= 4.0                          # strongly anisotropic
    return p, q, s


def _scene(p, q, s, opac=None, deg=0, dc=(0.3, 0.55, 0.8)):
    n = len(p)
    K = (deg + 1) ** 2
    sh = np.zeros((n, K, 3))
    sh[:, 0, :] = dc
    return sg.Scene(deg, np.zeros((0, 3)), np.zeros((0, 4)), np.zeros((0, 2)), np.zeros((0, K, 3)),
                    np.asarray(p, np.float64), np.asarray(q, np.float64), np.asarray(s, np.float64),
                    np.full(n, 0.8) if opac is None else np.asarray(opac, np.float64), sh)


def _pinhole(cam, t):
    return np.array([cam.fx * t[0] / t[2] + cam.cx, cam.fy * t[1] / t[2] + cam.cy])


def _jacobian_complex_step(cam, t, h=1e-30):
    J = np.empty((2, 3))
    for k in range(3):
        tt = np.asarray(t, np.complex128).copy()
        tt[k] += 1j * h
        J[:, k] = np.imag(_pinhole(cam, tt)) / h
    return J


def _sigma3(q, s):
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()   # scipy is scalar-last
    return R @ np.diag(np.asarray(s) ** 2) @ R.T


def _reference(cam, p, q, s, lowpass=0.3):
    Rc, tc = _w2c(cam)
    t = Rc @ p + tc
    J = _jacobian_complex_step(cam, t)
    S2 = J @ Rc @ _sigma3(q, s) @ Rc.T @ J.T + lowpass * np.eye(2)
    return t, S2, _pinhole(cam, t)


def test_offaxis_sigma2_conic_and_centre_match_the_complex_step_jacobian(oracle_lib):
    cam = _camera()
    p, q, s = _gaussians(cam)
    sc = _scene(p, q, s)
    n_far = 0
    for i in range(len(p)):
        t, S2, ctr = _reference(cam, p[i], q[i], s[i])
        n_far += abs(t[0] / t[2]) > 0.8 or abs(t[1] / t[2]) > 0.8
        info = oracle_lib.gauss_info(sc, cam, i)
        assert info["valid"]
        got = np.array([[info["sigma2"][0], info["sigma2"][1]], [info["sigma2"][1], info["sigma2"][2]]])
        np.testing.assert_allclose(got, S2, rtol=0, atol=1e-9 * np.abs(S2).max())
        conic = np.linalg.inv(S2)
        gc = np.array([[info["conic"][0], info["conic"][1]], [info["conic"][1], info["conic"][2]]])
        np.testing.assert_allclose(gc, conic, rtol=0, atol=1e-9 * np.abs(conic).max())
        assert info["px"] == pytest.approx(ctr[0], rel=1e-12, abs=1e-9)
        assert info["py"] == pytest.approx(ctr[1], rel=1e-12, abs=1e-9)
        assert info["d"] == pytest.approx(t[2], rel=1e-13)
    assert n_far >= 6   # the off-axis terms of J carry weight in many cases


def _gauss_hermite_projected_cov(cam, t, L, n=7):
    """Second central moment of the exact pinhole image of N(t, L L^T), by a
    tensor Gauss-Hermite rule (probabilists' weights)."""
    x, w = np.polynomial.hermite_e.hermegauss(n)
    w = w / w.sum()
    X = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1).reshape(-1, 3)
    Wt = np.einsum("i,j,k->ijk", w, w, w).reshape(-1)
    pts = t[None, :] + X @ L.T
    uv = np.stack([cam.fx * pts[:, 0] / pts[:, 2] + cam.cx, cam.fy * pts[:, 1] / pts[:, 2] + cam.cy], 1)
    m = (Wt[:, None] * uv).sum(0)
    d = uv - m
    return (Wt[:, None, None] * d[:, :, None] * d[:, None, :]).sum(0)


def test_offaxis_sigma2_is_the_first_order_projected_covariance(oracle_lib):
    """For a Gaussian small against its depth, the covariance of its exact
    projection equals the EWA Sigma2 (without the low-pass) up to
    O((s/z)^2): no derivative is taken anywhere on this side."""
    cam = _camera()
    p, q, s = _gaussians(cam, n=12, seed=9)
    Rc, tc = _w2c(cam)
    for i in range(len(p)):
        t = Rc @ p[i] + tc
        st = s[i] / s[i].max() * 1e-4 * t[2]            # largest axis 1e-4 of the depth
        sc = _scene(p[i:i + 1], q[i:i + 1], st[None, :])
        info = oracle_lib.gauss_info(sc, cam, 0, dict(lowpass=0.0))
        got = np.array([[info["sigma2"][0], info["sigma2"][1]], [info["sigma2"][1], info["sigma2"][2]]])
        R = Rotation.from_quat([q[i][1], q[i][2], q[i][3], q[i][0]]).as_matrix()
        L = Rc @ R @ np.diag(st)
        ref = _gauss_hermite_projected_cov(cam, t, L)
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-6 * np.abs(ref).max())


def test_offaxis_gaussian_image_brute_force(oracle_lib):
    """A lone off-axis Gaussian, no surfels, background 0: C = alpha c/(1 + alpha)
    with alpha = sigma exp(-q/2) where alpha >= 1/255 (Eq. 2-5), q from the
    numpy Sigma2, at every pixel away from the cut."""
    W, H = 160, 128
    cam = sg.look_at((0.4, 0.3, -3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), W, H, 90.0)
    Rc, tc = _w2c(cam)
    # camera-space centre at x/z = 0.62, y/z = -0.48: inside the image, off axis
    tcam = np.array([0.62 * 2.5, -0.48 * 2.5, 2.5])
    p = Rc.T @ (tcam - tc)
    q = np.array([0.8, 0.3, -0.4, 0.33])
    q /= np.linalg.norm(q)
    s = np.array([0.4, 0.15, 0.06])
    sigma, dc = 0.85, (0.4, 0.1, 0.7)
    sc = _scene(p[None], q[None], s[None], opac=[sigma], dc=dc)
    out = oracle_lib.render(sc, cam, culled=False)
    t, S2, ctr = _reference(cam, p, q, s)
    Ci = np.linalg.inv(S2)
    U, V = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    D = np.stack([U - ctr[0], V - ctr[1]], -1)
    qf = np.einsum("...i,ij,...j->...", D, Ci, D)
    a = sigma * np.exp(-0.5 * qf)
    Y00 = 0.5 / math.sqrt(math.pi)
    c = np.maximum(0.0, 0.5 + np.asarray(dc) * Y00)
    keep = a >= 1.0 / 255.0
    ref = np.where(keep[None], a[None] * c[:, None, None] / (1.0 + a[None]), 0.0)
    away = np.abs(a - 1.0 / 255.0) > 1e-7
    assert keep.sum() > 200 and (~keep).sum() > 200
    np.testing.assert_allclose(out["rgb"][:, away], ref[:, away], rtol=0, atol=1e-12)
    np.testing.assert_allclose(out["wg"][away], np.where(keep, a, 0.0)[away], rtol=0, atol=1e-12)
