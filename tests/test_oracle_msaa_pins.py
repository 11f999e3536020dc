"""Pins of the oracle's 4x multisampled surfel pass (Sec. 5) on the CPU.

Multisampling an opaque single-colour surfel pass equals supersampling it on
the 2x2 grid and box-filtering, so each test ties the samples=4 render to
something computed another way: the closed-form disc, the samples=1 render at
twice the resolution, brute force, and finite differences.
"""
import math

import numpy as np
import pytest

import scenegen as sg
from test_oracle_pins import _disc_scene, _loss_mode, _random_small, f64, ident_cam

MS = dict(samples=4)


def _sample_dirs(cam):
    """Sample rays of the 2x2 grid, [4, H, W] each, plane k = a + 2 b at
    (i + 0.25 + 0.5 a, j + 0.25 + 0.5 b)."""
    dx, dy = [], []
    for k in range(4):
        a, b = k & 1, k >> 1
        U, V = np.meshgrid(np.arange(cam.width) + 0.25 + 0.5 * a, np.arange(cam.height) + 0.25 + 0.5 * b)
        dx.append((U - cam.cx) / cam.fx)
        dy.append((V - cam.cy) / cam.fy)
    return np.stack(dx), np.stack(dy)


def _double(cam):
    """The same camera at twice the resolution: pixel (2i+a, 2j+b)'s centre is
    sample a + 2b of pixel (i, j)."""
    return sg.Camera(2 * cam.width, 2 * cam.height, 2 * cam.fx, 2 * cam.fy, 2 * cam.cx, 2 * cam.cy,
                     cam.world_to_cam, cam.znear, cam.bg)


def _planes(a):
    """[2H, 2W] -> [4, H, W] with plane a + 2b holding element (2j+b, 2i+a)."""
    H, W = a.shape[0] // 2, a.shape[1] // 2
    return a.reshape(H, 2, W, 2).transpose(1, 3, 0, 2).reshape(4, H, W)


def test_msaa_disc_closed_form(oracle_lib):
    """A lone fronto-parallel disc: a sample is covered iff it lies inside the
    projected circle; the pixel colour is the covered fraction of the disc's
    colour plus the rest of the background; D_s = z0 where any sample is
    covered."""
    bg = np.array([0.1, 0.2, 0.9])
    cam = ident_cam(48, 40, 50.0, cx=23.7, cy=19.3, bg=bg)
    z0, s = 2.0, 0.1
    r2 = oracle_lib.DEFAULT_OPTS["surfel_r2"]
    out = oracle_lib.render(_disc_scene(z0, s), cam, MS)
    dx, dy = _sample_dirs(cam)
    lhs = (dx ** 2 + dy ** 2) * (z0 / s) ** 2
    assert np.min(np.abs(lhs - r2)) > 1e-6
    inside = lhs <= r2
    np.testing.assert_array_equal(out["id"], np.where(inside, 0, -1))
    n_in = inside.sum(0)
    assert ((n_in > 0) & (n_in < 4)).sum() > 20   # partly covered rim pixels exist
    col = 0.5 + np.array([0.4, 0.6, 0.8]) / (2 * math.sqrt(math.pi))
    want = (n_in[None] * col[:, None, None] + (4 - n_in[None]) * bg[:, None, None]) / 4
    np.testing.assert_allclose(out["rgb"], want, rtol=0, atol=1e-15)
    np.testing.assert_array_equal(np.isinf(out["depth"]), n_in == 0)
    np.testing.assert_allclose(out["depth"][n_in > 0], z0, rtol=1e-14)
    ns, ng = oracle_lib.count_fragments(_disc_scene(z0, s), cam, MS)
    assert ns == int(inside.sum()) and ng == 0


@pytest.mark.parametrize("seed", [21, 22])
def test_msaa_equals_box_filtered_supersampling(oracle_lib, seed):
    """Surfels only: the samples=4 image is the 2x2 box filter of the
    samples=1 image at twice the resolution; ids are its pixels, D_s the
    nearest of them."""
    sc = _random_small(seed)
    cam = sg.look_at((0.1, 0.2, -2.6), (0, 0, 0), (0, 1, 0), 45, 31, 60.0, bg=(0.3, 0.1, 0.6))
    ms = oracle_lib.render(sc, cam, dict(mode=1, samples=4))
    ss = oracle_lib.render(sc, _double(cam), dict(mode=1))
    np.testing.assert_array_equal(ms["id"], _planes(ss["id"]))
    np.testing.assert_array_equal(ms["depth"], _planes(ss["depth"]).min(0))
    box = np.stack([_planes(ss["rgb"][ch]).mean(0) for ch in range(3)])
    np.testing.assert_allclose(ms["rgb"], box, rtol=0, atol=1e-15)
    assert (ms["id"] >= 0).any() and ((ms["id"] >= 0).sum(0) % 4 != 0).any()


def test_msaa_gaussians_at_pixel_centre_against_nearest_sample(oracle_lib):
    """Full render: the Gaussians are evaluated once, at the pixel centre, and
    depth-tested against the nearest sample's depth (Eq. 2-5).  W_G and C_G
    summed by brute force from each Gaussian's projected parameters."""
    sc = _random_small(23, n_s=40, n_g=120)
    cam = sg.look_at((0.1, -0.2, -2.6), (0, 0, 0), (0, 1, 0), 41, 33, 60.0)
    full = oracle_lib.render(sc, cam, MS)
    s_only = oracle_lib.render(sc, cam, dict(mode=1, samples=4))
    np.testing.assert_array_equal(full["depth"], s_only["depth"])
    np.testing.assert_array_equal(full["id"], s_only["id"])
    U, V = np.meshgrid(np.arange(cam.width) + 0.5, np.arange(cam.height) + 0.5)
    WG = np.zeros((cam.height, cam.width))
    CG = np.zeros((3, cam.height, cam.width))
    for k in range(sc.n_gaussians):
        g = oracle_lib.gauss_info(sc, cam, k)
        if not g["valid"]:
            continue
        du, dv = U - g["px"], V - g["py"]
        ca, cb, cc = g["conic"]
        a = g["sigma"] * np.exp(-0.5 * (ca * du * du + 2 * cb * du * dv + cc * dv * dv))
        x0, x1, y0, y1 = g["bbox"]
        box = np.zeros_like(a, bool)
        box[y0:y1 + 1, x0:x1 + 1] = True
        keep = box & (a >= 1 / 255) & (g["d"] < full["depth"] + g["eps"])
        WG += np.where(keep, a, 0.0)
        CG += np.where(keep, a, 0.0)[None] * g["rgb"][:, None, None]
    partial = (full["id"] >= 0).sum(0) % 4 != 0
    assert (WG > 0).mean() > 0.1 and np.isfinite(full["depth"]).mean() > 0.2 and (partial & (WG > 0)).sum() > 5
    np.testing.assert_allclose(full["wg"], WG, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(full["rgb"], (s_only["rgb"] + CG) / (1 + WG), rtol=0, atol=1e-13)


def test_msaa_culled_equals_brute_force_bitwise(oracle_lib):
    sc = _random_small(24)
    cams = [sg.look_at((0.0, 0.0, -2.6), (0, 0, 0), (0, 1, 0), 53, 37, 60.0),
            sg.look_at((0.2, 0.1, -0.5), (0, 0.1, 1), (0, 1, 0), 40, 29, 90.0)]
    for cam in cams:
        for mode in (0, 1):
            a = oracle_lib.render(sc, cam, dict(mode=mode, samples=4), culled=True)
            b = oracle_lib.render(sc, cam, dict(mode=mode, samples=4), culled=False)
            for k in a:
                np.testing.assert_array_equal(a[k], b[k], err_msg=f"{k} mode={mode}")


def test_msaa_id_check_per_sample(oracle_lib):
    """The id check runs on every sample's own ray: the render's planes pass;
    a plane shifted by one sample fails where that changes the clear answer."""
    sc, cams = sg.config_scene(0)
    cam = cams[0]
    ref = oracle_lib.render(sc, cam, MS)
    assert ref["id"].shape == (4, cam.height, cam.width)
    ok = oracle_lib.id_validity(sc, cam, ref, ref["id"], MS)
    assert ok.all()
    import ctypes
    lib = oracle_lib.load()
    pin = oracle_lib.oracle._Pinned(sc, cam, MS)
    swapped = np.ascontiguousarray(ref["id"][[3, 2, 1, 0]], np.int32)
    v = np.empty(swapped.shape, np.uint8)
    assert lib.ora_check_ids(ctypes.byref(pin.s), ctypes.byref(pin.c), ctypes.byref(pin.o),
                             swapped.ctypes.data, v.ctypes.data) == 0
    differs = swapped != ref["id"]
    clear = (ref["amb"] & 1) == 0
    assert differs.sum() > 50
    # an empty sample given a covering surfel's id or vice versa, away from any band, is wrong
    wrong = differs & clear[None] & ((swapped < 0) != (ref["id"] < 0))
    assert wrong.sum() > 10 and not v.astype(bool)[wrong].any()


@pytest.mark.parametrize("mode", [0, 1])
def test_msaa_backward_matches_central_differences(oracle_lib, mode):
    """Surfel SH gradients with 4 samples: each won sample carries 1/4 of the
    pixel's weight (and the Gaussian terms keep theirs)."""
    sc, cam = sg.crop_scene(7)
    sc = f64(sc)
    rng = np.random.default_rng(9)
    g = rng.standard_normal((3, cam.height, cam.width))
    opts = dict(mode=mode, samples=4)
    grads = oracle_lib.backward(sc, cam, g, opts)
    base = oracle_lib.render(sc, cam, opts)
    partial = ((base["id"] >= 0).sum(0) % 4 != 0).sum()
    assert partial > 10   # pixels whose samples disagree
    checks = ["s_sh"] + (["g_pos", "g_opac", "g_sh"] if mode == 0 else [])
    n_checked = 0
    for name in checks:
        flat = getattr(sc, name).reshape(-1)
        gmax = np.abs(grads[name]).max()
        idx = range(flat.size) if flat.size <= 150 else rng.choice(flat.size, 150, replace=False)
        for k in idx:
            h = 1e-6 * max(1.0, abs(flat[k]))
            old = flat[k]
            flat[k] = old + h
            lp, op = _loss_mode(oracle_lib, sc, cam, g, opts)
            flat[k] = old - h
            lm, om = _loss_mode(oracle_lib, sc, cam, g, opts)
            flat[k] = old
            if not (np.array_equal(op["ncontrib"], om["ncontrib"]) and np.array_equal(op["id"], om["id"])
                    and np.array_equal(op["ncontrib"], base["ncontrib"])):
                continue
            fd = (lp - lm) / (2 * h)
            an = grads[name].reshape(-1)[k]
            assert abs(fd - an) <= 2e-5 * abs(an) + 1e-6 * gmax + 1e-9, (name, k, fd, an)
            n_checked += 1
    assert n_checked > 100
