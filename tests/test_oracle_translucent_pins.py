"""Pins of the oracle's translucent-surfel render (Sec. 4.1, Eq. 6-7), its
backward, the covering score and the Gaussian contribution score (Eq. 9) on
the CPU: closed forms for one and two surfels, the front-first order, the
early stop, the paper's statement that at w = 255 the render equals the
z-buffer render, brute force, and central differences."""
import math

import numpy as np
import pytest

import scenegen as sg
from test_oracle_pins import _disc_scene, _one_gaussian, f64, ident_cam, mk_scene, pixel_dirs


def _col(dc):
    return 0.5 + np.asarray(dc) / (2 * math.sqrt(math.pi))


def _discs(z, s, dcs, pos_xy=None, rot=None):
    n = len(z)
    sh = np.zeros((n, 1, 3))
    sh[:, 0] = dcs
    pos = np.zeros((n, 3))
    pos[:, 2] = z
    if pos_xy is not None:
        pos[:, :2] = pos_xy
    return mk_scene(0, s_pos=pos, s_rot=rot if rot is not None else [[1.0, 0, 0, 0]] * n,
                    s_scale=[[si, si] for si in s], s_sh=sh)


@pytest.mark.parametrize("w", [0.1, 2.0, 255.0])
def test_single_disc_closed_form(oracle_lib, w):
    bg = np.array([0.1, 0.2, 0.3])
    cam = ident_cam(48, 40, 50.0, cx=23.7, cy=19.3, bg=bg)
    z0, s = 2.0, 0.08
    out = oracle_lib.render_translucent(_disc_scene(z0, s, dc=(0.4, 0.6, 0.8)), cam, [w])
    dx, dy = pixel_dirs(cam)
    G = np.exp(-0.5 * (dx ** 2 + dy ** 2) * (z0 / s) ** 2)
    a = np.minimum(1.0, w * G)
    keep = np.minimum(a, G) >= 1 / 255
    a = np.where(keep, a, 0.0)
    assert keep.sum() > 30
    want = _col((0.4, 0.6, 0.8))[:, None, None] * a + (1 - a) * bg[:, None, None]
    np.testing.assert_allclose(out["rgb"], want, rtol=0, atol=1e-14)
    np.testing.assert_allclose(out["T"], 1 - a, rtol=0, atol=1e-15)
    np.testing.assert_array_equal(out["front"], np.where(keep, 0, -1))


def test_two_discs_blend_in_centre_depth_order(oracle_lib):
    """Two fronto-parallel discs: the nearer centre blends first; equal centre
    depths blend the lower index first."""
    cam = ident_cam(40, 40, 40.0)
    c0, c1 = (0.9, 0.1, 0.1), (0.1, 0.1, 0.9)
    for z, first in (([2.0, 1.5], 1), ([2.0, 2.0], 0)):
        sc = _discs(z, [0.1, 0.12], [c0, c1], pos_xy=[[0.01, 0.0], [0.0, 0.01]])
        w = np.array([0.8, 0.6])
        out = oracle_lib.render_translucent(sc, cam, w, front_first=False)
        dx, dy = pixel_dirs(cam)
        al = []
        for k in range(2):
            G = np.exp(-0.5 * (((dx * z[k] - sc.s_pos[k, 0]) ** 2 + (dy * z[k] - sc.s_pos[k, 1]) ** 2) / sc.s_scale[k, 0] ** 2))
            a = np.minimum(1.0, w[k] * G)
            al.append(np.where(np.minimum(a, G) >= 1 / 255, a, 0.0))
        cols = [_col(c0)[:, None, None], _col(c1)[:, None, None]]
        f, b = first, 1 - first
        want = cols[f] * al[f] + (1 - al[f]) * cols[b] * al[b]
        np.testing.assert_allclose(out["rgb"], want, rtol=0, atol=1e-14)


def test_front_choice_is_ambiguous_only_within_the_depth_band(oracle_lib):
    """The frontmost contributor (least depth at the pixel) is a unique answer
    only when no other contributor lies within the depth band of it.  Two
    coplanar discs tie everywhere they overlap, which is flagged in both blend
    orders.  With one disc clearly nearer it is the front surfel, and the
    front choice adds no flag."""
    cam = ident_cam(40, 40, 40.0)
    c0, c1 = (0.9, 0.1, 0.1), (0.1, 0.1, 0.9)
    w = np.array([0.8, 0.6])
    tie = _discs([2.0, 2.0], [0.1, 0.12], [c0, c1], pos_xy=[[0.01, 0.0], [0.0, 0.01]])
    for ff in (False, True):
        out = oracle_lib.render_translucent(tie, cam, w, front_first=ff)
        both = out["nblend"] == 2
        assert both.sum() > 50
        assert np.all(out["amb"][both] != 0)
        if not ff:
            assert np.all((out["amb"][both] & 1) != 0)
    near = _discs([2.0, 1.5], [0.1, 0.12], [c0, c1], pos_xy=[[0.01, 0.0], [0.0, 0.01]])
    for ff in (False, True):
        out = oracle_lib.render_translucent(near, cam, w, front_first=ff)
        both = out["nblend"] == 2
        clear = both & (out["amb"] == 0)
        assert clear.sum() > 0.8 * both.sum() > 40
        assert np.all(out["front"][both] == 1)
        assert np.all((out["amb"][both] & 1) == 0)


def test_front_first_moves_the_nearest_fragment(oracle_lib):
    """A large tilted disc whose centre is behind a small fronto-parallel one
    but whose fragment is in front of it at some pixels: with front_first it
    blends first there, without it the centre order holds."""
    cam = ident_cam(40, 40, 40.0)
    ang = 1.2
    q = [math.cos(ang / 2), math.sin(ang / 2), 0.0, 0.0]
    sc = _discs([2.0, 2.1], [0.15, 0.6], [(0.9, 0.1, 0.1), (0.1, 0.9, 0.1)], rot=[[1.0, 0, 0, 0], q])
    sc = f64(sc)
    w = np.array([0.7, 0.7])
    a = oracle_lib.render_translucent(sc, cam, w, front_first=True)
    b = oracle_lib.render_translucent(sc, cam, w, front_first=False)
    both = (a["nblend"] == 2) & (a["amb"] == 0)
    moved = both & (a["front"] == 1)
    stay = both & (a["front"] == 0)
    assert moved.sum() > 10 and stay.sum() > 10
    np.testing.assert_array_equal(a["rgb"][:, stay], b["rgb"][:, stay])
    assert np.all(np.abs(a["rgb"][:, moved] - b["rgb"][:, moved]).max(0) > 1e-6)
    # the front entry really is the nearer fragment there
    j, i = np.nonzero(moved)
    z, rho, nd, ok = oracle_lib.surfel_eval(sc, cam, i, j, np.zeros_like(i))
    z1, _, _, _ = oracle_lib.surfel_eval(sc, cam, i, j, np.ones_like(i))
    assert np.all(z1 < z)


def test_early_stop_below_1e4(oracle_lib):
    """A stack of fronto-parallel discs of opacity 0.6 at the centre pixel: the
    blend stops after the first k with 0.4^k < 1e-4 (k = 11)."""
    cam = ident_cam(17, 17, 30.0, cx=8.5, cy=8.5)
    n = 20
    z = 1.0 + 0.05 * np.arange(n)
    sc = _discs(z, [0.5] * n, [(0.5, 0.5, 0.5)] * n)
    out = oracle_lib.render_translucent(sc, cam, np.full(n, 0.6))
    k = next(k for k in range(1, n + 1) if 0.4 ** k < 1e-4)
    assert out["nblend"][8, 8] == k == 11
    np.testing.assert_allclose(out["T"][8, 8], 0.4 ** k, rtol=1e-12)


def test_w255_front_first_equals_zbuffer_render(oracle_lib):
    """At w = 255 the frontmost surfel has alpha = 1 wherever it covers the
    pixel: the translucent render equals the opaque z-buffer render (Sec. 4.1:
    the end of the optimisation is consistent with the z-buffer rendering)."""
    sc, cams = sg.config_scene(0)
    cam = cams[0]
    t = oracle_lib.render_translucent(sc, cam, np.full(sc.n_surfels, 255.0), front_first=True)
    z = oracle_lib.render(sc, cam, dict(mode=1))
    ok = (t["amb"] == 0) & (z["amb"] == 0)
    assert ok.mean() > 0.95
    np.testing.assert_allclose(t["rgb"][:, ok], z["rgb"][:, ok], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(t["front"][ok], z["id"][ok])
    assert np.all(t["T"][ok & (z["id"] >= 0)] == 0.0)


def test_covering_counts_are_the_zbuffer_histogram_at_w255(oracle_lib):
    sc, cams = sg.config_scene(0)
    cam = cams[0]
    cnt = oracle_lib.covering_counts(sc, cam, np.full(sc.n_surfels, 255.0))
    ids = oracle_lib.render(sc, cam, dict(mode=1))["id"]
    hist = np.bincount(ids[ids >= 0], minlength=sc.n_surfels)
    amb = oracle_lib.render_translucent(sc, cam, np.full(sc.n_surfels, 255.0))["amb"] != 0
    assert np.abs(cnt - hist).sum() <= amb.sum()
    assert cnt.sum() == (ids >= 0).sum() and (cnt > 0).sum() > 100


def test_translucent_culled_equals_brute_force_bitwise(oracle_lib):
    sc = sg.random_scene(91, 80, 10, n_objects=4, box=1.0, sphere_r=(0.3, 0.6), plane_side=(0.6, 1.2),
                         surfel_scale=(0.05, 0.15))
    w = np.random.default_rng(3).uniform(0.05, 40.0, sc.n_surfels)
    cam = sg.look_at((0.0, 0.0, -2.6), (0, 0, 0), (0, 1, 0), 53, 37, 60.0)
    for ff in (False, True):
        a = oracle_lib.render_translucent(sc, cam, w, ff, culled=True)
        b = oracle_lib.render_translucent(sc, cam, w, ff, culled=False)
        for k in a:
            np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    assert (a["nblend"] > 1).mean() > 0.1


def _tloss(oracle_lib, sc, cam, w, g, ff):
    out = oracle_lib.render_translucent(sc, cam, w, ff, nthreads=1)
    return float(np.sum(out["rgb"] * g)), out


@pytest.mark.parametrize("ff", [False, True])
def test_translucent_backward_matches_central_differences(oracle_lib, ff):
    sc, cam = sg.crop_scene(7)
    sc = f64(sc)
    rng = np.random.default_rng(31)
    w = rng.uniform(0.3, 3.0, sc.n_surfels)
    g = rng.standard_normal((3, cam.height, cam.width))
    grads = oracle_lib.backward_translucent(sc, cam, w, g, ff)
    base = oracle_lib.render_translucent(sc, cam, w, ff)
    assert (base["nblend"] > 1).sum() > 100
    n_checked = 0
    for name in ("s_pos", "s_rot", "s_scale", "s_w", "s_sh"):
        if name == "s_w":
            flat = w
        else:
            flat = getattr(sc, name).reshape(-1)
        gmax = np.abs(grads[name]).max()
        idx = range(flat.size) if flat.size <= 150 else rng.choice(flat.size, 150, replace=False)
        for k in idx:
            h = 1e-6 * max(1.0, abs(flat[k])) if name != "s_scale" else 1e-6 * abs(flat[k])
            old = flat[k]
            flat[k] = old + h
            lp, op = _tloss(oracle_lib, sc, cam, w, g, ff)
            flat[k] = old - h
            lm, om = _tloss(oracle_lib, sc, cam, w, g, ff)
            flat[k] = old
            if not (np.array_equal(op["nblend"], om["nblend"]) and np.array_equal(op["front"], om["front"]) and
                    np.array_equal(op["nblend"], base["nblend"])):
                continue
            fd = (lp - lm) / (2 * h)
            an = grads[name].reshape(-1)[k]
            assert abs(fd - an) <= 2e-5 * abs(an) + 1e-6 * gmax + 1e-9, (name, k, fd, an)
            n_checked += 1
    assert n_checked > 300


def test_contribution_score_single_gaussian_and_brute_force(oracle_lib):
    """Eq. 9: one on-axis Gaussian over the background: the best pixel is the
    centre, s = c_max sigma / (1 + sigma); a random scene against a direct
    evaluation from each Gaussian's projected parameters."""
    f, z0, s, sig = 40.0, 2.0, 0.05, 0.7
    cam = ident_cam(65, 65, f, cx=32.5, cy=32.5)
    sc = _one_gaussian(z0, s, sig, dc=(0.3, 0.5, 0.7))
    sc_ = oracle_lib.contribution(sc, cam)
    np.testing.assert_allclose(sc_[0], _col((0.3, 0.5, 0.7)).max() * sig / (1 + sig), rtol=1e-13)
    rs = sg.random_scene(92, 60, 150, n_objects=4, box=1.0, sphere_r=(0.3, 0.6), plane_side=(0.6, 1.2),
                         surfel_scale=(0.05, 0.15), gauss_logscale=(-3.5, 0.4))
    cam = sg.look_at((0.1, -0.2, -2.6), (0, 0, 0), (0, 1, 0), 41, 33, 60.0)
    got = oracle_lib.contribution(rs, cam)
    ref = oracle_lib.render(rs, cam)
    U, V = np.meshgrid(np.arange(cam.width) + 0.5, np.arange(cam.height) + 0.5)
    for k in range(rs.n_gaussians):
        gi = oracle_lib.gauss_info(rs, cam, k)
        want = 0.0
        if gi["valid"]:
            du, dv = U - gi["px"], V - gi["py"]
            ca, cb, cc = gi["conic"]
            a = gi["sigma"] * np.exp(-0.5 * (ca * du * du + 2 * cb * du * dv + cc * dv * dv))
            x0, x1, y0, y1 = gi["bbox"]
            box = np.zeros_like(a, bool)
            box[y0:y1 + 1, x0:x1 + 1] = True
            m = box & (a >= 1 / 255) & (gi["d"] < ref["depth"] + gi["eps"])
            if m.any():
                want = float((gi["rgb"].max() * a / (1 + ref["wg"]))[m].max())
        assert abs(got[k] - want) <= 1e-12 * max(1.0, want), (k, got[k], want)
    assert (got > 0).sum() > 30
