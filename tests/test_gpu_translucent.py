"""Translucent-surfel render of the coarse stage (Sec. 4.1, Eq. 6-7) on the
GPU vs the FP64 oracle: forward, backward, covering score; and the Gaussian
contribution score (Eq. 9)."""
import json

import numpy as np
import pytest

import oracle
import scenegen as sg
from parity import COL_TOL, log_result

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3


@pytest.fixture(scope="module")
def R():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_17545_gb300 import render as R
    return R


def _scene_w(kind, seed):
    rng = np.random.default_rng(seed)
    if kind == "crop":
        sc, cam = sg.crop_scene(7)
    else:
        sc, cams = sg.config_scene(0)
        cam = cams[0]
    w = rng.uniform(0.3, 3.0, sc.n_surfels) if seed % 2 else rng.uniform(0.05, 60.0, sc.n_surfels)
    return sc, cam, w.astype(np.float32).astype(np.float64)


def _run(R, sc, cam, w, ff, cover=False):
    import torch
    gs = R.GESScene.from_arrays(sc)
    out = R.render_translucent(gs, cam, torch.as_tensor(w, dtype=torch.float32, device="cuda"), ff, cover=cover)
    return gs, out


def _fwd_compare(gpu, ref):
    ok = ref["amb"] == 0
    rgb = gpu["rgb"].cpu().numpy().astype(np.float64)
    res = dict(col_max=float(np.abs(rgb - ref["rgb"])[:, ok].max()),
               T_max=float(np.abs(gpu["T"].cpu().numpy() - ref["T"])[ok].max()),
               front_mismatch=int((gpu["front"].cpu().numpy() != ref["front"])[ok].sum()),
               compared=int(ok.sum()), masked_frac=float(1.0 - ok.mean()))
    res["pass"] = (res["col_max"] <= COL_TOL and res["T_max"] <= COL_TOL and res["front_mismatch"] == 0 and
                   res["masked_frac"] <= 0.1)
    log_result("translucent", res)
    return res


@pytest.mark.parametrize("kind,seed", [("crop", 1), ("crop", 2), ("cfg0", 3), ("cfg0", 4)])
@pytest.mark.parametrize("ff", [False, True])
def test_translucent_forward_matches_oracle(R, kind, seed, ff):
    sc, cam, w = _scene_w(kind, seed)
    gs, out = _run(R, sc, cam, w, ff)
    gs.close()
    ref = oracle.render_translucent(sc, cam, w, ff)
    res = _fwd_compare(out, ref)
    assert res["pass"], json.dumps(res)
    assert res["compared"] > 0.9 * cam.width * cam.height


@pytest.mark.parametrize("ff", [False, True])
def test_translucent_discs_at_and_behind_the_camera(R, ff):
    """The hand-placed discs at and behind the camera in the translucent
    render: centres behind the camera have negative camera depths, which
    must order before every other centre, and the walls reach through the
    near plane."""
    import camera_discs as cd
    cam, base = cd.camera(), cd.background()
    for discs, seed in ((cd.walls(), 37), (cd.tilted(), 38)):
        sc = cd.with_discs(base, discs, seed)
        w = np.random.default_rng(seed).uniform(0.3, 3.0, sc.n_surfels).astype(np.float32).astype(np.float64)
        gs, out = _run(R, sc, cam, w, ff)
        gs.close()
        ref = oracle.render_translucent(sc, cam, w, ff)
        res = _fwd_compare(out, ref)
        assert res["pass"], json.dumps(res)
        assert (ref["front"] == base.n_surfels).sum() > 50


def test_translucent_w255_equals_opaque_render(R):
    """At w = 255 with the front-first order the translucent render equals the
    z-buffer render (surfels only), as the paper states for the end of the
    coarse stage."""
    scene, cams = sg.config_scene(0)
    gs, out = _run(R, scene, cams[0], np.full(scene.n_surfels, 255.0), True, cover=True)
    op = R.render(gs, cams[0], dict(mode=1))
    ref = oracle.render_translucent(scene, cams[0], np.full(scene.n_surfels, 255.0), True)
    ok = (ref["amb"] == 0) & (oracle.render(scene, cams[0], dict(mode=1))["amb"] == 0)
    np.testing.assert_allclose(out["rgb"].cpu().numpy()[:, ok], op["rgb"].cpu().numpy()[:, ok], rtol=0, atol=1e-6)
    ids = op["id"].cpu().numpy()
    assert (out["front"].cpu().numpy()[ok] == ids[ok]).all()
    cov = out["cover"].cpu().numpy()
    fr = out["front"].cpu().numpy()
    np.testing.assert_array_equal(cov, np.bincount(fr[fr >= 0], minlength=scene.n_surfels))
    gs.close()


def test_translucent_1080p_orbit_camera(R):
    scene, cams = sg.config_scene(1)
    sc = scene.subset(g_idx=np.zeros(0, int))
    w = np.random.default_rng(5).uniform(0.5, 60.0, sc.n_surfels).astype(np.float32).astype(np.float64)
    gs, out = _run(R, sc, cams[4], w, True)
    gs.close()
    ref = oracle.render_translucent(sc, cams[4], w, True)
    res = _fwd_compare(out, ref)
    assert res["pass"], json.dumps(res)
    assert res["compared"] > 0.9 * cams[4].width * cams[4].height


def test_translucent_covering_counts_match_oracle(R):
    sc, cam, w = _scene_w("cfg0", 5)
    gs, out = _run(R, sc, cam, w, True, cover=True)
    gs.close()
    ref = oracle.covering_counts(sc, cam, w)
    amb = oracle.render_translucent(sc, cam, w, True)["amb"] != 0
    assert np.abs(out["cover"].cpu().numpy() - ref).sum() <= amb.sum()


def _bwd_check(gpu, ref, keep, keys):
    for k in keys:
        a = gpu[k][keep] if keep is not None else gpu[k]
        b = ref[k][keep] if keep is not None else ref[k]
        scale = max(np.abs(b).max(), 1e-12)
        err = float(np.abs(a - b).max())
        assert err <= GRAD_TOL * scale, (k, err, scale)


@pytest.mark.parametrize("kind,seed", [("crop", 1), ("cfg0", 3)])
@pytest.mark.parametrize("ff", [False, True])
def test_translucent_backward_matches_oracle(R, kind, seed, ff):
    import torch
    sc, cam, w = _scene_w(kind, seed)
    g = np.random.default_rng(seed + 10).standard_normal((3, cam.height, cam.width))
    gs, out = _run(R, sc, cam, w, ff)
    wt = torch.as_tensor(w, dtype=torch.float32, device="cuda")
    grads = R.render_translucent_backward(gs, cam, wt, out, torch.as_tensor(g, dtype=torch.float32, device="cuda"), ff)
    gpu = {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}
    gs.close()
    ref = oracle.backward_translucent(sc, cam, w, g, ff)
    amb = oracle.render_translucent(sc, cam, w, ff)["amb"] != 0
    st, _ = oracle.touching(sc, cam, amb)
    keep = ~st
    assert keep.mean() > 0.7
    _bwd_check(gpu, ref, keep, ["s_pos", "s_rot", "s_scale", "s_w", "s_sh"])


def test_translucent_deterministic_bitwise(R):
    import torch
    sc, cam, w = _scene_w("cfg0", 6)
    g = torch.as_tensor(np.random.default_rng(7).standard_normal((3, cam.height, cam.width)), dtype=torch.float32,
                        device="cuda")
    wt = torch.as_tensor(w, dtype=torch.float32, device="cuda")
    gs = R.GESScene.from_arrays(sc)
    a = R.render_translucent(gs, cam, wt, True)
    b = R.render_translucent(gs, cam, wt, True)
    ga = R.render_translucent_backward(gs, cam, wt, a, g, True)
    gb = R.render_translucent_backward(gs, cam, wt, b, g, True)
    for k in ("rgb", "T", "front", "last", "Tlast"):
        assert (a[k] == b[k]).all(), k
    for k in ga:
        assert (ga[k] == gb[k]).all(), k
    gs.close()


def test_translucent_rejects_bad_options(R):
    import torch
    from paper_2504_17545_gb300 import native as N
    sc, cam, w = _scene_w("crop", 1)
    gs = R.GESScene.from_arrays(sc)
    wt = torch.as_tensor(w, dtype=torch.float32, device="cuda")
    for bad in (dict(samples=4), dict(surfel_r2=4.0)):
        with pytest.raises(N.GesError) as ei:
            R.render_translucent(gs, cam, wt, True, opts=bad)
        assert ei.value.status == N.GES_ERR_INVALID_ARG
    gs.close()


def test_contribution_scores_match_oracle(R):
    scene, cams = sg.config_scene(0)
    gs = R.GESScene.from_arrays(scene)
    fwd = R.render(gs, cams[0])
    got = R.contribution_scores(gs, cams[0], fwd).cpu().numpy().astype(np.float64)
    gs.close()
    ref = oracle.contribution(scene, cams[0])
    amb = oracle.render(scene, cams[0])["amb"] != 0
    _, gt = oracle.touching(scene, cams[0], amb)
    keep = ~gt
    assert keep.mean() > 0.75 and (ref[keep] > 0).sum() > 100
    np.testing.assert_allclose(got[keep], ref[keep], rtol=2e-4, atol=1e-6)


def test_translucent_nonpositive_w_are_never_drawn(R):
    """w <= 0 (or a zero weight left by pruning) gives alpha = 0 everywhere:
    such surfels are never blended, never frontmost and get no gradient."""
    import torch
    sc, cam, w = _scene_w("cfg0", 11)
    rng = np.random.default_rng(12)
    off = rng.random(sc.n_surfels) < 0.3
    w = w.copy()
    w[off] = np.where(rng.random(off.sum()) < 0.5, 0.0, -1.0)
    gs, out = _run(R, sc, cam, w, True, cover=True)
    ref = oracle.render_translucent(sc, cam, w, True)
    res = _fwd_compare(out, ref)
    assert res["pass"], json.dumps(res)
    front = out["front"].cpu().numpy()
    assert not off[front[front >= 0]].any()
    assert (out["cover"].cpu().numpy()[off] == 0).all()
    g = torch.as_tensor(np.random.default_rng(13).standard_normal((3, cam.height, cam.width)), dtype=torch.float32,
                        device="cuda")
    wt = torch.as_tensor(w, dtype=torch.float32, device="cuda")
    gr = R.render_translucent_backward(gs, cam, wt, out, g, True)
    for k in ("s_pos", "s_rot", "s_scale", "s_w", "s_sh"):
        assert (gr[k].cpu().numpy()[off] == 0).all(), k
    gs.close()
