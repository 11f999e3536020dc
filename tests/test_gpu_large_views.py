"""Views of more than 32768 tiles (4096x2304: 256 x 144 = 36864).  The
per-CTA shared-memory bins of the preprocess and fill hold 32768 tile
counters, so the per-view path bins such views with global counters
(k_prep_atomic / k_fill_atomic).  Every render kind that goes through that
binning is compared with the oracle here; the batch graph, which only has
the shared-memory bins, refuses such views."""
import json

import numpy as np
import pytest

import oracle
import scenegen as sg
from parity import compare
from test_gpu_2dges import _flat
from test_gpu_translucent import _fwd_compare

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3   # of the largest |gradient| in each parameter group
LOCAL_MAX_TILES = 32768


@pytest.fixture(scope="module")
def R():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_17545_gb300 import render as R
    return R


def _big():
    return sg.look_at((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 4096, 2304, 60.0)


def _check_tiles(gs):
    s = gs.stats()
    assert s.tiles_x * s.tiles_y == 36864 > LOCAL_MAX_TILES


@pytest.mark.parametrize("opts", [None, dict(mode=1), dict(mode=2), dict(samples=4)])
def test_large_view_matches_oracle(R, opts):
    scene, _ = sg.config_scene(0)
    cam = _big()
    gs = R.GESScene.from_arrays(scene)
    out = R.render(gs, cam, opts)
    _check_tiles(gs)
    s = gs.stats()
    assert s.surfel_tile_pairs > 0 or (opts or {}).get("mode") == 2
    gs.close()
    ref = oracle.render(scene, cam, opts)
    res = compare(scene, cam, out, ref, opts)
    assert res["pass"], json.dumps(res, default=str)
    assert res["compared_px"] > 0.99 * cam.width * cam.height


def test_large_view_2d_gaussians_match_oracle(R):
    scene, _ = sg.config_scene(0)
    sc = _flat(scene)
    cam = _big()
    gs = R.GESScene.from_arrays(sc)
    out = R.render(gs, cam)
    _check_tiles(gs)
    gs.close()
    ref = oracle.render(sc, cam)
    res = compare(sc, cam, out, ref)
    assert res["pass"], json.dumps(res, default=str)
    assert (ref["wg"] > 0).mean() > 0.05


def test_large_view_backward_matches_oracle(R):
    """dL/dC is zero at the pixels the oracle flags as ambiguous (several
    forward answers are correct there), so every remaining contribution is
    one both sides agree on and all primitives are compared."""
    import torch
    scene, _ = sg.config_scene(0)
    cam = _big()
    amb = oracle.render(scene, cam)["amb"] != 0
    g = np.random.default_rng(12).standard_normal((3, cam.height, cam.width))
    g[:, amb] = 0.0
    gs = R.GESScene.from_arrays(scene)
    fwd = R.render(gs, cam)
    _check_tiles(gs)
    gr = R.render_backward(gs, cam, fwd, torch.as_tensor(g, dtype=torch.float32, device="cuda"))
    gpu = {k: v.cpu().numpy().astype(np.float64) for k, v in gr.items()}
    gs.close()
    ref = oracle.backward(scene, cam, g)
    for k in ("g_pos", "g_rot", "g_scale", "g_opac", "g_sh", "s_sh"):
        scale = max(np.abs(ref[k]).max(), 1e-12)
        err = float(np.abs(gpu[k] - ref[k]).max())
        assert err <= GRAD_TOL * scale, (k, err, scale)
        assert np.count_nonzero(ref[k]) > 0, k


@pytest.mark.parametrize("ff", [False, True])
def test_large_view_translucent_matches_oracle(R, ff):
    import torch
    scene, _ = sg.config_scene(0)
    cam = _big()
    w = np.random.default_rng(5).uniform(0.3, 3.0, scene.n_surfels).astype(np.float32).astype(np.float64)
    gs = R.GESScene.from_arrays(scene)
    out = R.render_translucent(gs, cam, torch.as_tensor(w, dtype=torch.float32, device="cuda"), ff)
    gs.close()
    ref = oracle.render_translucent(scene, cam, w, ff)
    res = _fwd_compare(out, ref)
    assert res["pass"], json.dumps(res)
    assert res["compared"] > 0.99 * cam.width * cam.height


def test_batch_refuses_views_beyond_the_shared_memory_bins(R):
    from paper_2504_17545_gb300 import native as N
    scene, cams = sg.config_scene(0)
    gs = R.GESScene.from_arrays(scene)
    with pytest.raises(N.GesError, match="tiles"):
        R.GESBatch([gs], [cams[0], _big()])
    # the scene is still usable afterwards
    out = R.render(gs, cams[0])
    assert out["rgb"].isfinite().all()
    gs.close()
