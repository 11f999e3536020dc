"""The batch graph (every phase one launch over all views, persistent raster
over (view, tile) items): bitwise the per-view render's images, for every
render mode, sample count and Gaussian kind, with empty, ragged and long tile
lists; and the timed 1080p orbit path itself against the oracle."""
import numpy as np
import pytest

import scenegen as sg
from test_gpu_2dges import _small2d
from test_gpu_forward import _small

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_17545_gb300 import render as R
    return R


def _views():
    return [sg.look_at((0.5, 0, -2.8), (0, 0, 0), (0, 1, 0), 301, 173, 60.0),
            sg.look_at((0, 0.3, -2.6), (0, 0, 0), (0, 1, 0), 128, 96, 50.0),
            sg.look_at((-0.4, 0.2, -2.2), (0, 0, 0), (0, 1, 0), 64, 200, 45.0),
            sg.look_at((0, 0, -2.5), (0, 0, 0), (0, 1, 0), 1, 1, 60.0),
            sg.look_at((0.1, 0.05, -0.6), (0, 0.1, 1), (0, 1, 0), 97, 61, 95.0)]


def _check(R, scenes, views, sov, opts, reps=2, shape=None):
    b = R.GESBatch(scenes, views, sov, opts=opts)
    if shape is not None:
        assert f"{b.info().tile_w}x{b.info().tile_h}" == shape
    for rep in range(reps):
        b.launch()
        b.sync()
        for v in range(len(views)):
            single = R.render(scenes[sov[v]], views[v], opts, with_aux=False)
            assert (b.rgb[v] == single["rgb"]).all(), (rep, v)
            assert (b.depth[v] == single["depth"]).all(), (rep, v)
    b.close()


@pytest.mark.parametrize("opts", [None, dict(mode=1), dict(mode=2), dict(samples=4)])
def test_batch_raster_equals_single_views(R, opts):
    scene, cams = sg.config_scene(0)
    other = _small(91, 2000, 6000)
    empty = other.subset(s_idx=np.zeros(0, int), g_idx=np.zeros(0, int))
    gs = [R.GESScene.from_arrays(x) for x in (scene, other, empty)]
    views = [cams[0]] + _views() + [cams[0]]
    sov = [0, 1, 0, 1, 0, 1, 2]
    _check(R, gs, views, sov, opts)
    for g in gs:
        g.close()


def test_batch_raster_long_tile_lists(R):
    """Thousands of entries per tile: many staged chunks (256 records) per tile."""
    dense = _small(92, 30000, 30000)
    gs = R.GESScene.from_arrays(dense)
    views = [sg.look_at((0, 0, -2.5), (0, 0, 0), (0, 1, 0), 48, 40, 60.0),
             sg.look_at((0.3, 0.2, -2.4), (0, 0, 0), (0, 1, 0), 33, 17, 50.0)]
    gs_stats = []
    for c in views:
        R.render(gs, c, with_aux=False)
        gs_stats.append(gs.stats())
    # the lists really are long: over 1000 entries per tile on average
    assert min(s.surfel_tile_pairs / (s.tiles_x * s.tiles_y) for s in gs_stats) > 1000
    _check(R, [gs], views, [0, 0], None)
    gs.close()


def test_batch_raster_2d_gaussians(R):
    ga, gb = R.GESScene.from_arrays(_small2d(93, 2000, 6000)), R.GESScene.from_arrays(_small2d(94, 500, 3000))
    views = _views()[:3]
    for opts in (None, dict(samples=4)):
        _check(R, [ga, gb], views, [0, 1, 0], opts, reps=1)
    ga.close()
    gb.close()


def test_batch_camera_discs_match_oracle(R):
    """The hand-placed discs at and behind the camera, and 2D splats reaching
    back through the near plane, through the batch graph (its own set-up and
    colour-pass kernels): two views of each scene, each against the oracle
    with the id map the batch writes."""
    import torch
    import oracle
    import camera_discs as cd
    from parity import compare
    cam0 = cd.camera()
    w2c = np.concatenate([np.eye(3), np.array([[0.01], [-0.005], [0.0]])], 1).astype(np.float32)
    cam1 = sg.Camera(cam0.width, cam0.height, cam0.fx, cam0.fy, cam0.cx, cam0.cy, w2c)
    base = cd.background()
    scenes = [cd.with_discs(base, cd.walls(), 37), cd.with_splats(cd.flat(base), cd.splats(), 40)]
    for sc in scenes:
        gs = R.GESScene.from_arrays(sc)
        b = R.GESBatch([gs], [cam0, cam1])
        ids = [torch.empty((cam0.height, cam0.width), dtype=torch.int32, device="cuda") for _ in range(2)]
        for v in range(2):
            b.set_id_output(v, ids[v])
        b.launch()
        b.sync()
        for v, cam in enumerate((cam0, cam1)):
            ref = oracle.render(sc, cam)
            res = compare(sc, cam, dict(rgb=b.rgb[v], depth=b.depth[v], id=ids[v]), ref, max_masked=0.1)
            assert res["pass"], res
            single = R.render(gs, cam)
            assert (b.rgb[v] == single["rgb"]).all() and (b.depth[v] == single["depth"]).all(), v
        b.close()
        gs.close()


def test_timed_orbit_path_matches_oracle(R):
    """The benchmark's own path: a batch graph over views of the 1M-surfel /
    300k-Gaussian 1080p orbit.  One view against the oracle directly (colour,
    depth and the surfel id map the batch writes when asked), every view
    bitwise equal to its per-view render (ids and W_G too where written), and
    the per-view completion stamps sane."""
    import torch
    import oracle
    from parity import MASKED_MAX, compare
    scene, cams = sg.config_scene(1)
    gs = R.GESScene.from_arrays(scene)
    views = [cams[k] for k in (0, 16, 33, 50)]
    b = R.GESBatch([gs], views)
    ids = {v: torch.empty((views[v].height, views[v].width), dtype=torch.int32, device="cuda") for v in (1, 2)}
    aux = torch.empty((views[2].height, views[2].width), device="cuda")
    b.set_id_output(1, ids[1])
    b.set_id_output(2, ids[2], aux)
    b.launch()
    b.sync()
    t = b.view_times()
    assert all(0.0 < x < 1000.0 for x in t), t
    for v in range(len(views)):
        single = R.render(gs, views[v], with_aux=True)
        assert (b.rgb[v] == single["rgb"]).all() and (b.depth[v] == single["depth"]).all(), v
        if v in ids:
            assert (ids[v] == single["id"]).all(), v
        if v == 2:
            assert (aux == single["aux"]).all()
    ref = oracle.render(scene, views[2])
    res = compare(scene, views[2], dict(rgb=b.rgb[2], depth=b.depth[2], id=ids[2]), ref)
    assert res["pass"], res
    assert res["masked_frac"] <= MASKED_MAX
    # switched off again: the next launch leaves the arrays alone
    b.set_id_output(1, None)
    ids[1].fill_(-7)
    b.launch()
    b.sync()
    assert (ids[1] == -7).all()
    b.close()
    gs.close()


@pytest.mark.parametrize("shape", ["16x16", "32x8", "8x32"])
def test_batch_tile_shapes_equal_single_views(R, monkeypatch, shape):
    """Every binning tile shape the autotuner tries gives bitwise the per-view
    (16x16) render, with ragged, tiny and empty views, 4 samples and 2D
    Gaussians: the shape moves work between CTAs, never the arithmetic."""
    monkeypatch.setenv("GES_BATCH_TILE", shape)
    scene, cams = sg.config_scene(0)
    other = _small(95, 2000, 6000)
    empty = other.subset(s_idx=np.zeros(0, int), g_idx=np.zeros(0, int))
    gs = [R.GESScene.from_arrays(x) for x in (scene, other, empty)]
    views = [cams[0]] + _views() + [cams[0]]
    sov = [0, 1, 0, 1, 0, 1, 2]
    for opts in (None, dict(samples=4)):
        _check(R, gs, views, sov, opts, reps=1, shape=shape)
    for g in gs:
        g.close()
    g2 = R.GESScene.from_arrays(_small2d(96, 2000, 6000))
    _check(R, [g2], _views()[:3], [0, 0, 0], None, reps=1, shape=shape)
    g2.close()


def test_batch_autotuner_candidates(R):
    scene, cams = sg.config_scene(0)
    gs = R.GESScene.from_arrays(scene)
    b = R.GESBatch([gs], [cams[0]])
    # 3 tile shapes x 5 preprocess ranges x 2 raster occupancies
    assert b.info().candidates == 30
    assert f"{b.info().tile_w}x{b.info().tile_h}" in ("16x16", "32x8", "8x32")
    b.launch()
    b.sync()
    single = R.render(gs, cams[0], with_aux=False)
    assert (b.rgb[0] == single["rgb"]).all() and (b.depth[0] == single["depth"]).all()
    b.close()
    gs.close()


def test_batch_2160p_orbit_view_matches_oracle(R):
    """The headline scene at 3840x2160 (32400 tiles, near the local-binning
    limit of 32768) through the batch graph: one view against the oracle, the
    other equal to its per-view render."""
    import dataclasses
    import oracle
    from parity import MASKED_MAX, compare
    scene, cams = sg.config_scene(1)
    big = [dataclasses.replace(c, width=2 * c.width, height=2 * c.height, fx=2 * c.fx, fy=2 * c.fy,
                               cx=2 * c.cx, cy=2 * c.cy) for c in (cams[5], cams[40])]
    gs = R.GESScene.from_arrays(scene)
    b = R.GESBatch([gs], big)
    b.launch()
    b.sync()
    ref = oracle.render(scene, big[0])
    single = R.render(gs, big[0])
    assert (b.rgb[0] == single["rgb"]).all() and (b.depth[0] == single["depth"]).all()
    res = compare(scene, big[0], single, ref)
    assert res["pass"], res
    assert res["masked_frac"] <= MASKED_MAX
    single1 = R.render(gs, big[1], with_aux=False)
    assert (b.rgb[1] == single1["rgb"]).all() and (b.depth[1] == single1["depth"]).all()
    b.close()
    gs.close()


@pytest.mark.parametrize("deg,dtype", [(0, "float32"), (1, "float32"), (2, "float16"), (3, "bfloat16")])
def test_batch_colour_pass_sh_degrees_and_storage(R, deg, dtype):
    """The batch's colour pass (Eq. 1 for all views of a scene, one SH read
    per primitive) stores the same bits as the inline colour of the per-view
    path, for every SH degree and storage type."""
    import torch
    sc = sg.random_scene(95, 1500, 4000, n_objects=5, box=1.0, sphere_r=(0.3, 0.6), plane_side=(0.6, 1.2),
                         surfel_scale=(0.03, 0.1), gauss_logscale=(-3.8, 0.4), sh_degree=deg)
    dt = getattr(torch, dtype)
    gs = R.GESScene.from_arrays(sc, attr_dtype=dt, sh_dtype=dt)
    _check(R, [gs], _views()[:3], [0, 0, 0], None, reps=1)
    gs.close()


def test_batch_colour_pass_groups_views_by_scene_arrays(R):
    """Views are grouped for the colour pass by the arrays their scenes view:
    two scene handles on the same tensors share one group, a scene with the
    same positions but other SH does not; ges_render_batch rebuilds its kept
    graph when the grouping of the same view pattern changes."""
    import torch
    sc = _small(96, 1500, 4000)
    ga = R.GESScene.from_arrays(sc)
    gb = R.GESScene(sc.sh_degree, **ga.t)                     # the same tensors
    t = dict(ga.t)
    t["s_sh"] = (t["s_sh"] * 0.5).contiguous()
    t["g_sh"] = (t["g_sh"] - 0.1).contiguous()
    gc = R.GESScene(sc.sh_degree, **t)                       # same positions, other colours
    views = _views()[:3]
    _check(R, [ga, gb, gc], views + views[:2], [0, 1, 2, 0, 2], None, reps=1)
    for scenes in ([ga, gb], [ga, gc], [ga, gb]):
        outs = R.render_batch(scenes, views[:2], [0, 1])
        torch.cuda.synchronize()
        for v in range(2):
            single = R.render(scenes[v], views[v], with_aux=False)
            assert (outs[v][0] == single["rgb"]).all() and (outs[v][1] == single["depth"]).all(), v
    for g in (ga, gb, gc):
        g.close()


def test_batch_colour_pass_more_views_than_one_staging_round(R):
    """A scene with 70 views: the colour pass stages the views' camera centres
    64 at a time, so a second round covers the last 6; every view's image
    equals its per-view render."""
    sc = _small(97, 800, 2000)
    gs = R.GESScene.from_arrays(sc)
    views = [sg.look_at((2.6 * np.sin(a), 0.3 * np.cos(3 * a), -2.6 * np.cos(a)), (0, 0, 0), (0, 1, 0), 40, 24, 55.0)
             for a in np.linspace(0.0, 2.0 * np.pi, 70, endpoint=False)]
    _check(R, [gs], views, [0] * 70, None, reps=1)
    gs.close()
