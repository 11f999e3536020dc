"""The batch graph's two raster kinds: CTA-staged, and pipelined (a producer
warp gathers each tile's records with bulk asynchronous copies into a ring of
shared-memory stages guarded by mbarriers; eight pixel warps consume them
without CTA-wide barriers).  Both must give bitwise the per-view render's
images, for every render mode, sample count and Gaussian kind, with empty,
ragged and multi-stage tile lists."""
import numpy as np
import pytest

import scenegen as sg
from test_gpu_2dges import _small2d
from test_gpu_forward import _small

pytestmark = pytest.mark.gpu

KINDS = ["classic", "pipelined"]


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


def _check(R, scenes, views, sov, opts, kind, reps=2):
    b = R.GESBatch(scenes, views, sov, opts=opts)
    assert b.info().raster_pipelined == (1 if kind == "pipelined" else 0)
    for rep in range(reps):
        b.launch()
        b.sync()
        for v in range(len(views)):
            single = R.render(scenes[sov[v]], views[v], opts, with_aux=False)
            assert (b.rgb[v] == single["rgb"]).all(), (kind, rep, v)
            assert (b.depth[v] == single["depth"]).all(), (kind, rep, v)
    b.close()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("opts", [None, dict(mode=1), dict(mode=2), dict(samples=4)])
def test_batch_raster_equals_single_views(R, monkeypatch, kind, opts):
    monkeypatch.setenv("GES_BATCH_RASTER", kind)
    scene, cams = sg.config_scene(0)
    other = _small(91, 2000, 6000)
    empty = other.subset(s_idx=np.zeros(0, int), g_idx=np.zeros(0, int))
    gs = [R.GESScene.from_arrays(x) for x in (scene, other, empty)]
    views = [cams[0]] + _views() + [cams[0]]
    sov = [0, 1, 0, 1, 0, 1, 2]
    _check(R, gs, views, sov, opts, kind)
    for g in gs:
        g.close()


@pytest.mark.parametrize("kind", KINDS)
def test_batch_raster_long_tile_lists(R, monkeypatch, kind):
    """Thousands of entries per tile: many stages (128 records each) and
    chunks (256) per tile, so the ring wraps inside one tile."""
    monkeypatch.setenv("GES_BATCH_RASTER", kind)
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
    _check(R, [gs], views, [0, 0], None, kind)
    gs.close()


@pytest.mark.parametrize("kind", KINDS)
def test_batch_raster_2d_gaussians(R, monkeypatch, kind):
    monkeypatch.setenv("GES_BATCH_RASTER", kind)
    ga, gb = R.GESScene.from_arrays(_small2d(93, 2000, 6000)), R.GESScene.from_arrays(_small2d(94, 500, 3000))
    views = _views()[:3]
    for opts in (None, dict(samples=4)):
        _check(R, [ga, gb], views, [0, 1, 0], opts, kind, reps=1)
    ga.close()
    gb.close()


def test_batch_raster_kinds_agree_on_the_1080p_orbit(R, monkeypatch):
    """Four views of the 1M-surfel / 300k-Gaussian 1080p orbit through both
    kinds: identical images, and identical to the per-view render."""
    scene, cams = sg.config_scene(1)
    gs = R.GESScene.from_arrays(scene)
    views = [cams[k] for k in (0, 16, 33, 50)]
    imgs = {}
    for kind in KINDS:
        monkeypatch.setenv("GES_BATCH_RASTER", kind)
        b = R.GESBatch([gs], views)
        assert b.info().raster_pipelined == (1 if kind == "pipelined" else 0)
        b.launch()
        b.sync()
        imgs[kind] = [(b.rgb[v].clone(), b.depth[v].clone()) for v in range(len(views))]
        t = b.view_times()
        assert all(0.0 < x < 1000.0 for x in t), t
        b.close()
    single = R.render(gs, views[2], with_aux=False)
    for v in range(len(views)):
        assert (imgs["classic"][v][0] == imgs["pipelined"][v][0]).all(), v
        assert (imgs["classic"][v][1] == imgs["pipelined"][v][1]).all(), v
    assert (imgs["pipelined"][2][0] == single["rgb"]).all() and (imgs["pipelined"][2][1] == single["depth"]).all()
    gs.close()


def test_batch_raster_auto_times_both_kinds(R, monkeypatch):
    monkeypatch.setenv("GES_BATCH_RASTER", "auto")
    scene, cams = sg.config_scene(0)
    gs = R.GESScene.from_arrays(scene)
    b = R.GESBatch([gs], [cams[0]])
    # 5 preprocess ranges x (2 classic + 2 pipelined) raster shapes
    assert b.info().candidates == 20
    b.launch()
    b.sync()
    single = R.render(gs, cams[0], with_aux=False)
    assert (b.rgb[0] == single["rgb"]).all() and (b.depth[0] == single["depth"]).all()
    b.close()
    gs.close()


def test_bounded_mbarrier_wait_gives_up(R):
    """The pipelined raster's shared-memory waits are bounded: on a barrier
    that nothing completes, the wait returns after its limit (device time)
    and the GPU stays usable.  No fault is involved."""
    from paper_2504_17545_gb300 import native as N
    ok, gave_up, us = N.ges_selftest_wait_timeout(50)
    assert ok and gave_up, (ok, gave_up, us)
    assert 50_000 <= us < 5_000_000, us
    # the context still works
    scene, cams = sg.config_scene(0)
    gs = R.GESScene.from_arrays(scene)
    out = R.render(gs, cams[0])
    assert out["rgb"].isfinite().all()
    gs.close()
    with pytest.raises(N.GesError):
        N.ges_selftest_wait_timeout(0)


def test_batch_2160p_orbit_view_matches_oracle(R):
    """The headline scene at 3840x2160 (32400 tiles, near the local-binning
    limit of 32768) through the batch graph: one view against the oracle, the
    other equal to its per-view render."""
    import dataclasses
    import oracle
    from parity import compare
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
    assert res["masked_frac"] < 0.01
    single1 = R.render(gs, big[1], with_aux=False)
    assert (b.rgb[1] == single1["rgb"]).all() and (b.depth[1] == single1["depth"]).all()
    b.close()
    gs.close()
