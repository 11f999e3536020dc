"""2D-GES (Sec. 6.4) and the geometry maps (Eq. 10-12) on the GPU vs the FP64
oracle: 2D Gaussians with planar depth and the object-space filter, N_s,
D_G, N_G, D_smooth, N_smooth for both Gaussian kinds, the batch graph."""
import json
import numpy as np
import pytest

import oracle
import scenegen as sg
from parity import MASKED_MAX, compare, compare_geom
from test_gpu_forward import _render, _small

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_17545_gb300 import render as R
    return R


def _assert(res):
    assert res["pass"], json.dumps(res, default=str)


def _flat(scene):
    """The same scene with 2D Gaussians (the first two axes of each)."""
    sc = scene.subset()
    sc.g_scale = np.ascontiguousarray(sc.g_scale[:, :2])
    return sc


def _small2d(seed, n_s=400, n_g=1500):
    return _flat(sg.random_scene(seed, n_s, n_g, n_objects=5, box=1.0, sphere_r=(0.3, 0.6), plane_side=(0.6, 1.2),
                                 surfel_scale=(0.03, 0.1), gauss_logscale=(-3.2, 0.4)))


def test_2d_parity_workload_128(R):
    scene, cams = sg.config_scene(0)
    sc = _flat(scene)
    ref = oracle.render(sc, cams[0])
    res = compare(sc, cams[0], _render(R, sc, cams[0]), ref)
    _assert(res)
    assert res["compared_px"] > 0.95 * 128 * 128 and (ref["wg"] > 0).mean() > 0.15


@pytest.mark.parametrize("opts", [dict(mode=0), dict(mode=2), dict(mode=0, samples=4),
                                  dict(mode=0, eps_mode=1), dict(mode=0, lowpass=1.0)])
def test_2d_parity_ragged_modes_options(R, opts):
    scene = _small2d(81)
    cams = [sg.look_at((0.2, 0.3, -2.8), (0, 0, 0), (0, 1, 0), 203, 141, 55.0),
            sg.look_at((0.1, 0.05, -0.6), (0, 0.1, 1), (0, 1, 0), 97, 61, 95.0)]   # inside the scene
    for cam in cams:
        ref = oracle.render(scene, cam, opts)
        _assert(compare(scene, cam, _render(R, scene, cam, opts), ref, opts))


def test_2d_parity_1080p_orbit_camera(R):
    scene, cams = sg.config_scene(1)
    sc = _flat(scene)
    gs = R.GESScene.from_arrays(sc)
    ref = oracle.render(sc, cams[24])
    res = compare(sc, cams[24], R.render(gs, cams[24]), ref)
    _assert(res)
    assert res["masked_frac"] <= MASKED_MAX
    gs.close()


def test_2d_fragment_counts_match_oracle(R):
    from paper_2504_17545_gb300 import native as N
    scene, cams = sg.config_scene(0)
    sc = _flat(scene)
    gs = R.GESScene.from_arrays(sc)
    ns, ng = N.ges_count_fragments(gs.handle, R.camera_struct(cams[0]), R.opts_struct(None))
    os_, og = oracle.count_fragments(sc, cams[0])
    assert abs(ns - os_) <= max(3, 1e-4 * os_) and abs(ng - og) <= max(3, 1e-4 * og), (ns, os_, ng, og)
    gs.close()


@pytest.mark.parametrize("dim", [3, 2])
def test_geometry_maps_workload_128(R, dim):
    scene, cams = sg.config_scene(0)
    sc = scene if dim == 3 else _flat(scene)
    gs = R.GESScene.from_arrays(sc)
    out = R.render_geom(gs, cams[0])
    gs.close()
    ref = oracle.render(sc, cams[0])
    geo = oracle.render_geom(sc, cams[0])
    _assert(compare(sc, cams[0], out, ref))
    res = compare_geom(out, geo, ref)
    _assert(res)
    assert res["compared_px"] > 0.9 * 128 * 128


@pytest.mark.parametrize("dim", [3, 2])
@pytest.mark.parametrize("opts", [dict(mode=0), dict(mode=1), dict(mode=2), dict(mode=0, samples=4)])
def test_geometry_maps_ragged(R, dim, opts):
    scene = _small(82) if dim == 3 else _small2d(82)
    cam = sg.look_at((0.2, 0.3, -2.8), (0, 0, 0), (0, 1, 0), 203, 141, 55.0)
    gs = R.GESScene.from_arrays(scene)
    out = R.render_geom(gs, cam, opts)
    gs.close()
    ref = oracle.render(scene, cam, opts)
    _assert(compare_geom(out, oracle.render_geom(scene, cam, opts), ref))


def test_2d_splats_reaching_through_the_near_plane(R):
    """2D Gaussians whose centre is in front of the camera but whose extent
    reaches back through the near plane (the set-up's reference pixel at the
    far point, near-clipped bboxes; Sec. 6.4's ray-splat hit): the render
    and the geometry maps against the oracle."""
    import camera_discs as cd
    cam, base = cd.camera(), cd.flat(cd.background())
    ref0 = oracle.render(base, cam)
    for k, sp in enumerate(cd.splats()):
        sc = cd.with_splats(base, [sp], 40 + k)
        ref = oracle.render(sc, cam)
        assert (np.abs(ref["wg"] - ref0["wg"]) > 1e-3).sum() > 300     # the splat contributes
        _assert(compare(sc, cam, _render(R, sc, cam), ref, max_masked=0.1))
        gs = R.GESScene.from_arrays(sc)
        out = R.render_geom(gs, cam)
        gs.close()
        _assert(compare_geom(out, oracle.render_geom(sc, cam), ref))


def test_geometry_maps_1080p_orbit_camera(R):
    scene, cams = sg.config_scene(1)
    gs = R.GESScene.from_arrays(scene)
    out = R.render_geom(gs, cams[40])
    gs.close()
    ref = oracle.render(scene, cams[40])
    _assert(compare_geom(out, oracle.render_geom(scene, cams[40]), ref))


def test_2d_deterministic_and_order_independent_bitwise(R):
    scene, cams = sg.config_scene(0)
    sc = _flat(scene)
    gs = R.GESScene.from_arrays(sc)
    a, b = R.render_geom(gs, cams[0]), R.render_geom(gs, cams[0])
    gs.close()
    perm = np.random.default_rng(15).permutation(sc.n_gaussians)
    gp = R.GESScene.from_arrays(sc.subset(g_idx=perm))
    c = R.render_geom(gp, cams[0])
    gp.close()
    for k in a:
        assert (a[k] == b[k]).all() and (a[k] == c[k]).all(), k


def test_2d_batch_graph_equals_single_views(R):
    from paper_2504_17545_gb300 import native as N
    scene, cams = sg.config_scene(0)
    sa, sb = _flat(scene), _small2d(83, 2000, 6000)
    ga, gb = R.GESScene.from_arrays(sa), R.GESScene.from_arrays(sb)
    views = [cams[0], sg.look_at((0.5, 0, -2.8), (0, 0, 0), (0, 1, 0), 301, 173, 60.0)]
    b = R.GESBatch([ga, gb], views, [0, 1])
    b.launch()
    b.sync()
    for v, g in enumerate((ga, gb)):
        single = R.render(g, views[v])
        assert (b.rgb[v] == single["rgb"]).all() and (b.depth[v] == single["depth"]).all(), v
    b.close()
    g3 = R.GESScene.from_arrays(scene)
    with pytest.raises(N.GesError) as ei:
        R.GESBatch([ga, g3], views, [0, 1])
    assert ei.value.status == N.GES_ERR_UNSUPPORTED
    ga.close()
    gb.close()
    g3.close()
