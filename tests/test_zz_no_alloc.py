"""ges_render_noalloc: the forward render for callers that cannot allocate
device memory (they manage a fixed budget themselves, or their render thread
must never block in cudaMalloc/cudaFree).  Its scratch is one fixed device
array shared by all calls, so these tests render different scenes in a row
through the C ABI and check each against ges_render_ex.  Both paths sum the
Gaussians in exact fixed point and take an order-independent z-buffer
minimum, so every output must match bit for bit although the two bin their
tiles differently."""
import ctypes as C

import numpy as np
import pytest

import scenegen as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_17545_gb300 import render as R
    return R


def _call(R, gs, cam, opts=None, with_outputs=True):
    import torch
    from paper_2504_17545_gb300 import native as N
    c = R.camera_struct(cam)
    o = R.opts_struct(opts)
    H, W = c.height, c.width
    out = dict(rgb=torch.empty((3, H, W), device="cuda"), depth=torch.empty((H, W), device="cuda"),
               id=torch.empty((H, W) if o.samples == 1 else (o.samples, H, W), device="cuda", dtype=torch.int32),
               aux=torch.empty((H, W), device="cuda"))
    lib = N.load()
    st = lib.ges_render_noalloc(C.byref(gs._desc), C.byref(c), C.byref(o), C.c_void_p(out["rgb"].data_ptr()),
                                C.c_void_p(out["depth"].data_ptr()), C.c_void_p(out["id"].data_ptr()),
                                C.c_void_p(out["aux"].data_ptr()),
                                C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, out


def _noalloc(R, gs, cam, opts=None):
    from paper_2504_17545_gb300 import native as N
    st, out = _call(R, gs, cam, opts)
    assert st == N.GES_OK, N.ges_last_error_message()
    return out


def _same(a, b):
    for k in ("id", "depth", "rgb", "aux"):
        assert bool((a[k] == b[k]).all()), k


def test_noalloc_matches_render_ex_on_two_calls_in_a_row(R):
    scene_a, cams_a = sg.config_scene(0)
    scene_b = sg.random_scene(41, 3000, 9000, n_objects=6, box=1.0, sphere_r=(0.3, 0.6), plane_side=(0.6, 1.2),
                              surfel_scale=(0.02, 0.08), gauss_logscale=(-3.8, 0.4))
    cam_b = sg.look_at((0.3, 0.2, -2.6), (0, 0, 0), (0, 1, 0), 203, 141, 55.0)
    ga, gb = R.GESScene.from_arrays(scene_a), R.GESScene.from_arrays(scene_b)
    first = _noalloc(R, ga, cams_a[0])
    second = _noalloc(R, gb, cam_b)        # different sizes: stale scratch would show here
    _same(first, R.render(ga, cams_a[0]))
    _same(second, R.render(gb, cam_b))
    third = _noalloc(R, ga, cams_a[0])     # and back again
    _same(third, first)
    ga.close()
    gb.close()


def test_noalloc_four_samples_and_mip_filters(R):
    """4x multisampling (one id plane per sample) and the Mip-GES filters
    (3D filter variance in the scene, screen filter in the options) through
    the allocation-free path, each against ges_render_ex."""
    scene, cams = sg.config_scene(0)
    gs = R.GESScene.from_arrays(scene)
    ms = dict(samples=4)
    _same(_noalloc(R, gs, cams[0], ms), R.render(gs, cams[0], ms))
    gs.update(g_filter3d=gs.compute_filter3d(cams, 0.2))
    mip = dict(filter=1, lowpass=0.1)
    _same(_noalloc(R, gs, cams[0], mip), R.render(gs, cams[0], mip))
    gs.close()


def test_noalloc_rejects_inputs_beyond_its_fixed_limits(R):
    import torch
    from paper_2504_17545_gb300 import native as N
    scene, cams = sg.config_scene(0)
    gs = R.GESScene.from_arrays(scene)
    lib = N.load()
    big = sg.look_at((0, 0, -3), (0, 0, 0), (0, 1, 0), 4096, 4096, 60.0)   # 65536 tiles > 16384
    out = torch.empty((3, 16, 16), device="cuda")
    st = lib.ges_render_noalloc(C.byref(gs._desc), C.byref(R.camera_struct(big)), None,
                                C.c_void_p(out.data_ptr()), None, None, None, None)
    assert st == N.GES_ERR_CAPACITY and "tiles" in N.ges_last_error_message()
    d = N.ges_scene_desc.from_buffer_copy(gs._desc)
    d.n_surfels = 70000
    st = lib.ges_render_noalloc(C.byref(d), C.byref(R.camera_struct(cams[0])), None,
                                C.c_void_p(out.data_ptr()), None, None, None, None)
    assert st == N.GES_ERR_CAPACITY and "surfels" in N.ges_last_error_message()
    gs.close()


def test_noalloc_reports_tile_entry_overflow_and_recovers(R):
    """A dense scene within the primitive limits whose tile entries exceed the
    fixed lists (device-side overflow flag -> GES_ERR_CAPACITY, no raster),
    then a normal call on the same array succeeds."""
    from paper_2504_17545_gb300 import native as N
    n = 1200
    rng = np.random.default_rng(7)
    K = 16
    s_pos = np.zeros((n, 3), np.float32)
    s_pos[:, :2] = rng.uniform(-0.05, 0.05, (n, 2))
    s_pos[:, 2] = rng.uniform(0.0, 0.5, n)
    s_rot = np.tile(np.array([1.0, 0.0, 0.0, 0.0], np.float32), (n, 1))
    s_scale = np.full((n, 2), 0.5, np.float32)              # each disc covers the whole 1024^2 view
    s_sh = np.zeros((n, K, 3), np.float32)
    z = np.zeros
    dense = sg.Scene(3, s_pos, s_rot, s_scale, s_sh, z((0, 3), np.float32), z((0, 4), np.float32),
                     z((0, 3), np.float32), z((0,), np.float32), z((0, K, 3), np.float32))
    cam = sg.look_at((0, 0, -3), (0, 0, 0), (0, 1, 0), 1024, 1024, 60.0)   # 4096 tiles x 1200 discs > 2^20
    gd = R.GESScene.from_arrays(dense)
    st, _ = _call(R, gd, cam)
    assert st == N.GES_ERR_CAPACITY and "tile entries" in N.ges_last_error_message()
    gd.close()
    scene, cams = sg.config_scene(0)
    gs = R.GESScene.from_arrays(scene)
    _same(_noalloc(R, gs, cams[0]), R.render(gs, cams[0]))
    gs.close()
