"""ges_render_noalloc: the forward render for callers that cannot allocate
device memory (they manage a fixed budget themselves, or their render thread
must never block in cudaMalloc/cudaFree).  Its scratch is one fixed device
array shared by all calls, so this test renders two different scenes in a
row through the C ABI and checks each against ges_render_ex."""
import ctypes as C

import numpy as np
import pytest

import scenegen as sg

pytestmark = pytest.mark.gpu

COL_TOL = 2e-4   # the colour tolerance of the parity tests


@pytest.fixture(scope="module")
def R():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_17545_gb300 import render as R
    return R


def _noalloc(R, gs, cam):
    import torch
    from paper_2504_17545_gb300 import native as N
    c = R.camera_struct(cam)
    H, W = c.height, c.width
    out = dict(rgb=torch.empty((3, H, W), device="cuda"), depth=torch.empty((H, W), device="cuda"),
               id=torch.empty((H, W), device="cuda", dtype=torch.int32), aux=torch.empty((H, W), device="cuda"))
    lib = N.load()
    st = lib.ges_render_noalloc(C.byref(gs._desc), C.byref(c), None, C.c_void_p(out["rgb"].data_ptr()),
                                C.c_void_p(out["depth"].data_ptr()), C.c_void_p(out["id"].data_ptr()),
                                C.c_void_p(out["aux"].data_ptr()),
                                C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == N.GES_OK, N.ges_last_error_message()
    return out


def _same(a, b):
    assert (a["id"] == b["id"]).all()
    assert (a["depth"] == b["depth"]).all()
    assert float((a["rgb"] - b["rgb"]).abs().max()) <= COL_TOL
    assert float((a["aux"] - b["aux"]).abs().max()) <= COL_TOL


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
