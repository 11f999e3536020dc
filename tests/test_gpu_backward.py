"""GPU backward pass vs the oracle's analytic FP64 gradients (which are pinned
to central finite differences by the CPU tests)."""
import numpy as np
import pytest

import oracle
import scenegen as sg

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3   # of the largest |gradient| in each parameter group


@pytest.fixture(scope="module")
def R():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_17545_gb300 import render as R
    return R


def _grads_gpu(R, scene, cam, g, opts=None):
    import torch
    gs = R.GESScene.from_arrays(scene)
    fwd = R.render(gs, cam, opts)
    gr = R.render_backward(gs, cam, fwd, torch.as_tensor(g, dtype=torch.float32, device="cuda"), opts)
    out = {k: v.cpu().numpy().astype(np.float64) for k, v in gr.items()}
    gs.close()
    return out, fwd


def _check(gpu, ref, keys, scene=None, cam=None, opts=None):
    """Per parameter group, max |gpu - oracle| <= GRAD_TOL * max |oracle|,
    leaving out primitives that touch a pixel the oracle flags as ambiguous
    (several forward answers are correct there; see parity.py)."""
    s_keep = g_keep = None
    if scene is not None:
        amb = oracle.render(scene, cam, opts)["amb"] != 0
        st, gt = oracle.touching(scene, cam, amb, opts)
        s_keep, g_keep = ~st, ~gt
        assert g_keep.mean() > 0.75 and s_keep.mean() > 0.75
    for k in keys:
        keep = s_keep if k == "s_sh" else g_keep
        a, b = (gpu[k], ref[k]) if keep is None else (gpu[k][keep], ref[k][keep])
        scale = max(np.abs(b).max(), 1e-12)
        err = np.abs(a - b).max()
        assert err <= GRAD_TOL * scale, (k, err, scale)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_backward_crop_matches_oracle(R, mode):
    scene, cam = sg.crop_scene(7)
    g = np.random.default_rng(8).standard_normal((3, cam.height, cam.width))
    opts = dict(mode=mode)
    ref = oracle.backward(scene, cam, g, opts)
    gpu, _ = _grads_gpu(R, scene, cam, g, opts)
    keys = {0: ["g_pos", "g_rot", "g_scale", "g_opac", "g_sh", "s_sh"], 1: ["s_sh"],
            2: ["g_pos", "g_rot", "g_scale", "g_opac", "g_sh"]}[mode]
    assert (oracle.render(scene, cam, opts)["amb"] == 0).all()   # nothing ambiguous: compare everything
    _check(gpu, ref, keys)
    if mode == 1:
        assert np.all(gpu["g_pos"] == 0) and np.all(gpu["g_sh"] == 0)
    if mode == 2:
        assert np.all(gpu["s_sh"] == 0)


def test_backward_discs_at_and_behind_the_camera(R):
    """Gradients with the hand-placed discs at and behind the camera (their
    SH gradients come from the pixels they win; the Gaussians behind the
    walls fail the depth test) and with 2D-Gaussian splats reaching back
    through the near plane (Sec. 4.2; Sec. 6.4)."""
    import camera_discs as cd
    cam, base = cd.camera(), cd.background()
    g = np.random.default_rng(12).standard_normal((3, cam.height, cam.width))
    keys = ["g_pos", "g_rot", "g_scale", "g_opac", "g_sh", "s_sh"]
    scenes = [cd.with_discs(base, cd.walls(), 37), cd.with_discs(base, cd.tilted(), 38)]
    scenes += [cd.with_splats(cd.flat(base), [sp], 40 + k) for k, sp in enumerate(cd.splats())]
    for sc in scenes:
        ref = oracle.backward(sc, cam, g)
        gpu, _ = _grads_gpu(R, sc, cam, g)
        _check(gpu, ref, keys, sc, cam)
    # the walls' SH gradients are not trivially zero
    ref = oracle.backward(scenes[0], cam, g)
    assert np.abs(ref["s_sh"][base.n_surfels]).max() > 1.0


def test_backward_parity_workload(R):
    scene, cams = sg.config_scene(0)
    g = np.random.default_rng(11).standard_normal((3, 128, 128))
    ref = oracle.backward(scene, cams[0], g)
    gpu, _ = _grads_gpu(R, scene, cams[0], g)
    _check(gpu, ref, ["g_pos", "g_rot", "g_scale", "g_opac", "g_sh", "s_sh"], scene, cams[0])


def test_backward_train_step_workload(R):
    """1600x1060, 500k surfels + 500k Gaussians, L1 loss against the render of
    a perturbed scene (the training-step workload).  dL/dC = sign(C - T)/(3HW)
    is formed from the oracle's C and T and fed to both sides."""
    scene, cams = sg.config_scene(3)
    cam = cams[0]
    target = oracle.render(sg.perturbed_scene(scene, 1003), cam)["rgb"]
    C = oracle.render(scene, cam)["rgb"]
    g = np.sign(C - target) / (3.0 * cam.width * cam.height)
    ref = oracle.backward(scene, cam, g)
    gpu, _ = _grads_gpu(R, scene, cam, g)
    _check(gpu, ref, ["g_pos", "g_rot", "g_scale", "g_opac", "g_sh", "s_sh"], scene, cam)


def test_backward_deterministic(R):
    scene, cams = sg.config_scene(0)
    g = np.random.default_rng(12).standard_normal((3, 128, 128))
    a, _ = _grads_gpu(R, scene, cams[0], g)
    b, _ = _grads_gpu(R, scene, cams[0], g)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_autograd_function_matches_explicit_backward(R):
    import torch
    scene, cam = sg.crop_scene(13)
    gs = R.GESScene.from_arrays(scene)
    for k in ("g_pos", "g_rot", "g_scale", "g_opac", "g_sh", "s_sh"):
        gs.t[k].requires_grad_(True)
    rgb, depth, sid, aux = R.render_differentiable(gs, cam)
    w = torch.randn_like(rgb)
    (rgb * w).sum().backward()
    fwd = dict(rgb=rgb.detach(), depth=depth, id=sid, aux=aux)
    ref = R.render_backward(gs, cam, fwd, w)
    for k in ref:
        assert torch.equal(gs.t[k].grad, ref[k]), k
    gs.close()


# ------------------------------------------- 2D Gaussians (Sec. 6.4, Eq. 17-18)

def _flat(scene):
    sc = scene.subset()
    sc.g_scale = np.ascontiguousarray(sc.g_scale[:, :2])
    return sc


def _unambiguous_g(scene, cam, g, opts=None):
    """dL/dC with the pixels the oracle flags as ambiguous set to zero.  Every
    gradient is a sum of per-pixel terms, each proportional to dL/dC there, so
    both sides then sum exactly the pixels whose forward decisions they share,
    and every primitive can be compared."""
    amb = oracle.render(scene, cam, opts)["amb"] != 0
    g = np.array(g, dtype=np.float64)
    g[:, amb] = 0.0
    return g


@pytest.mark.parametrize("opts", [dict(mode=0), dict(mode=2), dict(mode=0, samples=4, lowpass=1.0),
                                  dict(mode=0, eps_mode=1)])
def test_2d_backward_crop_matches_oracle(R, opts):
    """Every gradient of the 2D-GES backward (ray-splat hit, object-space
    filter factors, SH view direction) against the oracle's FP64 chain, which
    the CPU tests pin to central differences."""
    scene, cam = sg.crop_scene(11)
    sc = _flat(scene)
    g = _unambiguous_g(sc, cam, np.random.default_rng(12).standard_normal((3, cam.height, cam.width)), opts)
    ref = oracle.backward(sc, cam, g, opts)
    gpu, _ = _grads_gpu(R, sc, cam, g, opts)
    assert gpu["g_scale"].shape == (sc.n_gaussians, 2)
    keys = ["g_pos", "g_rot", "g_scale", "g_opac", "g_sh"] + (["s_sh"] if opts.get("mode", 0) == 0 else [])
    _check(gpu, ref, keys)


def test_2d_backward_parity_workload(R):
    """The 128x128 parity workload with its Gaussians flattened to splats
    (1k surfels, 4k 2D Gaussians)."""
    scene, cams = sg.config_scene(0)
    sc = _flat(scene)
    g = _unambiguous_g(sc, cams[0], np.random.default_rng(21).standard_normal((3, 128, 128)))
    ref = oracle.backward(sc, cams[0], g)
    gpu, _ = _grads_gpu(R, sc, cams[0], g)
    _check(gpu, ref, ["g_pos", "g_rot", "g_scale", "g_opac", "g_sh", "s_sh"])


def test_2d_backward_ragged_view_inside_scene(R):
    """A ragged 203x141 view and a camera inside the scene (near, grazing and
    partly clipped splats), Gaussians-only and full modes."""
    sc = _flat(sg.random_scene(81, 400, 1500, n_objects=5, box=1.0, sphere_r=(0.3, 0.6), plane_side=(0.6, 1.2),
                               surfel_scale=(0.03, 0.1), gauss_logscale=(-3.2, 0.4)))
    for cam, seed in ((sg.look_at((0.2, 0.3, -2.8), (0, 0, 0), (0, 1, 0), 203, 141, 55.0), 3),
                      (sg.look_at((0.1, 0.05, -0.6), (0, 0.1, 1), (0, 1, 0), 97, 61, 95.0), 4)):
        g = _unambiguous_g(sc, cam, np.random.default_rng(seed).standard_normal((3, cam.height, cam.width)))
        ref = oracle.backward(sc, cam, g)
        gpu, _ = _grads_gpu(R, sc, cam, g)
        _check(gpu, ref, ["g_pos", "g_rot", "g_scale", "g_opac", "g_sh", "s_sh"])


def test_2d_backward_train_step_workload(R):
    """The 1600x1060 training-step workload (500k surfels, 500k Gaussians)
    with 2D Gaussians: L1 loss against the render of a perturbed scene."""
    scene, cams = sg.config_scene(3)
    sc, cam = _flat(scene), cams[0]
    target = oracle.render(sg.perturbed_scene(sc, 1003), cam)["rgb"]
    C = oracle.render(sc, cam)["rgb"]
    g = _unambiguous_g(sc, cam, np.sign(C - target) / (3.0 * cam.width * cam.height))
    ref = oracle.backward(sc, cam, g)
    gpu, _ = _grads_gpu(R, sc, cam, g)
    _check(gpu, ref, ["g_pos", "g_rot", "g_scale", "g_opac", "g_sh", "s_sh"])


def test_2d_backward_deterministic_and_autograd(R):
    import torch
    scene, cam = sg.crop_scene(13)
    sc = _flat(scene)
    g = np.random.default_rng(5).standard_normal((3, cam.height, cam.width))
    a, _ = _grads_gpu(R, sc, cam, g)
    b, _ = _grads_gpu(R, sc, cam, g)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    gs = R.GESScene.from_arrays(sc)
    for k in ("g_pos", "g_rot", "g_scale", "g_opac", "g_sh", "s_sh"):
        gs.t[k].requires_grad_(True)
    rgb, depth, sid, aux = R.render_differentiable(gs, cam)
    w = torch.as_tensor(g, dtype=torch.float32, device="cuda")
    (rgb * w).sum().backward()
    assert gs.t["g_scale"].grad.shape == (sc.n_gaussians, 2)
    assert torch.equal(gs.t["g_scale"].grad.cpu(), torch.as_tensor(a["g_scale"], dtype=torch.float32))
    gs.close()
