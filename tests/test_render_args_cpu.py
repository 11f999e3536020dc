"""The torch layer checks every caller-supplied tensor (device, dtype, element
count, layout) before it hands a pointer to the C ABI, so a wrong tensor is a
ValueError on the host and never reaches a kernel.  Runs on the CPU: the scene
is a stand-in whose tensors live on the CPU, and the ABI calls are stubs that
record whether they were reached."""
import pytest

torch = pytest.importorskip("torch")

from paper_2504_17545_gb300 import native as N
from paper_2504_17545_gb300 import render as R

H, W, NS, NG, K = 6, 5, 7, 4, 16
CAM = dict(width=W, height=H, fx=5.0, fy=5.0, cx=2.5, cy=3.0,
           world_to_cam=[[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]], znear=0.01, bg=(0, 0, 0))


class _Scene:
    def __init__(self):
        self.t = {"s_pos": torch.zeros(NS, 3), "g_pos": torch.zeros(NG, 3), "s_sh": torch.zeros(NS, K, 3),
                  "g_sh": torch.zeros(NG, K, 3)}
        self.n_surfels, self.n_gaussians, self.sh_degree, self.gauss_dim, self.handle = NS, NG, 3, 3, None

    def bind_stream(self):
        pass


@pytest.fixture
def calls(monkeypatch):
    got = []
    for name in ("ges_render_backward", "ges_render_translucent", "ges_render_translucent_backward",
                 "ges_contribution_scores", "ges_render_batch", "ges_batch_set_id_output"):
        monkeypatch.setattr(N, name, lambda *a, _n=name: got.append(_n))
    return got


def _fwd():
    return dict(rgb=torch.zeros(3, H, W), depth=torch.zeros(H, W), id=torch.zeros(H, W, dtype=torch.int32),
                aux=torch.zeros(H, W), T=torch.zeros(H, W), front=torch.zeros(H, W, dtype=torch.int32),
                last=torch.zeros(H, W, dtype=torch.int32), Tlast=torch.zeros(H, W))


def test_backward_checks_its_inputs(calls):
    sc = _Scene()
    R.render_backward(sc, CAM, _fwd(), torch.zeros(3, H, W))
    assert calls == ["ges_render_backward"]
    bad = [("id", torch.zeros(H, W, dtype=torch.int64)), ("id", torch.zeros(H, W - 1, dtype=torch.int32)),
           ("aux", torch.zeros(H, W, dtype=torch.float64)), ("depth", torch.zeros(W, H).t()),
           ("rgb", torch.zeros(3, H, W, device="meta"))]
    for k, t in bad:
        f = _fwd()
        f[k] = t
        with pytest.raises(ValueError, match=k):
            R.render_backward(sc, CAM, f, torch.zeros(3, H, W))
    with pytest.raises(ValueError, match="dL_drgb"):
        R.render_backward(sc, CAM, _fwd(), torch.zeros(3, H, W + 1))
    with pytest.raises(ValueError, match="id"):           # four samples need [4,H,W] ids
        R.render_backward(sc, CAM, _fwd(), torch.zeros(3, H, W), dict(samples=4))
    assert calls == ["ges_render_backward"]


def test_translucent_calls_check_w_and_the_forward_maps(calls):
    sc = _Scene()
    R.render_translucent(sc, CAM, torch.ones(NS))
    R.render_translucent_backward(sc, CAM, torch.ones(NS), _fwd(), torch.zeros(3, H, W))
    assert calls == ["ges_render_translucent", "ges_render_translucent_backward"]
    with pytest.raises(ValueError, match="w"):
        R.render_translucent(sc, CAM, torch.ones(NS - 1))
    f = _fwd()
    f["front"] = torch.zeros(H, W)                          # float, not int32
    with pytest.raises(ValueError, match="front"):
        R.render_translucent_backward(sc, CAM, torch.ones(NS), f, torch.zeros(3, H, W))
    assert len(calls) == 2


def test_contribution_scores_and_render_batch_check_their_buffers(calls):
    sc = _Scene()
    R.contribution_scores(sc, CAM, _fwd())
    R.render_batch([sc], [CAM, CAM], outputs=[(torch.zeros(3, H, W), torch.zeros(H, W)),
                                              (torch.zeros(3, H, W), None)])
    assert calls == ["ges_contribution_scores", "ges_render_batch"]
    f = _fwd()
    f["aux"] = torch.zeros(H * W + 1)
    with pytest.raises(ValueError, match="aux"):
        R.contribution_scores(sc, CAM, f)
    with pytest.raises(ValueError, match="outputs"):
        R.render_batch([sc], [CAM, CAM], outputs=[(torch.zeros(3, H, W), torch.zeros(H, W))])
    with pytest.raises(ValueError, match=r"outputs\[1\]\[0\]"):
        R.render_batch([sc], [CAM, CAM], outputs=[(torch.zeros(3, H, W), None), (torch.zeros(3, W, H + 1), None)])
    assert len(calls) == 2


def test_batch_id_outputs_are_checked(calls):
    b = object.__new__(R.GESBatch)
    b.handle, b._sizes, b._samples, b.rgb = None, [(H, W), (H + 1, W)], 1, [torch.zeros(3, H, W)]
    b.set_id_output(1, torch.zeros(H + 1, W, dtype=torch.int32), torch.zeros(H + 1, W))
    b.set_id_output(0, None)
    assert calls == ["ges_batch_set_id_output"] * 2
    with pytest.raises(ValueError, match="out_id"):
        b.set_id_output(0, torch.zeros(H + 1, W, dtype=torch.int32))
    with pytest.raises(ValueError, match="aux"):
        b.set_id_output(0, None, torch.zeros(H, W, dtype=torch.float16))
    with pytest.raises(ValueError, match="out of range"):
        b.set_id_output(2, None)
    assert len(calls) == 2


def _scene_tensors(n=NS, m=NG, deg=3, gdim=3):
    k = (deg + 1) ** 2
    z = torch.zeros
    return dict(s_pos=z(n, 3), s_rot=z(n, 4), s_scale=z(n, 2), s_sh=z(n, k, 3), g_pos=z(m, 3), g_rot=z(m, 4),
                g_scale=z(m, gdim), g_opac=z(m), g_sh=z(m, k, 3))


def test_scene_layout_is_checked_against_the_abi():
    assert R._scene_layout(_scene_tensors(), 3) == 3
    assert R._scene_layout(_scene_tensors(gdim=2), 3) == 2
    assert R._scene_layout(_scene_tensors(n=0, m=0, deg=0), 0) == 3
    bad = [("s_sh", torch.zeros(NS, 9, 3)), ("s_rot", torch.zeros(NS - 1, 4)), ("g_opac", torch.zeros(NG, 1)),
           ("g_scale", torch.zeros(NG, 4)), ("g_pos", torch.zeros(NG, 4)), ("g_sh", torch.zeros(NG + 1, K, 3))]
    for k, v in bad:
        t = _scene_tensors()
        t[k] = v
        with pytest.raises(ValueError, match=k):
            R._scene_layout(t, 3)
    t = _scene_tensors()
    t["g_opac"] = torch.zeros(NG, dtype=torch.float16)
    with pytest.raises(TypeError, match="one dtype"):
        R._scene_layout(t, 3)
    t = _scene_tensors()
    t["g_pos"] = torch.zeros(NG, 3, dtype=torch.float16)
    with pytest.raises(TypeError, match="float32"):
        R._scene_layout(t, 3)
    t = _scene_tensors()
    t["g_sh"] = torch.zeros(NG, K, 3, device="meta")
    with pytest.raises(ValueError, match="g_sh"):
        R._scene_layout(t, 3)
    with pytest.raises(ValueError, match="sh_degree"):
        R._scene_layout(_scene_tensors(), 4)
