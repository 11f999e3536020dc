"""The C ABI without a GPU: the library loads, exports every symbol the header
declares, and rejects bad arguments before touching the device."""
import math
import os
import re

import pytest

from paper_2504_17545_gb300 import native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    hdr = open(os.path.join(ROOT, "include", "ges.h")).read()
    return re.findall(r"GES_API\s+[\w\s\*]+?\b(ges_\w+)\s*\(", hdr)


def test_library_exports_every_declared_symbol():
    lib = N.load()
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(N._SIGS), "binding and header disagree"


def test_default_opts_are_the_papers():
    o = N.ges_default_opts()
    assert o.eps_mode == N.GES_EPS_ADAPTIVE and o.eps_factor == 5.0          # Sec. 5
    assert o.alpha_min == pytest.approx(1 / 255, rel=1e-7)                  # Sec. 3, after Eq. 4
    assert o.surfel_r2 == pytest.approx(2 * math.log(255), rel=1e-7)       # Sec. 4.1
    assert o.lowpass == pytest.approx(0.3) and o.mode == N.GES_MODE_FULL
    assert N.ges_version() == 1


def _desc(**kw):
    d = N.ges_scene_desc()
    d.n_surfels, d.n_gaussians, d.sh_degree = 0, 0, 3
    for k, v in kw.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("kw,msg", [
    (dict(n_surfels=-1), "negative"),
    (dict(sh_degree=4), "sh_degree"),
    (dict(attr_dtype=7), "dtype"),
    (dict(n_surfels=5), "surfel attribute pointer"),
    (dict(n_gaussians=5), "Gaussian attribute pointer"),
])
def test_bad_scene_descriptions(kw, msg):
    with pytest.raises(N.GesError) as ei:
        N.ges_create_scene(_desc(**kw))
    assert ei.value.status == N.GES_ERR_INVALID_ARG
    assert msg in str(ei.value)


def test_null_handles():
    lib = N.load()
    assert lib.ges_create_scene(None, None) == N.GES_ERR_INVALID_ARG
    assert lib.ges_destroy_scene(None) == N.GES_OK
    assert lib.ges_render(None, None, None, None) == N.GES_ERR_INVALID_ARG
    assert "scene is NULL" in N.ges_last_error_message()
    assert lib.ges_get_stats(None, None) == N.GES_ERR_INVALID_ARG
    assert lib.ges_render_batch(None, None, None, 0, None, None, None) == N.GES_ERR_INVALID_ARG
    assert lib.ges_default_opts(None) == N.GES_ERR_INVALID_ARG
    assert lib.ges_batch_set_camera(None, 0, None) == N.GES_ERR_INVALID_ARG
    assert lib.ges_batch_set_id_output(None, 0, None, None) == N.GES_ERR_INVALID_ARG
    assert "batch is NULL" in N.ges_last_error_message()
    assert lib.ges_batch_launch(None, None) == N.GES_ERR_INVALID_ARG


def test_without_a_device_creation_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(N.GesError) as ei:
        N.ges_create_scene(_desc())
    assert ei.value.status in (N.GES_ERR_CUDA, N.GES_ERR_UNSUPPORTED)
