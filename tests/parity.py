"""Comparison of a GPU render with the FP64 oracle (test infrastructure).

Surfel ids must match bit-for-bit wherever the oracle did not flag the pixel
as ambiguous (competing depths within 1e-6 relative, a disc rim within 1e-5
relative of r^2, a near-plane or grazing fragment; with 4 samples, at any
sample of the pixel); at flagged pixels the GPU's
id must still be an acceptable answer (``oracle.id_validity``).  Depth must
match to ``depth_rel`` where the ids match; colour to ``col_tol`` max abs per
channel where the ids match and no Gaussian sits on the 1/255 clamp or the
depth-test threshold.
"""
import numpy as np

import oracle

COL_TOL = 2e-4       # spec colour tolerance for FP32 work
# GPU depth = 1/(iz0 + gu du + gv dv): iz0 carries the rounding of the
# double-float centre and of its reciprocal (~3u), the affine step ~2u, the
# final reciprocal 1u, and 16-bit quaternions renormalised in float32 a few u
# more; over millions of pixels the worst case reaches ~20u (u = 2^-24).
DEPTH_REL = 2e-6


def compare(scene, cam, gpu, ref, opts=None, col_tol=COL_TOL, depth_rel=DEPTH_REL, check_ids=True):
    rgb = gpu["rgb"].detach().cpu().numpy().astype(np.float64)
    depth = gpu["depth"].detach().cpu().numpy().astype(np.float64)
    out = {}
    amb_id = (ref["amb"] & 1) != 0
    amb_col = (ref["amb"] & 2) != 0
    if "id" in gpu and check_ids:
        ids = gpu["id"].detach().cpu().numpy()
        mism = ids != ref["id"]
        out["id_mismatch_unmasked"] = int((mism & ~amb_id).sum())
        valid = oracle.id_validity(scene, cam, ref, ids, opts)
        out["id_invalid"] = int((~valid).sum())
        same = ~mism if mism.ndim == 2 else ~mism.any(0)   # [samples,H,W]: every sample agrees
    else:
        same = np.ones(depth.shape, bool)
    hit = ref["id"] >= 0
    if hit.ndim == 3:
        hit = hit.any(0)
    cov = same & hit & ~amb_id     # grazing/rim/tie pixels: depth is ill-conditioned
    if cov.any():
        rel = np.abs(depth[cov] - ref["depth"][cov]) / ref["depth"][cov]
        out["depth_rel_max"] = float(rel.max())
    else:
        out["depth_rel_max"] = 0.0
    out["depth_inf_ok"] = bool(np.all(np.isinf(depth[same & ~hit])))
    ok = same & ~amb_col & ~amb_id
    err = np.abs(rgb - ref["rgb"])[:, ok]
    out["col_max"] = float(err.max()) if err.size else 0.0
    out["masked_frac"] = float((amb_id | amb_col).mean())
    out["compared_px"] = int(ok.sum())
    out["pass"] = (out.get("id_mismatch_unmasked", 0) == 0 and out.get("id_invalid", 0) == 0 and
                   out["depth_rel_max"] <= depth_rel and out["depth_inf_ok"] and out["col_max"] <= col_tol)
    return out
