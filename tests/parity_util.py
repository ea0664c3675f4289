"""Comparison rules of the GPU path against the FP64 oracle.

Tolerances (fixed by the specification of this path):
  * integer peak d*: identical, except where the oracle's own top-2 gap is
    below NEAR_TIE (then the two candidates are both valid maxima up to
    rounding; the frame is reported, not failed);
  * subpixel shift: |gpu - oracle| <= SHIFT_TOL px on every other frame;
  * corrected frames and summary images: ||gpu - oracle||_inf /
    ||oracle||_inf <= REL_TOL per image.
"""
import numpy as np

NEAR_TIE = 1e-6
SHIFT_TOL = 0.01
REL_TOL = 1e-4


def compare_shifts(gpu_shifts, gpu_info, ref):
    """Returns (near_tie_frames, max_shift_err over non-near-tie frames)."""
    gs = np.asarray(gpu_shifts, np.float64)
    gd = np.asarray(gpu_info, np.float64)[:, :2].astype(np.int64)
    rd = ref["dstar"].astype(np.int64)
    gap = ref["info"][:, 0] - ref["info"][:, 1]
    near = gap < NEAR_TIE
    same = np.all(gd == rd, axis=1)
    bad = (~same) & (~near)
    assert not bad.any(), f"integer peak differs on frames {np.nonzero(bad)[0][:10]}"
    ok = same & ~near
    err = np.abs(gs[ok] - ref["shifts"][ok]).max() if ok.any() else 0.0
    assert err <= SHIFT_TOL, f"subpixel shift differs by {err} px"
    return np.nonzero(near)[0], err


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def compare_images(gpu, ref, what, frames=None, tol=REL_TOL):
    """Per-image relative infinity-norm error, images along axis 0."""
    worst = 0.0
    idx = range(gpu.shape[0]) if frames is None else frames
    for i in idx:
        e = rel_err(gpu[i], ref[i])
        worst = max(worst, e)
        assert e <= tol, f"{what}[{i}] relative error {e:.3e} > {tol}"
    return worst
