"""FP64 CPU oracle of the whole-video summary images that VolPy feeds to its
Mask R-CNN, which Bando et al. (BIBM 2023, Sec. III-A and Fig. 2) compare with
their per-segment summaries: the temporal average image and the temporal
(local) correlation image of the motion-corrected video V(x, t).

TEST INFRASTRUCTURE ONLY (tests and the benchmark's CPU legs); the product
never imports it.  Plain numpy in double precision.

Readings (the paper names the two images without defining them):
  * average:     A(x) = (1/n) sum_t V(x, t) over every frame of the video;
  * correlation: C(x) = mean over the in-image 8-neighbours y of x of the
    Pearson correlation over time of V(x, .) and V(y, .); a pair in which
    either trace has zero variance correlates 0; border pixels average over
    their 3 or 5 neighbours.

Parity: pinned to numpy's corrcoef pair by pair (brute force), to closed forms
(identical traces -> 1, anti-correlated -> -1, per-pixel affine maps leave C
unchanged, a constant pixel -> 0), and to the mean (tests/test_oracle_video_summary.py).
"""
from __future__ import annotations

import numpy as np

# the 8 neighbour offsets (dy, dx)
NEIGHBOURS = [(-1, -1), (-1, 0), (-1, 1), (0, -1), (0, 1), (1, -1), (1, 0), (1, 1)]


def average_image(V):
    """V [n][H][W] -> A [H][W]."""
    return np.asarray(V, np.float64).mean(axis=0)


def pair_correlation(a, b):
    """Pearson correlation of two traces over time; 0 if either is constant."""
    a = np.asarray(a, np.float64) - np.mean(a)
    b = np.asarray(b, np.float64) - np.mean(b)
    den = np.sqrt((a * a).sum() * (b * b).sum())
    return float((a * b).sum() / den) if den > 0 else 0.0


def correlation_image(V):
    """V [n][H][W] -> C [H][W] (see the module's readings)."""
    V = np.asarray(V, np.float64)
    n, H, W = V.shape
    Z = V - V.mean(axis=0)
    norm = np.sqrt((Z * Z).sum(axis=0))
    Z = np.divide(Z, norm, out=np.zeros_like(Z), where=norm > 0)  # unit traces, 0 if constant
    total = np.zeros((H, W))
    count = np.zeros((H, W))
    for dy, dx in NEIGHBOURS:
        ys, ye = max(0, -dy), min(H, H - dy)   # pixels whose neighbour (y+dy, x+dx) exists
        xs, xe = max(0, -dx), min(W, W - dx)
        prod = (Z[:, ys:ye, xs:xe] * Z[:, ys + dy:ye + dy, xs + dx:xe + dx]).sum(axis=0)
        total[ys:ye, xs:xe] += prod
        count[ys:ye, xs:xe] += 1
    return total / count
