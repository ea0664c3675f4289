"""FP64 CPU oracle of the footprint reconstruction of Sec. III-D (Bando et al.,
BIBM 2023): per-segment probability maps p_i(x) -> binary masks -> cleanup by
shape -> OR over segments -> connected components -> NMF (Eq. 3, P ~ F A) on
each component.

TEST INFRASTRUCTURE ONLY (tests and the benchmark's CPU legs); the product
never imports it.  Plain numpy / scipy in double precision.

The paper gives the steps but not their constants; readings taken here:
  * b_i(x) = p_i(x) > 0.5;
  * components are 8-connected; a per-segment component is kept if
    area in [20, 1000] pixels, eccentricity <= 0.95 and concaveness <= 0.3,
    with eccentricity sqrt(1 - l2 / l1) of the pixel centres' population
    covariance (eigenvalues l1 >= l2; 0 when l1 = 0, a single pixel) and
    concaveness 1 - area / (area of the convex hull of the pixel squares);
  * b(x) = OR_i of the kept masks; its 8-connected components are the regions;
  * the kept per-segment components inside a region ("blobs", in segment
    order, then by smallest pixel index) are clustered greedily: a blob joins
    the first cluster whose first blob it overlaps with IoU >= 1/2 (the exact
    integer test 2 |a & b| >= |a | b|), else it starts a new cluster; N = the
    number of clusters (neurons that spike in different segments separate
    even where their footprints touch).  F column j starts as the indicator of
    the union of cluster j's blobs, A[j][i] as the mean of p_i over that
    union, floored at 1e-6;
  * every region is factorised, whatever its size and its N (the paper sets
    no limit; a GPU implementation may have capacity limits of its own, which
    it must report rather than change the answer);
  * NMF by Lee & Seung's multiplicative updates for the Frobenius loss,
    100 iterations of A <- A * (F'P) / (F'F A + 1e-9), then
    F <- F * (P A') / (F A A' + 1e-9), over the region's pixels (rows of P,
    in raster order) and all K segments (columns).

Parity: components pinned to scipy.ndimage.label, hull areas to
scipy.spatial.ConvexHull, moments to closed forms on ellipses and rectangles,
the NMF to its fixed points and to monotone loss decrease (tests/test_oracle_segmentation.py).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import ndimage

THRESHOLD = 0.5
AREA_MIN, AREA_MAX = 20, 1000
ECC_MAX = 0.95
CONCAVE_MAX = 0.3
NMF_ITERS = 100
NMF_EPS = 1e-9
A_FLOOR = 1e-6
EIGHT = np.ones((3, 3), bool)


def components(mask):
    """8-connected components: list of pixel index arrays (raster order),
    ordered by their smallest pixel index."""
    lab, n = ndimage.label(np.asarray(mask, bool), structure=EIGHT)
    flat = lab.ravel()
    comps = [np.nonzero(flat == k)[0] for k in range(1, n + 1)]
    comps.sort(key=lambda c: c[0])
    return comps


def moments(idx, W):
    """(area, cov_yy, cov_xx, cov_xy) of the pixel centres of a component, from
    exact integer sums: cov_uv = S_uv / n - (S_u / n)(S_v / n) in FP64."""
    y, x = np.divmod(np.asarray(idx, np.int64), W)
    n = int(y.size)
    sy, sx = int(y.sum()), int(x.sum())
    syy, sxx, sxy = int((y * y).sum()), int((x * x).sum()), int((y * x).sum())
    my, mx = sy / n, sx / n
    return n, syy / n - my * my, sxx / n - mx * mx, sxy / n - my * mx


def eccentricity(cyy, cxx, cxy):
    """sqrt(1 - l2 / l1) of the 2x2 covariance; 0 for a single pixel (l1 = 0)."""
    tr, det = cyy + cxx, cyy * cxx - cxy * cxy
    disc = math.sqrt(max(tr * tr / 4 - det, 0.0))
    l1, l2 = tr / 2 + disc, tr / 2 - disc
    if l1 <= 0:
        return 0.0
    return math.sqrt(max(0.0, 1.0 - max(l2, 0.0) / l1))


def hull_area(idx, W):
    """Area of the convex hull of the union of the pixel squares [x, x+1] x
    [y, y+1]: the hull of the squares' corners, by Andrew's monotone chain on
    each row's extreme corners, and the shoelace formula."""
    y, x = np.divmod(np.asarray(idx), W)
    pts = set()
    for r in np.unique(y):
        xs = x[y == r]
        lo, hi = int(xs.min()), int(xs.max()) + 1
        for px in (lo, hi):
            pts.add((px, int(r)))
            pts.add((px, int(r) + 1))
    P = sorted(pts)

    def cross(o, a, b):
        return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0])

    lower, upper = [], []
    for p in P:
        while len(lower) >= 2 and cross(lower[-2], lower[-1], p) <= 0:
            lower.pop()
        lower.append(p)
    for p in reversed(P):
        while len(upper) >= 2 and cross(upper[-2], upper[-1], p) <= 0:
            upper.pop()
        upper.append(p)
    hull = lower[:-1] + upper[:-1]
    s = 0
    for i in range(len(hull)):
        x0, y0 = hull[i]
        x1, y1 = hull[(i + 1) % len(hull)]
        s += x0 * y1 - x1 * y0
    return abs(s) / 2.0


def keep(idx, W):
    """The shape test of a per-segment component."""
    n, cyy, cxx, cxy = moments(idx, W)
    if n < AREA_MIN or n > AREA_MAX:
        return False
    if eccentricity(cyy, cxx, cxy) > ECC_MAX:
        return False
    return 1.0 - n / hull_area(idx, W) <= CONCAVE_MAX


def cleaned_masks(prob):
    """prob [K][H][W] -> kept per-segment components: list (per segment) of index arrays."""
    prob = np.asarray(prob, np.float64)
    K, H, W = prob.shape
    return [[c for c in components(prob[i] > THRESHOLD) if keep(c, W)] for i in range(K)]


def nmf(P, F, A, iters=NMF_ITERS):
    """Multiplicative updates (Frobenius loss): A first, then F, per iteration."""
    P, F, A = (np.asarray(v, np.float64).copy() for v in (P, F, A))
    for _ in range(iters):
        A *= (F.T @ P) / (F.T @ F @ A + NMF_EPS)
        F *= (P @ A.T) / (F @ (A @ A.T) + NMF_EPS)
    return F, A


def regions(prob):
    """prob [K][H][W] -> list of regions (by smallest pixel index): dict(pixels =
    raster indices of the region, blobs = kept per-segment components inside,
    unions = per cluster the union of its blobs' pixels, N = number of clusters).
    The structure of the factorisation, without the NMF itself."""
    prob = np.asarray(prob, np.float64)
    K, H, W = prob.shape
    kept = cleaned_masks(prob)
    b = np.zeros(H * W, bool)
    for segs in kept:
        for c in segs:
            b[c] = True
    out = []
    for region in components(b.reshape(H, W)):
        rset = set(region.tolist())
        blobs = [set(c.tolist()) for i in range(K) for c in kept[i] if int(c[0]) in rset]
        reps, unions = [], []
        for bl in blobs:
            for j, rep in enumerate(reps):
                if 2 * len(bl & rep) >= len(bl | rep):
                    unions[j] |= bl
                    break
            else:
                reps.append(bl)
                unions.append(set(bl))
        out.append(dict(pixels=region, blobs=len(blobs), unions=unions, N=len(reps)))
    return out


def factorise(prob, region):
    """NMF of one region (a dict of regions()): returns (F [M][N], A [N][K])."""
    prob = np.asarray(prob, np.float64)
    K, H, W = prob.shape
    pix = region["pixels"]
    N = region["N"]
    pos = {p: r for r, p in enumerate(pix)}
    P = prob.reshape(K, H * W)[:, pix].T  # [M][K]
    F0 = np.zeros((pix.size, N))
    A0 = np.zeros((N, K))
    for j, un in enumerate(region["unions"]):
        idx = np.array(sorted(un))
        F0[[pos[p] for p in idx], j] = 1.0
        A0[j] = np.maximum(prob.reshape(K, H * W)[:, idx].mean(axis=1), A_FLOOR)
    return nmf(P, F0, A0)


def footprints(prob):
    """prob [K][H][W] -> list of regions (by smallest pixel index): dict(pixels =
    raster indices of the region, N, F [M][N], A [N][K], blobs = kept
    per-segment components inside)."""
    out = []
    for r in regions(prob):
        F, A = factorise(prob, r)
        out.append(dict(pixels=r["pixels"], N=r["N"], F=F, A=A, blobs=r["blobs"]))
    return out
