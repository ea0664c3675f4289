"""Pins of the footprint-reconstruction oracle (Sec. III-D: threshold, shape
cleanup, OR over segments, connected components, NMF of Eq. 3)."""
import math

import numpy as np
from scipy import ndimage
from scipy.spatial import ConvexHull

import oracle.segmentation as SG

rng = np.random.default_rng(5)


def _flood(mask):
    """Brute-force 8-connected components by breadth-first search."""
    H, W = mask.shape
    seen = np.zeros_like(mask, bool)
    comps = []
    for y in range(H):
        for x in range(W):
            if mask[y, x] and not seen[y, x]:
                q, comp = [(y, x)], []
                seen[y, x] = True
                while q:
                    cy, cx = q.pop()
                    comp.append(cy * W + cx)
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            ny, nx = cy + dy, cx + dx
                            if 0 <= ny < H and 0 <= nx < W and mask[ny, nx] and not seen[ny, nx]:
                                seen[ny, nx] = True
                                q.append((ny, nx))
                comps.append(sorted(comp))
    return sorted(comps, key=lambda c: c[0])


def test_components_are_the_flood_fill_partition():
    for _ in range(5):
        m = rng.random((17, 23)) < 0.35
        got = [list(c) for c in SG.components(m)]
        assert got == _flood(m)


def _rect(y0, x0, h, w, W):
    return np.array([(y0 + i) * W + x0 + j for i in range(h) for j in range(w)])


def test_hull_area():
    W = 40
    assert SG.hull_area(_rect(3, 4, 5, 7, W), W) == 35.0
    assert SG.hull_area(np.array([5 * W + 6]), W) == 1.0
    # 3x3 square plus one pixel below its left column: hull (0,0) (3,0) (3,3)
    # (1,4) (0,4), shoelace 22 / 2
    L = np.concatenate([_rect(0, 0, 3, 3, W), _rect(3, 0, 1, 1, W)])
    assert SG.hull_area(L, W) == 11.0
    for _ in range(20):
        idx = np.unique(rng.integers(0, 30, 12) * W + rng.integers(0, 30, 12))
        y, x = np.divmod(idx, W)
        corners = np.array([(xx + a, yy + b) for yy, xx in zip(y, x) for a in (0, 1) for b in (0, 1)])
        assert abs(SG.hull_area(idx, W) - ConvexHull(corners).volume) < 1e-9


def test_moments_and_eccentricity():
    W = 100
    n, cyy, cxx, cxy = SG.moments(_rect(10, 10, 4, 4, W), W)
    assert n == 16 and abs(cyy - 1.25) < 1e-12 and abs(cxx - 1.25) < 1e-12 and cxy == 0.0
    assert SG.eccentricity(cyy, cxx, cxy) == 0.0
    line = _rect(5, 5, 1, 30, W)
    assert abs(SG.eccentricity(*SG.moments(line, W)[1:]) - 1.0) < 1e-12
    a, b = 20.0, 10.0
    yy, xx = np.mgrid[0:W, 0:W]
    ell = np.nonzero((((yy - 50) / b) ** 2 + ((xx - 50) / a) ** 2 <= 1).ravel())[0]
    e = SG.eccentricity(*SG.moments(ell, W)[1:])
    assert abs(e - math.sqrt(1 - (b / a) ** 2)) < 0.01
    assert SG.eccentricity(0.0, 0.0, 0.0) == 0.0


def test_shape_cleanup():
    W = 100
    assert SG.keep(_rect(10, 10, 6, 6, W), W)             # compact blob
    assert not SG.keep(_rect(10, 10, 3, 3, W), W)         # area 9 < 20
    assert not SG.keep(_rect(10, 10, 2, 40, W), W)        # elongated: eccentricity
    ring = np.array([p for p in _rect(20, 20, 12, 12, W)
                     if not (22 <= p // W < 30 and 22 <= p % W < 30)])
    assert not SG.keep(ring, W)                          # concave: 80 of 144 hull px


def test_nmf_fixed_point_and_descent():
    F = rng.random((50, 2))
    A = rng.random((2, 30))
    P = F @ A
    F1, A1 = SG.nmf(P, F, A, iters=5)
    assert np.allclose(F1, F, rtol=1e-6) and np.allclose(A1, A, rtol=1e-6)
    F0, A0 = rng.random((50, 2)), rng.random((2, 30))
    losses = [np.linalg.norm(P - F0 @ A0)]
    Fi, Ai = F0, A0
    for _ in range(30):
        Fi, Ai = SG.nmf(P, Fi, Ai, iters=1)
        losses.append(np.linalg.norm(P - Fi @ Ai))
    assert all(b <= a + 1e-12 for a, b in zip(losses, losses[1:]))
    assert losses[-1] < 0.2 * losses[0]


def test_footprints_on_planted_blobs():
    """Two lone discs, and a touching pair whose members spike in different
    segments and once together (one merged blob): three regions, the pair's
    with N = 2 (the merged blob joins the first member's cluster)."""
    K, H, W = 6, 64, 64
    yy, xx = np.mgrid[0:H, 0:W]
    disc = lambda cy, cx, r: ((yy - cy) ** 2 + (xx - cx) ** 2 <= r * r).astype(float)
    d1, d2 = disc(15, 15, 5), disc(45, 45, 5)
    d3, d4 = disc(15, 46, 5), disc(15, 55, 5)   # overlapping pair (9 px apart)
    prob = np.full((K, H, W), 0.05)
    prob[0] += 0.8 * d1
    prob[1] += 0.8 * d2
    prob[2] += 0.8 * d3
    prob[3] += 0.8 * d4
    prob[4] += 0.8 * np.clip(d3 + d4, 0, 1)
    prob = np.clip(prob, 0, 1)
    regions = SG.footprints(prob)
    assert len(regions) == 3
    assert sorted(r["N"] for r in regions) == [1, 1, 2]
    assert sorted(r["blobs"] for r in regions) == [1, 1, 3]
    for r in regions:
        assert r["F"].shape == (r["pixels"].size, r["N"]) and (r["F"] >= 0).all()
        assert (r["A"] >= 0).all()
        recon = r["F"] @ r["A"]
        P = prob.reshape(K, -1)[:, r["pixels"]].T
        assert np.linalg.norm(P - recon) < 0.1 * np.linalg.norm(P)


def test_touching_pair_separates_into_two_footprints():
    K, H, W = 6, 64, 64
    yy, xx = np.mgrid[0:H, 0:W]
    d3 = ((yy - 15) ** 2 + (xx - 46) ** 2 <= 25).astype(float)
    d4 = ((yy - 15) ** 2 + (xx - 55) ** 2 <= 25).astype(float)
    prob = np.full((K, H, W), 0.05)
    prob[2] += 0.8 * d3
    prob[3] += 0.8 * d4
    prob[4] += 0.8 * np.clip(d3 + d4, 0, 1)
    (r,) = SG.footprints(np.clip(prob, 0, 1))
    assert r["N"] == 2
    own = [d3.ravel()[r["pixels"]] > 0, d4.ravel()[r["pixels"]] > 0]
    for j in range(2):
        f = r["F"][:, j]
        mass = [f[o].sum() / f.sum() for o in own]
        assert max(mass) > 0.8            # each footprint concentrates on one disc
    m0 = [r["F"][own[0], j].sum() / r["F"][:, j].sum() for j in range(2)]
    assert (m0[0] > 0.8) != (m0[1] > 0.8)  # ... and on different discs


def test_no_capacity_limit_on_region_size_or_neuron_count():
    """The oracle factorises every region, however large and however many
    clusters it holds: a 24-disc chain of about 20,000 px and a 40-disc chain
    (N = 40) come out with one cluster per disc, and each footprint of the
    40-disc chain concentrates on its own disc."""
    from paper_2403_16438_gb300 import synth
    prob = synth.disc_chain_maps().double().numpy()
    K, H, W = prob.shape
    regs = SG.regions(prob)
    assert [r["N"] for r in regs] == [24, 40, 1]
    lab, n = ndimage.label(prob.max(axis=0) > 0.5, structure=np.ones((3, 3), bool))
    sizes = sorted(np.bincount(lab.ravel())[1:].tolist())
    assert sorted(r["pixels"].size for r in regs) == sizes and sizes[-1] > 16000
    big = regs[0]
    F, A = SG.factorise(prob, regs[1])
    assert F.shape == (regs[1]["pixels"].size, 40) and A.shape == (40, K)
    yy, xx = np.divmod(regs[1]["pixels"], W)
    for j in range(40):  # clusters in blob order: segment 0's discs, then segment 1's
        k = 2 * j if j < 20 else 2 * (j - 20) + 1
        own = (yy - 70) ** 2 + (xx - (10 + 6 * k)) ** 2 <= 16
        assert F[own, j].sum() > 0.5 * F[:, j].sum()
        assert A[j, k % 2] > 10 * A[j, 1 - k % 2]
    assert big["pixels"].size > 16000
