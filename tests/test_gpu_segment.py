"""Footprint reconstruction (Sec. III-D) on the GPU against the FP64 oracle.

Integer stages are compared exactly: the region map (OR of the kept blobs,
8-connected components) and the number of neurons per region follow from
thresholds on the same float32 maps, exact integer moments and exact hull
areas, decided in FP64 without contraction on both sides.  The NMF runs in
FP32 on the GPU and FP64 in the oracle: footprints and activities within 1e-3
of each neuron's maximum."""
import numpy as np
import pytest
import torch

import oracle.segmentation as SG
from paper_2403_16438_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def vimg():
    from paper_2403_16438_gb300 import vimg as v
    return v


# Capacity of the GPU's NMF kernel (vimg.h): larger regions are reported, not factorised.
CAP_PIXELS, CAP_CLUSTERS = 16000, 32


def _compare(vimg, prob):
    """GPU against the uncapped oracle: identical region map; each region's
    status is 0 exactly when it is within the kernel's capacity, else the
    matching VIMG_REGION_* code; every factorised region's footprints and
    activities equal the oracle's.  Returns (neurons, regions, status)."""
    K, H, W = prob.shape
    seg = vimg.Segmenter(H, W, K)
    foot, act, rmap, nreg = seg.run(prob.to(DEV), max_neurons=512)
    torch.cuda.synchronize()
    status = seg.status()
    seg.close()
    p64 = prob.double().numpy()
    regions = SG.regions(p64)
    # region map: every region of b in pixel order
    ref_map = -np.ones(H * W, np.int64)
    for k, r in enumerate(regions):
        ref_map[r["pixels"]] = k
    assert np.array_equal(rmap.cpu().numpy().ravel(), ref_map)
    assert nreg == len(regions) == len(status)
    expect = [vimg.REGION_TOO_LARGE if r["pixels"].size > CAP_PIXELS else
              vimg.REGION_TOO_MANY if r["N"] > CAP_CLUSTERS else 0 for r in regions]
    assert status == expect
    n_ref = sum(r["N"] for r, st in zip(regions, status) if st == 0)
    assert foot.shape[0] == n_ref
    f = foot.cpu().double().numpy().reshape(n_ref, H * W)
    a = act.cpu().double().numpy()
    k = 0
    for r, st in zip(regions, status):
        if st:
            continue
        F, A = SG.factorise(p64, r)
        for j in range(r["N"]):
            ref_f = np.zeros(H * W)
            ref_f[r["pixels"]] = F[:, j]
            scale_f = np.abs(ref_f).max()
            assert np.abs(f[k] - ref_f).max() <= 1e-3 * scale_f, (k, np.abs(f[k] - ref_f).max(), scale_f)
            scale_a = np.abs(A[j]).max()
            assert np.abs(a[k] - A[j]).max() <= 1e-3 * scale_a
            k += 1
    return n_ref, nreg, status


def test_planted_maps_match_the_oracle(vimg):
    cfg = synth.tiny_config(seed=3)
    prob = synth.planted_prob_maps(cfg, 24, seed=1)
    n, nreg, status = _compare(vimg, prob)
    assert n >= len(synth.roi_masks(cfg)) - 2 and nreg >= 1 and not any(status)


def test_ragged_size_and_touching_pair(vimg):
    K, H, W = 6, 70, 90
    yy, xx = np.mgrid[0:H, 0:W]
    d3 = ((yy - 15) ** 2 + (xx - 46) ** 2 <= 25).astype(np.float32)
    d4 = ((yy - 15) ** 2 + (xx - 55) ** 2 <= 25).astype(np.float32)
    d1 = ((yy - 50) ** 2 + (xx - 20) ** 2 <= 30).astype(np.float32)
    prob = np.full((K, H, W), 0.05, np.float32)
    prob[0] += 0.8 * d1
    prob[2] += 0.8 * d3
    prob[3] += 0.8 * d4
    prob[4] += 0.8 * np.clip(d3 + d4, 0, 1)
    prob[5, 60, 5:80] = 0.9          # a line: removed by eccentricity
    n, nreg, status = _compare(vimg, torch.from_numpy(np.clip(prob, 0, 1)))
    assert n == 3 and nreg == 2 and status == [0, 0]


def test_empty_maps(vimg):
    seg = vimg.Segmenter(64, 64, 4)
    foot, act, rmap, nreg = seg.run(torch.zeros((4, 64, 64), device=DEV))
    assert foot.shape[0] == 0 and nreg == 0 and bool((rmap == -1).all())
    assert seg.status() == []
    seg.close()


def test_regions_beyond_capacity_are_reported(vimg):
    """A 24-disc chain of about 20,000 px (too large) and a 40-disc chain with
    40 clusters (too many) are reported by their status and contribute no
    neuron; the ordinary disc beside them still equals the uncapped oracle."""
    n, nreg, status = _compare(vimg, synth.disc_chain_maps())
    assert nreg == 3 and status == [vimg.REGION_TOO_LARGE, vimg.REGION_TOO_MANY, 0] and n == 1


def test_tiling_blobs_form_one_region_too_large(vimg):
    K, H, W = 8, 160, 160
    prob = torch.zeros((K, H, W))
    yy, xx = torch.meshgrid(torch.arange(H), torch.arange(W), indexing="ij")
    for i in range(K):  # discs of radius 4 every 10 px, odd segments offset by (5, 5)
        off = 5 * (i % 2)
        for cy in range(6 + off, H, 10):
            for cx in range(6 + off, W, 10):
                prob[i] += (((yy - cy) ** 2 + (xx - cx) ** 2) <= 16).float() * 0.9
    n, nreg, status = _compare(vimg, prob.clamp(0, 1))
    assert n == 0 and nreg == 1 and status == [vimg.REGION_TOO_LARGE]
