"""Voltage traces on the GPU (Sec. II, third stage: the mean of each motion-
corrected frame within every neuron ROI), compared with the FP64 oracle.

The GPU sums V in 2^-20 fixed point inside the fused temporal pass, so traces
are also checked to be bit-identical across chunkings, across output choices
(traces alone, with corrected frames, with the high-pass output) and against a
plain mean of the GPU's own corrected frames up to the fixed-point rounding."""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_16438_gb300 import synth
from parity_util import compare_images, compare_shifts

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def vimg():
    from paper_2403_16438_gb300 import vimg as v
    return v


def _masks(cfg):
    """The scene's neuron footprints plus the degenerate ROIs: the whole image,
    an empty one, a single corner pixel, a band along the bottom and right
    borders, and one overlapping two footprints."""
    m = synth.roi_masks(cfg)
    H, W = cfg.H, cfg.W
    extra = torch.zeros((5, H, W), dtype=torch.bool)
    extra[0] = True
    extra[2, H - 1, W - 1] = True
    extra[3, H - 3:, :] = True
    extra[3, :, W - 2:] = True
    extra[4] = m[0] | m[1]
    return torch.cat([m, extra])


def _run(vimg, h, frames, n_rois, **out):
    n = frames.shape[0]
    tr = torch.full((n, n_rois), float("nan"), device=DEV)
    h.process(frames, traces=tr, **out)
    return tr


def test_traces_match_the_oracle(vimg):
    cfg = synth.tiny_config()
    n = 120  # two full segments and a partial one
    frames, _, T = synth.make_video(cfg, n)
    masks = _masks(cfg)
    h = vimg.Handle(cfg.H, cfg.W, max_chunk=64)
    h.set_template(T.to(DEV))
    h.set_rois(masks.to(DEV))
    shifts = torch.empty((n, 2), device=DEV)
    info = torch.empty((n, 4), device=DEV)
    corr = torch.empty((n, cfg.H, cfg.W), device=DEV)
    tr = _run(vimg, h, frames.to(DEV), masks.shape[0], shifts=shifts, peak_info=info,
              corrected=corr)
    torch.cuda.synchronize()
    h.close()
    o = oracle.Oracle(cfg.H, cfg.W)
    o.set_template(T.double().numpy())
    o.set_rois(masks.numpy())
    r = o.process(frames.numpy(), want_summary=False)
    compare_shifts(shifts.cpu().numpy(), info.cpu().numpy(), r)
    g = tr.cpu().double().numpy()
    assert np.isfinite(g).all()
    assert np.all(g[:, -4] == 0.0)  # the empty ROI
    compare_images(g, r["traces"], "traces")
    # the GPU's traces are the ROI means of its own corrected frames
    c = corr.cpu().double().numpy()
    mk = masks.numpy()
    for i in (0, 49, 50, 119):
        own = oracle.roi_means(c[i], mk)
        assert np.abs(g[i] - own).max() <= 1e-6 * np.abs(own).max() + 2e-6


def test_traces_identical_across_chunkings_and_outputs(vimg):
    cfg = synth.tiny_config(seed=11)
    n = 137
    frames, _, T = synth.make_video(cfg, n)
    fd = frames.to(DEV)
    masks = _masks(cfg).to(DEV)
    nr = masks.shape[0]

    def handle(**kw):
        h = vimg.Handle(cfg.H, cfg.W, **kw)
        h.set_template(T.to(DEV))
        h.set_rois(masks)
        return h

    h = handle()
    ref = _run(vimg, h, fd, nr, corrected=torch.empty((n, cfg.H, cfg.W), device=DEV))
    h.close()
    # traces alone, several calls of uneven length, small internal batches
    h = handle(max_chunk=16)
    parts = [_run(vimg, h, fd[a:b], nr) for a, b in ((0, 37), (37, 87), (87, 88), (88, n))]
    h.close()
    # high-pass output: the traces still come from V
    h = handle(hp_window=10, flags=vimg.OUT_HIGHPASS)
    hp = _run(vimg, h, fd, nr, corrected=torch.empty((n, cfg.H, cfg.W), device=DEV),
              summary=torch.empty((2, 2, cfg.H, cfg.W), device=DEV))
    h.close()
    torch.cuda.synchronize()
    assert torch.equal(torch.cat(parts), ref)
    assert torch.equal(hp, ref)


def test_roi_limits(vimg):
    cfg = synth.tiny_config()
    frames, _, T = synth.make_video(cfg, 5)
    h = vimg.Handle(cfg.H, cfg.W)
    h.set_template(T.to(DEV))
    ok = torch.zeros((2, cfg.H, cfg.W), dtype=torch.bool, device=DEV)
    ok[0, :10, :10] = True
    ok[1, 5:20, 5:20] = True
    h.set_rois(ok)
    five = torch.zeros((5, cfg.H, cfg.W), dtype=torch.bool, device=DEV)
    five[:, 40, 40] = True  # one pixel in five ROIs
    with pytest.raises(vimg.VimgError):
        h.set_rois(five)
    # the previous ROIs stay in force
    tr = torch.empty((5, 2), device=DEV)
    corr = torch.empty((5, cfg.H, cfg.W), device=DEV)
    h.process(frames.to(DEV), traces=tr, corrected=corr)
    torch.cuda.synchronize()
    c = corr.cpu().double().numpy()
    for i in range(5):
        own = oracle.roi_means(c[i], ok.cpu().numpy())
        assert np.abs(tr[i].cpu().double().numpy() - own).max() <= 1e-6 * np.abs(own).max()
    # clearing: traces requested with no ROIs write nothing and fail nothing
    h.set_rois(None)
    h.process(frames.to(DEV), traces=torch.empty((5, 0), device=DEV))
    torch.cuda.synchronize()
    h.close()
