"""Whole-video summary images on the GPU (VolPy's temporal average and local
correlation images, Sec. III-A / Fig. 2) against the FP64 oracle.

Both sides resample with the same given shifts, so V differs only by FP32
against FP64 bilinear rounding; the GPU sums d = V - T in FP32 within an
internal batch and in FP64 across batches.  Bars: average within 1e-5
relative, correlation within 1e-4 absolute."""
import numpy as np
import pytest
import torch

import oracle
import oracle.video_summary as VS
from paper_2403_16438_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def vimg():
    from paper_2403_16438_gb300 import vimg as v
    return v


def _shifts(n, seed, amp=3.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(-amp, amp, size=(n, 2))


def _oracle_v(frames, T, shifts):
    o = oracle.Oracle(T.shape[0], T.shape[1])
    o.set_template(T.double().numpy())
    return o.process(frames.numpy(), shifts_in=shifts, want_summary=False)["corrected"]


def _gpu(vimg, frames, T, shifts, splits, max_chunk=200):
    H, W = T.shape
    h = vimg.Handle(H, W, max_chunk=max_chunk, flags=vimg.VIDEO_SUMMARY)
    h.set_template(T.to(DEV))
    fd = frames.to(DEV)
    sd = torch.from_numpy(shifts).float().to(DEV)
    for a, b in splits:
        h.process(fd[a:b], shifts_in=sd[a:b])
    avg = torch.empty((H, W), device=DEV)
    corr = torch.empty((H, W), device=DEV)
    h.video_summary(avg, corr)
    torch.cuda.synchronize()
    h.close()
    return avg.cpu().double().numpy(), corr.cpu().double().numpy()


def test_summary_images_match_the_oracle(vimg):
    cfg = synth.tiny_config(dff_lo=0.3, dff_hi=0.3)
    n = 137
    frames, _, T = synth.make_video(cfg, n)
    sh = _shifts(n, 1)
    sh[5] = (-20.5, 30.25)   # far outside: clamped coordinates everywhere
    V = _oracle_v(frames, T, sh)
    ra, rc = VS.average_image(V), VS.correlation_image(V)
    ga, gc = _gpu(vimg, frames, T, sh, [(0, 37), (37, 100), (100, n)], max_chunk=48)
    assert np.abs(ga - ra).max() <= 1e-5 * np.abs(ra).max()
    assert np.abs(gc - rc).max() <= 1e-4, np.abs(gc - rc).max()
    # footprints correlate more than the background (the image is informative)
    m = synth.roi_masks(cfg).numpy().any(axis=0)
    assert gc[m].mean() > gc[~m].mean()


def test_ragged_size_and_batching(vimg):
    cfg = synth.scaled_config(100, 130, 60, seed=4)
    frames, _, T = synth.make_video(cfg, 60)
    sh = _shifts(60, 2, amp=1.5)
    V = _oracle_v(frames, T, sh)
    rc = VS.correlation_image(V)
    g1 = _gpu(vimg, frames, T, sh, [(0, 60)])
    g2 = _gpu(vimg, frames, T, sh, [(i, i + 1) for i in range(60)], max_chunk=7)
    for ga, gc in (g1, g2):
        assert np.abs(gc - rc).max() <= 1e-4
        assert np.abs(ga - VS.average_image(V)).max() <= 1e-5 * np.abs(V).max()


def test_constant_video_and_errors(vimg):
    """A constant video: every trace is constant, so C = 0 and A = the frame."""
    H = W = 64
    frames = torch.full((20, H, W), 1234, dtype=torch.uint16)
    T = torch.full((H, W), 1000.0)
    ga, gc = _gpu(vimg, frames, T, np.zeros((20, 2)), [(0, 20)])
    assert np.all(gc == 0.0) and np.allclose(ga, 1234.0, rtol=0, atol=1e-3)
    h = vimg.Handle(H, W)
    h.set_template(T.to(DEV))
    with pytest.raises(vimg.VimgError):
        h.video_summary(torch.empty((H, W), device=DEV))  # flag not set
    h.close()
    h = vimg.Handle(H, W, flags=vimg.VIDEO_SUMMARY)
    h.set_template(T.to(DEV))
    with pytest.raises(vimg.VimgError):
        h.video_summary(torch.empty((H, W), device=DEV))  # no frames yet
    h.process(frames.to(DEV), shifts_in=torch.zeros((20, 2), device=DEV))
    h.reset()
    with pytest.raises(vimg.VimgError):
        h.video_summary(torch.empty((H, W), device=DEV))  # reset cleared them
    h.close()
