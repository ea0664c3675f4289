"""Parity at the benchmark's full size and in its launch configuration, at a
larger frame size, and on degenerate inputs.

The 10,000-frame 512x512 video goes through vimg_process exactly as the
benchmark runs it (200-frame internal batches, corrected frames and summaries);
the oracle then recomputes, one by one, sampled frames at batch and segment
boundaries and two whole segments."""
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


def _oracle(T, H, W, **kw):
    o = oracle.Oracle(H, W, **kw)
    o.set_template(T.cpu().double().numpy())
    return o


def test_bench_size_and_launch_configuration(vimg):
    cfg = synth.paper_scale_config()
    n = cfg.n_frames
    frames, planted, T = synth.make_video(cfg, n, device=DEV)
    h = vimg.Handle(cfg.H, cfg.W, max_chunk=200)  # the benchmark's launch configuration
    h.set_template(T)
    shifts = torch.empty((n, 2), device=DEV)
    info = torch.empty((n, 4), device=DEV)
    corr = torch.empty((n, cfg.H, cfg.W), device=DEV)
    summ = torch.empty((n // 50, 2, cfg.H, cfg.W), device=DEV)
    assert h.process(frames, shifts=shifts, peak_info=info, corrected=corr, summary=summ) == n // 50
    torch.cuda.synchronize()
    h.close()
    # sampled frames: first and last of batches, segment ends, the last frame
    idx = np.array([0, 1, 199, 200, 4999, 5000, 9949, 9950, 9999])
    o = _oracle(T, cfg.H, cfg.W)
    sample = np.stack([frames[int(i)].cpu().numpy() for i in idx])  # no uint16 gather on CUDA
    r = o.process(sample, want_summary=False)
    compare_shifts(shifts[idx].cpu().numpy(), info[idx].cpu().numpy(), r)
    compare_images(corr[idx].cpu().numpy(), r["corrected"], "corrected")
    # two whole segments, the first and the last
    for seg in (0, n // 50 - 1):
        o = _oracle(T, cfg.H, cfg.W)
        rs = o.process(frames[50 * seg:50 * (seg + 1)].cpu().numpy(), want_corrected=False)
        compare_images(summ[seg].cpu().numpy(), rs["summary"][0], f"summary[{seg}]")
    # property at full size: every frame tracks the planted drift (the content
    # model moves by at most 12 px plus 3-px jumps)
    err = (shifts.cpu().double() - planted).abs().max().item()
    assert err < 1.0, err


def test_large_frames(vimg):
    cfg = synth.scaled_config(1024, 1024, 3, seed=77)
    frames, _, T = synth.make_video(cfg, 3)
    h = vimg.Handle(1024, 1024)
    h.set_template(T.to(DEV))
    s = torch.empty((3, 2), device=DEV)
    info = torch.empty((3, 4), device=DEV)
    surf = torch.empty((3, 33, 33), device=DEV, dtype=torch.float64)
    corr = torch.empty((3, 1024, 1024), device=DEV)
    h.process(frames.to(DEV), shifts=s, peak_info=info, surface=surf, corrected=corr)
    torch.cuda.synchronize()
    h.close()
    r = _oracle(T, 1024, 1024).process(frames.numpy(), want_surface=True, want_summary=False)
    assert np.abs(surf.cpu().numpy() - r["surface"]).max() < 2e-6
    compare_shifts(s.cpu().numpy(), info.cpu().numpy(), r)
    compare_images(corr.cpu().numpy(), r["corrected"], "corrected")


@pytest.mark.parametrize("R", [0, 1])
def test_smallest_search_windows(vimg, R):
    cfg = synth.tiny_config(clamp=1.0)
    frames, _, T = synth.make_video(cfg, 60)
    h = vimg.Handle(128, 128, search_radius=R)
    h.set_template(T.to(DEV))
    w = 2 * R + 1
    s = torch.empty((60, 2), device=DEV)
    info = torch.empty((60, 4), device=DEV)
    surf = torch.empty((60, w, w), device=DEV, dtype=torch.float64)
    summ = torch.empty((1, 2, 128, 128), device=DEV)
    h.process(frames.to(DEV), shifts=s, peak_info=info, surface=surf, summary=summ)
    torch.cuda.synchronize()
    h.close()
    r = _oracle(T, 128, 128, R=R).process(frames.numpy(), want_surface=True, want_corrected=False)
    assert np.abs(surf.cpu().numpy() - r["surface"]).max() < 2e-6
    compare_shifts(s.cpu().numpy(), info.cpu().numpy(), r)
    compare_images(summ.cpu().numpy().reshape(-1, 128, 128), r["summary"].reshape(-1, 128, 128),
                   "summary")


def test_segment_length_one_and_flat_template_patches(vimg):
    """L = 1: every frame is a segment, S = V and T = 0.  A template that is
    constant on its left half has zero-norm patches there, whose ZNCC is 0."""
    cfg = synth.tiny_config()
    frames, _, T = synth.make_video(cfg, 7)
    T = T.clone()
    T[:, :64] = 1500.0
    h = vimg.Handle(128, 128, segment_len=1)
    h.set_template(T.to(DEV))
    s = torch.empty((7, 2), device=DEV)
    info = torch.empty((7, 4), device=DEV)
    surf = torch.empty((7, 33, 33), device=DEV, dtype=torch.float64)
    corr = torch.empty((7, 128, 128), device=DEV)
    summ = torch.empty((7, 2, 128, 128), device=DEV)
    assert h.process(frames.to(DEV), shifts=s, peak_info=info, surface=surf, corrected=corr,
                     summary=summ) == 7
    torch.cuda.synchronize()
    h.close()
    r = _oracle(T, 128, 128, L=1).process(frames.numpy(), want_surface=True)
    assert np.abs(surf.cpu().numpy() - r["surface"]).max() < 2e-6
    compare_shifts(s.cpu().numpy(), info.cpu().numpy(), r)
    sm = summ.cpu().numpy()
    assert np.array_equal(sm[:, 0], corr.cpu().numpy())  # S_i = V for L = 1
    assert np.abs(sm[:, 1]).max() == 0.0                  # T_i = max - median = 0
    compare_images(sm.reshape(-1, 128, 128), r["summary"].reshape(-1, 128, 128), "summary")
