"""The fused temporal pass with the segment history in tensor memory and
TMA-staged frames (k_temporal_tm) against the FP64 oracle and against the
general kernel that keeps the history in shared memory (VIMG_TEMPORAL_SMEM).

Both kernels resample, smooth and take the max and median with the same FP32
operations in the same order, so the corrected frames and T_i must be equal
bit for bit; S_i adds the frames in two interleaved partial sums (one per
warp group) and may differ by FP32 rounding.  Against the oracle every output
is held to the 1e-4 relative bar.  The cases cover the tile and window
geometry: ragged heights, windows leaving the image on every side, windows
entirely outside it (given shifts far beyond the image), short segments,
segments split across calls (carried frames) and voltage traces."""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_16438_gb300 import synth
from parity_util import compare_images

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def vimg():
    from paper_2403_16438_gb300 import vimg as v
    return v


def _run(vimg, frames, T, shifts, flags=0, chunks=None, L=50, masks=None):
    n, H, W = frames.shape
    h = vimg.Handle(H, W, flags=flags, segment_len=L)
    h.set_template(T.to(DEV))
    if masks is not None:
        h.set_rois(masks.to(DEV))
    fd = frames.to(DEV)
    sd = shifts.to(DEV, torch.float32).contiguous()
    corr = torch.zeros((n, H, W), device=DEV)
    summ = torch.zeros((max(1, n // L), 2, H, W), device=DEV)
    tr = torch.zeros((n, masks.shape[0]), device=DEV) if masks is not None else None
    k_tot, t = 0, 0
    for c in (chunks or [n]):
        k_tot += h.process(fd[t:t + c], corrected=corr[t:t + c], summary=summ[k_tot:],
                           shifts_in=sd[t:t + c], traces=None if tr is None else tr[t:t + c])
        t += c
    assert h.synchronize() == 0
    h.close()
    return corr, summ[:k_tot], tr, k_tot


def _both(vimg, frames, T, shifts, **kw):
    a = _run(vimg, frames, T, shifts, **kw)
    b = _run(vimg, frames, T, shifts, flags=vimg.TEMPORAL_SMEM, **kw)
    assert a[3] == b[3]
    assert torch.equal(a[0], b[0]), "corrected frames differ between the kernels"
    if a[3]:
        assert torch.equal(a[1][:, 1], b[1][:, 1]), "T differs between the kernels"
        d = (a[1][:, 0] - b[1][:, 0]).abs().max() / b[1][:, 0].abs().max()
        assert d.item() <= 1e-6, d.item()
    if a[2] is not None:
        assert torch.equal(a[2], b[2])
    return a


def _oracle(frames, T, shifts, L=50, masks=None):
    n, H, W = frames.shape
    o = oracle.Oracle(H, W, L=L)
    o.set_template(T.double().numpy())
    if masks is not None:
        o.set_rois(masks.numpy())
    return o.process(frames.numpy(), shifts_in=shifts.to(torch.float32).double().numpy())


def _check_oracle(g, r):
    compare_images(g[0].cpu().numpy(), r["corrected"], "corrected")
    if g[3]:
        for s in range(g[3]):
            compare_images(g[1][s].cpu().numpy(), r["summary"][s], f"summary[{s}]")


@pytest.mark.parametrize("H,W,n,L,chunks", [
    (128, 128, 100, 50, None),        # two segments, every tile at the border
    (200, 136, 57, 50, [20, 37]),     # ragged height and width, a segment across calls
    (96, 256, 23, 7, [5, 9, 9]),      # short segments, odd frame counts per group
    (512, 512, 50, 50, None),         # interior tiles
])
def test_tensor_memory_kernel_matches_oracle_and_general_kernel(vimg, H, W, n, L, chunks):
    cfg = synth.scaled_config(H, W, n, seed=H * 7 + W)
    frames, planted, T = synth.make_video(cfg, n)
    g = _both(vimg, frames, T, planted, L=L, chunks=chunks)
    _check_oracle(g, _oracle(frames, T, planted, L=L))


def test_windows_outside_the_image(vimg):
    """Given shifts that move the source window past every border by up to the
    whole tile, and two far outside the image (every sample an edge pixel)."""
    cfg = synth.scaled_config(96, 160, 50, seed=5)
    frames, _, T = synth.make_video(cfg, 50)
    g = torch.Generator().manual_seed(6)
    s = (torch.rand((50, 2), generator=g) - 0.5) * 2 * 30.0
    s[7] = torch.tensor([-1000.25, 3.5])
    s[8] = torch.tensor([2.75, 4000.5])
    s[9] = torch.tensor([40.5, -45.75])
    out = _both(vimg, frames, T, s)
    _check_oracle(out, _oracle(frames, T, s))


def test_traces_with_the_tensor_memory_kernel(vimg):
    cfg = synth.tiny_config(seed=12)
    frames, planted, T = synth.make_video(cfg, 60)
    masks = synth.roi_masks(cfg)
    out = _both(vimg, frames, T, planted, chunks=[31, 29], masks=masks)
    r = _oracle(frames, T, planted, masks=masks)
    tr = out[2].cpu().double().numpy()
    assert np.abs(tr - r["traces"]).max() / np.abs(r["traces"]).max() <= 1e-4
