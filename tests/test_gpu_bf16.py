"""BF16 tensor-core (tcgen05) correlation: shifts and surfaces against the FP64
oracle and the FP32 path.  Its gate is the shift error against the oracle,
<= 0.05 px; the integer peak must agree except on near-ties."""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_16438_gb300 import synth
from parity_util import NEAR_TIE, compare_images

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def run(vimg, frames, T, flags, **kw):
    n, H, W = frames.shape
    h = vimg.Handle(H, W, flags=flags, **kw)
    h.set_template(T.to(DEV))
    fd = frames.to(DEV)
    s = torch.zeros((n, 2), device=DEV)
    info = torch.zeros((n, 4), device=DEV)
    surf = torch.zeros((n, 33, 33), device=DEV, dtype=torch.float64)
    corr = torch.zeros((n, H, W), device=DEV)
    h.process(fd, shifts=s, peak_info=info, surface=surf, corrected=corr)
    assert h.synchronize() == 0
    h.close()
    return s.cpu().numpy(), info.cpu().numpy(), surf.cpu().numpy(), corr.cpu().numpy()


@pytest.fixture(scope="module")
def vimg():
    from paper_2403_16438_gb300 import vimg as v
    return v


def test_bf16_against_oracle_paper_scale(vimg):
    cfg = synth.paper_scale_config(seed=77)
    frames, planted, T = synth.make_video(cfg, 20)
    s, info, surf, corr = run(vimg, frames, T, vimg.CORR_BF16)
    o = oracle.Oracle(cfg.H, cfg.W)
    o.set_template(T.double().numpy())
    r = o.process(frames.numpy(), want_surface=True)
    assert np.abs(surf - r["surface"]).max() < 2e-3
    gap = r["info"][:, 0] - r["info"][:, 1]
    same = np.all(info[:, :2].astype(int) == r["dstar"], axis=1)
    assert np.all(same | (gap < 1e-3))
    err = np.abs(s - r["shifts"]).max()
    assert err <= 0.05, err
    compare_images(corr, r["corrected"], "corrected", tol=1e-3)


@pytest.mark.parametrize("H,W,n,chunk", [(300, 250, 37, 24), (128, 128, 16, 24),
                                          (160, 203, 230, 200)])
def test_bf16_against_fp32_ragged(vimg, H, W, n, chunk):
    """Frame groups of 80 (N = 80) with ragged tails (N = 48, 32, 16), widths
    that are not multiples of 8, and several internal batches."""
    cfg = synth.scaled_config(H, W, n, seed=H + W)
    frames, _, T = synth.make_video(cfg, n)
    s16, i16, surf16, _ = run(vimg, frames, T, vimg.CORR_BF16, max_chunk=chunk)
    s32, i32, surf32, _ = run(vimg, frames, T, 0)
    assert np.abs(surf16 - surf32).max() < 2e-3
    assert np.abs(s16 - s32).max() <= 0.05
