"""The FP32 correlation's patch-group size (vimg_params.corr_group): every
supported size against the FP64 oracle on a frame whose patch rows (19 patches)
leave a ragged last group for each of them, and a batched call that mixes
handles of different group sizes against the same handles called one by one.
Only the offset c of each item's first patch moves with the group size, so the
surfaces stay within the oracle tolerance of the default size."""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_16438_gb300 import synth
from parity_util import compare_shifts

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def vimg():
    from paper_2403_16438_gb300 import vimg as v
    return v


@pytest.fixture(scope="module")
def video():
    # 96 x 448: 3 x 19 patches at R = 16 (groups of 7: 7, 7, 5; of 8: 8, 8, 3;
    # of 10: 10, 9; of 11: 11, 8)
    cfg = synth.scaled_config(96, 448, 12, seed=77)
    frames, planted, T = synth.make_video(cfg, 12)
    o = oracle.Oracle(96, 448, R=16)
    o.set_template(T.double().numpy())
    ref = o.process(frames.numpy(), want_surface=True)
    return frames, T, ref


def run(vimg, frames, T, cg):
    n, H, W = frames.shape
    h = vimg.Handle(H, W, corr_group=cg)
    h.set_template(T.to(DEV))
    sh = torch.zeros((n, 2), device=DEV)
    info = torch.zeros((n, 4), device=DEV)
    surf = torch.zeros((n, 33, 33), device=DEV, dtype=torch.float64)
    h.process(frames.to(DEV), shifts=sh, peak_info=info, surface=surf)
    torch.cuda.synchronize()
    h.close()
    return sh.cpu().numpy(), info.cpu().numpy(), surf.cpu().numpy()


@pytest.mark.parametrize("cg", [0, 7, 8, 10, 11])
def test_group_sizes_against_the_oracle(vimg, video, cg):
    frames, T, ref = video
    sh, info, surf = run(vimg, frames, T, cg)
    assert np.abs(surf - ref["surface"]).max() < 2e-6
    near, _ = compare_shifts(sh, info, ref)
    assert len(near) == 0


def test_default_group_is_eleven(vimg, video):
    frames, T, _ = video
    a = run(vimg, frames, T, 0)
    b = run(vimg, frames, T, 11)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_invalid_group_is_rejected(vimg):
    with pytest.raises(vimg.VimgError):
        vimg.Handle(96, 448, corr_group=9)


def test_batch_with_mixed_group_sizes(vimg):
    """Two videos with different group sizes in one batched call give the
    same shifts and summaries as each handle on its own."""
    vids = []
    for (H, W, seed, cg) in [(96, 448, 78, 7), (128, 256, 79, 11)]:
        cfg = synth.scaled_config(H, W, 60, seed=seed)
        f, _, T = synth.make_video(cfg, 60, device=DEV)
        vids.append((f, T, cg))
    singles = []
    for f, T, cg in vids:
        h = vimg.Handle(f.shape[1], f.shape[2], corr_group=cg)
        h.set_template(T)
        sh = torch.zeros((f.shape[0], 2), device=DEV)
        sm = torch.zeros((1, 2, f.shape[1], f.shape[2]), device=DEV)
        h.process(f, shifts=sh, summary=sm)
        torch.cuda.synchronize()
        singles.append((sh.cpu(), sm.cpu()))
        h.close()
    hs, shs, sms = [], [], []
    for f, T, cg in vids:
        h = vimg.Handle(f.shape[1], f.shape[2], corr_group=cg)
        h.set_template(T)
        hs.append(h)
        shs.append(torch.zeros((f.shape[0], 2), device=DEV))
        sms.append(torch.zeros((1, 2, f.shape[1], f.shape[2]), device=DEV))
    vimg.process_batch(hs, [v[0] for v in vids], shifts=shs, summary=sms)
    torch.cuda.synchronize()
    for (sh, sm), bsh, bsm in zip(singles, shs, sms):
        assert torch.equal(sh, bsh.cpu()) and torch.equal(sm, bsm.cpu())
    for h in hs:
        h.close()


@pytest.mark.parametrize("cg", [7, 11])
def test_group_sizes_at_a_smaller_radius(vimg, cg):
    """R = 8 (17 x 17 window, no 33rd-row pass; 20 patches per row: groups of 7
    give 7, 7, 6) against the oracle, on a width whose statistics take the TMA
    tiles."""
    cfg = synth.scaled_config(80, 448, 10, seed=91)
    frames, _, T = synth.make_video(cfg, 10)
    o = oracle.Oracle(80, 448, R=8)
    o.set_template(T.double().numpy())
    ref = o.process(frames.numpy(), want_surface=True)
    n, H, W = frames.shape
    h = vimg.Handle(H, W, corr_group=cg, search_radius=8)
    h.set_template(T.to(DEV))
    sh = torch.zeros((n, 2), device=DEV)
    info = torch.zeros((n, 4), device=DEV)
    surf = torch.zeros((n, 17, 17), device=DEV, dtype=torch.float64)
    h.process(frames.to(DEV), shifts=sh, peak_info=info, surface=surf)
    torch.cuda.synchronize()
    h.close()
    assert np.abs(surf.cpu().numpy() - ref["surface"]).max() < 2e-6
    near, _ = compare_shifts(sh.cpu().numpy(), info.cpu().numpy(), ref)
    assert len(near) == 0
