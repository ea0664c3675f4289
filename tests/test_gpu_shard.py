"""One video cut into time shards (paper_2403_16438_gb300.shard), each shard on
its own handle that starts with vimg_seek at the shard's first frame: the
concatenated shifts, corrected (or high-passed) frames, segment summaries and
traces equal one handle over the whole video bit for bit.  Without the
high-pass the tensor-memory temporal kernel runs, with it the general kernel."""
import pytest
import torch

from paper_2403_16438_gb300 import shard, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def vimg():
    from paper_2403_16438_gb300 import vimg as v
    return v


def _run(vimg, frames, T, sh, masks=None, **kw):
    n, H, W = frames.shape
    h = vimg.Handle(H, W, **kw)
    h.set_template(T)
    if masks is not None:
        h.set_rois(masks)
    h.seek(sh.start, frames[sh.hist_start:sh.start].contiguous() if sh.history else None)
    m = sh.frames
    s = torch.full((m, 2), float("nan"), device=DEV)
    c = torch.full((m, H, W), float("nan"), device=DEV)
    L = h.params.segment_len
    k_max = (sh.end // L) - (sh.start // L)
    summ = torch.full((max(1, k_max), 2, H, W), float("nan"), device=DEV)
    tr = torch.zeros((m, masks.shape[0]), device=DEV) if masks is not None else None
    k = h.process(frames[sh.start:sh.end].contiguous(), shifts=s, corrected=c, summary=summ,
                  traces=tr)
    assert k == k_max and h.frames_seen == sh.end
    assert h.synchronize() == 0
    h.close()
    return s, c, summ[:k], tr


@pytest.mark.parametrize("H,W,n,parts,hp", [(128, 128, 230, 3, 0), (128, 128, 230, 3, 9),
                                             (512, 512, 300, 2, 0), (96, 136, 175, 4, 5)])
def test_shards_reproduce_one_stream(vimg, H, W, n, parts, hp):
    cfg = synth.scaled_config(H, W, n, seed=H + W + n)
    frames, _, T = synth.make_video(cfg, n, device=DEV)
    masks = synth.roi_masks(cfg).to(DEV) if H == 128 else None
    kw = dict(hp_window=hp, flags=vimg.OUT_HIGHPASS if hp else 0)
    full = _run(vimg, frames, T, shard.Shard(0, n, 0), masks, **kw)
    plan = shard.plan(n, parts, 50, hp)
    assert len(plan) == parts
    pieces = [_run(vimg, frames, T, sh, masks, **kw) for sh in plan]
    for i, name in enumerate(("shifts", "corrected", "summary", "traces")):
        if full[i] is None:
            continue
        got = torch.cat([p[i] for p in pieces])
        assert torch.equal(got, full[i]), name


def test_seek_rejects_bad_positions(vimg):
    cfg = synth.tiny_config(seed=5)
    frames, _, T = synth.make_video(cfg, 60, device=DEV)
    h = vimg.Handle(cfg.H, cfg.W, hp_window=5)
    h.set_template(T)
    with pytest.raises(vimg.VimgError):
        h.seek(49, frames[:49].contiguous())   # not a segment boundary
    with pytest.raises(vimg.VimgError):
        h.seek(50, frames[48:50].contiguous())  # shorter than hp_window - 1
    h.seek(50, frames[46:50].contiguous())
    assert h.frames_seen == 50
    h.close()
