"""Stream-state checkpoint and restore (vimg_get_state / vimg_set_state): a
stream stopped inside a segment, with a high-pass history and whole-video sums,
continues on a fresh handle from the saved state exactly as one uninterrupted
stream; states of handles with other parameters, truncated or foreign buffers
are refused with the handle's state unchanged."""
import numpy as np
import pytest
import torch

from paper_2403_16438_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def vimg():
    from paper_2403_16438_gb300 import vimg as v
    return v


@pytest.fixture(scope="module")
def video():
    cfg = synth.tiny_config(seed=57)
    frames, _, T = synth.make_video(cfg, 130, device=DEV)
    return frames, T


def make(vimg, T, **kw):
    kw = dict(dict(hp_window=7, flags=vimg.OUT_HIGHPASS | vimg.VIDEO_SUMMARY, max_chunk=40), **kw)
    h = vimg.Handle(T.shape[0], T.shape[1], **kw)
    h.set_template(T)
    return h


def outputs(n, H, W):
    return (torch.zeros((n, 2), device=DEV), torch.zeros((n, H, W), device=DEV),
            torch.zeros((3, 2, H, W), device=DEV))


@pytest.mark.parametrize("cut", [70, 50, 1])
def test_restored_stream_continues_bit_for_bit(vimg, video, cut):
    frames, T = video
    n, H, W = frames.shape
    # one uninterrupted stream
    ref = make(vimg, T)
    s0, c0, m0 = outputs(n, H, W)
    k = ref.process(frames[:cut], shifts=s0[:cut], corrected=c0[:cut], summary=m0)
    ref.process(frames[cut:], shifts=s0[cut:], corrected=c0[cut:], summary=m0[k:])
    av0, cr0 = torch.zeros((H, W), device=DEV), torch.zeros((H, W), device=DEV)
    ref.video_summary(av0, cr0)
    torch.cuda.synchronize()
    # stop at `cut`, save, restore on a new handle, continue
    a = make(vimg, T)
    s1, c1, m1 = outputs(n, H, W)
    k1 = a.process(frames[:cut], shifts=s1[:cut], corrected=c1[:cut], summary=m1)
    state = a.get_state()
    a.close()
    b = make(vimg, T)
    b.set_state(state)
    assert b.frames_seen == cut
    b.process(frames[cut:], shifts=s1[cut:], corrected=c1[cut:], summary=m1[k1:])
    av1, cr1 = torch.zeros((H, W), device=DEV), torch.zeros((H, W), device=DEV)
    b.video_summary(av1, cr1)
    torch.cuda.synchronize()
    assert torch.equal(s0, s1) and torch.equal(c0, c1) and torch.equal(m0, m1)
    assert torch.equal(av0, av1) and torch.equal(cr0, cr1)
    b.close()
    ref.close()


def test_state_size_follows_the_open_segment(vimg, video):
    frames, T = video
    h = make(vimg, T, flags=0, hp_window=0)
    empty = len(h.get_state())
    h.process(frames[:30])
    assert len(h.get_state()) == empty + 30 * (h.H * h.W * 2 + 8)
    h.process(frames[30:50])  # a segment completes: nothing held
    assert len(h.get_state()) == empty
    h.close()


def test_foreign_states_are_refused(vimg, video):
    frames, T = video
    a = make(vimg, T)
    a.process(frames[:33])
    state = a.get_state()
    other = make(vimg, T, hp_window=5)
    with pytest.raises(vimg.VimgError):
        other.set_state(state)
    b = make(vimg, T)
    with pytest.raises(vimg.VimgError):
        b.set_state(state[:len(state) - 1])
    with pytest.raises(vimg.VimgError):
        b.set_state(bytes(len(state)))
    assert b.frames_seen == 0
    b.set_state(state)
    assert b.frames_seen == 33
    for h in (a, other, b):
        h.close()
