"""The allocation-free motion estimate (vimg_motion_noalloc) against the
handle-based vimg_process on the same frames, and against the FP64 oracle at
its largest documented frame size.

Callers that cannot allocate device memory (real-time acquisition loops that
forbid allocator calls, hosts with every byte of device memory reserved for
their own buffers) use that entry point; its scratch is one fixed static
device array that every call shares.  Both paths run the same kernels, and the
aggregated surface is an exact fixed-point sum, so shifts and peak
information must be identical bit for bit.  This file is collected last so
that a failure here never hides another test, and it passes both alone in a
fresh process and after the whole suite."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2403_16438_gb300 import synth
from parity_util import compare_shifts

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _handle_path(vimg, H, W, td, fd):
    n = fd.shape[0]
    h = vimg.Handle(H, W)
    h.set_template(td)
    s = torch.zeros((n, 2), device=DEV)
    info = torch.zeros((n, 4), device=DEV)
    h.process(fd, shifts=s, peak_info=info)
    torch.cuda.synchronize()
    h.close()
    return s, info


def _noalloc(vimg, H, W, td, fd, stream):
    n = fd.shape[0]
    s = torch.full((n, 2), 99.0, device=DEV)
    info = torch.full((n, 4), -7.0, device=DEV)
    rc = vimg.lib.vimg_motion_noalloc(_p(td), _p(fd), n, H, W, 16, _p(s), _p(info),
                                      ctypes.c_void_p(stream.cuda_stream))
    assert rc == vimg.OK
    torch.cuda.synchronize()
    return s, info


def test_noalloc_matches_handle_path_on_two_calls_in_a_row():
    from paper_2403_16438_gb300 import vimg
    cfg = synth.tiny_config(seed=4242)
    frames, _, T = synth.make_video(cfg, 40)
    fd = frames.to(DEV)
    td = T.to(DEV)
    ref_s, ref_i = _handle_path(vimg, cfg.H, cfg.W, td, fd)
    stream = torch.cuda.current_stream()
    # two calls in a row share the static scratch (the second starts from what
    # the first left behind); each must equal the handle path exactly
    for lo, hi in [(0, 23), (23, 40)]:
        s, info = _noalloc(vimg, cfg.H, cfg.W, td, fd[lo:hi].contiguous(), stream)
        assert torch.equal(s, ref_s[lo:hi])
        assert torch.equal(info, ref_i[lo:hi])


def test_noalloc_at_its_largest_frame_size_against_the_oracle():
    """1024 x 1024 at R = 16, the documented limit: two frames per launch, so
    five frames take three launches that reuse the array."""
    from paper_2403_16438_gb300 import vimg
    cfg = synth.scaled_config(1024, 1024, 5, seed=78)
    frames, _, T = synth.make_video(cfg, 5)
    fd = frames.to(DEV)
    td = T.to(DEV)
    stream = torch.cuda.current_stream()
    first = _noalloc(vimg, 1024, 1024, td, fd, stream)
    second = _noalloc(vimg, 1024, 1024, td, fd, stream)
    assert torch.equal(first[0], second[0]) and torch.equal(first[1], second[1])
    ref_s, ref_i = _handle_path(vimg, 1024, 1024, td, fd)
    assert torch.equal(first[0], ref_s) and torch.equal(first[1], ref_i)
    o = oracle.Oracle(1024, 1024)
    o.set_template(T.double().numpy())
    r = o.process(frames.numpy(), want_corrected=False, want_summary=False)
    compare_shifts(first[0].cpu().numpy(), first[1].cpu().numpy(), r)


def test_noalloc_rejects_frames_beyond_its_scratch():
    from paper_2403_16438_gb300 import vimg
    dummy = torch.zeros(1, device=DEV)
    rc = vimg.lib.vimg_motion_noalloc(_p(dummy), _p(dummy), 1, 2048, 2048, 16, _p(dummy), None,
                                      None)
    assert rc == vimg.ERR_SIZE
    rc = vimg.lib.vimg_motion_noalloc(_p(dummy), _p(dummy), 1, 1025, 512, 16, _p(dummy), None,
                                      None)
    assert rc == vimg.ERR_SIZE
    rc = vimg.lib.vimg_motion_noalloc(_p(dummy), _p(dummy), 1, 40, 40, 16, _p(dummy), None, None)
    assert rc == vimg.ERR_SIZE
    assert np.isfinite(dummy.cpu().numpy()).all()  # nothing was enqueued on it
