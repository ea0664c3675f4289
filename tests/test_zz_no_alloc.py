"""The allocation-free motion estimate (vimg_motion_noalloc) against the
handle-based vimg_process on the same frames.

Callers that cannot allocate device memory (inside a graph capture that must
not grow the pool, allocator-free acquisition loops, hosts with every byte
reserved) use that entry point; its scratch is a fixed static device array.
This file is collected last so that a failure here never hides another test,
and it passes both alone in a fresh process and after the whole suite."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2403_16438_gb300 import synth
from parity_util import SHIFT_TOL

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_handle_path_on_two_calls_in_a_row():
    from paper_2403_16438_gb300 import vimg
    cfg = synth.tiny_config(seed=4242)
    frames, _, T = synth.make_video(cfg, 40)
    fd = frames.to(DEV)
    td = T.to(DEV)
    stream = torch.cuda.current_stream()

    h = vimg.Handle(cfg.H, cfg.W)
    h.set_template(td)
    ref_s = torch.zeros((40, 2), device=DEV)
    ref_i = torch.zeros((40, 4), device=DEV)
    h.process(fd, shifts=ref_s, peak_info=ref_i)
    torch.cuda.synchronize()
    h.close()

    for lo, hi in [(0, 23), (23, 40)]:  # two calls in a row share the static scratch
        s = torch.full((hi - lo, 2), 99.0, device=DEV)
        info = torch.zeros((hi - lo, 4), device=DEV)
        rc = vimg.lib.vimg_motion_noalloc(_p(td), _p(fd[lo:hi]), hi - lo, cfg.H, cfg.W, 16,
                                          _p(s), _p(info), ctypes.c_void_p(stream.cuda_stream))
        assert rc == vimg.OK
        torch.cuda.synchronize()
        assert torch.equal(info[:, :2], ref_i[lo:hi, :2])  # integer peaks
        assert (s - ref_s[lo:hi]).abs().max().item() <= SHIFT_TOL
        np.testing.assert_allclose(info[:, 2].cpu().numpy(), ref_i[lo:hi, 2].cpu().numpy(),
                                   atol=1e-6)


def test_noalloc_rejects_frames_beyond_its_scratch():
    from paper_2403_16438_gb300 import vimg
    dummy = torch.zeros(1, device=DEV)
    rc = vimg.lib.vimg_motion_noalloc(_p(dummy), _p(dummy), 1, 2048, 2048, 16, _p(dummy), None,
                                      None)
    assert rc == vimg.ERR_SIZE
    rc = vimg.lib.vimg_motion_noalloc(_p(dummy), _p(dummy), 1, 40, 40, 16, _p(dummy), None, None)
    assert rc == vimg.ERR_SIZE
