"""Several videos per call (vimg_process_batch): one launch per kernel for the
videos of a step must give, bit for bit, what vimg_process gives per video;
the CUDA-graph form must give the same; rotating output slots, groups of more
than 8 videos and argument checks.  One video is also checked against the
FP64 oracle directly."""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_16438_gb300 import synth
from parity_util import NEAR_TIE, SHIFT_TOL, compare_images

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

# uneven sizes, ragged frame counts (not multiples of L = 50)
SIZES = [(96, 128, 130), (128, 96, 75), (160, 160, 61), (90, 110, 101)]


@pytest.fixture(scope="module")
def vimg():
    from paper_2403_16438_gb300 import vimg as v
    return v


@pytest.fixture(scope="module")
def videos():
    out = []
    for i, (H, W, n) in enumerate(SIZES):
        cfg = synth.scaled_config(H, W, n, seed=5000 + i, clamp=6.0)
        f, planted, T = synth.make_video(cfg, n, device=DEV)
        out.append((f, T))
    return out


def _outputs(H, W, n, L=50, ring=None):
    frames_out = n if ring is None else ring
    return (torch.full((n, 2), float("nan"), device=DEV),
            torch.full((frames_out, H, W), float("nan"), device=DEV),
            torch.full((max(1, n // L), 2, H, W), float("nan"), device=DEV))


def _handles(vimg, videos, **kw):
    hs = []
    for f, T in videos:
        h = vimg.Handle(f.shape[1], f.shape[2], **kw)
        h.set_template(T)
        hs.append(h)
    return hs


def _single(vimg, videos, **kw):
    res = []
    for f, T in videos:
        n, H, W = f.shape
        h = vimg.Handle(H, W, **kw)
        h.set_template(T)
        s, c, m = _outputs(H, W, n)
        k = h.process(f, shifts=s, corrected=c, summary=m)
        torch.cuda.synchronize()
        res.append((s, c, m[:k], k))
        h.close()
    return res


def _batched(vimg, videos, chunk, use_graph=False, calls=1, **kw):
    hs = _handles(vimg, videos, **kw)
    outs = [_outputs(f.shape[1], f.shape[2], f.shape[0]) for f, _ in videos]
    segs = None
    for _ in range(calls):
        for h in hs:
            h.reset()
        for o in outs:
            for t in o:
                t.fill_(float("nan"))
        segs = vimg.process_batch(hs, [f for f, _ in videos], shifts=[o[0] for o in outs],
                                  corrected=[o[1] for o in outs], summary=[o[2] for o in outs],
                                  chunk=chunk, use_graph=use_graph)
    torch.cuda.synchronize()
    for h in hs:
        h.close()
    return [(o[0], o[1], o[2][:k], k) for o, k in zip(outs, segs)]


def _assert_same(a, b):
    for (s1, c1, m1, k1), (s2, c2, m2, k2) in zip(a, b):
        assert k1 == k2
        assert torch.equal(s1, s2)
        assert torch.equal(c1, c2)
        assert torch.equal(m1, m2)


@pytest.mark.parametrize("chunk", [32, 64, 128])
def test_batch_equals_per_video(vimg, videos, chunk):
    ref = _single(vimg, videos)
    got = _batched(vimg, videos, chunk)
    _assert_same(got, ref)


def test_batch_highpass_equals_per_video(vimg, videos):
    kw = dict(hp_window=9, flags=vimg.OUT_HIGHPASS)
    ref = _single(vimg, videos, **kw)
    got = _batched(vimg, videos, 40, **kw)
    _assert_same(got, ref)


def test_graph_replay_equals_direct(vimg, videos):
    ref = _batched(vimg, videos, 64)
    # first call captures and launches the graph, the second replays it
    got = _batched(vimg, videos, 64, use_graph=True, calls=2)
    _assert_same(got, ref)


def test_ring_slots(vimg, videos):
    chunk, ring = 50, 2
    ref = _single(vimg, videos)
    hs = _handles(vimg, videos)
    rings = [torch.full((ring * chunk, f.shape[1], f.shape[2]), float("nan"), device=DEV)
             for f, _ in videos]
    vimg.process_batch(hs, [f for f, _ in videos], corrected=rings, chunk=chunk,
                       ring_chunks=ring)
    torch.cuda.synchronize()
    for (f, _), r, (s, c, m, k) in zip(videos, rings, ref):
        n = f.shape[0]
        steps = (n + chunk - 1) // chunk
        # the last `ring` steps are still in the ring
        for st in range(max(0, steps - ring), steps):
            a, b = st * chunk, min(n, (st + 1) * chunk)
            slot = (st % ring) * chunk
            assert torch.equal(r[slot:slot + b - a], c[a:b])
    for h in hs:
        h.close()


def test_more_videos_than_one_launch_holds(vimg):
    vids = []
    for i in range(10):
        H, W = 80 + 4 * i, 96 - 2 * i
        cfg = synth.scaled_config(H, W, 55, seed=6000 + i, clamp=5.0)
        f, _, T = synth.make_video(cfg, 55, device=DEV)
        vids.append((f, T))
    _assert_same(_batched(vimg, vids, 50), _single(vimg, vids))


def test_batch_against_oracle(vimg, videos):
    f, T = videos[2]
    s, c, m, k = _batched(vimg, [videos[0], videos[2]], 64)[1]
    o = oracle.Oracle(f.shape[1], f.shape[2], R=16)
    o.set_template(T.cpu().double().numpy())
    r = o.process(f.cpu().numpy())
    near = (r["info"][:, 0] - r["info"][:, 1]) < NEAR_TIE
    err = np.abs(s.cpu().numpy() - r["shifts"])[~near].max()
    assert err <= SHIFT_TOL, err
    compare_images(c.cpu().numpy(), r["corrected"], "corrected")
    assert k == r["summary"].shape[0]
    compare_images(m.cpu().numpy().reshape(-1, f.shape[1], f.shape[2]),
                   r["summary"].reshape(-1, f.shape[1], f.shape[2]), "summary")


def test_batch_argument_checks(vimg, videos):
    f, T = videos[0]
    h1 = vimg.Handle(f.shape[1], f.shape[2])
    h1.set_template(T)
    hb = vimg.Handle(f.shape[1], f.shape[2], flags=vimg.CORR_BF16)
    with pytest.raises(vimg.VimgError):
        vimg.process_batch([h1, h1], [f, f])  # repeated handle
    with pytest.raises(vimg.VimgError):
        vimg.process_batch([h1], [f], chunk=h1.params.max_chunk + 1)
    hb.set_template(T)
    with pytest.raises(vimg.VimgError):
        vimg.process_batch([h1, hb], [f, f])  # tensor-core handles are per-video only
    h2 = vimg.Handle(f.shape[1], f.shape[2])  # no template
    with pytest.raises(vimg.VimgError):
        vimg.process_batch([h1, h2], [f, f])
    for h in (h1, hb, h2):
        h.close()
