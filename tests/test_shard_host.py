"""Time shards of one video (paper_2403_16438_gb300.shard) on CPU: the planner's
cuts, the FP64 oracle's seek (a stream that starts at an absolute frame index
with high-pass history) against one stream over the whole video, and two gloo
ranks that each run the oracle on their shard -- the concatenated shifts,
corrected (high-passed) frames and segment summaries equal the one-rank run
bit for bit."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2403_16438_gb300 import shard, synth  # noqa: E402

HP = 7  # high-pass window of the shard tests (its history crosses shard cuts)


@pytest.mark.parametrize("n,k,L,hp", [(10000, 8, 50, 0), (10000, 3, 50, 9), (120, 2, 50, 7),
                                      (37, 4, 50, 0), (500, 7, 50, 64), (1000, 1, 50, 5),
                                      (230, 5, 7, 3)])
def test_plan_cuts_on_segment_boundaries(n, k, L, hp):
    s = shard.plan(n, k, L, hp)
    assert 1 <= len(s) <= k
    assert s[0].start == 0 and s[-1].end == n
    for a, b in zip(s, s[1:]):
        assert a.end == b.start                       # contiguous, no overlap
    for x in s:
        assert x.start % L == 0 and x.frames > 0      # whole segments
        assert x.history == min(x.start, max(0, hp - 1))
    units = [-(-x.frames // L) for x in s]
    assert max(units) - min(units) <= 1                # as even as whole segments allow
    assert len(s) == min(k, -(-n // L))


def test_plan_rejects_bad_requests():
    for args in [(-1, 2), (10, 0), (10, 2, 0), (10, 2, 50, -1)]:
        with pytest.raises(ValueError):
            shard.plan(*args)
    assert shard.shard_of(shard.plan(40, 4), 3) is None  # fewer segments than ranks


def _video(n=120):
    cfg = synth.tiny_config(seed=31)
    frames, _, T = synth.make_video(cfg, n)
    return cfg, frames.numpy(), T.double().numpy()


def _oracle_run(cfg, frames, T, sh):
    o = oracle.Oracle(cfg.H, cfg.W, hp_window=HP, flags=oracle.FLAG_OUT_HIGHPASS)
    o.set_template(T)
    o.seek(sh.start, frames[sh.hist_start:sh.start])
    r = o.process(frames[sh.start:sh.end])
    return r["shifts"], r["corrected"], r["summary"]


def test_oracle_seek_equals_one_stream():
    """Pins the oracle's seek to its own one-stream run: the shard after a cut
    reproduces that run's outputs exactly (shifts, high-passed frames, the
    segments after the cut)."""
    cfg, frames, T = _video()
    o = oracle.Oracle(cfg.H, cfg.W, hp_window=HP, flags=oracle.FLAG_OUT_HIGHPASS)
    o.set_template(T)
    full = o.process(frames)
    s, c, m = _oracle_run(cfg, frames, T, shard.Shard(50, 120, 50 - (HP - 1)))
    assert np.array_equal(s, full["shifts"][50:])
    assert np.array_equal(c, full["corrected"][50:])
    assert np.array_equal(m, full["summary"][1:])
    # too short a history changes the high-pass of the first frames: the seek
    # is not a no-op, the history matters
    s2, c2, _ = _oracle_run(cfg, frames, T, shard.Shard(50, 120, 50 - 2))
    assert np.array_equal(s2, s) and not np.array_equal(c2[:HP], c[:HP])
    with pytest.raises(ValueError):
        o.seek(49, frames[:49])  # not on a segment boundary


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), OMP_NUM_THREADS="2")
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    cfg, frames, T = _video()
    sh = shard.shard_of(shard.plan(frames.shape[0], ws, 50, HP), rank)
    res = _oracle_run(cfg, frames, T, sh)
    gathered = [None] * ws
    dist.all_gather_object(gathered, res)  # the host-side concatenation
    if rank == 0:
        out["shifts"] = np.concatenate([g[0] for g in gathered])
        out["corrected"] = np.concatenate([g[1] for g in gathered])
        out["summary"] = np.concatenate([g[2] for g in gathered])
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_one_rank_run():
    cfg, frames, T = _video()
    o = oracle.Oracle(cfg.H, cfg.W, hp_window=HP, flags=oracle.FLAG_OUT_HIGHPASS)
    o.set_template(T)
    full = o.process(frames)
    ws = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(ws, _free_port(), out), nprocs=ws, join=True)
        for key in ("shifts", "corrected", "summary"):
            assert np.array_equal(out[key], full[key]), key
