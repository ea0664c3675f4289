"""Time shards of one video for several GPUs (or several handles on one GPU).

Frames are independent given the template (Sec. II: each frame is registered
to the template on its own), and the segment summaries of Sec. III-B cover
fixed ranges of L frames at absolute indices.  So a video cuts into
contiguous shards whose boundaries are multiples of L: no segment straddles
two shards, and nothing is exchanged per frame.  The one state that crosses a
boundary is the trailing high-pass window: a shard that starts at frame s > 0
re-reads the hp_window - 1 frames before s as history (vimg_seek / Handle.seek)
and discards their outputs.  The concatenated shifts, corrected frames,
segment summaries and traces then equal one stream over the whole video, bit
for bit.
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass(frozen=True)
class Shard:
    start: int       # first frame the shard outputs (a multiple of L, or 0)
    end: int         # one past its last frame
    hist_start: int  # first history frame it reads before `start`

    @property
    def frames(self) -> int:
        return self.end - self.start

    @property
    def history(self) -> int:
        return self.start - self.hist_start


def plan(n_frames: int, n_shards: int, segment_len: int = 50, hp_window: int = 0) -> list[Shard]:
    """Cuts frames [0, n_frames) into at most n_shards contiguous shards with
    boundaries on multiples of segment_len, as even as those allow: the
    ceil(n_frames / segment_len) segments (the last one possibly partial) are
    spread over the shards.  Shards that would be empty are dropped."""
    if n_frames < 0 or n_shards < 1 or segment_len < 1 or hp_window < 0:
        raise ValueError("bad shard request")
    units = -(-n_frames // segment_len)
    out = []
    start = 0
    for k in range(n_shards):
        # segments [k units / n, (k + 1) units / n) go to shard k
        end = min(n_frames, ((k + 1) * units) // n_shards * segment_len)
        if end > start:
            need = min(start, max(0, hp_window - 1))
            out.append(Shard(start, end, start - need))
        start = max(start, end)
    return out


def shard_of(shards: list[Shard], rank: int) -> Shard | None:
    """The rank's shard (None when the video has fewer shards than ranks)."""
    return shards[rank] if rank < len(shards) else None
