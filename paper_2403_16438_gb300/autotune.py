"""Autotuner of the batched path's step shape.

The batched call (vimg_process_batch) advances all videos together in steps of
`chunk` frames per video; the step is the time extent of every launch (frames
per window-statistics, correlation, peak and temporal launch), so it sets how
full the GPU is at the end of each launch, how much of a step's frames are
still in L2 when the temporal pass re-reads them, and how many launches the
whole call makes.  Candidates are the chunk sizes {64, 128, 256, 512}
(shortened by the library to end on segment boundaries), each with and
without CUDA-graph replay.

The one spatial tile shape with a choice is the FP32 correlation's patch group
(vimg_params.corr_group: patches per work item, 11, 10, 8 or 7): a row of nx
patches takes ceil(nx / g) items, so the best g depends on the frame width (22
patches per row fill groups of 11, 35 fill groups of 7), while smaller groups
spend more of each item on its shared region and its 33rd-row warp.
`tune_groups` times the correlation stage of every video with every group size
on a probe and picks the fastest per video; the other kernels' tiles are fixed
by their shared-memory and tensor-memory budgets.

`tune` is the pure selection (any `run(candidate) -> seconds`); `tune_batch`
times candidates on the device with CUDA events on a probe prefix of the
videos; `load`/`store` keep the choice per device and video set in a JSON file.
"""
from __future__ import annotations

import json
import os

CHUNKS = (64, 128, 256, 512)
GROUPS = (11, 10, 8, 7)


def candidates(max_chunk: int, chunks=CHUNKS, graphs=(False, True)):
    """(chunk, use_graph) pairs allowed by the handles' workspace size."""
    return [(c, g) for c in chunks if c <= max_chunk for g in graphs]


def pick(timings: dict):
    """Fastest candidate; ties go to the smaller chunk, then to no graph."""
    if not timings:
        raise ValueError("no timings")
    return min(timings, key=lambda c: (timings[c], c[0], c[1]))


def tune(cands, run, reps: int = 2):
    """Times every candidate `reps` times (best of) and returns (best, table)."""
    table = {}
    for c in cands:
        table[c] = min(run(c) for _ in range(reps))
    return pick(table), table


def key_of(device_name: str, shapes) -> str:
    """Cache key: device and the (H, W, frames) of every video."""
    return device_name + "|" + ";".join(f"{H}x{W}x{n}" for H, W, n in shapes)


def load(path: str, key: str):
    try:
        with open(path) as f:
            c = json.load(f).get(key)
    except (OSError, ValueError):
        return None
    return None if c is None else (int(c["chunk"]), bool(c["use_graph"]))


def store(path: str, key: str, choice, table=None):
    data = {}
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        data = {}
    entry = {"chunk": int(choice[0]), "use_graph": bool(choice[1])}
    if table:
        entry["seconds"] = {f"{c}/{'graph' if g else 'direct'}": t for (c, g), t in table.items()}
    data[key] = entry
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune_batch(handles, frames, probe_frames: int = 500, reps: int = 2, chunks=CHUNKS,
               outputs=None, cache_path: str | None = None):
    """Picks (chunk, use_graph) for these handles by timing the batched call on
    the first `probe_frames` frames of every video (same work for every
    candidate).  outputs: dict of per-video lists for process_batch (shifts,
    corrected, summary) sized for the probe; the corrected buffers may be rings
    of 2 slots of the largest chunk.  Returns (choice, table)."""
    import torch

    from . import vimg

    dev = torch.cuda.current_device()
    shapes = [(h.H, h.W, int(f.shape[0])) for h, f in zip(handles, frames)]
    key = key_of(torch.cuda.get_device_name(dev), shapes)
    if cache_path:
        hit = load(cache_path, key)
        if hit is not None:
            return hit, None
    probe = [f[:min(probe_frames, f.shape[0])] for f in frames]
    outputs = outputs or {}
    stream = handles[0].stream
    max_chunk = min(h.params.max_chunk for h in handles)

    def run(c):
        chunk, graph = c
        for h in handles:
            h.reset()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ring = 2 if outputs.get("corrected") is not None else 0
        e0.record(stream)
        vimg.process_batch(handles, probe, chunk=chunk, use_graph=graph, ring_chunks=ring,
                           **outputs)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / 1000.0

    cands = candidates(max_chunk, chunks)
    for c in cands:  # warm-up (and graph capture) of every candidate
        run(c)
    choice, table = tune(cands, run, reps)
    for h in handles:
        h.reset()
    if cache_path:
        store(cache_path, key, choice, table)
    return choice, table


def pick_group(timings: dict) -> int:
    """Fastest group size; ties go to the larger group."""
    if not timings:
        raise ValueError("no timings")
    return min(timings, key=lambda g: (timings[g], -g))


def tune_groups(frames, templates, probe_frames: int = 200, groups=GROUPS, reps: int = 2,
                stream=None):
    """Per video, the correlation group size whose correlation stage (CUDA
    events around its launches, vimg_profile_*) is fastest on the first
    `probe_frames` frames.  frames: list of cuda uint16 [n, H, W]; templates:
    list of cuda float32 [H, W].  Returns (groups per video, {video: {g: s}})."""
    import torch

    from . import vimg

    chosen, table = [], {}
    for i, (f, T) in enumerate(zip(frames, templates)):
        probe = f[:min(probe_frames, f.shape[0])]
        times = {}
        for g in groups:
            h = vimg.Handle(f.shape[1], f.shape[2], stream=stream, max_chunk=probe.shape[0],
                            corr_group=g)
            h.set_template(T)
            h.process(probe)  # warm-up
            h.profile(True)
            best = None
            for _ in range(reps):
                h.profile_read(reset=True)
                h.reset()
                h.process(probe)
                ms = h.profile_read(reset=True)["corr"][0]
                best = ms if best is None else min(best, ms)
            h.profile(False)
            torch.cuda.synchronize()
            h.close()
            times[g] = best / 1000.0
        chosen.append(pick_group(times))
        table[i] = times
    return chosen, table
