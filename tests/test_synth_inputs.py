"""The seeded input generator against the workload recipes it stands in for
(CPU).  The configs carry the stated parameters; the drawn scenes, drift,
activity and noise follow them statistically; a frame shows the scene moved by
its planted shift; and the same seed gives the same video."""
import math

import numpy as np
import pytest
import torch

from paper_2403_16438_gb300 import synth


def test_configs_carry_the_workload_recipes():
    t = synth.tiny_config()
    assert (t.H, t.W, t.n_frames, t.fps, t.n_neurons) == (128, 128, 1000, 741.0, 8)
    assert (t.r_lo, t.r_hi, t.overlap_max, t.bg_amp) == (4.0, 8.0, 0.30, 2000.0)
    assert (t.rate_lo, t.rate_hi, t.dff_lo, t.dff_hi, t.decay) == (10.0, 10.0, 0.05, 0.05, 3.0)
    assert (t.read_sigma, t.walk_sigma, t.clamp, t.jump_frac) == (20.0, 0.3, 8.0, 0.0)
    p = synth.paper_scale_config()
    assert (p.H, p.W, p.n_frames, p.fps, p.n_neurons) == (512, 512, 10000, 741.0, 40)
    assert (p.r_lo, p.r_hi, p.overlap_max, p.bg_amp) == (5.0, 10.0, 0.40, 4000.0)
    assert (p.rate_lo, p.rate_hi, p.dff_lo, p.dff_hi) == (5.0, 20.0, 0.02, 0.08)
    assert (p.read_sigma, p.walk_sigma, p.clamp, p.jump_frac, p.jump_px) == (30.0, 0.5, 12.0, 0.01, 3.0)
    s = synth.scaled_config(1024, 1024, 5000, seed=5)
    assert s.n_neurons == 160 and (s.H, s.W, s.n_frames) == (1024, 1024, 5000)


def test_scenes_respect_count_radii_overlap_and_ranges():
    for cfg in (synth.tiny_config(), synth.paper_scale_config()):
        sc = synth.make_scene(cfg, torch.Generator().manual_seed(cfg.seed))
        assert len(sc.neurons) == cfg.n_neurons
        for (cy, cx, a, b, th, f0) in sc.neurons:
            assert cfg.r_lo * 0.85 <= a <= cfg.r_hi * 1.15 and cfg.r_lo * 0.85 <= b <= cfg.r_hi * 1.15
            m = max(a, b) + 2
            assert m <= cy <= cfg.H - m and m <= cx <= cfg.W - m
            assert f0 == 0.25 * cfg.bg_amp
        for i, (y1, x1, a1, b1, _, _) in enumerate(sc.neurons):
            for (y2, x2, a2, b2, _, _) in sc.neurons[:i]:
                ov = synth._disc_overlap(math.sqrt(a1 * b1), math.sqrt(a2 * b2), math.hypot(y1 - y2, x1 - x2))
                assert ov <= cfg.overlap_max + 1e-12
        assert all(cfg.rate_lo <= r <= cfg.rate_hi for r in sc.rates)
        assert all(cfg.dff_lo <= d <= cfg.dff_hi for d in sc.dffs)


def test_disc_overlap_closed_forms():
    assert synth._disc_overlap(3.0, 2.0, 5.0) == 0.0      # touching
    assert synth._disc_overlap(3.0, 1.0, 1.5) == 1.0      # contained
    # equal discs at distance r: lens area 2 r^2 acos(1/2) - (r^2 / 2) sqrt(3)
    r = 2.0
    lens = 2 * r * r * math.acos(0.5) - 0.5 * r * r * math.sqrt(3)
    assert abs(synth._disc_overlap(r, r, r) - lens / (math.pi * r * r)) < 1e-12


def test_drift_walk_clamp_and_jumps():
    p = synth.paper_scale_config()
    s = synth.planted_shifts(p, 10000, torch.Generator().manual_seed(3)).numpy()
    assert np.abs(s).max() <= p.clamp and np.all(s[0] == 0)
    d = np.diff(s, axis=0)
    free = np.all(np.abs(s[1:]) < p.clamp, axis=1) & np.all(np.abs(s[:-1]) < p.clamp, axis=1)
    mag = np.hypot(d[:, 0], d[:, 1])
    jumps = (mag > 2.2) & free
    n_free = int(free.sum())
    # 1 % of frames jump by 3 px in a random direction (binomial, +-5 sd)
    exp = p.jump_frac * n_free
    assert abs(jumps.sum() - exp) <= 5 * math.sqrt(exp), (jumps.sum(), exp)
    steps = d[free & ~(mag > 2.2)]
    assert abs(steps.std() - p.walk_sigma) < 0.05 * p.walk_sigma
    t = synth.tiny_config()
    st = synth.planted_shifts(t, 5000, torch.Generator().manual_seed(4)).numpy()
    dt = np.diff(st, axis=0)
    ok = np.all(np.abs(st[1:]) < t.clamp, axis=1) & np.all(np.abs(st[:-1]) < t.clamp, axis=1)
    assert np.abs(st).max() <= t.clamp
    assert abs(dt[ok].std() - t.walk_sigma) < 0.05 * t.walk_sigma
    assert np.hypot(dt[:, 0], dt[:, 1]).max() < 2.0  # no jumps in the tiny recipe


def test_activity_is_poisson_spikes_with_three_frame_decay():
    p = synth.paper_scale_config()
    sc = synth.make_scene(p, torch.Generator().manual_seed(p.seed))
    n = 10000
    act = synth.activity(sc, n, torch.Generator().manual_seed(9)).double().numpy()
    dff = np.array(sc.dffs)
    cur = act / dff
    dec = math.exp(-1.0 / p.decay)
    spikes = cur.copy()
    spikes[1:] -= dec * cur[:-1]
    # recovered spike counts are non-negative integers
    assert np.abs(spikes - np.round(spikes)).max() < 1e-3 and spikes.min() > -1e-3
    counts = np.round(spikes).sum(axis=0)
    expect = np.array(sc.rates) / p.fps * n
    assert np.all(np.abs(counts - expect) <= 5 * np.sqrt(expect) + 1), (counts, expect)
    # a single spike decays by exp(-1/3) per frame
    one = synth.Scene(p, sc.bg, sc.neurons[:1], [p.fps], [1.0])
    a1 = synth.activity(one, 40, torch.Generator().manual_seed(1)).double().numpy()[:, 0]
    s1 = a1.copy()
    s1[1:] -= dec * a1[:-1]
    assert np.abs(s1 - np.round(s1)).max() < 1e-3


def test_noise_model_shot_plus_read():
    g = torch.Generator().manual_seed(5)
    e = torch.full((200, 64, 64), 1000.0)
    f = synth.add_noise(e, 20.0, g).to(torch.int32).double()
    assert abs(f.mean().item() - 1000.0) < 1.0
    assert abs(f.var().item() / (1000.0 + 400.0) - 1.0) < 0.02
    hi = synth.add_noise(torch.full((4, 8, 8), 70000.0), 20.0, g).to(torch.int32)
    lo = synth.add_noise(torch.full((4, 8, 8), -50.0), 20.0, g).to(torch.int32)
    assert int(hi.min()) == 65535 and int(lo.max()) <= 100 and int(lo.min()) >= 0


def test_frame_shows_the_scene_moved_by_its_planted_shift():
    """Frame t is Scene(x - s_t): with an integer shift the rendered frame is
    the unshifted render moved by s_t (interior pixels, no noise)."""
    cfg = synth.tiny_config()
    sc = synth.make_scene(cfg, torch.Generator().manual_seed(cfg.seed))
    act = torch.zeros((2, len(sc.neurons)))
    sh = torch.tensor([[0.0, 0.0], [3.0, -5.0]], dtype=torch.float64)
    out = synth.render(sc, sh, act, "cpu", margin_px=12).double()
    a, b = out[0], out[1]
    # b[y, x] = a[y - 3, x + 5]
    assert torch.allclose(b[3:, :-5], a[:-3, 5:], rtol=0, atol=1e-2)


def test_same_seed_same_video():
    cfg = synth.tiny_config()
    f1, s1, t1 = synth.make_video(cfg, 12)
    f2, s2, t2 = synth.make_video(cfg, 12)
    assert torch.equal(f1.to(torch.int32), f2.to(torch.int32)) and torch.equal(s1, s2)
    assert torch.equal(t1, t2)
    f3, s3, _ = synth.make_video(synth.tiny_config(seed=7), 12)
    assert not torch.equal(f1.to(torch.int32), f3.to(torch.int32)) and not torch.equal(s1, s3)


def test_frame_range_of_one_video():
    """make_video_range: the planted drift of a range is that slice of the whole
    video's drift, the template does not depend on the range, and frames of a
    range follow the same content (mean counts close to the whole video's)."""
    cfg = synth.tiny_config(seed=77)
    n = 240
    _, full_shifts, _ = synth.ground_truth(cfg, n)
    f0, s0, T0 = synth.make_video_range(cfg, n, 0, 100)
    f1, s1, T1 = synth.make_video_range(cfg, n, 100, 240)
    assert torch.equal(s0, full_shifts[:100]) and torch.equal(s1, full_shifts[100:])
    assert torch.equal(T0, T1)
    ref, _, _ = synth.make_video(cfg, n)
    m_ref = ref.double().mean().item()
    assert abs(f1.double().mean().item() - m_ref) < 0.02 * m_ref
    with pytest.raises(ValueError):
        synth.make_video_range(cfg, n, 200, 100)
