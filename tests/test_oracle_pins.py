"""Pins of the FP64 oracle against facts fixed outside the oracle itself:
library routines for the special cases they cover (Pearson correlation,
scipy's Gaussian filter and linear spline shift, numpy's median), closed
forms (filter impulse and sinusoid responses, quadratic peaks, spike
responses), invariants (affine invariance, self-registration, exact
copies), and brute force on tiny inputs.  Each test names the passage of the
paper (Bando et al., BIBM 2023) or the reading it pins.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import ndimage

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rng(seed=0):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- constants
def test_paper_constants_fixture():
    """Sec. II: 21x21 patches; Sec. III-B: L = 50, sigma = 3 px."""
    with open(os.path.join(GOLDEN, "paper_constants.json")) as f:
        c = json.load(f)
    assert c["patch"]["value"] == 21
    assert c["segment_len"]["value"] == 50
    assert c["gauss_sigma"]["value"] == 3.0
    # Fig. 1: 10,000 frames recorded in 13.5 s at 741 fps.
    fig1 = c["fig1_timings"]
    assert abs(fig1["frames"] / fig1["fps"] - fig1["recording_s"]) < 0.05
    assert abs(sum(fig1["stage_s"]) - fig1["total_s"]) < 1e-9


# ---------------------------------------------------------------- patch grid
def test_patch_grid_hand_values():
    # (512-32)=480 -> 22 patches (462 px), 18 px left -> 9 each side -> y0 = 16+9.
    assert oracle.patch_grid(512, 512, 16) == (22, 22, 25, 25)
    # (128-32)=96 -> 4 patches (84), 12 left -> y0 = 16+6.
    assert oracle.patch_grid(128, 128, 16) == (4, 4, 22, 22)
    # The paper's 450x138 video: 106 -> 5 (105) -> y0=16; 418 -> 19 (399) -> x0=16+9.
    assert oracle.patch_grid(138, 450, 16) == (5, 19, 16, 25)
    with pytest.raises(ValueError):
        oracle.patch_grid(52, 512, 16)


@pytest.mark.parametrize("H,W,R", [(53, 53, 16), (100, 77, 5), (257, 300, 16), (64, 64, 0)])
def test_patch_grid_windows_in_bounds(H, W, R):
    ny, nx, y0, x0 = oracle.patch_grid(H, W, R)
    assert y0 - R >= 0 and x0 - R >= 0
    assert y0 + ny * 21 + R <= H and x0 + nx * 21 + R <= W
    assert (H - 2 * R) // 21 == ny  # as many patches as fit


# ---------------------------------------------------------------- ZNCC
def test_zncc_is_pearson_correlation():
    """Sec. II ZNCC == Pearson correlation coefficient (numpy's corrcoef)."""
    r = rng(1)
    F = r.integers(0, 4000, (70, 80)).astype(np.uint16)
    T = r.normal(1000, 300, (70, 80))
    for (ty, tx, dy, dx) in [(20, 25, 0, 0), (20, 25, -3, 4), (10, 30, 5, -7), (25, 20, 2, 2)]:
        a = T[ty:ty + 21, tx:tx + 21].ravel()
        b = F[ty + dy:ty + dy + 21, tx + dx:tx + dx + 21].astype(float).ravel()
        ref = np.corrcoef(a, b)[0, 1]
        assert abs(oracle.zncc(F, T, ty, tx, 21, dy, dx) - ref) < 1e-12


def test_zncc_invariants():
    r = rng(2)
    F = r.integers(0, 1000, (60, 60)).astype(np.uint16)
    T = F.astype(float)  # exact copy at d = 0
    assert abs(oracle.zncc(F, T, 20, 20, 21, 0, 0) - 1.0) < 1e-12
    # affine invariance: ZNCC(aF + b) = ZNCC(F) for a > 0
    G = (3 * F.astype(np.int64) + 100).astype(np.uint16)
    Tn = r.normal(0, 1, (60, 60))
    for d in [(0, 0), (3, -2), (-5, 5)]:
        z1 = oracle.zncc(F, Tn, 20, 20, 21, *d)
        z2 = oracle.zncc(G, Tn, 20, 20, 21, *d)
        assert abs(z1 - z2) < 1e-12 and -1 - 1e-12 <= z1 <= 1 + 1e-12
    # a negated pattern correlates at -1
    Tneg = -F.astype(float)
    assert abs(oracle.zncc(F, Tneg, 20, 20, 21, 0, 0) + 1.0) < 1e-12
    # zero-variance window or patch -> 0 (reading)
    C = np.full((60, 60), 7, np.uint16)
    assert oracle.zncc(C, Tn, 20, 20, 21, 1, 1) == 0.0
    assert oracle.zncc(F, np.ones((60, 60)), 20, 20, 21, 1, 1) == 0.0


def test_surface_brute_force_tiny():
    """Aggregated surface = mean over patches (reading of Sec. II) of the
    per-patch Pearson correlation, by brute force over every displacement."""
    r = rng(3)
    H, W, R = 58, 62, 4
    F = r.integers(0, 3000, (H, W)).astype(np.uint16)
    T = ndimage.uniform_filter(r.normal(0, 1, (H, W)), 3) * 500 + 2000
    ny, nx, y0, x0 = oracle.patch_grid(H, W, R)
    C, Z = oracle.surface(F, T, R, per_patch=True)
    ref = np.zeros((2 * R + 1, 2 * R + 1))
    for py in range(ny):
        for px in range(nx):
            ty, tx = y0 + 21 * py, x0 + 21 * px
            a = T[ty:ty + 21, tx:tx + 21].ravel()
            for dy in range(-R, R + 1):
                for dx in range(-R, R + 1):
                    b = F[ty + dy:ty + dy + 21, tx + dx:tx + dx + 21].astype(float).ravel()
                    z = np.corrcoef(a, b)[0, 1]
                    assert abs(Z[py * nx + px, dy + R, dx + R] - z) < 1e-12
                    ref[dy + R, dx + R] += z
    ref /= ny * nx
    assert np.max(np.abs(C - ref)) < 1e-12
    # a sub-window reproduces the same values (narrow windows equal full ones)
    Cw = oracle.surface(F, T, R, window=(-1, 2, 3, 2))
    assert np.array_equal(Cw, C[-1 + R:2 + R, 2 + R:4 + R])


# ---------------------------------------------------------------- peak
def _texture(shape, seed):
    r = rng(seed)
    return ndimage.gaussian_filter(r.normal(0, 1, shape), 1.5) * 800 + 3000


def test_self_registration_zero_shift():
    T = _texture((96, 96), 4)
    F = np.round(T).astype(np.uint16)
    C = oracle.surface(F, np.round(T), 8)
    s, d, info = oracle.peak(C, -8, -8)
    assert tuple(d) == (0, 0)
    assert abs(info[0] - 1.0) < 1e-12
    assert np.all(np.abs(s) < 0.5)


@pytest.mark.parametrize("sy,sx", [(3, -5), (-8, 8), (0, 1), (-2, -7)])
def test_planted_integer_shift_noise_free(sy, sx):
    """F(x) = T(x - s): the window at d = s is an exact copy -> ZNCC = 1,
    the unique maximum, so d* = s exactly (test (a) of the oracle plan)."""
    m = 10
    S = np.round(_texture((80 + 2 * m, 84 + 2 * m), 5))
    T = S[m:m + 80, m:m + 84]
    F = S[m - sy:m - sy + 80, m - sx:m - sx + 84].astype(np.uint16)
    C = oracle.surface(F, T, 8)
    s, d, info = oracle.peak(C, -8, -8)
    assert tuple(d) == (sy, sx)
    assert abs(info[0] - 1.0) < 1e-12 and info[1] < 1.0 - 1e-3


def test_narrow_center_rounding_and_clamp():
    """Round to nearest, halves to even (as the proposal is rounded on the GPU);
    clamp so the 7x7 window stays in [-R, R]; non-finite -> 0."""
    c = oracle.narrow_center
    assert c((2.5, -2.5), 16) == (2, -2) and c((3.5, -0.49), 16) == (4, 0)
    assert c((14.0, -30.0), 16) == (13, -13) and c((float("nan"), float("inf")), 16) == (0, 0)
    assert c((1.6, 5.0), 4) == (1, 1)


def test_narrow_window_agrees_with_the_full_window_near_the_truth():
    """Noise-free integer shift with a proposal within 2 px of it: the full
    window's peak lies inside the narrow window, off its border, so the narrow
    estimate uses the same three values per axis as the full window and gives
    its shift exactly, without falling back."""
    m = 12
    S = np.round(_texture((90 + 2 * m, 94 + 2 * m), 9))
    T = S[m:m + 90, m:m + 94]
    for (sy, sx), prop in [((3, -5), (4.2, -3.6)), ((-6, 7), (-6.4, 8.9)), ((0, 0), (1.1, 0.3))]:
        F = S[m - sy:m - sy + 90, m - sx:m - sx + 94].astype(np.uint16)
        r = oracle.narrow_estimate(F, T, 10, prop)
        C = oracle.surface(F, T, 10)
        s, d, info = oracle.peak(C, -10, -10)
        assert not r["fallback"] and tuple(r["dstar"]) == (sy, sx) == tuple(d)
        assert np.array_equal(r["shifts"], s)
        cy, cx = r["center"]
        assert np.array_equal(r["narrow"], C[cy - 3 + 10:cy + 4 + 10, cx - 3 + 10:cx + 4 + 10])


def test_narrow_window_falls_back_far_from_the_truth_or_below_threshold():
    """A proposal 7 px off puts the narrow peak on the window border (the
    surface rises towards the true shift); a threshold above 1 rejects every
    peak: both fall back to exactly the full window's estimate."""
    m = 12
    S = np.round(_texture((90 + 2 * m, 94 + 2 * m), 10))
    T = S[m:m + 90, m:m + 94]
    F = S[m - 4:m - 4 + 90, m + 2:m + 2 + 94].astype(np.uint16)
    s, d, info = oracle.peak(oracle.surface(F, T, 10), -10, -10)
    for prop, thr in [((-3.0, -2.0), 0.5), ((4.0, -2.0), 1.01)]:
        r = oracle.narrow_estimate(F, T, 10, prop, thresh=thr)
        assert r["fallback"] and tuple(r["dstar"]) == (4, -2) == tuple(d)
        assert np.array_equal(r["shifts"], s)
    r = oracle.narrow_estimate(F, T, 10, (4.0, -2.0), thresh=0.5)
    assert not r["fallback"] and tuple(r["dstar"]) == (4, -2)


def test_constant_frame_gives_zero_surface_and_origin():
    F = np.full((64, 64), 1234, np.uint16)
    C = oracle.surface(F, _texture((64, 64), 6), 5)
    assert np.all(C == 0.0)
    s, d, info = oracle.peak(C, -5, -5)
    assert tuple(d) == (0, 0) and tuple(s) == (0.0, 0.0)


def test_tie_break_rule():
    """Reading: exact ties -> smallest dy^2+dx^2, then smallest dy, then dx."""
    R = 4
    C = np.zeros((9, 9))
    for (dy, dx) in [(0, 3), (2, 1), (1, -2), (-1, 2), (-2, 1), (-2, -1)]:
        C[dy + R, dx + R] = 0.75
    s, d, info = oracle.peak(C, -R, -R)
    assert tuple(d) == (-2, -1)


def test_parabola_exact_on_separable_quadratic():
    """Reading of the subpixel step: a 3-point parabola per axis is exact on
    a separable quadratic surface."""
    ys, xs = np.meshgrid(np.arange(-6, 7), np.arange(-6, 7), indexing="ij")
    for (py, px) in [(1.3, -2.25), (-0.49, 0.0), (2.0, 3.45)]:
        C = 0.9 - 0.02 * (ys - py) ** 2 - 0.035 * (xs - px) ** 2
        s, d, info = oracle.peak(C, -6, -6)
        assert abs(s[0] - py) < 1e-12 and abs(s[1] - px) < 1e-12
        assert info[2] == 0


def test_parabola_border_symmetric_and_clamp():
    ys, xs = np.meshgrid(np.arange(-3, 4), np.arange(-3, 4), indexing="ij")
    # symmetric neighbours -> delta = 0 exactly
    C = 1.0 - 0.1 * ys ** 2 - 0.1 * xs ** 2
    s, d, _ = oracle.peak(C, -3, -3)
    assert tuple(s) == (0.0, 0.0)
    # peak on the window border -> no refinement on that axis, flagged
    C = -0.1 * (ys - 5.0) ** 2 - 0.1 * (xs - 0.3) ** 2
    s, d, info = oracle.peak(C, -3, -3)
    assert d[0] == 3 and s[0] == 3.0 and int(info[2]) & 1
    assert abs(s[1] - 0.3) < 1e-12
    # a kink (c- - 2 c0 + c+ < 0) refines; a flat neighbourhood (= 0) does not
    C = -0.01 * np.abs(xs) - 0.02 * np.abs(ys)
    s, d, _ = oracle.peak(C, -3, -3)
    assert tuple(s) == (0.0, 0.0)
    C = np.where(np.abs(xs) <= 1, 0.0, -1.0) - 0.02 * np.abs(ys)
    s, d, _ = oracle.peak(C, -3, -3)
    assert tuple(d) == (0, 0) and tuple(s) == (0.0, 0.0)  # 3-way tie, zero curvature


# ---------------------------------------------------------------- resample
def test_resample_matches_scipy_linear_shift():
    """Reading: bilinear with clamped coordinates == scipy's order-1 spline
    shift with 'nearest' extension; V(x) = F(x + s) is a shift by -s."""
    r = rng(7)
    F = r.integers(0, 5000, (37, 53)).astype(np.uint16)
    for (sy, sx) in [(1.37, -2.61), (-0.5, 0.25), (12.9, -15.2), (0.0, 0.0), (-40.0, 3.3)]:
        V = oracle.resample(F, sy, sx)
        ref = ndimage.shift(F.astype(float), (-sy, -sx), order=1, mode="nearest", prefilter=False)
        assert np.max(np.abs(V - ref)) < 1e-8


def test_resample_integer_shift_and_ramp():
    r = rng(8)
    F = r.integers(0, 5000, (40, 40)).astype(np.uint16)
    V = oracle.resample(F, 3, -2)
    assert np.array_equal(V[:37, 2:], F[3:, :38].astype(float))
    ys, xs = np.meshgrid(np.arange(40), np.arange(40), indexing="ij")
    ramp = (3 * ys + 5 * xs + 10).astype(np.uint16)
    V = oracle.resample(ramp, 1.25, 2.5)
    inner = (slice(0, 38), slice(0, 37))
    assert np.allclose(V[inner], (3 * (ys + 1.25) + 5 * (xs + 2.5) + 10)[inner], atol=1e-12)


# ---------------------------------------------------------------- Gaussian
def test_gauss_matches_scipy():
    """Eq. 2 pre-smoothing, sigma = 3 px; reading: radius ceil(4 sigma) = 12,
    mirror border == scipy gaussian_filter(mode='reflect', truncate=4)."""
    r = rng(9)
    V = r.normal(2000, 300, (70, 90))
    out = oracle.gauss(V, 3.0)
    ref = ndimage.gaussian_filter(V, 3.0, mode="reflect", truncate=4.0)
    assert np.max(np.abs(out - ref)) < 1e-9


def test_gauss_constant_and_impulse():
    out = oracle.gauss(np.full((40, 50), 1234.5), 3.0)
    assert np.max(np.abs(out - 1234.5)) < 1e-9
    imp = np.zeros((41, 41))
    imp[20, 20] = 1.0
    out = oracle.gauss(imp, 3.0)
    k = np.arange(-12, 13)
    w = np.exp(-k ** 2 / 18.0)
    w /= w.sum()
    ref = np.zeros((41, 41))
    ref[8:33, 8:33] = np.outer(w, w)
    assert np.max(np.abs(out - ref)) < 1e-15


# ---------------------------------------------------------------- median
def test_median_even_count():
    assert oracle.median([4.0, 1.0, 3.0, 2.0]) == 2.5
    r = rng(10)
    for n in (49, 50, 51):
        v = r.normal(0, 1, n)
        assert oracle.median(v) == np.median(v)


# ---------------------------------------------------------------- pipeline
def _run(frames, hp=0, flags=0, shifts=None, chunks=None, L=50):
    n, H, W = frames.shape
    o = oracle.Oracle(H, W, R=4, L=L, hp_window=hp, flags=flags)
    o.set_template(np.zeros((H, W)) + np.arange(W)[None, :])
    sh = np.zeros((n, 2)) if shifts is None else shifts
    outs, t = [], 0
    for c in (chunks or [n]):
        outs.append(o.process(frames[t:t + c], shifts_in=sh[t:t + c]))
        t += c
    corr = np.concatenate([x["corrected"] for x in outs])
    summ = np.concatenate([x["summary"] for x in outs if x["k"] > 0]) if any(
        x["k"] for x in outs) else np.zeros((0, 2, H, W))
    return corr, summ


def test_highpass_impulse_response_and_dc():
    """Reading of the high-pass: trailing boxcar baseline subtraction,
    h[0] = 1 - 1/W, h[1..W-1] = -1/W, 0 after; DC -> 0 from t = 0."""
    Whp, t0, a, c = 8, 20, 500, 1000
    n = 40
    frames = np.full((n, 30, 30), c, np.uint16)
    frames[t0] += a
    corr, _ = _run(frames, hp=Whp, flags=oracle.FLAG_OUT_HIGHPASS)
    y = corr[:, 15, 15]
    h = np.zeros(n)
    h[t0] = 1 - 1 / Whp
    h[t0 + 1:t0 + Whp] = -1 / Whp
    assert np.max(np.abs(y - a * h)) < 1e-9
    assert np.max(np.abs(corr[:t0])) < 1e-12


def test_highpass_sinusoid_steady_state():
    """Closed form of the boxcar high-pass on cos(wt):
    y = cos wt - (1/W) sin(wW/2)/sin(w/2) cos(w(t - (W-1)/2)).
    Inputs are rounded to integers, so |error| <= 0.5 (1 + 1)."""
    Whp, A, c, w = 10, 20000.0, 30000.0, 2 * math.pi / 23
    n = 120
    t = np.arange(n)
    x = np.round(c + A * np.cos(w * t))
    frames = np.broadcast_to(x[:, None, None], (n, 30, 30)).astype(np.uint16).copy()
    corr, _ = _run(frames, hp=Whp, flags=oracle.FLAG_OUT_HIGHPASS)
    y = corr[Whp:, 15, 15]
    tt = t[Whp:]
    ref = A * (np.cos(w * tt) - (1 / Whp) * math.sin(w * Whp / 2) / math.sin(w / 2) * np.cos(
        w * (tt - (Whp - 1) / 2)))
    assert np.max(np.abs(y - ref)) <= 1.0


def test_constant_video_summaries():
    """Eq. 1 and Eq. 2 on a constant video: S = c, T = 0."""
    frames = np.full((100, 30, 34), 777, np.uint16)
    corr, summ = _run(frames)
    assert summ.shape == (2, 2, 30, 34)
    assert np.max(np.abs(summ[:, 0] - 777)) < 1e-9
    assert np.max(np.abs(summ[:, 1])) < 1e-9


def test_single_spike_max_median_response():
    """Eq. 2: one frame with an impulse of a on a constant video -> median =
    c, max - median = a * (Gaussian impulse response), from scipy; Eq. 1: the
    mean picks up a / L at the impulse pixel."""
    c, a, L = 1000, 400, 50
    frames = np.full((L, 41, 41), c, np.uint16)
    frames[17, 20, 20] += a
    corr, summ = _run(frames)
    imp = np.zeros((41, 41))
    imp[20, 20] = a
    ref = ndimage.gaussian_filter(imp, 3.0, mode="reflect", truncate=4.0)
    assert np.max(np.abs(summ[0, 1] - ref)) < 1e-9
    S = np.full((41, 41), float(c))
    S[20, 20] += a / L
    assert np.max(np.abs(summ[0, 0] - S)) < 1e-9


def test_T_invariant_to_static_offsets():
    r = rng(11)
    frames = r.integers(1000, 1200, (50, 30, 30)).astype(np.int64)
    off = r.integers(0, 300, (30, 30))
    _, s1 = _run(frames.astype(np.uint16))
    _, s2 = _run((frames + off[None]).astype(np.uint16))
    assert np.max(np.abs(s1[0, 1] - s2[0, 1])) < 1e-9
    assert np.max(np.abs(s2[0, 0] - s1[0, 0] - off)) < 1e-9


def test_rechunked_stream_is_bit_identical():
    r = rng(12)
    frames = r.integers(500, 3000, (130, 30, 30)).astype(np.uint16)
    sh = r.uniform(-3, 3, (130, 2))
    c1, s1 = _run(frames, hp=6, flags=oracle.FLAG_OUT_HIGHPASS, shifts=sh)
    c2, s2 = _run(frames, hp=6, flags=oracle.FLAG_OUT_HIGHPASS, shifts=sh, chunks=[7, 50, 13, 1, 59])
    assert s1.shape[0] == 2 and np.array_equal(c1, c2) and np.array_equal(s1, s2)


def test_planted_shifts_synthetic_video():
    """Test (a) of the oracle plan on the tiny synthetic video: the estimate
    follows the planted drift."""
    import torch
    from paper_2403_16438_gb300 import synth
    cfg = synth.tiny_config()
    frames, planted, T = synth.make_video(cfg, 24)
    o = oracle.Oracle(cfg.H, cfg.W, R=16)
    o.set_template(T.double().numpy())
    out = o.process(frames.numpy(), want_corrected=False, want_summary=False)
    err = np.abs(out["shifts"] - planted.numpy())
    assert err.max() < 0.25 and err.mean() < 0.08, err


def test_paper_scale_scene_registers_within_0_05_px_without_noise():
    """On noise-free, activity-free frames of the paper-scale scene the ZNCC
    estimate follows the planted drift within 0.05 px (mean); read noise alone
    (sigma 30 plus shot noise) moves it by a near-constant offset of about a
    tenth to a fifth of a pixel -- the bias of the window-variance
    normalisation of ZNCC under additive noise, a property of the method, not
    of an implementation."""
    from paper_2403_16438_gb300 import synth
    import torch
    cfg = synth.paper_scale_config()
    n = 12
    g = torch.Generator().manual_seed(cfg.seed)
    scene = synth.make_scene(cfg, g)
    shifts = synth.planted_shifts(cfg, n, g)
    act0 = torch.zeros((n, len(scene.neurons)))
    T = synth.render(scene, torch.zeros((1, 2), dtype=torch.float64), act0[:1], "cpu")[0]
    exp_ = synth.render(scene, shifts, act0, "cpu")
    clean = torch.clamp(torch.round(exp_), 0, 65535).to(torch.int32).to(torch.uint16)
    noisy = synth.add_noise(exp_, cfg.read_sigma, torch.Generator().manual_seed(5))
    o = oracle.Oracle(cfg.H, cfg.W)
    o.set_template(T.double().numpy())
    e_clean = o.process(clean.numpy(), want_corrected=False, want_summary=False)["shifts"] - \
        shifts.numpy()
    e_noisy = o.process(noisy.numpy(), want_corrected=False, want_summary=False)["shifts"] - \
        shifts.numpy()
    assert np.abs(e_clean).mean() < 0.05 and np.abs(e_clean).max() < 0.1
    offset = e_noisy.mean(axis=0)
    assert np.abs(offset).max() > 0.1                      # the noise-induced offset
    assert np.abs(e_noisy - offset).max() < 0.2            # near-constant over the frames
