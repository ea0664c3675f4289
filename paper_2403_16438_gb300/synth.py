"""Seeded synthetic voltage-imaging videos with planted rigid shifts.

This module only makes inputs.  It holds none of the motion-correction or
summary arithmetic, and both the CUDA path's tests and the CPU oracle's tests
take their inputs from it.

Content model (the workloads the paper evaluates on are not available, so
these stand in for them; shapes and rates follow the paper's Fig. 1 video and
its datasets table):
  * background: two axis-aligned anisotropic 2-D Gaussians on a pedestal;
  * neurons: ellipses with a 1-px logistic edge, baseline brightness 25 % of
    the background amplitude, limited pairwise overlap;
  * activity: Poisson spike trains; each spike adds dF/F * exp(-k/3) for
    k >= 0 frames after it (3-frame decay);
  * noise: Poisson shot noise on the expected counts plus Gaussian read
    noise, rounded and clamped to uint16;
  * motion: rigid 2-D Gaussian random walk clamped to +-clamp px, optional
    3-px jumps; frame t shows Scene(x - s_t), so the planted shift s_t is
    what registration against the template Scene(x) should return.
The scene is evaluated analytically at the shifted coordinates, so subpixel
shifts carry no interpolation bias.  Everything runs through torch on either
device; a torch.Generator seeded from the config makes it reproducible.
"""
from __future__ import annotations

import dataclasses
import math

import torch


@dataclasses.dataclass
class VideoConfig:
    H: int = 128
    W: int = 128
    n_frames: int = 1000
    fps: float = 741.0
    n_neurons: int = 8
    r_lo: float = 4.0
    r_hi: float = 8.0
    overlap_max: float = 0.30
    bg_amp: float = 2000.0
    rate_lo: float = 10.0  # spikes/s
    rate_hi: float = 10.0
    dff_lo: float = 0.05
    dff_hi: float = 0.05
    decay: float = 3.0  # frames
    read_sigma: float = 20.0
    walk_sigma: float = 0.3  # px/frame
    clamp: float = 8.0
    jump_frac: float = 0.0
    jump_px: float = 3.0
    template_frames: int = 200
    seed: int = 1001


def tiny_config(**kw) -> VideoConfig:
    """128x128, 1,000 frames, 8 neurons (r 4-8 px, <=30 % overlap), background
    2,000 counts, 10 Hz spikes of 5 % dF/F, read noise 20, walk 0.3 px clamped
    at +-8 px."""
    return dataclasses.replace(VideoConfig(), **kw)


def paper_scale_config(**kw) -> VideoConfig:
    """512x512, 10,000 frames, 40 neurons (r 5-10 px, <=40 % overlap),
    background 4,000 counts, 5-20 Hz spikes of 2-8 % dF/F, read noise 30, walk
    0.5 px clamped at +-12 px, 1 % of frames with 3-px jumps."""
    base = VideoConfig(H=512, W=512, n_frames=10000, n_neurons=40, r_lo=5.0, r_hi=10.0,
                       overlap_max=0.40, bg_amp=4000.0, rate_lo=5.0, rate_hi=20.0, dff_lo=0.02,
                       dff_hi=0.08, read_sigma=30.0, walk_sigma=0.5, clamp=12.0, jump_frac=0.01,
                       seed=1002)
    return dataclasses.replace(base, **kw)


def scaled_config(H: int, W: int, n_frames: int, seed: int, **kw) -> VideoConfig:
    """Paper-scale content at another size, neuron count scaled to area."""
    n = max(1, round(40 * H * W / (512 * 512)))
    return paper_scale_config(H=H, W=W, n_frames=n_frames, n_neurons=n, seed=seed, **kw)


@dataclasses.dataclass
class Scene:
    cfg: VideoConfig
    bg: list  # per Gaussian: (weight, cy, cx, sy, sx)
    neurons: list  # per neuron: (cy, cx, a, b, theta, f0)
    rates: list
    dffs: list


def make_scene(cfg: VideoConfig, gen: torch.Generator) -> Scene:
    def u(lo=0.0, hi=1.0):
        return lo + (hi - lo) * torch.rand((), generator=gen).item()

    H, W = cfg.H, cfg.W
    bg = []
    for wgt in (1.0, 0.6):
        bg.append((wgt, u(0.2, 0.8) * H, u(0.2, 0.8) * W, u(0.25, 0.5) * H, u(0.25, 0.5) * W))
    neurons, tries = [], 0
    while len(neurons) < cfg.n_neurons and tries < 20000:
        tries += 1
        r = u(cfg.r_lo, cfg.r_hi)
        a, b = r * u(0.85, 1.15), r * u(0.85, 1.15)
        m = max(a, b) + 2
        cy, cx = u(m, H - m), u(m, W - m)
        ok = True
        for (py, px, pa, pb, _, _) in neurons:
            ov = _disc_overlap(math.sqrt(a * b), math.sqrt(pa * pb), math.hypot(cy - py, cx - px))
            if ov > cfg.overlap_max:
                ok = False
                break
        if ok:
            neurons.append((cy, cx, a, b, u(0, math.pi), 0.25 * cfg.bg_amp))
    rates = [u(cfg.rate_lo, cfg.rate_hi) for _ in neurons]
    dffs = [u(cfg.dff_lo, cfg.dff_hi) for _ in neurons]
    return Scene(cfg, bg, neurons, rates, dffs)


def _disc_overlap(r1: float, r2: float, d: float) -> float:
    """Intersection area of two discs over the smaller disc's area."""
    if d >= r1 + r2:
        return 0.0
    if d <= abs(r1 - r2):
        return 1.0
    a1 = r1 * r1 * math.acos((d * d + r1 * r1 - r2 * r2) / (2 * d * r1))
    a2 = r2 * r2 * math.acos((d * d + r2 * r2 - r1 * r1) / (2 * d * r2))
    a3 = 0.5 * math.sqrt(max(0.0, (-d + r1 + r2) * (d + r1 - r2) * (d - r1 + r2) * (d + r1 + r2)))
    return (a1 + a2 - a3) / (math.pi * min(r1, r2) ** 2)


def planted_shifts(cfg: VideoConfig, n: int, gen: torch.Generator) -> torch.Tensor:
    """Rigid drift (dy, dx) per frame, float64 [n, 2]."""
    steps = torch.randn((n, 2), generator=gen, dtype=torch.float64) * cfg.walk_sigma
    if cfg.jump_frac > 0:
        jumps = torch.rand((n,), generator=gen, dtype=torch.float64) < cfg.jump_frac
        ang = torch.rand((n,), generator=gen, dtype=torch.float64) * 2 * math.pi
        steps[:, 0] += jumps * cfg.jump_px * torch.sin(ang)
        steps[:, 1] += jumps * cfg.jump_px * torch.cos(ang)
    s = torch.zeros((n, 2), dtype=torch.float64)
    cur = torch.zeros(2, dtype=torch.float64)
    for t in range(n):
        if t > 0:
            cur = torch.clamp(cur + steps[t], -cfg.clamp, cfg.clamp)
        s[t] = cur
    return s


def activity(scene: Scene, n: int, gen: torch.Generator) -> torch.Tensor:
    """dF/F per neuron and frame, float32 [n, n_neurons]."""
    cfg = scene.cfg
    k = len(scene.neurons)
    if k == 0:
        return torch.zeros((n, 0))
    rate = torch.tensor(scene.rates, dtype=torch.float32) / cfg.fps
    spikes = torch.poisson(rate.expand(n, k).contiguous(), generator=gen)
    act = torch.zeros((n, k))
    cur = torch.zeros(k)
    dec = math.exp(-1.0 / cfg.decay)
    for t in range(n):
        cur = cur * dec + spikes[t]
        act[t] = cur
    return act * torch.tensor(scene.dffs, dtype=torch.float32)


def render(scene: Scene, shifts: torch.Tensor, act: torch.Tensor, device, crop=None,
           margin_px=None) -> torch.Tensor:
    """Expected counts float32 [n, H, W] of frames showing Scene(x - s_t).
    crop = (y0, x0, h, w) renders only that window of the frame."""
    cfg = scene.cfg
    H, W = cfg.H, cfg.W
    cy0, cx0 = 0, 0
    if crop is not None:
        cy0, cx0, H, W = crop
    n = shifts.shape[0]
    sy = shifts[:, 0].to(device=device, dtype=torch.float32).view(n, 1, 1)
    sx = shifts[:, 1].to(device=device, dtype=torch.float32).view(n, 1, 1)
    ys = torch.arange(cy0, cy0 + H, device=device, dtype=torch.float32).view(1, H, 1)
    xs = torch.arange(cx0, cx0 + W, device=device, dtype=torch.float32).view(1, 1, W)
    out = torch.full((n, H, W), 0.3 * cfg.bg_amp, device=device)
    for (wgt, cy, cx, gy, gx) in scene.bg:
        ey = torch.exp(-0.5 * ((ys - sy - cy) / gy) ** 2)
        ex = torch.exp(-0.5 * ((xs - sx - cx) / gx) ** 2)
        out += (0.7 * cfg.bg_amp * wgt) * ey * ex
    act = act.to(device)
    if margin_px is None:
        margin_px = cfg.clamp + 4 * cfg.jump_px * (cfg.jump_frac > 0)
    margin = int(math.ceil(max(margin_px, 1))) + 4
    for j, (cy, cx, a, b, th, f0) in enumerate(scene.neurons):
        half = int(math.ceil(max(a, b))) + margin
        y0, y1 = max(0, int(cy) - half - cy0), min(H, int(cy) + half + 1 - cy0)
        x0, x1 = max(0, int(cx) - half - cx0), min(W, int(cx) + half + 1 - cx0)
        if y0 >= y1 or x0 >= x1:
            continue
        yy = ys[:, y0:y1, :] - sy - cy
        xx = xs[:, :, x0:x1] - sx - cx
        c, s = math.cos(th), math.sin(th)
        u = (c * xx + s * yy) / a
        v = (-s * xx + c * yy) / b
        rho = torch.sqrt(u * u + v * v)
        fp = torch.sigmoid((1.0 - rho) * math.sqrt(a * b))  # ~1-px logistic edge
        out[:, y0:y1, x0:x1] += (f0 * (1.0 + act[:, j])).view(n, 1, 1) * fp
    return out


def add_noise(expected: torch.Tensor, read_sigma: float, gen: torch.Generator) -> torch.Tensor:
    shot = torch.poisson(expected.clamp_min(0), generator=gen)
    read = torch.randn(expected.shape, generator=gen, device=expected.device) * read_sigma
    return torch.clamp(torch.round(shot + read), 0, 65535).to(torch.int32).to(torch.uint16)


def ground_truth(cfg: VideoConfig, n_frames: int | None = None):
    """(scene, planted shifts, activity) exactly as make_video draws them."""
    n = cfg.n_frames if n_frames is None else n_frames
    g_cpu = torch.Generator().manual_seed(cfg.seed)
    scene = make_scene(cfg, g_cpu)
    shifts = planted_shifts(cfg, n, g_cpu)
    act = activity(scene, n, g_cpu)
    return scene, shifts, act


def roi_masks(cfg: VideoConfig) -> torch.Tensor:
    """Footprint interiors (rho < 1) of the scene's neurons at zero shift, bool
    [n_neurons][H][W]: the synthetic stand-in for segmented neuron ROIs."""
    scene = make_scene(cfg, torch.Generator().manual_seed(cfg.seed))
    H, W = cfg.H, cfg.W
    ys = torch.arange(H, dtype=torch.float32).view(H, 1)
    xs = torch.arange(W, dtype=torch.float32).view(1, W)
    masks = torch.zeros((len(scene.neurons), H, W), dtype=torch.bool)
    for j, (cy, cx, a, b, th, _) in enumerate(scene.neurons):
        c, s = math.cos(th), math.sin(th)
        u = (c * (xs - cx) + s * (ys - cy)) / a
        v = (-s * (xs - cx) + c * (ys - cy)) / b
        masks[j] = (u * u + v * v) < 1.0
    return masks


def make_video(cfg: VideoConfig, n_frames: int | None = None, device="cpu", chunk: int = 256,
               out: torch.Tensor | None = None):
    """Returns (frames uint16 [n,H,W], planted shifts float64 [n,2] (CPU),
    template float32 [H,W]) on `device`.  `out` may be a preallocated frames
    tensor (e.g. pinned host memory)."""
    n = cfg.n_frames if n_frames is None else n_frames
    device = torch.device(device)
    g_cpu = torch.Generator().manual_seed(cfg.seed)
    scene = make_scene(cfg, g_cpu)
    shifts = planted_shifts(cfg, n, g_cpu)
    act = activity(scene, n, g_cpu)
    g_dev = torch.Generator(device=device).manual_seed(cfg.seed + 7919)
    frames = out if out is not None else torch.empty((n, cfg.H, cfg.W), dtype=torch.uint16,
                                                     device=device)
    for t0 in range(0, n, chunk):
        t1 = min(n, t0 + chunk)
        exp_ = render(scene, shifts[t0:t1], act[t0:t1], device)
        frames[t0:t1].copy_(add_noise(exp_, cfg.read_sigma, g_dev))
    # Template: mean of template_frames noisy frames at zero shift.
    nt = cfg.template_frames
    act_t = activity(scene, nt, g_cpu)
    acc = torch.zeros((cfg.H, cfg.W), dtype=torch.float64, device=device)
    for t0 in range(0, nt, chunk):
        t1 = min(nt, t0 + chunk)
        exp_ = render(scene, torch.zeros((t1 - t0, 2), dtype=torch.float64), act_t[t0:t1], device)
        acc += add_noise(exp_, cfg.read_sigma, g_dev).to(torch.float64).sum(0)
    template = (acc / nt).to(torch.float32)
    return frames, shifts, template


def training_batch(scenes, n: int, gen: torch.Generator, device, crop: int = 128,
                   max_shift: float = 12.0):
    """A batch of (frame crop uint16 [n,crop,crop], template crop float32
    [n,crop,crop], planted shift float32 [n,2]) for the learned shift
    proposal: random scene, uniform shift in [-max_shift, max_shift]^2, the
    centre crop of the frame; the template crop is that scene's template.
    `scenes` is a list of (Scene, template crop float32 [crop,crop] on device)."""
    k = len(scenes)
    idx = torch.randint(0, k, (n,), generator=gen)
    shifts = (torch.rand((n, 2), generator=gen, dtype=torch.float64) * 2 - 1) * max_shift
    frames = torch.empty((n, crop, crop), dtype=torch.int32, device=device)
    tmpl = torch.empty((n, crop, crop), dtype=torch.float32, device=device)
    g_dev = torch.Generator(device=device).manual_seed(int(torch.randint(0, 2**31 - 1, (1,), generator=gen)))
    for s_i in range(k):
        sel = (idx == s_i).nonzero().flatten()
        if sel.numel() == 0:
            continue
        scene, tcrop = scenes[s_i]
        cfg = scene.cfg
        y0, x0 = (cfg.H - crop) // 2, (cfg.W - crop) // 2
        act = activity(scene, sel.numel(), gen)
        exp_ = render(scene, shifts[sel], act, device, crop=(y0, x0, crop, crop),
                      margin_px=max_shift + 2)
        frames[sel.to(device)] = add_noise(exp_, cfg.read_sigma, g_dev).to(torch.int32)
        tmpl[sel.to(device)] = tcrop
    return frames.to(torch.uint16), tmpl, shifts.to(torch.float32)


def training_scenes(n_scenes: int, seed: int, device, crop: int = 128):
    """Paper-scale scenes (config-2 content) with their template centre crops."""
    out = []
    for i in range(n_scenes):
        cfg = paper_scale_config(seed=seed + i, template_frames=100)
        g = torch.Generator().manual_seed(cfg.seed)
        scene = make_scene(cfg, g)
        y0, x0 = (cfg.H - crop) // 2, (cfg.W - crop) // 2
        g_dev = torch.Generator(device=device).manual_seed(cfg.seed + 17)
        act = activity(scene, cfg.template_frames, g)
        exp_ = render(scene, torch.zeros((cfg.template_frames, 2), dtype=torch.float64), act,
                      device, crop=(y0, x0, crop, crop), margin_px=2)
        t = add_noise(exp_, cfg.read_sigma, g_dev).to(torch.float64).mean(0).to(torch.float32)
        out.append((scene, t))
    return out


def training_pool(n_frames: int, n_scenes: int, seed: int, device, crop: int = 128,
                  max_shift: float = 12.0):
    """A pool of n_frames training samples from n_scenes paper-scale scenes:
    (frame crops uint16 [n,crop,crop], per-sample scene index int64 [n],
    template crops float32 [n_scenes,crop,crop], planted shifts float32 [n,2])."""
    dev = torch.device(device)
    gen = torch.Generator().manual_seed(seed)
    per = (n_frames + n_scenes - 1) // n_scenes
    frames = torch.empty((n_frames, crop, crop), dtype=torch.uint16, device=dev)
    shifts = torch.empty((n_frames, 2), dtype=torch.float32)
    scene_idx = torch.empty((n_frames,), dtype=torch.int64)
    tmpls = torch.empty((n_scenes, crop, crop), dtype=torch.float32, device=dev)
    g_dev = torch.Generator(device=dev).manual_seed(seed + 31)
    t = 0
    for i in range(n_scenes):
        cfg = paper_scale_config(seed=seed + 1000 + i, template_frames=64)
        scene = make_scene(cfg, gen)
        y0, x0 = (cfg.H - crop) // 2, (cfg.W - crop) // 2
        act_t = activity(scene, cfg.template_frames, gen)
        exp_t = render(scene, torch.zeros((cfg.template_frames, 2), dtype=torch.float64), act_t,
                       dev, crop=(y0, x0, crop, crop), margin_px=2)
        tmpls[i] = add_noise(exp_t, cfg.read_sigma, g_dev).to(torch.float32).mean(0)
        m = min(per, n_frames - t)
        if m <= 0:
            break
        sh = (torch.rand((m, 2), generator=gen, dtype=torch.float64) * 2 - 1) * max_shift
        act = activity(scene, m, gen)
        exp_ = render(scene, sh, act, dev, crop=(y0, x0, crop, crop), margin_px=max_shift + 2)
        frames[t:t + m] = add_noise(exp_, cfg.read_sigma, g_dev)
        shifts[t:t + m] = sh.to(torch.float32)
        scene_idx[t:t + m] = i
        t += m
    return frames, scene_idx, tmpls, shifts


def augmented_batch(pool, n: int, gen: torch.Generator):
    """Random samples of a training pool under a random element of the square's
    symmetry group (flips and transposition), applied alike to frame, template
    and shift.  Returns (frames uint16, templates float32, shifts float32 [n,2])."""
    frames, scene_idx, tmpls, shifts = pool
    dev = frames.device
    idx = torch.randint(0, frames.shape[0], (n,), generator=gen)
    f = frames.view(torch.int16)[idx.to(dev)]  # same bits; uint16 indexing is not on every device
    t = tmpls[scene_idx[idx].to(dev)]
    s = shifts[idx].clone()
    op = int(torch.randint(0, 8, (1,), generator=gen))
    if op & 1:  # flip y
        f, t, s[:, 0] = f.flip(1), t.flip(1), -s[:, 0]
    if op & 2:  # flip x
        f, t, s[:, 1] = f.flip(2), t.flip(2), -s[:, 1]
    if op & 4:  # transpose
        f, t, s = f.transpose(1, 2), t.transpose(1, 2), s[:, [1, 0]]
    return f.contiguous().view(torch.uint16), t.contiguous(), s.contiguous()


def unet_params(layers, seed: int = 0) -> torch.Tensor:
    """Seeded random-initialised weights for a network given as [(kind, cin,
    cout)] with kind 'conv' (3x3), 'up' (2x2 stride-2 transposed) or 'out'
    (1x1): weights N(0, 2 / fan_in) (He), biases U(-0.1, 0.1), flat float32 in
    layer order, weights before biases.  A stand-in for trained weights (none
    are available)."""
    g = torch.Generator().manual_seed(seed)
    parts = []
    for kind, ci, co in layers:
        taps = {"conv": 9, "up": 4, "out": 1}[kind]
        fan_in = ci * taps if kind != "up" else ci
        gain = 2.0 if kind != "out" else 1.0
        parts.append(torch.randn(ci * co * taps, generator=g, dtype=torch.float64)
                     * math.sqrt(gain / fan_in))
        parts.append((torch.rand(co, generator=g, dtype=torch.float64) - 0.5) * 0.2)
    return torch.cat(parts).to(torch.float32)


def summary_pair(cfg: VideoConfig, k: int, seed: int = 0) -> torch.Tensor:
    """[k][2][H][W] float32 stand-ins for segment summaries: S = the scene's
    resting image plus read noise, T = Gaussian blobs at the neurons that
    spike in the segment plus a small noise floor (the shape of Eq. 1 / Eq. 2
    outputs, without running the temporal pass)."""
    g = torch.Generator().manual_seed(seed)
    scene = make_scene(cfg, torch.Generator().manual_seed(cfg.seed))
    H, W = cfg.H, cfg.W
    ys = torch.arange(H, dtype=torch.float64).view(H, 1)
    xs = torch.arange(W, dtype=torch.float64).view(1, W)
    base = torch.full((H, W), float(cfg.bg_amp), dtype=torch.float64)
    blobs = []
    for (cy, cx, a, b, th, amp) in scene.neurons:
        c, s = math.cos(th), math.sin(th)
        u = (c * (xs - cx) + s * (ys - cy)) / a
        v = (-s * (xs - cx) + c * (ys - cy)) / b
        fp = torch.exp(-0.5 * (u * u + v * v) * 4.0)
        base += amp * fp
        blobs.append(fp)
    out = torch.zeros((k, 2, H, W), dtype=torch.float64)
    for i in range(k):
        out[i, 0] = base + torch.randn((H, W), generator=g, dtype=torch.float64) * cfg.read_sigma
        t = torch.rand((H, W), generator=g, dtype=torch.float64) * 5.0
        for fp in blobs:
            if torch.rand(1, generator=g).item() < 0.5:
                t += 60.0 * fp
        out[i, 1] = t
    return out.to(torch.float32)


def planted_prob_maps(cfg: VideoConfig, K: int, seed: int = 0) -> torch.Tensor:
    """[K][H][W] float32 stand-ins for U-Net probability maps: a background of
    uniform values below 0.35; in each segment every neuron of the scene spikes
    with probability 0.4 and then shows its footprint interior at 0.6-0.95; a
    few thin vessel-like lines and 2x2 specks appear above 0.5 as well (shapes
    the cleanup has to remove)."""
    g = torch.Generator().manual_seed(seed)
    masks = roi_masks(cfg).to(torch.float32)
    H, W = cfg.H, cfg.W
    out = torch.rand((K, H, W), generator=g) * 0.35
    for i in range(K):
        for m in masks:
            if torch.rand(1, generator=g).item() < 0.4:
                level = 0.6 + 0.35 * torch.rand(1, generator=g).item()
                out[i] = torch.maximum(out[i], m * level)
        if torch.rand(1, generator=g).item() < 0.5:  # a vessel: 1 px wide, 40 px long
            y = int(torch.randint(2, H - 2, (1,), generator=g))
            x = int(torch.randint(0, max(1, W - 40), (1,), generator=g))
            out[i, y, x:x + 40] = 0.9
        for _ in range(2):  # specks
            y = int(torch.randint(0, H - 2, (1,), generator=g))
            x = int(torch.randint(0, W - 2, (1,), generator=g))
            out[i, y:y + 2, x:x + 2] = 0.8
    return out


def disc_chain_maps() -> torch.Tensor:
    """[2][96][760] float32 probability maps that stress the footprint
    reconstruction's region size and neuron count.  Background 0.05; discs at
    0.85 lighting up in alternate segments (disc k in segment k mod 2), so that
    neighbours, which overlap, are separate blobs of different segments:
      * a chain of 24 discs of radius 17 (908 px each) along row 24, centres
        every 30 px from x = 20: one region of about 20,000 px made of 24 blobs;
      * a chain of 40 discs of radius 4 (49 px each) along row 70, centres every
        6 px from x = 10: one region of about 1,700 px made of 40 blobs;
      * a lone disc of radius 6 at (75, 500) in segment 0: an ordinary region."""
    H, W = 96, 760
    yy, xx = torch.meshgrid(torch.arange(H), torch.arange(W), indexing="ij")
    out = torch.full((2, H, W), 0.05)

    def disc(cy, cx, r):
        return ((yy - cy) ** 2 + (xx - cx) ** 2) <= r * r

    for k in range(24):
        out[k % 2][disc(24, 20 + 30 * k, 17)] = 0.85
    for k in range(40):
        out[k % 2][disc(70, 10 + 6 * k, 4)] = 0.85
    out[0][disc(75, 500, 6)] = 0.85
    return out


def make_video_range(cfg: VideoConfig, n_total: int, t0: int, t1: int, device="cpu",
                     chunk: int = 256):
    """Frames [t0, t1) of one n_total-frame video (for a time shard): the scene,
    drift and activity of the whole video, rendered only over the range, with
    the noise drawn for the range (generator seeded by the seed and t0), and
    the video's template (independent of the range).  Returns (frames uint16
    [t1 - t0, H, W], planted shifts float64 [t1 - t0, 2], template float32)."""
    if not 0 <= t0 <= t1 <= n_total:
        raise ValueError("bad frame range")
    device = torch.device(device)
    g_cpu = torch.Generator().manual_seed(cfg.seed)
    scene = make_scene(cfg, g_cpu)
    shifts = planted_shifts(cfg, n_total, g_cpu)
    act = activity(scene, n_total, g_cpu)
    g_dev = torch.Generator(device=device).manual_seed(cfg.seed + 7919 + 1000003 * t0)
    frames = torch.empty((t1 - t0, cfg.H, cfg.W), dtype=torch.uint16, device=device)
    for a in range(t0, t1, chunk):
        b = min(t1, a + chunk)
        exp_ = render(scene, shifts[a:b], act[a:b], device)
        frames[a - t0:b - t0].copy_(add_noise(exp_, cfg.read_sigma, g_dev))
    g_t = torch.Generator(device=device).manual_seed(cfg.seed + 104729)
    nt = cfg.template_frames
    act_t = activity(scene, nt, torch.Generator().manual_seed(cfg.seed + 1))
    acc = torch.zeros((cfg.H, cfg.W), dtype=torch.float64, device=device)
    for a in range(0, nt, chunk):
        b = min(nt, a + chunk)
        exp_ = render(scene, torch.zeros((b - a, 2), dtype=torch.float64), act_t[a:b], device)
        acc += add_noise(exp_, cfg.read_sigma, g_t).to(torch.float64).sum(0)
    return frames, shifts[t0:t1], (acc / nt).to(torch.float32)
