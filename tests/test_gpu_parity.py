"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the
same seeded inputs.  Sizes span several tiles, patch groups and segments, with
ragged tails; one test runs the paper-scale 512x512 configuration on sampled
frames."""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_16438_gb300 import synth
from parity_util import REL_TOL, compare_images, compare_shifts, rel_err

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def vimg():
    from paper_2403_16438_gb300 import vimg as v
    return v


def run_gpu(vimg, frames, T, chunks=None, want_surface=False, shifts_in=None, **kw):
    n, H, W = frames.shape
    h = vimg.Handle(H, W, **kw)
    h.set_template(T.to(DEV))
    L = h.params.segment_len
    R = h.params.search_radius
    fd = frames.to(DEV)
    shifts = torch.zeros((n, 2), device=DEV)
    info = torch.zeros((n, 4), device=DEV)
    corrected = torch.zeros((n, H, W), device=DEV)
    summary = torch.zeros((max(1, n // L), 2, H, W), device=DEV)
    surface = torch.zeros((n, 2 * R + 1, 2 * R + 1), device=DEV,
                          dtype=torch.float64) if want_surface else None
    sin = None if shifts_in is None else shifts_in.to(DEV, torch.float32).contiguous()
    k_tot, t = 0, 0
    for c in (chunks or [n]):
        k = h.process(fd[t:t + c], shifts=shifts[t:t + c], corrected=corrected[t:t + c],
                      summary=summary[k_tot:], peak_info=info[t:t + c],
                      surface=None if surface is None else surface[t:t + c],
                      shifts_in=None if sin is None else sin[t:t + c])
        k_tot += k
        t += c
    torch.cuda.synchronize()
    out = dict(shifts=shifts.cpu().numpy(), info=info.cpu().numpy(),
               corrected=corrected.cpu().numpy(), summary=summary[:k_tot].cpu().numpy(), k=k_tot)
    if surface is not None:
        out["surface"] = surface.cpu().numpy()
    h.close()
    return out


def run_oracle(frames, T, shifts_in=None, want_surface=False, R=16, **kw):
    n, H, W = frames.shape
    o = oracle.Oracle(H, W, R=R, **kw)
    o.set_template(T.double().numpy())
    sin = None if shifts_in is None else shifts_in.to(torch.float32).double().numpy()
    return o.process(frames.numpy(), shifts_in=sin, want_surface=want_surface)


@pytest.fixture(scope="module")
def tiny():
    cfg = synth.tiny_config()
    frames, planted, T = synth.make_video(cfg, 130)
    return frames, planted, T


def test_library_loads_and_version(vimg):
    assert "sm_103a" in vimg.version()


def test_surface_and_shift_parity_tiny(vimg, tiny):
    frames, planted, T = tiny
    f = frames[:24]
    g = run_gpu(vimg, f, T, want_surface=True)
    r = run_oracle(f, T, want_surface=True)
    assert np.abs(g["surface"] - r["surface"]).max() < 2e-6
    near, err = compare_shifts(g["shifts"], g["info"], r)
    assert len(near) == 0
    # against the planted drift (content model, not parity)
    assert np.abs(g["shifts"] - planted[:24].numpy()).mean() < 0.1


def test_full_pipeline_parity_tiny(vimg, tiny):
    frames, _, T = tiny
    g = run_gpu(vimg, frames, T)
    r = run_oracle(frames, T)
    compare_shifts(g["shifts"], g["info"], r)
    assert g["k"] == r["k"] == 2
    compare_images(g["corrected"], r["corrected"], "corrected")
    compare_images(g["summary"][:, 0], r["summary"][:, 0], "S")
    compare_images(g["summary"][:, 1], r["summary"][:, 1], "T")


def test_stream_rechunking_is_bitwise_identical(vimg, tiny):
    frames, _, T = tiny
    a = run_gpu(vimg, frames, T, hp_window=7, flags=vimg.OUT_HIGHPASS)
    b = run_gpu(vimg, frames, T, hp_window=7, flags=vimg.OUT_HIGHPASS, chunks=[3, 47, 1, 60, 19])
    c = run_gpu(vimg, frames, T, hp_window=7, flags=vimg.OUT_HIGHPASS, max_chunk=17)
    for x in (b, c):
        assert np.array_equal(a["shifts"], x["shifts"])
        assert np.array_equal(a["corrected"], x["corrected"])
        assert np.array_equal(a["summary"], x["summary"])


@pytest.mark.parametrize("hp", [0, 1, 9])
def test_temporal_stage_with_given_shifts(vimg, tiny, hp):
    """The temporal stage alone: both sides apply the same planted shifts."""
    frames, planted, T = tiny
    sh = planted.to(torch.float32)
    flags = vimg.OUT_HIGHPASS if hp else 0
    g = run_gpu(vimg, frames, T, shifts_in=sh, hp_window=hp, flags=flags, chunks=[70, 60])
    r = run_oracle(frames, T, shifts_in=sh, hp_window=hp, flags=oracle.FLAG_OUT_HIGHPASS if hp else 0)
    if hp == 1:
        assert np.abs(g["corrected"]).max() == 0.0 and np.abs(r["corrected"]).max() == 0.0
    else:
        compare_images(g["corrected"], r["corrected"], "corrected")
    compare_images(g["summary"][:, 0], r["summary"][:, 0], "S")
    compare_images(g["summary"][:, 1], r["summary"][:, 1], "T")


def test_wide_range_blocks(vimg, tiny):
    """Window statistics sum squares in 32 bits when a staged block's pixels lie
    within 3,100 of the middle of their range, in 64 bits otherwise.  Scaling
    the left half of the video (and template) by 10 puts blocks of both kinds
    in one frame: those straddling column 64 span > 15,000 counts, those right
    of it keep the tiny video's range."""
    frames, _, T = tiny
    f = np.clip(frames[:12].numpy().astype(np.int64) * np.where(np.arange(128) < 64, 10, 1),
                0, 65535)
    assert f[:, :, 60:68].max() - f[:, :, 60:68].min() > 15000
    f = torch.from_numpy(f.astype(np.uint16))
    T2 = T.clone()
    T2[:, :64] *= 10
    g = run_gpu(vimg, f, T2, want_surface=True)
    r = run_oracle(f, T2, want_surface=True)
    # Ten times larger pixel terms: the FP32 numerators (441 products each) carry
    # more rounding than on the plain video; bound = 441 u, u = 2^-24, the
    # worst-case relative error of an FP32 sum of 441 terms.
    assert np.abs(g["surface"] - r["surface"]).max() < 441 * 2.0 ** -24
    compare_shifts(g["shifts"], g["info"], r)


@pytest.mark.parametrize("H,W,R,L", [(75, 100, 8, 50), (97, 61, 5, 13), (53, 53, 16, 50)])
def test_ragged_sizes_and_radii(vimg, H, W, R, L):
    cfg = synth.tiny_config(H=H, W=W, seed=77 + H, clamp=min(8.0, R))
    frames, _, T = synth.make_video(cfg, 2 * L + 3)
    g = run_gpu(vimg, frames, T, search_radius=R, segment_len=L)
    r = run_oracle(frames, T, R=R, L=L)
    compare_shifts(g["shifts"], g["info"], r)
    compare_images(g["corrected"], r["corrected"], "corrected")
    assert g["k"] == r["k"] == 2
    compare_images(g["summary"][:, 0], r["summary"][:, 0], "S")
    compare_images(g["summary"][:, 1], r["summary"][:, 1], "T")


def test_paper_scale_sampled(vimg):
    """512x512, R = 16 (484 patches, 1089 displacements): the launch
    configuration the benchmark times, checked on 3 frames."""
    cfg = synth.paper_scale_config()
    frames, planted, T = synth.make_video(cfg, 3)
    g = run_gpu(vimg, frames, T, want_surface=True)
    r = run_oracle(frames, T, want_surface=True)
    assert np.abs(g["surface"] - r["surface"]).max() < 2e-6
    compare_shifts(g["shifts"], g["info"], r)
    compare_images(g["corrected"], r["corrected"], "corrected")


def test_edge_cases(vimg):
    H = W = 64
    T = torch.rand((H, W)) * 1000 + 1000
    h = vimg.Handle(H, W, search_radius=8)
    with pytest.raises(vimg.VimgError) as e:
        h.process(torch.zeros((1, H, W), dtype=torch.uint16, device=DEV))
    assert e.value.code == vimg.ERR_NO_TEMPLATE
    h.set_template(T.to(DEV))
    assert h.process(torch.zeros((0, H, W), dtype=torch.uint16, device=DEV)) == 0
    # constant frame: every ZNCC is 0 -> d* = (0, 0) by the tie-break, no refinement
    const = torch.full((2, H, W), 1234, dtype=torch.uint16, device=DEV)
    s = torch.full((2, 2), 7.0, device=DEV)
    info = torch.zeros((2, 4), device=DEV)
    corr = torch.zeros((2, H, W), device=DEV)
    h.process(const, shifts=s, peak_info=info, corrected=corr)
    torch.cuda.synchronize()
    assert s.abs().max().item() == 0.0 and info[:, 2].abs().max().item() == 0.0
    assert (corr == 1234.0).all()
    # the template registered to itself gives zero integer shift and C = 1
    tf = torch.round(T).to(torch.uint16).to(DEV).unsqueeze(0)
    h.set_template(torch.round(T).to(DEV))
    h.process(tf, shifts=s[:1], peak_info=info[:1])
    torch.cuda.synchronize()
    assert info[0, :2].abs().max().item() == 0.0 and abs(info[0, 2].item() - 1.0) < 1e-5
    h.close()
    with pytest.raises(vimg.VimgError):
        vimg.Handle(40, 40, search_radius=16)  # 40 < 2R + 21


@pytest.mark.parametrize("max_chunk,split", [(40, None), (10, None), (10, 70)])
def test_host_buffer_entry_point(vimg, tiny, max_chunk, split):
    """vimg_process_host against the device-buffer path, bit for bit: batches of
    max_chunk frames through the ring of upload stages and the pair of download
    stages (max_chunk = 10 wraps both several times), and the stream split
    over two calls at frame `split` (the second call's uploads and downloads
    follow the first's)."""
    frames, _, T = tiny
    n, H, W = frames.shape
    h = vimg.Handle(H, W, max_chunk=max_chunk)
    h.set_template(T.to(DEV))
    fh = frames.pin_memory()
    sh = torch.zeros((n, 2)).pin_memory()
    sm = torch.zeros((n // 50, 2, H, W)).pin_memory()
    if split is None:
        k = h.process_host(fh, shifts_host=sh, summary_host=sm)
    else:
        k1 = h.process_host(fh[:split], shifts_host=sh[:split], summary_host=sm)
        k = k1 + h.process_host(fh[split:], shifts_host=sh[split:], summary_host=sm[k1:])
    assert k == 2
    g = run_gpu(vimg, frames, T)
    assert np.array_equal(sh.numpy(), g["shifts"])
    assert np.array_equal(sm.numpy(), g["summary"])
    h.close()


def test_fma_rate_is_plausible(vimg):
    """The measured FP32 FMA rate (the FP32 correlation's ALU roofline): below
    the nominal 128 FMA lanes x 2 FLOP x the maximum clock of every SM, and far
    above a small fraction of it."""
    rate = vimg.fma_rate()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = sms * 128 * 2 * 2.2e9
    assert 0.3 * nominal < rate <= nominal, (rate, nominal)
