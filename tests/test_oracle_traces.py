"""Pins of the oracle's voltage traces (Sec. II, third stage: the mean pixel
intensity within each neuron ROI of every motion-corrected frame)."""
import numpy as np
import torch

import oracle
from paper_2403_16438_gb300 import synth


def test_closed_forms():
    rng = np.random.default_rng(3)
    H, W = 20, 30
    V = rng.uniform(0, 5000, (H, W))
    m = np.zeros((4, H, W), bool)
    m[0, 3, 7] = True                       # single pixel
    m[1, 2:9, 4:11] = True                  # block
    m[2, 12:18, 20:29] = True               # disjoint block
    # m[3] empty
    out = oracle.roi_means(V, m)
    assert out[0] == V[3, 7]
    assert out[3] == 0.0
    # constant frame -> the constant in every non-empty ROI
    assert np.allclose(oracle.roi_means(np.full((H, W), 1234.5), m)[:3], 1234.5, rtol=0, atol=1e-12)
    # affine maps commute with the mean
    a, b = 3.5, -17.0
    assert np.allclose(oracle.roi_means(a * V + b, m)[:3], a * out[:3] + b, rtol=1e-12)
    # disjoint union: count-weighted mean of the parts
    u = (m[1] | m[2])[None]
    n1, n2 = m[1].sum(), m[2].sum()
    assert np.isclose(oracle.roi_means(V, u)[0], (n1 * out[1] + n2 * out[2]) / (n1 + n2), rtol=1e-12)


def test_traces_of_the_streaming_oracle_are_roi_means_of_its_corrected_frames():
    cfg = synth.tiny_config()
    frames, _, T = synth.make_video(cfg, 12)
    masks = synth.roi_masks(cfg).numpy()
    o = oracle.Oracle(cfg.H, cfg.W)
    o.set_template(T.double().numpy())
    o.set_rois(masks)
    r = o.process(frames.numpy())
    for i in range(12):
        assert np.array_equal(r["traces"][i], oracle.roi_means(r["corrected"][i], masks))


def test_traces_follow_the_planted_activity():
    """Noise-free, drift-free video, zero shifts applied: the corrected frames
    are the frames, so each neuron's trace is an affine function of its planted
    activity, up to the overlap with neighbouring footprints and integer rounding."""
    cfg = synth.tiny_config(read_sigma=0.0, walk_sigma=0.0)
    n = 150
    scene, shifts, act = synth.ground_truth(cfg, n)
    exp_ = synth.render(scene, shifts, act, "cpu")
    frames = torch.clamp(torch.round(exp_), 0, 65535).to(torch.int32).to(torch.uint16)
    T = synth.render(scene, torch.zeros((1, 2), dtype=torch.float64), torch.zeros((1, act.shape[1])),
                     "cpu")[0]
    masks = synth.roi_masks(cfg).numpy()
    o = oracle.Oracle(cfg.H, cfg.W)
    o.set_template(T.double().numpy())
    o.set_rois(masks)
    # zero shifts given: the corrected frames are exactly the frames
    r = o.process(frames.numpy(), shifts_in=np.zeros((n, 2)), want_summary=False)
    assert np.array_equal(r["corrected"], frames.numpy().astype(np.float64))
    tr = r["traces"]
    corr = [np.corrcoef(tr[:, j], act[:, j].numpy())[0, 1] for j in range(act.shape[1])
            if act[:, j].std() > 0]
    assert min(corr) > 0.9 and np.median(corr) > 0.99, corr
