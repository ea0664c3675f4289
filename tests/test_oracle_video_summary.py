"""Pins of the oracle's whole-video summary images (VolPy's temporal average and
temporal correlation images, Sec. III-A / Fig. 2)."""
import numpy as np

import oracle
import oracle.video_summary as VS
from paper_2403_16438_gb300 import synth

rng = np.random.default_rng(11)


def test_correlation_image_is_the_mean_of_corrcoef_over_neighbours():
    V = rng.normal(size=(40, 5, 6)) + rng.normal(size=(1, 5, 6))
    V[:, 1:3, 2:4] += rng.normal(size=(40, 1, 1)) * 2.0  # a correlated patch
    C = VS.correlation_image(V)
    H, W = V.shape[1:]
    for y in range(H):
        for x in range(W):
            vals = [np.corrcoef(V[:, y, x], V[:, y + dy, x + dx])[0, 1]
                    for dy, dx in VS.NEIGHBOURS if 0 <= y + dy < H and 0 <= x + dx < W]
            assert abs(C[y, x] - np.mean(vals)) < 1e-12
    assert len([1 for dy, dx in VS.NEIGHBOURS if 0 <= dy < H and 0 <= dx < W]) == 3  # corner


def test_closed_forms():
    t = rng.normal(size=50)
    same = np.broadcast_to(t[:, None, None], (50, 4, 7)).copy()
    assert np.allclose(VS.correlation_image(same), 1.0, atol=1e-12)
    # columns alternating t, -t: an interior pixel's six neighbours in the
    # adjacent columns correlate -1, the two in its own column +1
    alt = same.copy()
    alt[:, :, 1::2] *= -1.0
    C = VS.correlation_image(alt)
    assert abs(C[1, 3] - (6 * -1 + 2 * 1) / 8) < 1e-12
    # per-pixel positive affine maps leave C unchanged; the mean follows them
    V = rng.normal(size=(30, 6, 5))
    a = rng.uniform(0.5, 3.0, size=(6, 5))
    b = rng.uniform(-100, 100, size=(6, 5))
    assert np.allclose(VS.correlation_image(a * V + b), VS.correlation_image(V), atol=1e-12)
    assert np.allclose(VS.average_image(a * V + b), a * V.mean(0) + b, atol=1e-12)
    # a constant pixel correlates 0 with everything, and its neighbours average it in
    V[:, 2, 2] = 7.0
    C = VS.correlation_image(V)
    assert C[2, 2] == 0.0
    ref = np.mean([VS.pair_correlation(V[:, 1, 1], V[:, 1 + dy, 1 + dx]) for dy, dx in VS.NEIGHBOURS])
    assert abs(C[1, 1] - ref) < 1e-12
    assert VS.pair_correlation(V[:, 2, 2], V[:, 1, 1]) == 0.0


def test_independent_noise_correlates_near_zero():
    V = rng.normal(size=(4000, 8, 8))
    C = VS.correlation_image(V)
    assert np.abs(C).max() < 5 / np.sqrt(4000)


def test_on_the_oracles_corrected_video():
    """Neuron footprints share their activity: pixels inside a footprint
    correlate more with their neighbours than background pixels do."""
    cfg = synth.tiny_config(read_sigma=5.0, walk_sigma=0.0, dff_lo=0.3, dff_hi=0.3)
    frames, _, T = synth.make_video(cfg, 300)
    o = oracle.Oracle(cfg.H, cfg.W)
    o.set_template(T.double().numpy())
    r = o.process(frames.numpy(), shifts_in=np.zeros((300, 2)), want_summary=False)
    C = VS.correlation_image(r["corrected"])
    m = synth.roi_masks(cfg).numpy().any(axis=0)
    assert C[m].mean() > C[~m].mean() + 0.1
    assert np.allclose(VS.average_image(r["corrected"]), frames.numpy().mean(0), atol=1e-9)
