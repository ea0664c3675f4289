"""GB300-native frame-stream hot path of real-time voltage-imaging analysis.

Per-frame rigid motion correction by patch-tiled ZNCC against a template,
fused with the per-segment summary images (Eq. 1 temporal mean, Eq. 2
max-minus-median of the Gaussian-smoothed video) and a temporal high-pass,
after Bando et al., "Real-time Neuron Segmentation for Voltage Imaging"
(BIBM 2023), Sec. II and Sec. III-B.

The compute runs in hand-written CUDA kernels for sm_103a behind a C ABI
(``include/vimg.h``); ``vimg`` is the thin ctypes binding.  Import of the
binding is lazy so that the input generator (``synth``) works without a GPU.
"""
