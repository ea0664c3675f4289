"""Thin ctypes binding of libvimg (include/vimg.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  torch supplies device memory and the stream.  There is no CPU
fallback: if the library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libvimg.so")

OK = 0
ERR_ARG, ERR_NO_TEMPLATE, ERR_CUDA, ERR_TIMEOUT, ERR_OOM, ERR_SIZE = -1, -2, -3, -4, -5, -6
REGION_TOO_LARGE, REGION_TOO_MANY = 1, 2  # vimg_segment_status
CORR_BF16, PROPOSAL_CNN, OUT_HIGHPASS, VIDEO_SUMMARY, TEMPORAL_SMEM = 1, 2, 4, 8, 16


class Params(ctypes.Structure):
    _fields_ = [
        ("search_radius", ctypes.c_int),
        ("patch", ctypes.c_int),
        ("segment_len", ctypes.c_int),
        ("gauss_sigma", ctypes.c_float),
        ("hp_window", ctypes.c_int),
        ("flags", ctypes.c_int),
        ("fallback_zncc", ctypes.c_float),
        ("narrow_radius", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("timeout_spins", ctypes.c_longlong),
        ("max_chunk", ctypes.c_int),
        ("corr_group", ctypes.c_int),
    ]


class IO(ctypes.Structure):
    _fields_ = [
        ("shifts", ctypes.c_void_p),
        ("corrected", ctypes.c_void_p),
        ("summary", ctypes.c_void_p),
        ("peak_info", ctypes.c_void_p),
        ("surface", ctypes.c_void_p),
        ("shifts_in", ctypes.c_void_p),
        ("traces", ctypes.c_void_p),
        ("prob", ctypes.c_void_p),
        ("proposal", ctypes.c_void_p),
    ]


class BatchOpts(ctypes.Structure):
    _fields_ = [
        ("chunk", ctypes.c_int),
        ("ring_chunks", ctypes.c_int),
        ("use_graph", ctypes.c_int),
        ("reserved", ctypes.c_int),
    ]


# Every symbol include/vimg.h declares (checked by the host-only tests).
EXPORTS = [
    "vimg_default_params", "vimg_create", "vimg_destroy", "vimg_set_template", "vimg_process",
    "vimg_process_io", "vimg_process_host", "vimg_frames_seen", "vimg_reset", "vimg_seek",
    "vimg_last_error",
    "vimg_version", "vimg_profile_enable", "vimg_profile_read", "vimg_motion_noalloc",
    "vimg_cnn_param_count", "vimg_cnn_workspace_floats", "vimg_cnn_prepare", "vimg_cnn_pack_bf16",
    "vimg_cnn_forward", "vimg_cnn_loss", "vimg_cnn_backward", "vimg_cnn_adam", "vimg_load_proposal",
    "vimg_proposal_stats", "vimg_synchronize", "vimg_process_batch", "vimg_set_rois",
    "vimg_unet_param_count", "vimg_unet_layers", "vimg_unet_create", "vimg_unet_destroy",
    "vimg_unet_last_error", "vimg_unet_load", "vimg_unet_run", "vimg_unet_synchronize",
    "vimg_unet_profile", "vimg_unet_profile_read", "vimg_attach_unet", "vimg_unet_activation",
    "vimg_video_summary", "vimg_segmenter_create", "vimg_segmenter_destroy",
    "vimg_segmenter_last_error", "vimg_segment", "vimg_segment_status", "vimg_fma_rate",
    "vimg_state_bytes", "vimg_get_state", "vimg_set_state",
]
NSTAGES = 7
STAGES = ["stats", "corr", "peak", "temporal", "proposal", "carry_copy", "downstream"]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libvimg.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    P, i, vp = ctypes.POINTER, ctypes.c_int, ctypes.c_void_p
    L.vimg_default_params.argtypes = [P(Params)]
    L.vimg_default_params.restype = None
    L.vimg_create.argtypes = [i, i, P(Params)]
    L.vimg_create.restype = vp
    L.vimg_destroy.argtypes = [vp]
    L.vimg_destroy.restype = None
    L.vimg_set_template.argtypes = [vp, vp]
    L.vimg_set_template.restype = i
    L.vimg_seek.argtypes = [vp, ctypes.c_longlong, vp, i]
    L.vimg_seek.restype = i
    L.vimg_fma_rate.argtypes = [vp, P(ctypes.c_double)]
    L.vimg_fma_rate.restype = i
    L.vimg_state_bytes.argtypes = [vp]
    L.vimg_state_bytes.restype = ctypes.c_longlong
    L.vimg_get_state.argtypes = [vp, vp, ctypes.c_longlong]
    L.vimg_get_state.restype = i
    L.vimg_set_state.argtypes = [vp, vp, ctypes.c_longlong]
    L.vimg_set_state.restype = i
    L.vimg_segmenter_create.argtypes = [i, i, i, vp]
    L.vimg_segmenter_create.restype = vp
    L.vimg_segmenter_destroy.argtypes = [vp]
    L.vimg_segmenter_destroy.restype = None
    L.vimg_segmenter_last_error.argtypes = [vp]
    L.vimg_segmenter_last_error.restype = ctypes.c_char_p
    L.vimg_segment.argtypes = [vp, vp, i, vp, vp, i, vp, P(i)]
    L.vimg_segment.restype = i
    L.vimg_segment_status.argtypes = [vp, vp, i]
    L.vimg_segment_status.restype = i
    L.vimg_video_summary.argtypes = [vp, vp, vp]
    L.vimg_video_summary.restype = i
    L.vimg_set_rois.argtypes = [vp, vp, i]
    L.vimg_set_rois.restype = i
    L.vimg_unet_param_count.argtypes = []
    L.vimg_unet_param_count.restype = i
    L.vimg_unet_layers.argtypes = [vp, vp, vp, i]
    L.vimg_unet_layers.restype = i
    L.vimg_unet_create.argtypes = [i, i, i, vp]
    L.vimg_unet_create.restype = vp
    L.vimg_unet_destroy.argtypes = [vp]
    L.vimg_unet_destroy.restype = None
    L.vimg_unet_last_error.argtypes = [vp]
    L.vimg_unet_last_error.restype = ctypes.c_char_p
    L.vimg_unet_load.argtypes = [vp, vp]
    L.vimg_unet_load.restype = i
    L.vimg_unet_run.argtypes = [vp, vp, i, vp]
    L.vimg_unet_run.restype = i
    L.vimg_unet_synchronize.argtypes = [vp]
    L.vimg_unet_synchronize.restype = i
    L.vimg_unet_profile.argtypes = [vp, i]
    L.vimg_unet_profile.restype = i
    L.vimg_unet_profile_read.argtypes = [vp, vp, vp, vp, i]
    L.vimg_unet_profile_read.restype = i
    L.vimg_unet_activation.argtypes = [vp, i, vp, vp, vp, vp]
    L.vimg_unet_activation.restype = i
    L.vimg_attach_unet.argtypes = [vp, vp]
    L.vimg_attach_unet.restype = i
    L.vimg_process.argtypes = [vp, vp, i, vp, vp, vp]
    L.vimg_process.restype = i
    L.vimg_process_io.argtypes = [vp, vp, i, P(IO)]
    L.vimg_process_io.restype = i
    L.vimg_process_host.argtypes = [vp, vp, i, vp, vp, vp]
    L.vimg_process_host.restype = i
    L.vimg_frames_seen.argtypes = [vp]
    L.vimg_frames_seen.restype = ctypes.c_longlong
    L.vimg_reset.argtypes = [vp]
    L.vimg_reset.restype = i
    L.vimg_last_error.argtypes = [vp]
    L.vimg_last_error.restype = ctypes.c_char_p
    L.vimg_profile_enable.argtypes = [vp, i]
    L.vimg_profile_enable.restype = i
    L.vimg_profile_read.argtypes = [vp, vp, vp, i]
    L.vimg_profile_read.restype = i
    L.vimg_motion_noalloc.argtypes = [vp, vp, i, i, i, i, vp, vp, vp]
    L.vimg_motion_noalloc.restype = i
    L.vimg_cnn_param_count.argtypes = []
    L.vimg_cnn_param_count.restype = i
    L.vimg_cnn_workspace_floats.argtypes = [i]
    L.vimg_cnn_workspace_floats.restype = ctypes.c_size_t
    L.vimg_cnn_prepare.argtypes = [vp, i, i, i, vp, ctypes.c_longlong, vp, vp]
    L.vimg_cnn_prepare.restype = i
    L.vimg_cnn_pack_bf16.argtypes = [vp, vp, vp]
    L.vimg_cnn_pack_bf16.restype = i
    L.vimg_cnn_forward.argtypes = [vp, vp, vp, i, vp, vp]
    L.vimg_cnn_forward.restype = i
    L.vimg_cnn_loss.argtypes = [vp, vp, i, vp, vp, vp]
    L.vimg_cnn_loss.restype = i
    L.vimg_cnn_backward.argtypes = [vp, vp, vp, vp, i, vp, vp, vp]
    L.vimg_cnn_backward.restype = i
    L.vimg_cnn_adam.argtypes = [vp, vp, vp, vp, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                ctypes.c_float, i, vp]
    L.vimg_cnn_adam.restype = i
    L.vimg_load_proposal.argtypes = [vp, vp]
    L.vimg_load_proposal.restype = i
    L.vimg_proposal_stats.argtypes = [vp, vp, vp]
    L.vimg_proposal_stats.restype = i
    L.vimg_synchronize.argtypes = [vp]
    L.vimg_synchronize.restype = i
    L.vimg_process_batch.argtypes = [vp, i, vp, vp, vp, vp, vp, vp, P(BatchOpts)]
    L.vimg_process_batch.restype = i
    L.vimg_version.argtypes = []
    L.vimg_version.restype = ctypes.c_char_p
    return L


lib = _load()


class VimgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"vimg error {code}: {msg}")
        self.code = code


def fma_rate(stream=None) -> float:
    """Measured FP32 FMA rate of the current device, FLOP/s (vimg_fma_rate)."""
    if stream is None:
        stream = torch.cuda.current_stream()
    out = ctypes.c_double()
    rc = lib.vimg_fma_rate(ctypes.c_void_p(stream.cuda_stream), ctypes.byref(out))
    if rc < 0:
        raise VimgError(rc, "vimg_fma_rate failed")
    return out.value


def default_params() -> Params:
    p = Params()
    lib.vimg_default_params(ctypes.byref(p))
    return p


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Handle:
    """One stream of frames of one H x W video (see vimg_create)."""

    def __init__(self, H, W, stream=None, **kw):
        p = default_params()
        for k, v in kw.items():
            if not hasattr(p, k):
                raise TypeError(f"unknown parameter {k}")
            setattr(p, k, v)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        p.stream = ctypes.c_void_p(stream.cuda_stream)
        self.params = p
        self.H, self.W = H, W
        self.n_rois = 0
        self._h = lib.vimg_create(H, W, ctypes.byref(p))
        if not self._h:
            raise VimgError(ERR_ARG, lib.vimg_last_error(None).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib.vimg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc < 0:
            raise VimgError(rc, lib.vimg_last_error(self._h).decode())
        return rc

    @property
    def frames_seen(self) -> int:
        return lib.vimg_frames_seen(self._h)

    def segments_for(self, n: int) -> int:
        L = self.params.segment_len
        return (self.frames_seen % L + n) // L

    def set_template(self, template: torch.Tensor):
        assert template.is_cuda and template.dtype == torch.float32
        assert template.shape == (self.H, self.W) and template.is_contiguous()
        self._template = template
        self._check(lib.vimg_set_template(self._h, _ptr(template)))

    def get_state(self) -> bytes:
        """The stream state (vimg_get_state) as bytes: position, open segment,
        high-pass history, whole-video sums, proposal counters."""
        n = lib.vimg_state_bytes(self._h)
        if n < 0:
            self._check(int(n))
        buf = ctypes.create_string_buffer(int(n))
        self._check(lib.vimg_get_state(self._h, buf, n))
        return buf.raw

    def set_state(self, state: bytes):
        """Restores a state from get_state of a handle with the same parameters."""
        buf = ctypes.create_string_buffer(bytes(state), len(state))
        self._check(lib.vimg_set_state(self._h, buf, len(state)))

    def seek(self, t_start: int, history: torch.Tensor | None = None):
        """Starts the stream at absolute frame t_start (a multiple of the segment
        length); history: cuda uint16 [n, H, W], the frames just before it
        (vimg_seek)."""
        n = 0 if history is None else history.shape[0]
        if history is not None:
            assert history.is_cuda and history.dtype == torch.uint16 and history.is_contiguous()
        self._check(lib.vimg_seek(self._h, int(t_start), _ptr(history), n))

    def reset(self):
        self._check(lib.vimg_reset(self._h))

    def set_rois(self, masks: torch.Tensor):
        """masks: cuda uint8 or bool [n_rois, H, W] (nonzero = in the ROI), or
        None to clear.  Traces of later process(traces=...) calls are the mean
        corrected intensity per ROI and frame."""
        if masks is None or masks.shape[0] == 0:
            self.n_rois = 0
            self._check(lib.vimg_set_rois(self._h, None, 0))
            return
        assert masks.is_cuda and masks.dtype in (torch.uint8, torch.bool)
        assert masks.shape[1:] == (self.H, self.W)
        m = masks.to(torch.uint8).contiguous()
        self._check(lib.vimg_set_rois(self._h, _ptr(m), m.shape[0]))
        self.n_rois = m.shape[0]

    def video_summary(self, average=None, correlation=None):
        """Whole-video average and local correlation images (handle created with
        flags=VIDEO_SUMMARY) into cuda float32 [H, W] tensors."""
        self._check(lib.vimg_video_summary(self._h, _ptr(average), _ptr(correlation)))

    def attach_unet(self, unet):
        """Attach a Unet of the same size (None detaches): process(prob=...)
        then gives each completed segment's spiking-probability map."""
        self._unet = unet
        self._check(lib.vimg_attach_unet(self._h, None if unet is None else unet._u))

    def process(self, frames, shifts=None, corrected=None, summary=None, peak_info=None,
                surface=None, shifts_in=None, traces=None, prob=None, proposal=None) -> int:
        """frames: cuda uint16 [n,H,W].  Outputs are optional preallocated cuda
        tensors (see vimg_io; traces: float32 [n, n_rois]; prob: float32
        [k, H, W], needs summary; proposal: float32 [n, 2], learned proposals in
        px).  Returns k, the segments written."""
        assert frames.is_cuda and frames.dtype == torch.uint16 and frames.is_contiguous()
        n = frames.shape[0]
        io = IO(_ptr(shifts), _ptr(corrected), _ptr(summary), _ptr(peak_info), _ptr(surface),
                _ptr(shifts_in), _ptr(traces), _ptr(prob), _ptr(proposal))
        return self._check(lib.vimg_process_io(self._h, _ptr(frames), n, ctypes.byref(io)))

    def process_host(self, frames_host, shifts_host=None, summary_host=None,
                     corrected=None) -> int:
        """frames_host: CPU uint16 [n,H,W] (pinned for overlap)."""
        assert not frames_host.is_cuda and frames_host.is_contiguous()
        n = frames_host.shape[0]
        return self._check(lib.vimg_process_host(self._h, _ptr(frames_host), n,
                                                 _ptr(shifts_host), _ptr(summary_host),
                                                 _ptr(corrected)))


    def load_proposal(self, params: torch.Tensor):
        assert params.is_cuda and params.dtype == torch.float32 and params.is_contiguous()
        self._check(lib.vimg_load_proposal(self._h, _ptr(params)))

    def proposal_stats(self):
        fr, fb = ctypes.c_longlong(), ctypes.c_longlong()
        self._check(lib.vimg_proposal_stats(self._h, ctypes.byref(fr), ctypes.byref(fb)))
        return fr.value, fb.value

    def synchronize(self):
        return self._check(lib.vimg_synchronize(self._h))

    def profile(self, on: bool = True):
        self._check(lib.vimg_profile_enable(self._h, 1 if on else 0))

    def profile_read(self, reset: bool = True):
        """{stage: (ms, launches)} summed since the last reset."""
        ms = (ctypes.c_double * NSTAGES)()
        cnt = (ctypes.c_longlong * NSTAGES)()
        self._check(lib.vimg_profile_read(self._h, ms, cnt, 1 if reset else 0))
        return {STAGES[i]: (ms[i], cnt[i]) for i in range(NSTAGES)}


def _ptr_array(ts):
    """ctypes array of device pointers (None -> NULL), or None if ts is None."""
    if ts is None:
        return None
    return (ctypes.c_void_p * len(ts))(*[None if t is None else t.data_ptr() for t in ts])


def process_batch(handles, frames, shifts=None, corrected=None, summary=None, chunk=0,
                  ring_chunks=0, use_graph=False):
    """Several videos per call (vimg_process_batch).  handles: list of Handle;
    frames: list of cuda uint16 [n_v, H_v, W_v]; shifts/corrected/summary: lists
    of preallocated cuda tensors (entries may be None) or None.  Runs on the
    first handle's stream.  Returns the list of segments written per video."""
    k = len(handles)
    if k == 0 or len(frames) != k:
        raise ValueError("one frames tensor per handle")
    for h, f in zip(handles, frames):
        assert f.is_cuda and f.dtype == torch.uint16 and f.is_contiguous()
        assert f.shape[1:] == (h.H, h.W)
    for outs in (shifts, corrected, summary):
        assert outs is None or len(outs) == k
    hs = (ctypes.c_void_p * k)(*[h._h for h in handles])
    ns = (ctypes.c_int * k)(*[f.shape[0] for f in frames])
    segs = (ctypes.c_int * k)()
    opts = BatchOpts(chunk, ring_chunks, 1 if use_graph else 0, 0)
    rc = lib.vimg_process_batch(hs, k, _ptr_array(frames), ns, _ptr_array(shifts),
                                _ptr_array(corrected), _ptr_array(summary), segs,
                                ctypes.byref(opts))
    handles[0]._check(rc)
    return list(segs)


def version() -> str:
    return lib.vimg_version().decode()


def unet_param_count() -> int:
    return lib.vimg_unet_param_count()


def unet_layers():
    """[(kind, cin, cout)] in parameter order, kind 'conv', 'up' or 'out'."""
    n = lib.vimg_unet_layers(None, None, None, 0)
    k, ci, co = (ctypes.c_int * n)(), (ctypes.c_int * n)(), (ctypes.c_int * n)()
    lib.vimg_unet_layers(k, ci, co, n)
    names = {0: "conv", 1: "up", 2: "out"}
    return [(names[k[i]], ci[i], co[i]) for i in range(n)]


class Unet:
    """Spiking-pixel U-Net on summary pairs (see vimg_unet_create)."""

    def __init__(self, H, W, max_segments=4, stream=None):
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.H, self.W = H, W
        self._u = lib.vimg_unet_create(H, W, max_segments, ctypes.c_void_p(stream.cuda_stream))
        if not self._u:
            raise VimgError(ERR_ARG, lib.vimg_unet_last_error(None).decode())

    def close(self):
        if getattr(self, "_u", None):
            lib.vimg_unet_destroy(self._u)
            self._u = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc < 0:
            raise VimgError(rc, lib.vimg_unet_last_error(self._u).decode())
        return rc

    def load(self, params: torch.Tensor):
        assert params.is_cuda and params.dtype == torch.float32 and params.is_contiguous()
        assert params.numel() == unet_param_count()
        self._params = params
        self._check(lib.vimg_unet_load(self._u, _ptr(params)))

    def run(self, summary: torch.Tensor, prob: torch.Tensor):
        """summary: cuda float32 [k, 2, H, W]; prob: cuda float32 [k, H, W]."""
        assert summary.is_cuda and summary.dtype == torch.float32 and summary.is_contiguous()
        k = summary.shape[0]
        assert summary.shape == (k, 2, self.H, self.W) and prob.shape == (k, self.H, self.W)
        self._check(lib.vimg_unet_run(self._u, _ptr(summary), k, _ptr(prob)))

    def synchronize(self):
        self._check(lib.vimg_unet_synchronize(self._u))

    def activation(self, i: int) -> torch.Tensor:
        """Activation i of the last internal pass (see vimg_unet_activation):
        bfloat16 [n, side, side, C] for i <= 22, float32 [n, 64, 64] for 23."""
        n, sd, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(lib.vimg_unet_activation(self._u, i, None, ctypes.byref(n), ctypes.byref(sd),
                                             ctypes.byref(c)))
        if c.value == 1 and i > 0:
            out = torch.empty((n.value, sd.value, sd.value), device="cuda", dtype=torch.float32)
        else:
            out = torch.empty((n.value, sd.value, sd.value, c.value), device="cuda",
                              dtype=torch.bfloat16)
        self._check(lib.vimg_unet_activation(self._u, i, _ptr(out), None, None, None))
        self.synchronize()
        return out

    def profile(self, on: bool = True):
        self._check(lib.vimg_unet_profile(self._u, 1 if on else 0))

    def profile_read(self, reset: bool = True):
        """(tensor-core ms, whole-run ms, tensor-core launches) since the last reset."""
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_longlong()
        self._check(lib.vimg_unet_profile_read(self._u, ctypes.byref(a), ctypes.byref(b),
                                               ctypes.byref(c), 1 if reset else 0))
        return a.value, b.value, c.value


class Segmenter:
    """Footprint reconstruction from probability maps (see vimg_segment)."""

    def __init__(self, H, W, max_segments, stream=None):
        if stream is None:
            stream = torch.cuda.current_stream()
        self.H, self.W = H, W
        self._s = lib.vimg_segmenter_create(H, W, max_segments,
                                            ctypes.c_void_p(stream.cuda_stream))
        if not self._s:
            raise VimgError(ERR_OOM, "vimg_segmenter_create failed")

    def close(self):
        if getattr(self, "_s", None):
            lib.vimg_segmenter_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, prob: torch.Tensor, max_neurons: int = 256):
        """prob: cuda float32 [K, H, W] -> (footprints [n, H, W], activity [n, K],
        region map int32 [H, W], number of regions)."""
        assert prob.is_cuda and prob.dtype == torch.float32 and prob.is_contiguous()
        K = prob.shape[0]
        foot = torch.zeros((max_neurons, self.H, self.W), device=prob.device)
        act = torch.zeros((max_neurons, K), device=prob.device)
        rmap = torch.empty((self.H, self.W), device=prob.device, dtype=torch.int32)
        nreg = ctypes.c_int()
        n = lib.vimg_segment(self._s, _ptr(prob), K, _ptr(foot), _ptr(act), max_neurons,
                             _ptr(rmap), ctypes.byref(nreg))
        if n < 0:
            raise VimgError(n, lib.vimg_segmenter_last_error(self._s).decode())
        m = min(n, max_neurons)
        return foot[:m], act[:m], rmap, nreg.value

    def status(self):
        """Per-region status of the last run: 0 factorised, REGION_TOO_LARGE or
        REGION_TOO_MANY (beyond the NMF kernel's capacity, not factorised)."""
        n = lib.vimg_segment_status(self._s, None, 0)
        if n < 0:
            raise VimgError(n, "vimg_segment_status failed")
        out = (ctypes.c_int * max(n, 1))()
        lib.vimg_segment_status(self._s, out, n)
        return [out[i] for i in range(n)]
