"""Plain FP64 CPU oracle for the voltage-imaging frame-stream hot path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product package never
imports this module.  It shares no code with the CUDA path; its arithmetic
lives in ``vimg_oracle.c`` (plain loops, double precision, the paper's
definitions written out; each function there cites the passage it follows).

Paper: Bando et al., "Real-time Neuron Segmentation for Voltage Imaging",
BIBM 2023 -- Sec. II (ZNCC motion correction on 21x21 patches), Sec. III-B
(segments of L = 50 frames, Eq. 1 spatial summary, Eq. 2 max-median summary
with a sigma = 3 px Gaussian).

Parity status per function (pins live in ``tests/test_oracle_pins.py``):
  patch_grid, zncc, surface, peak (integer part), resample, gauss, median,
  highpass, segments: pinned.
  peak (subpixel parabola): pinned to its closed form on exact quadratics;
  the paper itself prints no subpixel method, so agreement with the paper is
  a reading, not a pin.
  narrow_center, narrow_estimate (learned-proposal window and fallback rule):
  pinned to the full window's values and decisions; a reading of the task's
  configuration, not of the paper.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vimg_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")

FLAG_OUT_HIGHPASS = 4


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP, -O2, IEEE arithmetic)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i, d = ctypes.c_int, ctypes.c_double
        L.orc_num_threads.restype = i
        L.orc_set_num_threads.argtypes = [i]
        L.orc_patch_grid.argtypes = [i, i, i, i, P]
        L.orc_patch_grid.restype = i
        L.orc_zncc.argtypes = [P, i, i, P, i, i, i, i, i]
        L.orc_zncc.restype = d
        L.orc_surface.argtypes = [P, i, i, P, i, i, i, i, i, i, P, P]
        L.orc_surface.restype = i
        L.orc_peak.argtypes = [P, i, i, i, i, P, P, P]
        L.orc_resample.argtypes = [P, i, i, d, d, P]
        L.orc_gauss.argtypes = [P, i, i, d, P]
        L.orc_gauss.restype = i
        L.orc_median.argtypes = [P, i]
        L.orc_median.restype = d
        L.orc_create.argtypes = [i, i, i, i, i, d, i, i]
        L.orc_create.restype = P
        L.orc_destroy.argtypes = [P]
        L.orc_set_template.argtypes = [P, P]
        L.orc_seek.argtypes = [P, ctypes.c_longlong, P, i]
        L.orc_seek.restype = i
        L.orc_frames_seen.argtypes = [P]
        L.orc_frames_seen.restype = ctypes.c_longlong
        L.orc_process.argtypes = [P, P, i, P, P, P, P, P, P, P, P]
        L.orc_set_rois.argtypes = [P, P, i]
        L.orc_set_rois.restype = i
        L.orc_roi_means.argtypes = [P, i, i, P, i, P]
        L.orc_process.restype = i
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _u16(a):
    return np.ascontiguousarray(a, dtype=np.uint16)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    lib().orc_set_num_threads(int(n))


def patch_grid(H, W, R, P=21):
    out = np.zeros(4, np.int32)
    if lib().orc_patch_grid(H, W, R, P, _p(out)):
        raise ValueError("no patch fits")
    return tuple(int(v) for v in out)


def zncc(F, T, ty, tx, P, dy, dx) -> float:
    F, T = _u16(F), _f64(T)
    H, W = F.shape
    return lib().orc_zncc(_p(F), H, W, _p(T), ty, tx, P, dy, dx)


def surface(F, T, R, P=21, window=None, per_patch=False):
    """C[wy][wx] over window (dy0, dx0, wy, wx); default the full +-R window."""
    F, T = _u16(F), _f64(T)
    H, W = F.shape
    dy0, dx0, wy, wx = window if window is not None else (-R, -R, 2 * R + 1, 2 * R + 1)
    C = np.zeros((wy, wx), np.float64)
    Z = None
    if per_patch:
        g = patch_grid(H, W, R, P)
        Z = np.zeros((g[0] * g[1], wy, wx), np.float64)
    if lib().orc_surface(_p(F), H, W, _p(T), R, P, dy0, dx0, wy, wx, _p(C), _p(Z)):
        raise ValueError("bad window")
    return (C, Z) if per_patch else C


def peak(C, dy0, dx0):
    C = _f64(C)
    wy, wx = C.shape
    s = np.zeros(2, np.float64)
    d = np.zeros(2, np.int32)
    info = np.zeros(3, np.float64)
    lib().orc_peak(_p(C), dy0, dx0, wy, wx, _p(s), _p(d), _p(info))
    return s, d, info


def narrow_center(proposal_px, R, half=3):
    """Centre of the narrow window: the proposal (dy, dx) in px rounded to the
    nearest integer (halves to even), then clamped so that the window of
    +-half stays inside [-R, R]; a non-finite proposal counts as 0."""
    lim = R - half
    c = []
    for v in proposal_px:
        v = float(v)
        v = float(np.rint(min(64.0, max(-64.0, v)))) if np.isfinite(v) else 0.0
        c.append(int(max(-lim, min(lim, v))))
    return tuple(c)


def narrow_estimate(F, T, R, proposal_px, thresh=0.5, half=3, P=21):
    """Learned-proposal reading (task config 4; not in the paper): the surface
    on the (2 half + 1)^2 displacements around narrow_center(proposal), its peak
    and parabola (the peak() rules on that window); when d* lies on the window's
    border (no neighbour for the parabola) or C(d*) < thresh, the full +-R
    window decides instead.  Returns dict(center, fallback, shifts, dstar, info,
    narrow = the window's surface)."""
    cy, cx = narrow_center(proposal_px, R, half)
    w = 2 * half + 1
    Cn = surface(F, T, R, P, window=(cy - half, cx - half, w, w))
    s, d, info = peak(Cn, cy - half, cx - half)
    edge = int(info[2]) != 0
    out = dict(center=(cy, cx), narrow=Cn, fallback=bool(edge or info[0] < thresh))
    if out["fallback"]:
        s, d, info = peak(surface(F, T, R, P), -R, -R)
    out.update(shifts=s, dstar=d, info=info)
    return out


def resample(F, sy, sx):
    F = _u16(F)
    H, W = F.shape
    V = np.zeros((H, W), np.float64)
    lib().orc_resample(_p(F), H, W, float(sy), float(sx), _p(V))
    return V


def gauss(V, sigma=3.0):
    V = _f64(V)
    H, W = V.shape
    out = np.zeros_like(V)
    if lib().orc_gauss(_p(V), H, W, float(sigma), _p(out)):
        raise ValueError("image smaller than the Gaussian radius")
    return out


def roi_means(V, masks):
    """Mean of the frame V [H][W] within each mask [n_rois][H][W] (0 if empty)."""
    V = _f64(V)
    m = np.ascontiguousarray(np.asarray(masks) != 0, dtype=np.uint8)
    out = np.zeros(m.shape[0], np.float64)
    lib().orc_roi_means(_p(V), V.shape[0], V.shape[1], _p(m), m.shape[0], _p(out))
    return out


def median(v) -> float:
    v = _f64(v)
    return lib().orc_median(_p(v), v.size)


class Oracle:
    """Streaming FP64 pipeline: the same contract as the library's handle."""

    def __init__(self, H, W, R=16, P=21, L=50, sigma=3.0, hp_window=0, flags=0):
        self.H, self.W, self.R, self.P, self.L = H, W, R, P, L
        self._h = lib().orc_create(H, W, R, P, L, float(sigma), hp_window, flags)
        if not self._h:
            raise ValueError("bad oracle parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    @property
    def frames_seen(self) -> int:
        return lib().orc_frames_seen(self._h)

    def set_template(self, T):
        T = _f64(T)
        assert T.shape == (self.H, self.W)
        lib().orc_set_template(self._h, _p(T))

    def seek(self, t_start, history=None):
        """Starts the stream at absolute frame t_start (a multiple of L) with the
        frames before it, history [n][H][W], as high-pass history only."""
        h = None if history is None else _u16(history)
        n = 0 if h is None else h.shape[0]
        if lib().orc_seek(self._h, int(t_start), _p(h), n):
            raise ValueError("bad seek")

    def set_rois(self, masks):
        """ROI masks [n_rois][H][W] (nonzero = in the ROI) for the voltage traces."""
        m = np.ascontiguousarray(np.asarray(masks) != 0, dtype=np.uint8)
        assert m.ndim == 3 and m.shape[1:] == (self.H, self.W)
        self.n_rois = m.shape[0]
        if lib().orc_set_rois(self._h, _p(m), self.n_rois) != 0:
            raise MemoryError("oracle ROI masks")

    def process(self, frames, shifts_in=None, want_surface=False, want_corrected=True,
                want_summary=True):
        frames = _u16(frames)
        n = frames.shape[0]
        H, W, L = self.H, self.W, self.L
        w = 2 * self.R + 1
        kmax = (self.frames_seen % L + n) // L
        out = {
            "shifts": np.zeros((n, 2), np.float64),
            "dstar": np.zeros((n, 2), np.int32),
            "info": np.zeros((n, 3), np.float64),
        }
        out["surface"] = np.zeros((n, w, w), np.float64) if want_surface else None
        out["corrected"] = np.zeros((n, H, W), np.float64) if want_corrected else None
        summ = np.zeros((max(kmax, 1), 2, H, W), np.float64) if want_summary else None
        nr = getattr(self, "n_rois", 0)
        out["traces"] = np.zeros((n, nr), np.float64) if nr else None
        sin = None if shifts_in is None else _f64(shifts_in).reshape(n, 2)
        k = lib().orc_process(self._h, _p(frames), n, _p(sin), _p(out["shifts"]),
                              _p(out["dstar"]), _p(out["info"]), _p(out["surface"]),
                              _p(out["corrected"]), _p(summ), _p(out["traces"]))
        if k < 0:
            raise RuntimeError("oracle process failed")
        assert k == kmax
        out["summary"] = summ[:k] if summ is not None else None
        out["k"] = k
        return out
