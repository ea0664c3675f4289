"""Host-only checks of the C ABI: the library loads without a GPU, exports
every function include/vimg.h declares, and rejects bad arguments before any
CUDA call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def vimg():
    from paper_2403_16438_gb300 import build
    build.build()
    from paper_2403_16438_gb300 import vimg as v
    return v


def declared_functions():
    src = open(os.path.join(ROOT, "include", "vimg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vimg_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(vimg):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(vimg.lib, n), n
    assert sorted(vimg.EXPORTS) == names


def test_struct_layouts_match_header(vimg, tmp_path):
    """The binding's structs against the header itself: a C program built with
    gcc from include/vimg.h prints the sizes and member offsets."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    src = tmp_path / "layout.c"
    fields = {"vimg_params": [f for f, _ in vimg.Params._fields_],
              "vimg_io": [f for f, _ in vimg.IO._fields_],
              "vimg_batch_opts": [f for f, _ in vimg.BatchOpts._fields_]}
    body = "".join(
        f'  printf("{t} %zu", sizeof({t}));' + "".join(
            f' printf(" %zu", offsetof({t}, {f}));' for f in fs) + ' printf("\\n");\n'
        for t, fs in fields.items())
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "vimg.h"\n'
                   "int main(void) {\n" + body + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src),
                           "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    for line, (cls, t) in zip(out, [(vimg.Params, "vimg_params"), (vimg.IO, "vimg_io"),
                                    (vimg.BatchOpts, "vimg_batch_opts")]):
        name, size, *offs = line.split()
        assert name == t and int(size) == ctypes.sizeof(cls)
        assert [int(o) for o in offs] == [getattr(cls, f).offset for f, _ in cls._fields_]


def test_defaults(vimg):
    p = vimg.default_params()
    assert (p.search_radius, p.patch, p.segment_len, p.gauss_sigma) == (16, 21, 50, 3.0)
    assert p.hp_window == 0 and p.flags == 0 and abs(p.fallback_zncc - 0.5) < 1e-7
    assert p.narrow_radius == 2 and p.max_chunk > 0


@pytest.mark.parametrize("field,value,H,W", [
    ("search_radius", 17, 512, 512), ("search_radius", -1, 512, 512), ("patch", 15, 512, 512),
    ("segment_len", 0, 512, 512), ("segment_len", 51, 512, 512), ("gauss_sigma", 3.5, 512, 512),
    ("gauss_sigma", 0.0, 512, 512), ("hp_window", 65, 512, 512), ("max_chunk", 0, 512, 512),
    ("flags", 64, 512, 512), ("search_radius", 16, 52, 512), ("search_radius", 16, 0, 512),
])
def test_create_rejects_bad_parameters(vimg, field, value, H, W):
    p = vimg.default_params()
    setattr(p, field, value)
    h = vimg.lib.vimg_create(H, W, ctypes.byref(p))
    assert not h
    assert len(vimg.lib.vimg_last_error(None)) > 0


def test_null_handle_calls(vimg):
    L = vimg.lib
    L.vimg_destroy(None)
    assert L.vimg_process(None, None, 0, None, None, None) == vimg.ERR_ARG
    assert L.vimg_set_template(None, None) == vimg.ERR_ARG
    assert L.vimg_reset(None) == vimg.ERR_ARG
    assert L.vimg_frames_seen(None) == -1
    assert L.vimg_state_bytes(None) == vimg.ERR_ARG
    assert L.vimg_get_state(None, None, 0) == vimg.ERR_ARG
    assert L.vimg_set_state(None, None, 0) == vimg.ERR_ARG
    assert b"sm_103a" in L.vimg_version()


def test_unet_architecture_matches_the_oracle(vimg):
    """The library's U-Net (parameter layout and layer list) is the oracle's reading."""
    import oracle.unet as U
    assert vimg.unet_layers() == U.architecture()
    assert vimg.unet_param_count() == U.param_count()


def test_unet_create_rejects_small_images(vimg):
    assert not vimg.lib.vimg_unet_create(63, 128, 4, None)
    assert b"64" in vimg.lib.vimg_unet_last_error(None)
    assert vimg.lib.vimg_unet_load(None, None) == vimg.ERR_ARG


def test_downstream_calls_reject_null_handles(vimg):
    """Argument checks before any CUDA call: traces, summaries, U-Net and
    footprint entry points on NULL handles."""
    L = vimg.lib
    assert L.vimg_set_rois(None, None, 0) == vimg.ERR_ARG
    assert L.vimg_video_summary(None, None, None) == vimg.ERR_ARG
    assert L.vimg_attach_unet(None, None) == vimg.ERR_ARG
    assert L.vimg_unet_run(None, None, 0, None) == vimg.ERR_ARG
    assert L.vimg_unet_activation(None, 0, None, None, None, None) == vimg.ERR_ARG
    assert L.vimg_segment(None, None, 1, None, None, 0, None, None) == vimg.ERR_ARG
    assert not L.vimg_segmenter_create(0, 64, 4, None)


def test_remaining_entry_points_reject_bad_arguments(vimg):
    """Argument checks that run before any CUDA call, for the entry points not
    covered above: host-buffer, batch, profiling, proposal, CNN training and
    allocation-free calls.  Every case returns before a pointer is used on the
    device (checked by reading each function's validation order)."""
    import numpy as np
    L = vimg.lib
    ARG, SIZE = vimg.ERR_ARG, vimg.ERR_SIZE
    assert L.vimg_process_io(None, None, 0, None) == ARG
    assert L.vimg_process_host(None, None, 0, None, None, None) == ARG
    assert L.vimg_profile_enable(None, 1) == ARG
    assert L.vimg_profile_read(None, None, None, 1) == ARG
    assert L.vimg_synchronize(None) == ARG
    assert L.vimg_load_proposal(None, None) == ARG
    assert L.vimg_proposal_stats(None, None, None) == ARG
    # several videos per call: no handles, too few / too many, null frame tables
    nulls = (ctypes.c_void_p * 65)()
    assert L.vimg_process_batch(None, 1, None, None, None, None, None, None, None) == ARG
    assert L.vimg_process_batch(nulls, 0, None, None, None, None, None, None, None) == ARG
    assert L.vimg_process_batch(nulls, 65, nulls, nulls, None, None, None, None, None) == ARG
    assert L.vimg_process_batch(nulls, 1, None, None, None, None, None, None, None) == ARG
    counts = (ctypes.c_int * 1)(0)
    assert L.vimg_process_batch(nulls, 1, nulls, counts, None, None, None, None, None) == ARG
    # proposal network training calls
    assert L.vimg_cnn_prepare(None, -1, 128, 128, None, 0, None, None) == ARG
    assert L.vimg_cnn_prepare(None, 0, 64, 128, None, 0, None, None) == ARG
    assert L.vimg_cnn_pack_bf16(None, None, None) == ARG
    assert L.vimg_cnn_forward(None, None, None, 1, None, None) == ARG
    assert L.vimg_cnn_loss(None, None, 1, None, None, None) == ARG
    assert L.vimg_cnn_backward(None, None, None, None, 1, None, None, None) == ARG
    assert L.vimg_cnn_adam(None, None, None, None, 1e-3, 0.9, 0.999, 1e-8, 0, None) == ARG
    # allocation-free motion estimate: a host buffer stands in for the template
    # pointer; every case below returns before it is used
    buf = np.zeros(16, np.float32)
    tp = ctypes.c_void_p(buf.ctypes.data)
    assert L.vimg_motion_noalloc(None, None, 0, 128, 128, 16, None, None, None) == ARG
    assert L.vimg_motion_noalloc(tp, None, -1, 128, 128, 16, None, None, None) == ARG
    assert L.vimg_motion_noalloc(tp, None, 1, 128, 128, 16, None, None, None) == ARG
    assert L.vimg_motion_noalloc(tp, None, 0, 128, 128, 17, None, None, None) == ARG
    assert L.vimg_motion_noalloc(tp, None, 0, 52, 128, 16, None, None, None) == SIZE
    assert L.vimg_motion_noalloc(tp, None, 0, 1 << 20, 128, 16, None, None, None) == SIZE
    # U-Net stage
    assert L.vimg_unet_synchronize(None) == ARG
    assert L.vimg_unet_profile(None, 1) == ARG
    assert L.vimg_unet_profile_read(None, None, None, None, 1) == ARG
