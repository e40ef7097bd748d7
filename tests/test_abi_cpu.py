"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every entry
point include/dqo.h declares; the Python binding declares exactly those names."""
import ctypes
import os
import re

from paper_2503_02223_gb300 import build as b

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "dqo.h")).read()
    return sorted(set(re.findall(r"^DQO_API\s+[\w\s\*]+?\b(dqo_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_abi():
    fns = header_functions()
    for want in ("dqo_create", "dqo_destroy", "dqo_render_forward", "dqo_render_backward", "dqo_quadric_project",
                 "dqo_quadric_bbox_loss", "dqo_settings_default", "dqo_get_buffer"):
        assert want in fns


def test_library_loads_and_exports_every_declared_symbol():
    path = b.build()
    lib = ctypes.CDLL(path)
    for fn in header_functions():
        assert hasattr(lib, fn), fn
    # pure host entry points work without a device
    assert lib.dqo_version() >= 100
    lib.dqo_status_str.restype = ctypes.c_char_p
    assert lib.dqo_status_str(1) == b"invalid argument"


def test_binding_matches_header():
    from paper_2503_02223_gb300 import dqo
    assert sorted(dqo._SIGS) == header_functions()


def test_settings_defaults_through_the_abi():
    from paper_2503_02223_gb300 import dqo
    s = dqo.settings()
    assert (s.tile_w, s.tile_h, s.batch, s.og_filter) == (16, 16, 256, 1)
    assert abs(s.alpha_clamp - 0.99) < 1e-7 and abs(s.alpha_min - 1 / 255) < 1e-9
    assert abs(s.t_stop - 1e-4) < 1e-10 and abs(s.znear - 0.2) < 1e-7 and abs(s.lowpass - 0.3) < 1e-7


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        return
    from paper_2503_02223_gb300 import dqo
    lib = dqo.load()
    h = ctypes.c_void_p()
    assert lib.dqo_create(ctypes.byref(h), 0) == dqo.DQO_ECUDA
    assert lib.dqo_create(None, 0) == dqo.DQO_EINVAL
