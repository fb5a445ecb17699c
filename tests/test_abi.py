"""The C-ABI library loads on a machine without a GPU, exports every entry
point that include/sg.h declares, and rejects bad arguments before touching
the device (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:sg_status|const char\*)\s+(sg_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("sg_volume_create", "sg_upload_bricks", "sg_set_transfer_function", "sg_select_lod", "sg_render"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1804_08197_b300 import sg
    lib = ctypes.CDLL(sg.LIB_PATH)
    for n in _declared():
        assert hasattr(lib, n), n
    assert set(_declared()) <= set(sg.EXPORTS) | {"sg_last_error", "sg_version"}
    assert "sm_103a" in sg.sg_version()


def test_invalid_arguments_are_rejected_on_the_host():
    from paper_1804_08197_b300 import sg
    lib = sg.lib
    assert lib.sg_volume_create(None, None) == sg.SG_ERR_INVALID_ARG
    assert "NULL" in lib.sg_last_error().decode()
    d = sg.sg_volume_desc()
    d.dims[:] = [64, 64, 64]
    d.dtype, d.channels, d.timepoints, d.brick_size, d.apron, d.lod_levels = 3, 1, 1, 32, 1, 2
    h = ctypes.c_void_p()
    assert lib.sg_volume_create(ctypes.byref(d), ctypes.byref(h)) == sg.SG_ERR_INVALID_ARG  # dtype 3
    d.dtype, d.brick_size = sg.SG_U8, 12
    assert lib.sg_volume_create(ctypes.byref(d), ctypes.byref(h)) == sg.SG_ERR_INVALID_ARG  # not a multiple of 8
    d.brick_size, d.apron = 32, 2
    assert lib.sg_volume_create(ctypes.byref(d), ctypes.byref(h)) == sg.SG_ERR_INVALID_ARG  # apron must be 1
    d.apron = 1
    for bad_skip, brick in [(3, 32), (64, 64), (16, 24), (4, 256)]:  # not 2/4/8/16, not dividing, > 32 cells
        d.skip_block, d.brick_size = bad_skip, brick
        assert lib.sg_volume_create(ctypes.byref(d), ctypes.byref(h)) == sg.SG_ERR_INVALID_ARG, (bad_skip, brick)
        assert "skip_block" in lib.sg_last_error().decode()
    assert lib.sg_render(None, None, None, None, None) == sg.SG_ERR_INVALID_ARG
    assert lib.sg_select_lod(None, None, None, None) == sg.SG_ERR_INVALID_ARG
    assert lib.sg_volume_destroy(None) == sg.SG_OK


def test_no_cpu_fallback_when_the_library_is_missing(tmp_path, monkeypatch):
    import importlib.util
    from paper_1804_08197_b300 import sg
    spec = importlib.util.spec_from_file_location("sg_copy", sg.__file__)
    mod = importlib.util.module_from_spec(spec)
    monkeypatch.setattr(os.path, "exists", lambda p: False if p.endswith("libsg.so") else os.path.isfile(p))
    with pytest.raises(ImportError):
        spec.loader.exec_module(mod)


def test_autotuner_cache_round_trip(tmp_path):
    """The autotuner's pick survives the process: store appends, lookup finds
    the latest line for a key, other keys and a missing file give nothing,
    unsupported shapes and bad keys are refused (host only, no GPU)."""
    from paper_1804_08197_b300 import sg
    path = tmp_path / "tuned.txt"
    assert sg.sg_render_config_lookup(path, "B300 bench") is None
    a = dict(persistent=1, tile_w=8, tile_h=8, rays_per_thread=1)
    b = dict(persistent=0, tile_w=16, tile_h=16, rays_per_thread=2)
    sg.sg_render_config_store(path, "B300 bench", a)
    sg.sg_render_config_store(path, "B300 other", b)
    assert sg.sg_render_config_lookup(path, "B300 bench") == a
    sg.sg_render_config_store(path, "B300 bench", b)
    assert sg.sg_render_config_lookup(path, "B300 bench") == b
    assert sg.sg_render_config_lookup(path, "B200 bench") is None
    with pytest.raises(sg.SGError):
        sg.sg_render_config_store(path, "bad", dict(persistent=0, tile_w=7, tile_h=8, rays_per_thread=1))
    with pytest.raises(sg.SGError):
        sg.sg_render_config_store(path, "tab\there", a)
