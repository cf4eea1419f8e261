"""The C-ABI library loads and exports every entry point include/vuda.h
declares (CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "vuda.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(vuda_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def built():
    from paper_2605_01352_b300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("vuda_env_create", "vuda_sim_step", "vuda_render", "vuda_coschedule", "vuda_coschedule_reset",
              "vuda_pipeline_run", "vuda_wait", "vuda_env_get_state", "vuda_env_set_state", "vuda_env_status",
              "vuda_raster_screen_tris", "vuda_status_str"):
        assert n in names


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu(built):
    from paper_2605_01352_b300 import vuda
    assert vuda.lib.vuda_abi_version() == 2
    assert vuda.lib.vuda_status_str(0) == b"ok"
    assert b"invalid" in vuda.lib.vuda_status_str(1)


def test_invalid_arguments_are_rejected_without_gpu(built):
    """Validation happens before any device call."""
    from paper_2605_01352_b300 import vuda
    assert vuda.lib.vuda_env_create(None, None, None, None) == vuda.ERR_INVALID
    assert vuda.lib.vuda_raster_screen_tris(None, None, 0, 0, 8, None, None, None, None) == vuda.ERR_INVALID
    assert vuda.lib.vuda_sim_step(None, 1, None, None) == vuda.ERR_INVALID
