"""The C-ABI library loads and exports every entry point include/vuda.h
declares (CPU only: no compute calls)."""
import ctypes
import os
import re
import subprocess

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
    assert vuda.lib.vuda_abi_version() == 3
    assert vuda.lib.vuda_status_str(0) == b"ok"
    assert b"invalid" in vuda.lib.vuda_status_str(1)


def test_invalid_arguments_are_rejected_without_gpu(built):
    """Validation happens before any device call."""
    from paper_2605_01352_b300 import vuda
    assert vuda.lib.vuda_env_create(None, None, None, None) == vuda.ERR_INVALID
    assert vuda.lib.vuda_raster_screen_tris(None, None, 0, 0, 8, None, None, None, None) == vuda.ERR_INVALID
    assert vuda.lib.vuda_sim_step(None, 1, None, None) == vuda.ERR_INVALID


def test_binding_structs_match_the_c_header(built, tmp_path):
    """Every struct of the binding has the size and field offsets that a C
    compiler gives the header's struct (gcc, host only)."""
    import ctypes as C

    from paper_2605_01352_b300 import vuda
    pairs = [("vuda_sim_params", vuda.SimParams), ("vuda_scene", vuda.Scene), ("vuda_env_opts", vuda.EnvOpts),
             ("vuda_env_info", vuda.EnvInfo), ("vuda_frame", vuda.Frame), ("vuda_state", vuda.State),
             ("vuda_timing", vuda.Timing), ("vuda_tune_opts", vuda.TuneOpts), ("vuda_tune_result", vuda.TuneResult),
             ("vuda_cosched_opts", vuda.CoschedOpts), ("vuda_cosched_info", vuda.CoschedInfo),
             ("vuda_serve_opts", vuda.ServeOpts), ("vuda_result", vuda.Result),
             ("vuda_serve_stats", vuda.ServeStats)]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "vuda.h"', "int main(void) {"]
    expect = []
    for cname, py in pairs:
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        expect.append((cname, "sizeof", C.sizeof(py)))
        for f in py._fields_:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {f[0]}));')
            expect.append((cname, f[0], getattr(py, f[0]).offset))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert len(got) == len(expect)
    bad = [(e, g) for e, g in zip(expect, got) if e[2] != g]
    assert not bad, bad


def test_noalloc_rejects_a_missing_body_bound_without_gpu(built):
    """The allocation-free step refuses max_bodies <= 0 for a non-empty batch
    on the host, before any device call (the kernel sizes its shared-memory
    layout from it)."""
    import ctypes as C

    from paper_2605_01352_b300 import scene as S
    from paper_2605_01352_b300 import vuda
    prm = vuda.sim_params(S.SimParams())
    fake = C.c_void_p(0x1000)   # never dereferenced: the call returns before any device work
    for mb in (0, -3):
        st = vuda.lib.vuda_sim_step_noalloc(4, 32, mb, fake, fake, fake, fake, fake, fake, fake, fake, fake, None,
                                            C.byref(prm), 1, fake, fake, fake, 0, None)
        assert st == vuda.ERR_INVALID
        if mb == 0:
            assert b"max_bodies" in vuda.lib.vuda_last_error()
    # an empty batch needs no bound and launches nothing
    assert vuda.lib.vuda_sim_step_noalloc(0, 0, 0, None, None, None, None, None, None, None, None, None, None,
                                          C.byref(prm), 1, None, None, None, 0, None) == vuda.OK


def test_noalloc_refuses_hull_contacts_without_gpu(built):
    """Hull contacts read the batch's meshes, which the allocation-free step
    does not have: it refuses the option on the host."""
    import ctypes as C
    import dataclasses

    from paper_2605_01352_b300 import scene as S
    from paper_2605_01352_b300 import vuda
    prm = vuda.sim_params(dataclasses.replace(S.SimParams(), hull_contacts=1))
    fake = C.c_void_p(0x1000)   # never dereferenced: the call returns before any device work
    st = vuda.lib.vuda_sim_step_noalloc(4, 32, 8, fake, fake, fake, fake, fake, fake, fake, fake, fake, None,
                                        C.byref(prm), 1, fake, fake, fake, 0, None)
    assert st == vuda.ERR_INVALID
    assert b"hull" in vuda.lib.vuda_last_error()
