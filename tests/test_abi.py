"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports
every entry point include/stencil.h declares, and rejects bad arguments on
the host before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def stencil():
    from paper_2303_08365_gb300 import build
    build.build()
    import paper_2303_08365_gb300 as st
    st.lib()
    return st


def declared_functions():
    text = open(os.path.join(ROOT, "include", "stencil.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(stencil_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported_and_bound(stencil):
    names = declared_functions()
    assert len(names) >= 15
    lib = ctypes.CDLL(stencil.LIB_PATH)
    bound = {n for n, _, _ in stencil.SIGNATURES}
    for n in names:
        assert hasattr(lib, n), n
        assert n in bound, n


def test_header_compiles_as_c(tmp_path):
    src = tmp_path / "t.c"
    src.write_text('#include "stencil.h"\nint main(void){stencil_plan p=0;(void)p;return 0;}\n')
    import subprocess
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        "-c", str(src), "-o", str(tmp_path / "t.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_create_rejects_bad_arguments_on_host(stencil):
    w = np.ones(9) / 9
    for dims, radius, weights, boundary in [((0, 5), 1, w, 0), ((4, 4), 3, np.ones(49), 0),
                                            ((4, 4), 1, w, 7), ((4, 4, 4, 4), 1, np.ones(81), 0)]:
        with pytest.raises(stencil.StencilError) as ei:
            stencil.stencil_create(dims, radius, weights, boundary)
        assert ei.value.code == stencil.ERR_ARG
    bad = w.copy()
    bad[4] = np.nan
    with pytest.raises(stencil.StencilError):
        stencil.stencil_create((4, 4), 1, bad, 0)


def test_plan_lifecycle_and_tuning_checks_on_host(stencil):
    h = stencil.stencil_create((8, 9), 1, np.ones(9) / 9, stencil.PERIODIC)
    assert stencil.stencil_get_tuning(h) == (8, stencil.VARIANT_PERSISTENT)  # small 2D grid
    with pytest.raises(stencil.StencilError):
        stencil.stencil_set_tuning(h, 3, 0)
    with pytest.raises(stencil.StencilError):
        stencil.stencil_set_tuning(h, 2, 99)
    stencil.stencil_set_tuning(h, 2, stencil.VARIANT_TEMPORAL)
    assert stencil.stencil_get_tuning(h) == (2, stencil.VARIANT_TEMPORAL)
    stencil.stencil_set_tuning(h, 0, 0)
    assert stencil.stencil_get_tuning(h) == (8, stencil.VARIANT_PERSISTENT)
    mid = stencil.stencil_create((1024, 1024), 1, np.array([0, .1, 0, .1, .6, .1, 0, .1, 0]),
                                 stencil.DIRICHLET_ZERO)
    assert stencil.stencil_get_tuning(mid) == (4, stencil.VARIANT_PERSISTENT)
    stencil.stencil_destroy(mid)
    big = stencil.stencil_create((2048, 1024), 1, np.ones(9) / 9, stencil.PERIODIC)
    assert stencil.stencil_get_tuning(big) == (1, stencil.VARIANT_STREAM)
    stencil.stencil_destroy(big)
    r2 = stencil.stencil_create((9, 10, 11), 2, np.ones(125) / 125, stencil.PERIODIC)
    assert stencil.stencil_get_tuning(r2) == (1, stencil.VARIANT_DIRECT)
    stencil.stencil_destroy(r2)
    assert stencil.stencil_variant_name(stencil.VARIANT_STREAM) == "stream"
    stencil.stencil_destroy(h)
    hv = stencil.stencil_create_varcoef((4, 5, 6), stencil.PERIODIC)
    stencil.stencil_destroy(hv)
    with pytest.raises(stencil.StencilError):
        stencil.stencil_create_varcoef((4,), stencil.PERIODIC)
