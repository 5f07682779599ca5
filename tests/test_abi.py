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
    assert stencil.stencil_get_tuning(h) == (4, stencil.VARIANT_PERSISTENT)  # small 2D grid
    with pytest.raises(stencil.StencilError):
        stencil.stencil_set_tuning(h, 3, 0)
    with pytest.raises(stencil.StencilError):
        stencil.stencil_set_tuning(h, 2, 99)
    stencil.stencil_set_tuning(h, 2, stencil.VARIANT_TEMPORAL)
    assert stencil.stencil_get_tuning(h) == (2, stencil.VARIANT_TEMPORAL)
    stencil.stencil_set_tuning(h, 0, 0)
    assert stencil.stencil_get_tuning(h) == (4, stencil.VARIANT_PERSISTENT)
    mid = stencil.stencil_create((1024, 1024), 1, np.array([0, .1, 0, .1, .6, .1, 0, .1, 0]),
                                 stencil.DIRICHLET_ZERO)
    assert stencil.stencil_get_tuning(mid) == (1, stencil.VARIANT_PERSISTENT)
    stencil.stencil_destroy(mid)
    heat = np.array([0, .1, 0, .1, .6, .1, 0, .1, 0])
    for dims, want in [((512, 512), (4, stencil.VARIANT_PERSISTENT)),
                       ((2048, 1536), (1, stencil.VARIANT_PERSISTENT)),
                       ((2048, 2048), (1, stencil.VARIANT_STREAM))]:
        q = stencil.stencil_create(dims, 1, heat, stencil.DIRICHLET_ZERO)
        assert stencil.stencil_get_tuning(q) == want, dims
        stencil.stencil_destroy(q)
    big = stencil.stencil_create((2048, 1024), 1, np.ones(9) / 9, stencil.PERIODIC)
    assert stencil.stencil_get_tuning(big) == (1, stencil.VARIANT_STREAM)  # box: no one-step persistent form
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


def test_tuning_record_file_is_read(tmp_path):
    """A record in STENCIL_TUNE_CACHE (key: GPU name, ndim, dims, radius,
    stencil class, boundary) sets the choice of a new plan with that key;
    STENCIL_TUNE=off ignores it.  Runs in child processes (the record is read
    once per process)."""
    import subprocess
    import sys
    code = ("import numpy as np, paper_2303_08365_gb300 as st\n"
            "h = st.stencil_create((16, 32, 64), 1, np.ones(27) / 27, st.PERIODIC)\n"
            "print(*st.stencil_get_tuning(h))\n")
    cache = tmp_path / "tune.txt"
    # without a GPU the device name reads 'unknown'
    cache.write_text("unknown/d3/16x32x64/r1/boxeq/b1 2 3 0 12.5\n")
    env = dict(os.environ, STENCIL_TUNE_CACHE=str(cache), PYTHONPATH=ROOT)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    if out.stdout.split() == ["1", "2"]:
        pytest.skip("a CUDA device is visible: the key carries its name")
    assert out.stdout.split() == ["2", "3"]
    env["STENCIL_TUNE"] = "off"
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, cwd=ROOT)
    assert out.stdout.split() == ["1", "2"]


def test_plan_is_a_context_manager(stencil):
    with stencil.Plan((6, 7), 1, np.ones(9) / 9, stencil.PERIODIC) as p:
        assert p.handle
        assert p.get_tuning() == (4, stencil.VARIANT_PERSISTENT)
    assert p.handle is None
    p.close()  # closing twice is harmless


def test_default_goes_direct_for_shapes_the_streaming_kernels_cannot_take(stencil):
    heat3 = np.zeros((3, 3, 3))
    heat3[1, 1, 1] = 0.4
    for d in range(3):
        for e in (0, 2):
            i = [1, 1, 1]
            i[d] = e
            heat3[tuple(i)] = 0.1
    cases = [((64, 64, 64), heat3, stencil.PERIODIC, stencil.VARIANT_STREAM),
             ((63, 63, 63), heat3, stencil.DIRICHLET_ZERO, stencil.VARIANT_DIRECT),   # odd nx
             ((64, 64, 96), heat3, stencil.PERIODIC, stencil.VARIANT_DIRECT),         # nx % 64 != 0
             ((2048, 2047), np.ones(9) / 9, stencil.DIRICHLET_ZERO, stencil.VARIANT_DIRECT),
             ((2048, 2048), np.ones(9) / 9, stencil.DIRICHLET_ZERO, stencil.VARIANT_STREAM)]
    for dims, w, boundary, want in cases:
        with stencil.Plan(dims, 1, w, boundary) as p:
            assert p.get_tuning() == (1, want), dims


def test_tile_setting_is_checked_on_host(stencil):
    p = stencil.Plan((8, 32, 128), 1, np.ones(27) / 27, stencil.PERIODIC)
    for bad in ((32, 16), (64, 12), (0, 64)):
        with pytest.raises(stencil.StencilError):
            p.set_tile(*bad)
    p.set_tile(64, 8)
    p.set_tile(0, 0)
    p.close()


def test_old_four_field_tuning_records_are_read(tmp_path):
    """Records written before the tile field (key Tb variant rate) still apply."""
    import subprocess
    import sys
    code = ("import numpy as np, paper_2303_08365_gb300 as st\n"
            "h = st.stencil_create((16, 32, 64), 1, np.ones(27) / 27, st.PERIODIC)\n"
            "print(*st.stencil_get_tuning(h))\n")
    cache = tmp_path / "tune.txt"
    cache.write_text("unknown/d3/16x32x64/r1/boxeq/b1 4 3 9.5\n")
    env = dict(os.environ, STENCIL_TUNE_CACHE=str(cache), PYTHONPATH=ROOT)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    if out.stdout.split() == ["1", "2"]:
        pytest.skip("a CUDA device is visible: the key carries its name")
    assert out.stdout.split() == ["4", "3"]


def test_fixed_tb_without_variant_keeps_its_tb(stencil):
    """set_tuning(Tb, 0) keeps the Tb: a fused kernel for Tb > 1 (the
    exchange kernel where its tiling fits -- on a host without a GPU the SM
    count reads as 1, so the overlapped kernel), a one-step kernel for Tb = 1."""
    heat2 = np.array([0, .1, 0, .1, .6, .1, 0, .1, 0])
    heat3 = np.zeros(27)
    heat3[[4, 10, 12, 13, 14, 16, 22]] = [.1, .1, .1, .4, .1, .1, .1]
    cases = [((24, 64, 128), heat3, 1, 4, (stencil.VARIANT_TEMPORAL, stencil.VARIANT_EXCHANGE)),
             ((10, 20, 70), heat3, 0, 2, (stencil.VARIANT_TEMPORAL, stencil.VARIANT_EXCHANGE)),  # ragged nx
             ((10, 20, 70), heat3, 1, 2, (stencil.VARIANT_TEMPORAL,)),       # periodic, nx off the tiles
             ((96, 96), heat2, 0, 8, (stencil.VARIANT_PERSISTENT,)),        # small 2D grid
             ((1024, 1024), heat2, 0, 4, (stencil.VARIANT_TEMPORAL,)),
             ((5000,), np.array([.25, .5, .25]), 0, 2, (stencil.VARIANT_TEMPORAL,)),
             ((5000,), np.array([.25, .5, .25]), 0, 1, (stencil.VARIANT_DIRECT,)),
             ((8, 9), np.ones(9) / 9, 1, 1, (stencil.VARIANT_DIRECT,)),         # odd nx: no streaming
             ((96, 96), heat2, 0, 1, (stencil.VARIANT_PERSISTENT,))]          # one-step persistent
    for dims, w, bnd, tb, want in cases:
        h = stencil.stencil_create(dims, 1, w, bnd)
        stencil.stencil_set_tuning(h, tb, 0)
        got_tb, got_v = stencil.stencil_get_tuning(h)
        assert got_tb == tb and got_v in want, (dims, tb, got_tb, got_v)
        stencil.stencil_destroy(h)


def _bands_rows(ny, nx, periodic, Tb, sms):
    """The band cut the exchange kernel documents: one band when 32-row
    tiles over sms // (nx / 64) tile rows cover the plane, else near-equal
    owned ranges with Tb - 1 margin rows on each side toward a neighbour."""
    ty_max = sms // -(-nx // 64)
    max_rows = ty_max * 32
    if ny <= max_rows:
        return 1, ny
    H = Tb - 1
    nb = -(-ny // (max_rows - 2 * H))
    margins = H * (2 * nb if periodic else 2 * (nb - 1))
    return nb, ny + margins


def test_exchange_layout_reports_the_band_cut(stencil):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count if torch.cuda.is_available() else 1
    heat3 = np.zeros(27)
    heat3[[4, 10, 12, 13, 14, 16, 22]] = [.1, .1, .1, .4, .1, .1, .1]
    for dims, bnd in [((4, 100, 64), 0), ((4, 100, 64), 1), ((3, 1024, 1024), 0), ((3, 1024, 1024), 1),
                      ((2, 40, 64 * 152), 1), ((5, 7, 128), 1), ((4, 300, 1000), 0), ((4, 300, 1000), 1),
                      ((4, 30, 99), 0)]:
        h = stencil.stencil_create(dims, 1, heat3, bnd)
        for Tb in (2, 4, 8):
            # nx even (a multiple of 64 when periodic), at most one 64-column tile column per SM
            fits = dims[2] % 2 == 0 and (bnd == 0 or dims[2] % 64 == 0) and -(-dims[2] // 64) <= sms
            if not fits:
                with pytest.raises(stencil.StencilError) as ei:
                    stencil.stencil_exchange_layout(h, Tb)
                assert ei.value.code == stencil.ERR_UNSUPPORTED
                continue
            assert stencil.stencil_exchange_layout(h, Tb) == _bands_rows(dims[1], dims[2], bnd == 1, Tb, sms)
        with pytest.raises(stencil.StencilError):
            stencil.stencil_exchange_layout(h, 3)
        stencil.stencil_destroy(h)
    h2 = stencil.stencil_create((64, 64), 1, np.ones(9) / 9, 1)
    with pytest.raises(stencil.StencilError) as ei:
        stencil.stencil_exchange_layout(h2, 4)
    assert ei.value.code == stencil.ERR_UNSUPPORTED
    stencil.stencil_destroy(h2)
