"""Host-only checks of the C ABI: the library loads, exports every entry point
include/supra.h declares, and rejects invalid parameters before it touches a
device (parameter system with valid ranges, Sec. 2)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1711_06127_b300 as supra
import phantom
from paper_1711_06127_b300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return supra.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "supra.h")).read()
    return sorted(set(re.findall(r"SUPRA_API\s+[\w\s\*]+?\b(supra_\w+)\s*\(", text)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    assert set(supra.EXPORTS) == set(names), names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_checked_build_exports_every_declared_symbol():
    """The checked test variant (-DSUPRA_CHECKED) has the same ABI."""
    path = build.build(checked=True)
    checked = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(checked, name), name
    assert checked.supra_selftest_bounded_wait(0, None) == supra.EINVAL


def test_library_override_selects_another_build():
    """SUPRA_LIBRARY points the binding at another build of the library."""
    import subprocess
    import sys

    path = build.build(checked=True)
    code = "import paper_1711_06127_b300 as s; print(s.LIB_PATH)"
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=dict(os.environ, SUPRA_LIBRARY=path),
                         capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == path


def test_strerror_and_version(lib):
    assert supra.strerror(0) == "ok"
    assert supra.strerror(supra.EINVAL) == "invalid argument"
    assert "sm_103a" in supra.version()


def _params(**over):
    p = phantom.config1().params()
    p.update(over)
    return p


@pytest.mark.parametrize("over", [
    dict(c=0.0), dict(c=-1.0), dict(fs=0.0), dict(fc=30e6), dict(fnumber=0.0), dict(min_half_aperture=0.0),
    dict(fir_taps=62), dict(fir_taps=65), dict(fir_taps=129), dict(fir_taps=0), dict(dyn_range_db=0.0), dict(log_ref=-1.0),
    dict(n_depth=0), dict(n_samples=0), dict(window=7), dict(depth_step=0.0), dict(depth0=-1e-3),
    dict(line_tx=np.full(64, 64, np.int32)), dict(line_tx=np.full(64, -1, np.int32)),
    dict(line_dir=np.tile([0.0, 0.0, 2.0], (64, 1))), dict(fir_cutoff=25e6), dict(c=float("nan")),
    dict(n_bands=5, band_step=1e6), dict(n_bands=3, band_step=20e6), dict(n_bands=2, band_step=float("nan")),
    dict(n_bands=3, band_step=-1e6),
])
def test_invalid_parameters_are_rejected(lib, over):
    with pytest.raises(supra.SupraError) as e:
        supra.Plan(**_params(**over))
    assert e.value.code == supra.EINVAL


@pytest.mark.parametrize("grid_over", [
    dict(n=(0, 1, 10)),
    dict(n=(10, 1, 10), origin=(float("inf"), 0, 0)),
])
def test_invalid_grid_is_rejected(lib, grid_over):
    p = _params()
    g = {"n": (10, 1, 10), "origin": (0.0, 0.0, 0.0), "spacing": (1e-4, 1.0, 1e-4)}
    g.update(grid_over)
    p["grid"] = g
    with pytest.raises(supra.SupraError) as e:
        supra.Plan(**p)
    assert e.value.code == supra.EINVAL


def test_grid_layout_must_match_geometry(lib):
    # uneven line spacing under the linear layout
    p = _params()
    lo = p["line_origin"].copy()
    lo[5, 0] += 1e-4
    p.update(line_origin=lo, grid={"n": (10, 1, 10), "origin": (0.0, 0.0, 0.0), "spacing": (1e-4, 1.0, 1e-4)})
    with pytest.raises(supra.SupraError) as e:
        supra.Plan(**p)
    assert e.value.code == supra.EINVAL
    # a pyramid whose line count does not factor as lines_x * lines_y
    s = phantom.pyramid_setup(4, 4, 0.3e-3, 3, 3, 30.0, 64, grid_n=(8, 8, 8))
    q = s.params()
    q["lines_x"] = 4
    with pytest.raises(supra.SupraError) as e:
        supra.Plan(**q)
    assert e.value.code == supra.EINVAL


def test_null_arguments_are_rejected(lib):
    P = ctypes.c_void_p
    assert lib.supra_plan_create(None, None, None, None, None, None) == supra.EINVAL
    assert lib.supra_beamform(None, None, None, None) == supra.EINVAL
    assert lib.supra_envelope(None, None, None, None) == supra.EINVAL
    assert lib.supra_logcompress(None, None, None, None) == supra.EINVAL
    assert lib.supra_scanconvert(None, None, None, None) == supra.EINVAL
    assert lib.supra_bmode(None, None, None, None, 0, None) == supra.EINVAL
    assert lib.supra_bmode_batched(0, None, None, None, None, 0, None) == supra.EINVAL
    assert lib.supra_plan_get_info(None, None) == supra.EINVAL
    assert lib.supra_bmode_workspace_size(0, None) == 0
    lib.supra_plan_destroy(None)


def test_selftest_budget_out_of_range_is_rejected_before_any_cuda_call(lib):
    assert lib.supra_selftest_bounded_wait(0, None) == supra.EINVAL
    assert lib.supra_selftest_bounded_wait(1 << 9, None) == supra.EINVAL
    assert lib.supra_selftest_bounded_wait((1 << 31) + 1, None) == supra.EINVAL
