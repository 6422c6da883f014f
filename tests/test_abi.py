"""CPU-side checks of the C ABI library: it builds for sm_103a, loads, and exports every
function include/sonar.h declares; the binding's structs match the header's layout."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sonar.h")).read()
    return sorted(set(re.findall(r"^SONAR_API\s+[\w\s\*]+?\b(sonar_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2606_06130_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("sonar_create", "sonar_destroy", "sonar_scene_upload", "sonar_ping", "sonar_ping_batch",
              "sonar_get_hits", "sonar_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol(libpath):
    from paper_2606_06130_gb300 import sonar
    assert set(declared_functions()) == set(sonar._SIGS)


def test_struct_sizes_match_header_layout():
    from paper_2606_06130_gb300 import sonar
    assert ctypes.sizeof(sonar.sonar_pose) == 56
    assert ctypes.sizeof(sonar.sonar_point) == 24
    assert ctypes.sizeof(sonar.sonar_hit) == 32
    assert sonar.POINT_DTYPE.itemsize == 24 and sonar.HIT_DTYPE.itemsize == 32


def test_create_without_gpu_fails_cleanly(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2606_06130_gb300 import sonar
    h = ctypes.c_void_p()
    rc = sonar.lib().sonar_create(ctypes.byref(h), 0, None)
    assert rc in (sonar.SONAR_E_CUDA, sonar.SONAR_E_UNSUPPORTED)
    assert not h.value
    assert sonar.lib().sonar_destroy(None) == sonar.SONAR_OK


def test_params_marshalling_names():
    from paper_2606_06130_gb300 import inputs, sonar
    p = sonar.make_params(inputs.sensor_params("c2"), "bf16")
    assert p.nx == 32 and p.n_beam_az == 128 and p.n_range == 1024 and p.n_sub == 4
    assert abs(p.r_max_m - 15.0) < 1e-12 and p.precision == sonar.SONAR_BF16
