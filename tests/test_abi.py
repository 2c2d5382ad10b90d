"""The C-ABI library loads, exports every entry point that include/lbm3.h declares, and rejects
bad arguments before touching the GPU (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2102_04709_gb300 import build, lbm3
    build.build()
    return lbm3.load()


def header_functions():
    txt = open(os.path.join(ROOT, "include", "lbm3.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm3_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_binding_names():
    from paper_2102_04709_gb300 import lbm3
    assert header_functions() == sorted(lbm3.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    from paper_2102_04709_gb300 import lbm3
    out = subprocess.run(["nm", "-D", "--defined-only", lbm3.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (lbm3_\w+)", out))
    for name in header_functions():
        assert name in exported, name
        assert hasattr(lib, name)


def test_library_is_built_for_sm103a_only():
    """Every translation unit is compiled for sm_103a and nothing else: the one -gencode pair of
    the build (no PTX for other targets, no other SASS); the GPU tests then run it on a GB300."""
    from paper_2102_04709_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert not any(f.startswith("-arch") or f.startswith("--gpu-architecture") for f in build.FLAGS)


def _create(lib, **over):
    from paper_2102_04709_gb300 import lbm3
    nx, ny = over.pop("nx", 16), over.pop("ny", 12)
    solid = over.pop("solid", None)
    if solid is None:
        solid = np.zeros((ny, nx), np.uint8)
        solid[0] = solid[-1] = 1
    ang = over.pop("angles", np.full((ny, nx, 3), 90.0))
    sigma = np.array(over.pop("sigma", (0.01, 0.01, 0.01)))
    nu = np.array(over.pop("nu", (0.1, 0.1, 0.1)))
    g = lbm3.lbm3_grid(nx, ny, over.pop("periodic_y", 0), over.pop("bc_x", 0),
                       over.pop("u_in", 0.0), over.pop("rho_out", 1.0), over.pop("precision", 0))
    h = ctypes.c_void_p()
    D = ctypes.POINTER(ctypes.c_double)
    solid = np.ascontiguousarray(solid, np.uint8)
    ang = np.ascontiguousarray(ang, np.float64)
    code = lib.lbm3_create(ctypes.byref(h), ctypes.byref(g),
                           solid.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                           ang.ctypes.data_as(D), sigma.ctypes.data_as(D), nu.ctypes.data_as(D),
                           over.pop("beta0", 0.7), None)
    return code, h, lib.lbm3_last_error(None).decode()


@pytest.mark.parametrize("over,needle", [
    (dict(nx=4), "8x8"),
    (dict(nx=16, ny=5_000_000), "2^31"),
    (dict(bc_x=7), "bc_x"),
    (dict(nu=(0.1, -1.0, 0.1)), "nu"),
    (dict(sigma=(0.01, 0.0, 0.01)), "sigma"),
    (dict(beta0=-1.0), "beta0"),
    (dict(solid=np.zeros((12, 16), np.uint8)), "wall side"),        # walls in y missing
    (dict(bc_x=2, periodic_y=0), "Zou-He"),
    (dict(bc_x=1, sigma=(0.01, 0.01, 0.02)), "sigma_01"),
    (dict(angles=np.full((12, 16, 3), 180.0)), "angles"),
    (dict(precision=9), "precision"),
])
def test_create_rejects_bad_arguments(lib, over, needle):
    code, h, msg = _create(lib, **over)
    assert code == -1 and not h.value
    assert needle in msg


def test_null_handle_calls(lib):
    assert lib.lbm3_step(None, 1) == -1
    assert lib.lbm3_n_wall(None) == -1
    lib.lbm3_destroy(None)


def test_diag_fields_argument_checks(lib):
    """lbm3_diag_fields rejects NULL buffers, empty grids and grids beyond its fixed scratch
    before it touches the GPU."""
    from paper_2102_04709_gb300 import lbm3
    fake = 256  # never dereferenced: every case below is rejected first
    assert lib.lbm3_diag_fields(None, fake, fake, 8, 8, fake, None) == lbm3.LBM3_ERR_INVALID
    assert lib.lbm3_diag_fields(fake, fake, fake, 0, 8, fake, None) == lbm3.LBM3_ERR_INVALID
    assert lib.lbm3_diag_fields(fake, fake, fake, 65536, 65536, fake, None) == lbm3.LBM3_ERR_TOO_LARGE
