"""The C ABI without a GPU: libcgks.so builds for sm_103a, loads, exports every function that
include/cgks.h declares, and the Python binding declares the same set; context-free argument checks
answer without touching a device."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cgks.h")


def declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:cgks_status|const char\*)\s+(cgks_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2402_02075_gb300 import build
    return ctypes.CDLL(build.build())


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    import paper_2402_02075_gb300 as cg
    assert sorted(cg.EXPORTS) == declared()


def test_context_free_checks_need_no_device(lib):
    import paper_2402_02075_gb300 as cg
    L = cg.load()
    p = cg.Params()
    assert L.cgks_default_params(ctypes.byref(p)) == 0
    assert abs(p.gamma - 1.4) < 1e-15 and p.n_levels == 3 and p.pre == 1 and p.post == 0
    assert p.compression_factor == 1 and p.adjoint_recompute == 0 and p.agglo_seed == 0
    assert ctypes.sizeof(cg.Params) == 14 * 8 + 12 * 4 + 8  # the C struct: no padding, seed last
    assert L.cgks_default_params(None) == 1
    assert L.cgks_destroy(None) == 0
    assert L.cgks_density_norm_noalloc(None, None, 10, None, None) == 1
    # the adjoint entry points refuse a NULL context before any device work
    assert L.cgks_linearize(None) == 1
    assert L.cgks_residual_vjp(None, None, None, None, None) == 1
    assert L.cgks_wall_force(None, 1, None, None) == 1
    assert L.cgks_adjoint_solve(None, None, 1, 10, 1e-10, None, None, None) == 1
    assert L.cgks_adjoint(None, 1, None, 0, 1e-6, 1e-6, 1, 10, 1e-10, None, None, None, None) == 1
    assert b"NULL" in L.cgks_last_error(None)
