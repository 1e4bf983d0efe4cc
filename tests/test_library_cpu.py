"""The CUDA library builds for sm_103a, loads, exports every entry point of
include/lbm.h, and validates its arguments on the host (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lbm_lib):
    lib = lbm_lib.library()
    declared = _declared()
    assert len(declared) >= 20
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(lbm_lib.EXPORTS) == declared


def test_status_strings(lbm_lib):
    assert lbm_lib.lbm_strerror(0) == "ok"
    assert lbm_lib.lbm_strerror(-1) == "invalid argument"
    assert lbm_lib.lbm_strerror(-4) == "simulation diverged"


@pytest.mark.parametrize("field,value", [("theta_deg", 0.0), ("theta_deg", 180.0), ("d0", 1.0), ("d0", 0.0),
                                         ("W", -1.0), ("sigma", 0.0), ("eta_hat", 0.0), ("s_free_ns", 2.0),
                                         ("kappa", -1.5)])
def test_invalid_parameters_rejected_before_any_device_call(lbm_lib, field, value):
    p = lbm_lib.lbm_default_params(**{field: value})
    with pytest.raises(lbm_lib.LbmError) as e:
        lbm_lib.lbm_create(lbm_lib.LBM_D2Q9, 32, 32, 1, 3, p)
    assert e.value.status == -1


def test_invalid_shapes_rejected(lbm_lib):
    p = lbm_lib.lbm_default_params()
    for args in [(0, 32, -1, 1, 3), (0, 32, 32, 2, 3), (0, 1, 32, 1, 2), (0, 0, 32, 1, 3), (5, 8, 8, 1, 3)]:
        with pytest.raises(lbm_lib.LbmError) as e:
            lbm_lib.lbm_create(*args, p)
        assert e.value.status == -1
    # D3Q19 needs d0 < 1/2
    with pytest.raises(lbm_lib.LbmError):
        lbm_lib.lbm_create(lbm_lib.LBM_D3Q19, 8, 8, 8, 7, lbm_lib.lbm_default_params(d0=0.5))


def test_null_arguments(lbm_lib):
    lib = lbm_lib.library()
    assert lib.lbm_default_params(None) == -1
    assert lib.lbm_step(None, 1) == -1
    assert lib.lbm_sync(None) == -1
    assert lib.lbm_set_wait_limit(None, 0) == -1
    lib.lbm_destroy(None)


def test_build_targets_sm_103a():
    import importlib
    B = importlib.import_module("paper_2311_05091_gb300.build")
    assert "arch=compute_103a,code=sm_103a" in " ".join(B.ARCH)
    assert "-lineinfo" in B.FLAGS


def test_storage_options_validated_on_the_host(lbm_lib):
    L = lbm_lib
    p = [L.lbm_default_params()]
    with pytest.raises(L.LbmError) as e:
        L.lbm_create_ex(L.LBM_D3Q19, 20, 16, 16, 7, p, L.LBM_STORE_G_F16)
    assert e.value.status == -1          # nx % 8 != 0 (3D)
    with pytest.raises(L.LbmError) as e:
        L.lbm_create_multi(L.LBM_D3Q19, [(16, 16), (32, 16)], 3, p * 2)
    assert e.value.status == -7          # instances of different sizes: D2Q9 only
    with pytest.raises(L.LbmError) as e:
        L.lbm_create_ex(L.LBM_D2Q9, 20, 16, 1, 3, p, L.LBM_STORE_G_F16)
    assert e.value.status == -1          # nx % 8 != 0
    with pytest.raises(L.LbmError) as e:
        L.lbm_create_ex(L.LBM_D2Q9, 16, 16, 1, 3, p, 2)
    assert e.value.status == -1          # unknown flag


def test_create_alloc_needs_both_callbacks(lbm_lib):
    """The callbacks are checked before any device call."""
    import ctypes
    lib = lbm_lib.library()
    p = lbm_lib.lbm_default_params()
    out = ctypes.c_void_p()
    alloc = lbm_lib.lbm_alloc_fn(lambda n, s, u: None)
    st = lib.lbm_create_alloc(lbm_lib.LBM_D2Q9, 16, 8, 1, 3, 1, ctypes.byref(p), 0, None, alloc, lbm_lib.lbm_free_fn(),
                              None, ctypes.byref(out))
    assert st == -1 and not out.value
    st = lib.lbm_create_alloc(lbm_lib.LBM_D2Q9, 16, 8, 1, 3, 0, ctypes.byref(p), 0, None, alloc,
                              lbm_lib.lbm_free_fn(lambda a, b, c, d: None), None, ctypes.byref(out))
    assert st == -1                                   # nbatch 0


def test_public_headers_are_plain_c(tmp_path):
    """include/lbm.h and include/lbm_nn.h compile as strict C11 (a C caller needs no C++ compiler)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_headers.c"
    src.write_text('#include "lbm.h"\n#include "lbm_nn.h"\n'
                   "int main(void) { lbm_params p; lbm_flux f; (void)f; return lbm_default_params(&p); }\n")
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
