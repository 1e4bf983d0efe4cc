"""The warm-start kernels of include/lbm_nn.h are exported by the built
library and reject invalid arguments on the host, before any launch (no GPU
needed)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lbm_nn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_nn_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lbm_lib):
    from paper_2311_05091_gb300 import _nn
    lib = _nn.library()
    declared = _declared()
    assert len(declared) == 14
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(_nn.EXPORTS) == declared


def test_invalid_arguments_rejected(lbm_lib):
    from paper_2311_05091_gb300 import _nn
    lib = _nn.library()
    p = 256            # a non-null pointer value; never dereferenced because validation fails first
    # channel counts the tensor-core tiles cannot take
    assert lib.lbm_nn_conv3x3(p, p, None, p, 1, 8, 8, 24, 32, 0, None) == -1
    assert lib.lbm_nn_conv3x3(p, p, None, p, 1, 8, 8, 16, 48, 0, None) == -1
    assert lib.lbm_nn_conv3x3(None, p, None, p, 1, 8, 8, 16, 32, 0, None) == -1
    assert lib.lbm_nn_conv3x3(p, p, None, p, 0, 8, 8, 16, 32, 0, None) == -1
    # weight gradient: shape rules and a workspace that is too small
    ws = lib.lbm_nn_wgrad_workspace(2, 64, 64, 32, 32)
    assert ws >= 9 * 32 * 32 + 32
    assert lib.lbm_nn_conv3x3_wgrad(p, p, p, p, p, ws - 1, 2, 64, 64, 32, 32, None) == -1
    assert lib.lbm_nn_conv3x3_wgrad(p, p, p, p, p, ws, 2, 64, 64, 8, 32, None) == -1
    assert lib.lbm_nn_conv3x3_wgrad(p, p, p, p, p, ws, 2, 64, 64, 32, 24, None) == -1
    # pooling needs even sizes
    assert lib.lbm_nn_pool2(p, p, 1, 7, 8, 4, 0, None) == -1
    assert lib.lbm_nn_up2(p, p, 1, 0, 8, 4, 0, None) == -1
    assert lib.lbm_nn_adam(p, p, p, p, None, 10, 1e-3, 0.9, 0.999, 1e-8, 0, None) == -1
    assert lib.lbm_nn_mse_residual(p, 32, p, p, p, p, 1, p, 1000, None) == -1
    assert lib.lbm_nn_project(p, 32, p, p, p, p, 191, 1, 8, 8, None) == -1
    assert lib.lbm_nn_relu_bwd(None, p, p, 4, None) == -1
    assert lib.lbm_nn_add(p, p, None, 1.0, 4, None) == -1


def test_wgrad_plan_fits_one_wave(lbm_lib):
    # the weight gradient's partial-sum chunks times its channel tiles never exceed the four CTAs per SM (of 152)
    # that the TMEM allocation of 128 columns lets reside at once, so no CTA runs in a second wave
    from paper_2311_05091_gb300 import _nn
    lib = _nn.library()
    for n, h, w, cin, cout in [(16, 256, 256, 32, 32), (16, 256, 256, 16, 32), (16, 128, 128, 64, 64),
                               (16, 64, 64, 128, 128), (16, 32, 32, 256, 256), (16, 64, 64, 256, 128), (1, 1, 3, 16, 16)]:
        ws = lib.lbm_nn_wgrad_workspace(n, h, w, cin, cout)
        bias_chunks = -(-n * h * w // 4096)
        chunks, rem = divmod(ws - bias_chunks * cout, 9 * cin * cout)
        assert rem == 0 and chunks >= 1, (n, h, w, cin, cout, ws)
        tiles = (-(-cout // 32)) * (-(-cin // 32)) if cout <= 64 else (-(-cout // 128)) * 3 * (-(-cin // 32))
        assert chunks * tiles <= 4 * 152, (n, h, w, cin, cout, chunks, tiles)
