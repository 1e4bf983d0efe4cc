"""ctypes binding of the warm-start kernels (``include/lbm_nn.h``): argument marshalling only.

Every function takes device pointers (ints, e.g. ``tensor.data_ptr()``) and
raises :class:`NNError` on a non-zero status.
"""
from __future__ import annotations

import ctypes

from . import _lbm

c_int, c_float, c_ll, P = ctypes.c_int, ctypes.c_float, ctypes.c_longlong, ctypes.c_void_p

# every symbol include/lbm_nn.h declares
EXPORTS = ["lbm_nn_conv3x3", "lbm_nn_wgrad_workspace", "lbm_nn_conv3x3_wgrad", "lbm_nn_flip_transpose",
           "lbm_nn_relu_bwd", "lbm_nn_pool2", "lbm_nn_up2", "lbm_nn_add", "lbm_nn_pack_input",
           "lbm_nn_mse_residual", "lbm_nn_adam", "lbm_nn_to_bf16", "lbm_nn_project", "lbm_nn_check"]

_SIG = {
    "lbm_nn_conv3x3": (c_int, [P, P, P, P, c_int, c_int, c_int, c_int, c_int, c_int, P]),
    "lbm_nn_wgrad_workspace": (c_ll, [c_int, c_int, c_int, c_int, c_int]),
    "lbm_nn_conv3x3_wgrad": (c_int, [P, P, P, P, P, c_ll, c_int, c_int, c_int, c_int, c_int, P]),
    "lbm_nn_flip_transpose": (c_int, [P, P, c_int, c_int, P]),
    "lbm_nn_relu_bwd": (c_int, [P, P, P, c_ll, P]),
    "lbm_nn_pool2": (c_int, [P, P, c_int, c_int, c_int, c_int, c_int, P]),
    "lbm_nn_up2": (c_int, [P, P, c_int, c_int, c_int, c_int, c_int, P]),
    "lbm_nn_add": (c_int, [P, P, P, c_float, c_ll, P]),
    "lbm_nn_pack_input": (c_int, [P, P, P, P, c_int, c_int, c_int, P]),
    "lbm_nn_mse_residual": (c_int, [P, c_int, P, P, P, P, c_ll, P, c_ll, P]),
    "lbm_nn_adam": (c_int, [P, P, P, P, P, c_ll, c_float, c_float, c_float, c_float, c_int, P]),
    "lbm_nn_to_bf16": (c_int, [P, P, c_ll, P]),
    "lbm_nn_project": (c_int, [P, c_int, P, P, P, P, c_ll, c_int, c_int, c_int, P]),
    "lbm_nn_check": (c_int, []),
}

_LIB = None


class NNError(RuntimeError):
    pass


def library():
    global _LIB
    if _LIB is None:
        lib = _lbm.library()          # the same shared library; raises if it was not built
        for name, (res, args) in _SIG.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def _call(name, *args):
    st = getattr(library(), name)(*args)
    if st != 0:
        raise NNError(f"{name} returned {st}")


def conv3x3(x, wt, bias, y, n, h, w, cin, cout, relu, stream=0):
    _call("lbm_nn_conv3x3", x, wt, bias, y, n, h, w, cin, cout, int(relu), stream)


def wgrad_workspace(n, h, w, cin, cout):
    return int(library().lbm_nn_wgrad_workspace(n, h, w, cin, cout))


def conv3x3_wgrad(x, dy, dw, db, work, work_len, n, h, w, cin, cout, stream=0):
    _call("lbm_nn_conv3x3_wgrad", x, dy, dw, db, work, work_len, n, h, w, cin, cout, stream)


def flip_transpose(wt, wf, cin, cout, stream=0):
    _call("lbm_nn_flip_transpose", wt, wf, cin, cout, stream)


def relu_bwd(dy, y, dx, n, stream=0):
    _call("lbm_nn_relu_bwd", dy, y, dx, n, stream)


def pool2(x, y, n, h, w, c, backward=False, stream=0):
    _call("lbm_nn_pool2", x, y, n, h, w, c, int(backward), stream)


def up2(x, y, n, h, w, c, backward=False, stream=0):
    _call("lbm_nn_up2", x, y, n, h, w, c, int(backward), stream)


def add(z, x, y, a, n, stream=0):
    _call("lbm_nn_add", z, x, y, a, n, stream)


def pack_input(phi0, phi1, costh, x, n, h, w, stream=0):
    _call("lbm_nn_pack_input", phi0, phi1, costh, x, n, h, w, stream)


def mse_residual(out, cpad, base, target, dout, work, work_len, loss, P_, stream=0):
    _call("lbm_nn_mse_residual", out, cpad, base, target, dout, work, work_len, loss, P_, stream)


def adam(w, m, v, grad, w_bf16, n, lr, b1, b2, eps, t, stream=0):
    _call("lbm_nn_adam", w, m, v, grad, w_bf16, n, lr, b1, b2, eps, t, stream)


def to_bf16(a, b, n, stream=0):
    _call("lbm_nn_to_bf16", a, b, n, stream)


def project(out, cpad, phi0, phi1, field, work, work_len, n, h, w, stream=0):
    _call("lbm_nn_project", out, cpad, phi0, phi1, field, work, work_len, n, h, w, stream)


def check():
    """Raise if a convolution gave up waiting for the tensor cores since the last check."""
    _call("lbm_nn_check")
