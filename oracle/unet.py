"""FP64 oracle of the learned reconstruction network (test infrastructure).

Wraps oracle/unet.c: forward, loss + hand-derived gradients, bilinear 2x;
and the BF16 network (BF16 rounding at the points the learned path's
precision fixes) with the per-element standard deviation of an
FP32-accumulating implementation's difference from it: bf16_forward,
bf16_loss_grad, bf16.
Arrays are NHWC float64; parameters are laid out per layer as W[Cout][9][Cin]
then b[Cout] (layers c1a c1b c2a c2b c3a c3b d2a d2b d1a d1b head)."""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "unet.c")
_LIB = os.path.join(_HERE, "libunet_oracle.so")
_lib = None

CIN = [16, 32, 32, 64, 64, 128, 192, 64, 96, 32, 32]
COUT = [32, 32, 64, 64, 128, 128, 64, 64, 32, 32, 16]
NAMES = ["c1a", "c1b", "c2a", "c2b", "c3a", "c3b", "d2a", "d2b", "d1a", "d1b", "head"]


def build(force=False):
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC", _SRC,
                               "-o", _LIB, "-lm"])
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        vp, i32 = ctypes.c_void_p, ctypes.c_int
        L.ou_param_count.restype = ctypes.c_int64
        L.ou_forward.argtypes = [vp, vp, i32, i32, i32, vp]
        L.ou_loss_grad.argtypes = [vp, vp, vp, i32, i32, i32, vp, vp]
        L.ou_loss_grad.restype = ctypes.c_double
        L.ou_bilinear2x.argtypes = [vp, i32, i32, i32, i32, vp]
        L.ou_bf16.argtypes = [ctypes.c_double]
        L.ou_bf16.restype = ctypes.c_double
        L.ou_bf16_forward.argtypes = [vp, vp, i32, i32, i32, vp, vp]
        L.ou_bf16_loss_grad.argtypes = [vp, vp, vp, i32, i32, i32, vp, vp, vp, vp]
        L.ou_bf16_loss_grad.restype = ctypes.c_double
        _lib = L
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def param_count():
    return _load().ou_param_count()


def layer_slices():
    """(weight slice, bias slice) per layer in the flat parameter vector."""
    out, off = [], 0
    for ci, co in zip(CIN, COUT):
        w = slice(off, off + co * 9 * ci)
        off += co * 9 * ci
        b = slice(off, off + co)
        off += co
        out.append((w, b))
    return out


def forward(params, x):
    """x: (N, h, w, 4) -> (N, 2h, 2w, 4)."""
    x = np.ascontiguousarray(x, np.float64)
    p = np.ascontiguousarray(params, np.float64)
    N, h, w, _ = x.shape
    out = np.zeros((N, 2 * h, 2 * w, 4))
    _load().ou_forward(_p(p), _p(x), N, h, w, _p(out))
    return out


def loss_grad(params, x, target):
    x = np.ascontiguousarray(x, np.float64)
    t = np.ascontiguousarray(target, np.float64)
    p = np.ascontiguousarray(params, np.float64)
    N, h, w, _ = x.shape
    out = np.zeros((N, 2 * h, 2 * w, 4))
    g = np.zeros(param_count())
    loss = _load().ou_loss_grad(_p(p), _p(x), _p(t), N, h, w, _p(out), _p(g))
    return loss, g, out


def bilinear2x(x):
    x = np.ascontiguousarray(x, np.float64)
    N, h, w, C = x.shape
    out = np.zeros((N, 2 * h, 2 * w, C))
    _load().ou_bilinear2x(_p(x), N, h, w, C, _p(out))
    return out


def bf16(v):
    """Round to the nearest BF16 value (ties to even), elementwise."""
    f = _load().ou_bf16
    a = np.asarray(v, np.float64)
    return np.vectorize(f, otypes=[np.float64])(a) if a.ndim else f(float(a))


def bf16_forward(params, x):
    """The BF16 network's output and the per-element standard deviation of
    an FP32-accumulating implementation's difference from it: (out, sigma),
    both (N, 2h, 2w, 4). params: the weights the implementation multiplies
    with (BF16 values) and FP32 biases; x: FP32 values."""
    x = np.ascontiguousarray(x, np.float64)
    p = np.ascontiguousarray(params, np.float64)
    N, h, w, _ = x.shape
    out = np.zeros((N, 2 * h, 2 * w, 4))
    eout = np.zeros_like(out)
    _load().ou_bf16_forward(_p(p), _p(x), N, h, w, _p(out), _p(eout))
    return out, eout


def bf16_loss_grad(params, x, target):
    """(loss, grad, grad_sigma, out, out_sigma) of the BF16 network."""
    x = np.ascontiguousarray(x, np.float64)
    t = np.ascontiguousarray(target, np.float64)
    p = np.ascontiguousarray(params, np.float64)
    N, h, w, _ = x.shape
    out = np.zeros((N, 2 * h, 2 * w, 4))
    eout = np.zeros_like(out)
    g = np.zeros(param_count())
    eg = np.zeros_like(g)
    loss = _load().ou_bf16_loss_grad(_p(p), _p(x), _p(t), N, h, w, _p(out), _p(eout), _p(g), _p(eg))
    return loss, g, eg, out, eout
