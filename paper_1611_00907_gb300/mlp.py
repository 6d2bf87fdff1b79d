"""Python side of the BF16 multilayer perceptron (lbm_mlp_* in the C ABI):
parameter layout, initialisation, and training / prediction on CUDA tensors.

The network and its kernels live in the library; this module only holds the
host-side bookkeeping (layout, Xavier initialisation, input/output scaling).
"""
import ctypes as C

import numpy as np

from . import _lib

LAYERS = [(16, 128), (128, 128), (128, 128), (128, 16)]  # (k, n) per layer


def param_count():
    return int(_lib.load().lbm_mlp_param_count())


def layout():
    """[(weight slice, (k, n)), ...], [bias slice, ...] in the flat array."""
    w, off = [], 0
    for k, n in LAYERS:
        w.append((slice(off, off + k * n), (k, n)))
        off += k * n
    b = []
    for _, n in LAYERS:
        b.append(slice(off, off + n))
        off += n
    assert off == param_count()
    return w, b


def init_params(seed=0):
    """Xavier-uniform weights, zero biases (FP32)."""
    rng = np.random.default_rng(seed)
    p = np.zeros(param_count(), dtype=np.float32)
    for sl, (k, n) in layout()[0]:
        lim = np.sqrt(6.0 / (k + n))
        p[sl] = rng.uniform(-lim, lim, k * n).astype(np.float32)
    return p


class Mlp:
    """The network on one GPU.  X, T, Y are CUDA float32 tensors [B, nin] /
    [B, nout]; inputs and targets are standardised by the caller."""

    def __init__(self, params=None, device=None, seed=0):
        self._lib = _lib.load()
        p = np.ascontiguousarray(init_params(seed) if params is None else params,
                                 dtype=np.float32)
        h = C.c_void_p()
        from . import _default_device
        _lib.check_mlp(self._lib.lbm_mlp_create(_default_device(device), p.ctypes.data,
                                                C.byref(h)))
        self._m = h

    def close(self):
        if getattr(self, "_m", None):
            self._lib.lbm_mlp_destroy(self._m)
            self._m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def train(self, X, T, iters, lr=1e-3):
        loss = C.c_float()
        _lib.check_mlp(self._lib.lbm_mlp_train(
            self._m, X.data_ptr(), X.shape[1], T.data_ptr(), T.shape[1],
            X.shape[0], int(iters), float(lr), C.byref(loss)), self._m)
        return loss.value

    def gradient(self, X, T):
        """Full-batch gradient of the training loss at the current
        parameters (FP32 numpy array of param_count() values) and the
        loss; the network is not updated."""
        g = np.empty(param_count(), dtype=np.float32)
        loss = C.c_float()
        _lib.check_mlp(self._lib.lbm_mlp_gradient(
            self._m, X.data_ptr(), X.shape[1], T.data_ptr(), T.shape[1],
            X.shape[0], g.ctypes.data, C.byref(loss)), self._m)
        return g, loss.value

    def predict(self, X, nout):
        import torch
        Y = torch.empty((X.shape[0], nout), dtype=torch.float32,
                        device=X.device)
        _lib.check_mlp(self._lib.lbm_mlp_predict(
            self._m, X.data_ptr(), X.shape[1], Y.data_ptr(), nout, X.shape[0]),
            self._m)
        return Y

    def params(self):
        out = np.empty(param_count(), dtype=np.float32)
        _lib.check_mlp(self._lib.lbm_mlp_get_params(self._m, out.ctypes.data),
                       self._m)
        return out
