"""Python face of the candidate classifier (C ABI dd_nn_*): a small bf16 CNN
over 64x64 snippets, trained on the GPU by the library's own kernels."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from .dedisp import _stream_handle

NN_PARAMS = 191553
SHAPES = [("conv1.w", (16, 1, 3, 3)), ("conv1.b", (16,)), ("conv2.w", (32, 16, 3, 3)), ("conv2.b", (32,)),
          ("conv3.w", (64, 32, 3, 3)), ("conv3.b", (64,)), ("conv4.w", (64, 64, 3, 3)), ("conv4.b", (64,)),
          ("fc1.w", (128, 1024)), ("fc1.b", (128,)), ("fc2.w", (1, 128)), ("fc2.b", (1,))]


def init_params(seed: int) -> np.ndarray:
    """He-normal weights, zero biases (float32, flat)."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        if name.endswith(".w"):
            parts.append(rng.standard_normal(k) * np.sqrt(2.0 / int(np.prod(shp[1:]))))
        else:
            parts.append(np.zeros(k))
    return np.concatenate(parts).astype(np.float32)


class Classifier:
    def __init__(self, max_batch: int = 1024, params=None, seed: int = 0):
        self._L = _lib.load()
        self._h = ctypes.c_void_p()
        _lib.check(self._L.dd_nn_create(ctypes.byref(self._h), max_batch), "dd_nn_create")
        self.max_batch = max_batch
        self.set_params(init_params(seed) if params is None else params)

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == NN_PARAMS
        _lib.check(self._L.dd_nn_set_params(self._h, p.ctypes.data), "dd_nn_set_params")

    def params(self) -> np.ndarray:
        out = np.empty(NN_PARAMS, dtype=np.float32)
        _lib.check(self._L.dd_nn_get_params(self._h, out.ctypes.data), "dd_nn_get_params")
        return out

    def forward(self, x, out=None, stream=None, tensor_cores=False):
        """x: bfloat16 CUDA tensor [n, 64, 64] -> float32 logits [n].  The
        default is the fixed-order CUDA-core forward (bit-reproducible, the
        one training uses); tensor_cores=True runs the convolutions as tcgen05
        implicit GEMMs (faster; logits agree to about 1e-2)."""
        import torch

        n = x.shape[0]
        if out is None:
            out = torch.empty(n, dtype=torch.float32, device=x.device)
        fn = self._L.dd_nn_forward_tc if tensor_cores else self._L.dd_nn_forward
        _lib.check(fn(self._h, ctypes.c_void_p(x.data_ptr()), n, ctypes.c_void_p(out.data_ptr()),
                      _stream_handle(stream)), "dd_nn_forward")
        return out

    def status(self) -> int:
        """Error flags of the tensor-core forward (0 when all is well)."""
        f = ctypes.c_uint()
        _lib.check(self._L.dd_nn_status(self._h, ctypes.byref(f)), "dd_nn_status")
        return f.value

    def backward(self, x, labels, stream=None):
        _lib.check(self._L.dd_nn_backward(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(labels.data_ptr()),
                                          x.shape[0], _stream_handle(stream)), "dd_nn_backward")

    def loss(self, stream=None) -> float:
        v = ctypes.c_float()
        _lib.check(self._L.dd_nn_get_loss(self._h, ctypes.byref(v), _stream_handle(stream)), "dd_nn_get_loss")
        return v.value

    def grads(self, stream=None) -> np.ndarray:
        out = np.empty(NN_PARAMS, dtype=np.float32)
        _lib.check(self._L.dd_nn_get_grads(self._h, out.ctypes.data, _stream_handle(stream)), "dd_nn_get_grads")
        return out

    def set_grads(self, g):
        g = np.ascontiguousarray(g, dtype=np.float32)
        _lib.check(self._L.dd_nn_set_grads(self._h, g.ctypes.data), "dd_nn_set_grads")

    def adamw(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.01, stream=None):
        _lib.check(self._L.dd_nn_adamw(self._h, lr, beta1, beta2, eps, wd, _stream_handle(stream)), "dd_nn_adamw")

    def train_step(self, x, labels, lr, **kw):
        self.backward(x, labels, stream=kw.pop("stream", None))
        self.adamw(lr, **kw)

    def state(self):
        m = np.empty(NN_PARAMS, np.float32)
        v = np.empty(NN_PARAMS, np.float32)
        b = np.empty(NN_PARAMS, np.uint16)
        st = ctypes.c_int()
        _lib.check(self._L.dd_nn_get_state(self._h, m.ctypes.data, v.ctypes.data, b.ctypes.data, ctypes.byref(st)),
                   "dd_nn_get_state")
        return m, v, b, st.value

    def save(self, path: str):
        _lib.check(self._L.dd_nn_save(self._h, path.encode()), "dd_nn_save")

    def load(self, path: str):
        _lib.check(self._L.dd_nn_load(self._h, path.encode()), "dd_nn_load")

    def close(self):
        if self._h:
            self._L.dd_nn_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
