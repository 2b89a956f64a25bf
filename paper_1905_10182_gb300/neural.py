"""Python face of the neural-operator entry points (lbm_no_* of include/cmlbm.h), marshalling only."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native as nat


class NeuralOperator:
    def __init__(self, D=64, width=32, modes=12, layers=4, in_ch=4, out_ch=4, max_batch=4, seed=0, stream=None):
        self._lib = nat.lib()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        h = ctypes.c_void_p()
        st = self._lib.lbm_no_create(D, width, modes, layers, in_ch, out_ch, max_batch, ctypes.c_ulonglong(seed),
                                     ctypes.c_void_p(int(stream)) if stream else None, ctypes.byref(h))
        if st != nat.LBM_OK:
            raise nat.LbmError(st, "lbm_no_create failed")
        self._h = h
        self.D, self.width, self.modes, self.layers = D, width, modes, layers
        self.in_ch, self.out_ch, self.max_batch = in_ch, out_ch, max_batch

    def _check(self, st):
        if st != nat.LBM_OK:
            raise nat.LbmError(st, self._lib.lbm_no_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_no_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def param_count(self):
        return self._lib.lbm_no_param_count(self._h)

    def get_params(self):
        out = np.empty(self.param_count, dtype=np.float32)
        self._check(self._lib.lbm_no_params(self._h, nat.ptr(out), 0))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32) if not hasattr(p, "data_ptr") else p.contiguous()
        self._check(self._lib.lbm_no_params(self._h, nat.ptr(p), 1))

    def get_grads(self):
        out = np.empty(self.param_count, dtype=np.float32)
        self._check(self._lib.lbm_no_grads(self._h, nat.ptr(out)))
        return out

    def forward(self, inp, out):
        """inp: [B, in_ch, D, D, D], out: [B, out_ch, D, D, D] float32 (torch CUDA tensors or numpy)."""
        self._check(self._lib.lbm_no_forward(self._h, int(inp.shape[0]), nat.ptr(inp), nat.ptr(out)))
        return out

    def backward(self, dout):
        self._check(self._lib.lbm_no_backward(self._h, nat.ptr(dout)))

    def use_graphs(self, enable=True):
        """Replay the training step as a CUDA graph (default) or run it eagerly."""
        self._check(self._lib.lbm_no_use_graphs(self._h, 1 if enable else 0))

    def train_step(self, inp, target, lr):
        loss = ctypes.c_double()
        self._check(self._lib.lbm_no_train_step(self._h, int(inp.shape[0]), nat.ptr(inp), nat.ptr(target),
                                                ctypes.c_float(lr), ctypes.byref(loss)))
        return loss.value
