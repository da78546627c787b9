"""Thin Python front ends of the regime classifier (hyb_model_* in
include/hyb.h), the field surrogate (hyb_surrogate_*) and the per-cell
SwitchNet classifier (hyb_switchnet_*).

Argument marshalling only: weights and patches are handed to libhyb.so,
which runs every layer on the GPU.
"""
import ctypes as C

import numpy as np

from . import _abi
from ._abi import check

LAYERS = [(6, 32), (32, 32), (32, 16), (16, 1)]


class Classifier:
    """3D CNN 6->32->32->16->1 (3x3x3, ReLU, dropout, sigmoid) on the GPU."""

    def __init__(self, dropout=0.2, mc_passes=16, seed=7, mean=None, std=None, lr=1e-3, energy_weight=0.1,
                 stream=None):
        self._lib = _abi.load()
        d = _abi.hyb_model_desc()
        d.dropout, d.mc_passes, d.seed = dropout, mc_passes, seed
        mean = [0.0] * 6 if mean is None else mean
        std = [1.0] * 6 if std is None else std
        for c in range(6):
            d.mean[c] = float(mean[c])
            d.std[c] = float(std[c])
        d.lr, d.energy_weight = lr, energy_weight
        if stream is None:
            import torch
            cur = torch.cuda.current_stream()
            if cur.cuda_stream == 0:
                cur = torch.cuda.Stream()
            self.torch_stream = cur
            stream = cur.cuda_stream
        d.stream = stream
        self.desc = d
        h = C.c_void_p()
        check(self._lib.hyb_model_create(C.byref(d), C.byref(h)))
        self._m = h

    @property
    def handle(self):
        return self._m

    def close(self):
        if getattr(self, "_m", None):
            self._lib.hyb_model_destroy(self._m)
            self._m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_layer(self, layer, w, b):
        ci, co = LAYERS[layer]
        w = np.ascontiguousarray(w, dtype=np.float32).reshape(co, ci, 3, 3, 3)
        b = np.ascontiguousarray(b, dtype=np.float32).reshape(co)
        check(self._lib.hyb_model_set_layer(self._m, layer, w.ctypes.data, b.ctypes.data))

    def get_layer(self, layer):
        ci, co = LAYERS[layer]
        w = np.empty((co, ci, 3, 3, 3), np.float32)
        b = np.empty(co, np.float32)
        check(self._lib.hyb_model_get_layer(self._m, layer, w.ctypes.data, b.ctypes.data))
        return w, b

    def forward(self, x, pass_index=-1):
        """x: torch CUDA tensor [B, 6, D, H, W] FP32 -> logits [B, D, H, W] (torch CUDA)."""
        import torch
        x = x.contiguous().float()
        B, _, D, H, W = x.shape
        out = torch.empty((B, D, H, W), dtype=torch.float32, device=x.device)
        torch.cuda.current_stream().synchronize()
        check(self._lib.hyb_model_forward(self._m, x.data_ptr(), B, D, H, W, int(pass_index), out.data_ptr()))
        return out

    def train_step(self, x, y):
        """One Adam step on patches x [B, 6, D, H, W] and labels y [B, D, H, W]
        (torch CUDA tensors).  Returns the step statistics."""
        import torch
        x = x.contiguous().float()
        y = y.contiguous().float()
        B, _, D, H, W = x.shape
        st = _abi.hyb_train_stats()
        torch.cuda.current_stream().synchronize()
        check(self._lib.hyb_train_step(self._m, x.data_ptr(), y.data_ptr(), B, D, H, W, C.byref(st)))
        return {"loss": st.loss, "bce": st.bce, "accuracy": st.accuracy, "step": st.step}

    def get_grad(self, layer):
        ci, co = LAYERS[layer]
        w = np.empty((co, ci, 3, 3, 3), np.float32)
        b = np.empty(co, np.float32)
        check(self._lib.hyb_model_get_grad(self._m, layer, w.ctypes.data, b.ctypes.data))
        return w, b


SURROGATE_LAYERS = [(10, 13), (13, 32), (32, 64), (64, 128), (128, 32), (32, 10)]


def _model_stream(stream):
    import torch
    if stream is not None:
        return None, stream
    cur = torch.cuda.current_stream()
    if cur.cuda_stream == 0:
        cur = torch.cuda.Stream()
    return cur, cur.cuda_stream


class Surrogate:
    """The field surrogate (3D CNN 10->13->32->64->128->32->10 with identity
    shortcuts and dropout; hyb_surrogate_* in include/hyb.h) on the GPU."""

    def __init__(self, dropout=0.1, mc_passes=16, seed=11, mean=None, std=None, lr=1e-3, huber_delta=0.01,
                 energy_weight=0.1, stream=None, dstd=None):
        self._lib = _abi.load()
        d = _abi.hyb_surrogate_desc()
        d.seed, d.dropout, d.mc_passes = seed, dropout, mc_passes
        d.lr, d.huber_delta, d.energy_weight = lr, huber_delta, energy_weight
        mean = [0.0] * 10 if mean is None else mean
        std = [1.0] * 10 if std is None else std
        dstd = [0.0] * 10 if dstd is None else dstd
        for c in range(10):
            d.mean[c] = float(mean[c])
            d.std[c] = float(std[c])
            d.dstd[c] = float(dstd[c])
        self.torch_stream, d.stream = _model_stream(stream)
        self.desc = d
        h = C.c_void_p()
        check(self._lib.hyb_surrogate_create(C.byref(d), C.byref(h)))
        self._m = h

    def close(self):
        if getattr(self, "_m", None):
            self._lib.hyb_surrogate_destroy(self._m)
            self._m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_layer(self, layer, w, b):
        ci, co = SURROGATE_LAYERS[layer]
        w = np.ascontiguousarray(w, dtype=np.float32).reshape(co, ci, 3, 3, 3)
        b = np.ascontiguousarray(b, dtype=np.float32).reshape(co)
        check(self._lib.hyb_surrogate_set_layer(self._m, layer, w.ctypes.data, b.ctypes.data))

    def get_layer(self, layer):
        ci, co = SURROGATE_LAYERS[layer]
        w = np.empty((co, ci, 3, 3, 3), np.float32)
        b = np.empty(co, np.float32)
        check(self._lib.hyb_surrogate_get_layer(self._m, layer, w.ctypes.data, b.ctypes.data))
        return w, b

    def get_grad(self, layer):
        ci, co = SURROGATE_LAYERS[layer]
        w = np.empty((co, ci, 3, 3, 3), np.float32)
        b = np.empty(co, np.float32)
        check(self._lib.hyb_surrogate_get_grad(self._m, layer, w.ctypes.data, b.ctypes.data))
        return w, b

    def _sync_in(self):
        import torch
        torch.cuda.current_stream().synchronize()

    def _sync_out(self):
        import torch
        if self.torch_stream is not None:
            torch.cuda.current_stream().wait_stream(self.torch_stream)

    def forward(self, x, pass_index=-1):
        """x: torch CUDA tensor [B, 10, D, H, W] FP32 -> prediction of the same shape."""
        import torch
        x = x.contiguous().float()
        B, _, D, H, W = x.shape
        out = torch.empty_like(x)
        self._sync_in()
        check(self._lib.hyb_surrogate_forward(self._m, x.data_ptr(), B, D, H, W, int(pass_index), out.data_ptr()))
        self._sync_out()
        return out

    def mc(self, x):
        """MC-dropout mean and standard deviation of the prediction."""
        import torch
        x = x.contiguous().float()
        B, _, D, H, W = x.shape
        pm, ps = torch.empty_like(x), torch.empty_like(x)
        self._sync_in()
        check(self._lib.hyb_surrogate_mc(self._m, x.data_ptr(), B, D, H, W, pm.data_ptr(), ps.data_ptr()))
        self._sync_out()
        return pm, ps

    def train_step(self, x, t):
        """One Adam step on states x and targets t ([B, 10, D, H, W] torch CUDA)."""
        x = x.contiguous().float()
        t = t.contiguous().float()
        B, _, D, H, W = x.shape
        st = _abi.hyb_surrogate_stats()
        self._sync_in()
        check(self._lib.hyb_surrogate_train_step(self._m, x.data_ptr(), t.data_ptr(), B, D, H, W, C.byref(st)))
        return {"loss": st.loss, "huber": st.huber, "energy": st.energy, "step": st.step}


SWITCHNET_LAYERS = [(10, 128), (128, 256), (256, 256), (256, 256), (256, 1)]


class SwitchNet:
    """The per-cell regime classifier of the paper's Table 1 (hyb_switchnet_*)
    on the GPU: features [10, n] (the node channels E, B, J, rho) -> logits [n]."""

    def __init__(self, dropout=0.2, mc_passes=16, seed=13, mean=None, std=None, lr=1e-3, energy_weight=0.1,
                 stream=None):
        self._lib = _abi.load()
        d = _abi.hyb_switchnet_desc()
        d.seed, d.dropout, d.mc_passes, d.lr, d.energy_weight = seed, dropout, mc_passes, lr, energy_weight
        mean = [0.0] * 10 if mean is None else mean
        std = [1.0] * 10 if std is None else std
        for c in range(10):
            d.mean[c] = float(mean[c])
            d.std[c] = float(std[c])
        self.torch_stream, d.stream = _model_stream(stream)
        self.desc = d
        h = C.c_void_p()
        check(self._lib.hyb_switchnet_create(C.byref(d), C.byref(h)))
        self._m = h

    def close(self):
        if getattr(self, "_m", None):
            self._lib.hyb_switchnet_destroy(self._m)
            self._m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_layer(self, layer, w, b):
        ci, co = SWITCHNET_LAYERS[layer]
        w = np.ascontiguousarray(w, dtype=np.float32).reshape(co, ci)
        b = np.ascontiguousarray(b, dtype=np.float32).reshape(co)
        check(self._lib.hyb_switchnet_set_layer(self._m, layer, w.ctypes.data, b.ctypes.data))

    def get_layer(self, layer):
        ci, co = SWITCHNET_LAYERS[layer]
        w = np.empty((co, ci), np.float32)
        b = np.empty(co, np.float32)
        check(self._lib.hyb_switchnet_get_layer(self._m, layer, w.ctypes.data, b.ctypes.data))
        return w, b

    def get_grad(self, layer):
        ci, co = SWITCHNET_LAYERS[layer]
        w = np.empty((co, ci), np.float32)
        b = np.empty(co, np.float32)
        check(self._lib.hyb_switchnet_get_grad(self._m, layer, w.ctypes.data, b.ctypes.data))
        return w, b

    def _sync_in(self):
        import torch
        torch.cuda.current_stream().synchronize()

    def _sync_out(self):
        import torch
        if self.torch_stream is not None:
            torch.cuda.current_stream().wait_stream(self.torch_stream)

    def forward(self, x, pass_index=-1):
        """x: torch CUDA tensor [10, n] FP32 -> logits [n]."""
        import torch
        x = x.contiguous().float()
        out = torch.empty(x.shape[1], dtype=torch.float32, device=x.device)
        self._sync_in()
        check(self._lib.hyb_switchnet_forward(self._m, x.data_ptr(), x.shape[1], int(pass_index), out.data_ptr()))
        self._sync_out()
        return out

    def mc(self, x):
        import torch
        x = x.contiguous().float()
        pm = torch.empty(x.shape[1], dtype=torch.float32, device=x.device)
        ps = torch.empty_like(pm)
        self._sync_in()
        check(self._lib.hyb_switchnet_mc(self._m, x.data_ptr(), x.shape[1], pm.data_ptr(), ps.data_ptr()))
        self._sync_out()
        return pm, ps

    def train_step(self, x, y):
        x = x.contiguous().float()
        y = y.contiguous().float()
        st = _abi.hyb_train_stats()
        self._sync_in()
        check(self._lib.hyb_switchnet_train_step(self._m, x.data_ptr(), y.data_ptr(), x.shape[1], C.byref(st)))
        return {"loss": st.loss, "bce": st.bce, "accuracy": st.accuracy, "step": st.step}
