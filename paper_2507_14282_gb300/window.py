"""Differentiable window of the 1D faux-shock box (ctypes binding of the
fs_window_* calls in include/fs.h) and its torch.autograd.Function.

The loss is the upstream magnetic fluctuation energy at the end of a window
of hybrid steps; theta = (a_1..a_M, u_cr, u2) holds the seeded transverse-B
mode amplitudes, the cosmic-ray drift speed and the faux-shock kick. The
forward and the adjoint both run in libfs.so's CUDA kernels; this module
only marshals arguments. There is no CPU path.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import fs as _fs


class FauxShockWindow:
    """A window of `steps` steps of one 1D faux-shock box, checkpointed
    every `ckpt` steps. x0: initial positions in cells (X = i + f), v0:
    [n, 3] velocities; phases: the M mode phases."""

    def __init__(self, x0, v0, phases, steps: int = 200, ckpt: int = 20, loss_i0: int = 0,
                 device: str = "cuda:0", **params):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("FauxShockWindow needs a CUDA device; there is no CPU path")
        self.device = torch.device(device)
        params.setdefault("dim", 1)
        self._p = _fs.make_params(**params)
        self.n_modes = len(phases)
        x0 = np.ascontiguousarray(x0, np.float64)
        v0 = np.ascontiguousarray(v0, np.float64).reshape(-1, 3)
        ph = np.ascontiguousarray(phases, np.float64)
        n = len(x0)
        L = _fs.lib()
        nbytes = C.c_size_t()
        _fs._check(L.fs_window_query(C.byref(self._p), steps, ckpt, n, self.n_modes,
                                     C.byref(nbytes)), "fs_window_query")
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.current_stream()
            self._mem = torch.empty(int(nbytes.value) + 256, dtype=torch.uint8,
                                    device=self.device)
            base = self._mem.data_ptr()
            base += (-base) % 256
            h = C.c_void_p()
            _fs._check(L.fs_window_init(C.byref(self._p), steps, ckpt, n, _fs._ptr(x0),
                                        _fs._ptr(v0), self.n_modes, _fs._ptr(ph), loss_i0,
                                        C.c_void_p(base), nbytes,
                                        C.c_void_p(self.stream.cuda_stream), C.byref(h)),
                       "fs_window_init")
        self._h = h
        self.bytes = int(nbytes.value)

    def forward(self, theta) -> float:
        t = np.ascontiguousarray(theta, np.float64)
        assert t.size == self.n_modes + 2
        loss = C.c_double()
        _fs._check(_fs.lib().fs_window_forward(self._h, _fs._ptr(t), C.byref(loss)),
                   "fs_window_forward")
        return loss.value

    def backward(self, dloss: float = 1.0) -> np.ndarray:
        g = np.zeros(self.n_modes + 2)
        _fs._check(_fs.lib().fs_window_backward(self._h, float(dloss), _fs._ptr(g)),
                   "fs_window_backward")
        return g

    def loss_and_grad(self, theta):
        L = self.forward(theta)
        return L, self.backward(1.0)

    def counts(self) -> dict:
        c = np.zeros(5, np.int64)
        _fs._check(_fs.lib().fs_window_counts(self._h, _fs._ptr(c)), "fs_window_counts")
        return dict(zip(("incident", "reflected", "transmitted", "escaped", "injected"),
                        c.tolist()))

    def close(self):
        if getattr(self, "_h", None):
            _fs.lib().fs_window_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def window_loss(win: FauxShockWindow, theta):
    """The window's loss as a differentiable function of a float64 tensor
    theta (autograd runs the CUDA adjoint)."""
    import torch

    class _WindowLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, th):
            L = win.forward(th.detach().cpu().numpy())
            return th.new_tensor(L)

        @staticmethod
        def backward(ctx, gout):
            g = win.backward(float(gout))
            return torch.as_tensor(g, dtype=gout.dtype, device=gout.device)

    return _WindowLoss.apply(theta)
