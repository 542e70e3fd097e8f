"""ctypes binding of include/hfs_fno.h (the FNO surrogate) -- marshalling
only; ``Fno`` owns the caller-side buffers (parameters and workspace as
torch tensors on the current CUDA device)."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

from . import hfs

EXPORTS = ("hfs_fno_create", "hfs_fno_destroy", "hfs_fno_set_stream", "hfs_fno_param_count",
           "hfs_fno_workspace_size", "hfs_fno_bind", "hfs_fno_init_params", "hfs_fno_forward",
           "hfs_fno_loss_grad", "hfs_fno_train_step", "hfs_fno_set_gemm_engine",
           "hfs_fno_sync_status")
HFS_FNO_GEMM_MMA_SYNC, HFS_FNO_GEMM_TCGEN05 = 0, 1


class hfs_fno_config(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_int32), ("width", ctypes.c_int32), ("modes", ctypes.c_int32),
                ("layers", ctypes.c_int32), ("in_ch", ctypes.c_int32), ("proj", ctypes.c_int32),
                ("out_ch", ctypes.c_int32)]


@dataclass
class FnoConfig:
    grid: int = 256
    width: int = 64
    modes: int = 32
    layers: int = 4
    in_ch: int = 7
    proj: int = 128
    out_ch: int = 2

    def c(self) -> hfs_fno_config:
        return hfs_fno_config(self.grid, self.width, self.modes, self.layers, self.in_ch, self.proj, self.out_ch)


_sig_done = False


def _lib():
    global _sig_done
    L = hfs.lib()
    if not _sig_done:
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        sig = {
            "hfs_fno_create": [ctypes.POINTER(vp), ctypes.POINTER(hfs_fno_config), i32, i32],
            "hfs_fno_destroy": [vp],
            "hfs_fno_set_stream": [vp, vp],
            "hfs_fno_param_count": [vp, ctypes.POINTER(i64)],
            "hfs_fno_workspace_size": [vp, ctypes.POINTER(ctypes.c_size_t)],
            "hfs_fno_bind": [vp, vp, vp, ctypes.c_size_t],
            "hfs_fno_init_params": [vp, ctypes.c_uint64],
            "hfs_fno_forward": [vp, vp, vp, i32],
            "hfs_fno_loss_grad": [vp, vp, vp, i32, vp, ctypes.POINTER(ctypes.c_float)],
            "hfs_fno_train_step": [vp, vp, vp, i32, ctypes.c_float, ctypes.POINTER(ctypes.c_float)],
            "hfs_fno_set_gemm_engine": [vp, i32],
            "hfs_fno_sync_status": [vp],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.hfs_fno_destroy.restype = None
        _sig_done = True
    return L


def _check(code, where):
    if code != hfs.HFS_OK:
        raise hfs.HfsError(code, where)


class Fno:
    """One surrogate model; params is an FP32 torch tensor in the layout of
    include/hfs_fno.h."""

    def __init__(self, cfg: FnoConfig, max_batch: int, train: bool = True, seed: int | None = 0, stream=None):
        import torch
        self.torch = torch
        self.cfg = cfg
        self.max_batch = max_batch
        L = _lib()
        self.h = ctypes.c_void_p()
        cc = cfg.c()
        _check(L.hfs_fno_create(ctypes.byref(self.h), ctypes.byref(cc), max_batch, 1 if train else 0), "hfs_fno_create")
        self.stream = stream if stream is not None else torch.cuda.Stream()
        _check(L.hfs_fno_set_stream(self.h, ctypes.c_void_p(self.stream.cuda_stream)), "hfs_fno_set_stream")
        n = ctypes.c_int64()
        _check(L.hfs_fno_param_count(self.h, ctypes.byref(n)), "hfs_fno_param_count")
        self.nparams = n.value
        wb = ctypes.c_size_t()
        _check(L.hfs_fno_workspace_size(self.h, ctypes.byref(wb)), "hfs_fno_workspace_size")
        self.params = torch.zeros(self.nparams, dtype=torch.float32, device="cuda")
        self.work = torch.empty(wb.value, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        _check(L.hfs_fno_bind(self.h, ctypes.c_void_p(self.params.data_ptr()), ctypes.c_void_p(self.work.data_ptr()),
                              wb.value), "hfs_fno_bind")
        if seed is not None:
            _check(L.hfs_fno_init_params(self.h, seed), "hfs_fno_init_params")
        self.stream.synchronize()

    def set_params(self, vec):
        """Load a parameter vector (host or device) and rebuild the BF16 copies."""
        torch = self.torch
        t = torch.as_tensor(vec, dtype=torch.float32)
        self.params.copy_(t.to(self.params.device))
        torch.cuda.synchronize()
        _check(_lib().hfs_fno_bind(self.h, ctypes.c_void_p(self.params.data_ptr()),
                                   ctypes.c_void_p(self.work.data_ptr()), self.work.numel()), "hfs_fno_bind")
        self.stream.synchronize()

    def forward(self, x):
        torch = self.torch
        x = x.contiguous().float().cuda()
        B = x.shape[0]
        y = torch.empty((B, self.cfg.grid, self.cfg.out_ch), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        _check(_lib().hfs_fno_forward(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), B),
               "hfs_fno_forward")
        self.stream.synchronize()
        return y

    def loss_grad(self, x, y):
        torch = self.torch
        x = x.contiguous().float().cuda()
        y = y.contiguous().float().cuda()
        g = torch.empty(self.nparams, dtype=torch.float32, device="cuda")
        loss = ctypes.c_float()
        torch.cuda.synchronize()
        _check(_lib().hfs_fno_loss_grad(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                        x.shape[0], ctypes.c_void_p(g.data_ptr()), ctypes.byref(loss)),
               "hfs_fno_loss_grad")
        return loss.value, g

    def train_step(self, x, y, lr: float, want_loss: bool = True):
        loss = ctypes.c_float()
        _check(_lib().hfs_fno_train_step(self.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                         x.shape[0], lr, ctypes.byref(loss) if want_loss else None),
               "hfs_fno_train_step")
        return loss.value if want_loss else None

    def set_gemm_engine(self, engine: int):
        _check(_lib().hfs_fno_set_gemm_engine(self.h, int(engine)), "hfs_fno_set_gemm_engine")

    def status(self) -> int:
        """Device-side status since the last call (0, or HFS_ERR_DEVICE_TIMEOUT = 9)."""
        return _lib().hfs_fno_sync_status(self.h)

    def close(self):
        if getattr(self, "h", None) is not None:
            self.stream.synchronize()
            _lib().hfs_fno_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
