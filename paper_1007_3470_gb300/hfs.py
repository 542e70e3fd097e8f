"""ctypes binding of the C ABI in include/hfs.h (libhfs.so).

Functions named ``hfs_*`` mirror the C entry points one to one and only
marshal arguments; ``Solver`` is a convenience owner of the caller-side
buffers (state and workspace as torch tensors on the current CUDA device)
around those calls.  Every step of the computation runs in the library's
CUDA kernels; if the library has not been built this module raises instead
of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhfs.so")

HFS_OK = 0
HFS_ERR_WORKSPACE = 8
HFS_C64, HFS_C128 = 0, 1
HFS_OMEGA_CONST, HFS_OMEGA_SIN, HFS_OMEGA_COS_SQ, HFS_OMEGA_PULSE = 0, 1, 2, 3
HFS_VI_NONE, HFS_VI_X4, HFS_VI_COS = 0, 1, 2
HFS_SPLIT_HO, HFS_SPLIT_FOURIER = 0, 1
HFS_FLOW_LEMMA2, HFS_FLOW_CF4, HFS_FLOW_M6 = 0, 1, 2
HFS_COMP_STRANG, HFS_COMP_SRKN6_4, HFS_COMP_NI4_82, HFS_COMP_NI5_84, HFS_COMP_CUSTOM = 0, 1, 2, 3, 4
HFS_MODE_RESIDENT, HFS_MODE_STREAMING = 0, 1
HFS_DFT_SIMT, HFS_DFT_TENSOR_3XTF32 = 0, 1
HFS_PLAN_ALT_ORDER = 0x100

COMPOSITIONS = {"strang": HFS_COMP_STRANG, "srkn6_4": HFS_COMP_SRKN6_4, "ni4_82": HFS_COMP_NI4_82,
                "ni5_84": HFS_COMP_NI5_84, "custom": HFS_COMP_CUSTOM}

# every symbol include/hfs.h declares
EXPORTS = ("hfs_create", "hfs_destroy", "hfs_set_stream", "hfs_state_size", "hfs_instance_offset",
           "hfs_workspace_size", "hfs_bind", "hfs_set_schedule", "hfs_set_mode", "hfs_set_norm_projection",
           "hfs_set_dft_engine", "hfs_set_graphs", "hfs_set_schedule_reuse", "hfs_set_time", "hfs_get_time", "hfs_set_psi", "hfs_get_psi",
           "hfs_step", "hfs_norm", "hfs_energy", "hfs_sync_status", "hfs_set_plan", "hfs_set_occupancy",
           "hfs_autotune", "hfs_autotune_cache", "hfs_set_profiling", "hfs_last_step_kernel_ms",
           "hfs_step1d_noalloc", "hfs_error_string")


class hfs_instance(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32 * 3),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("mu", ctypes.c_double),
        ("omega_law", ctypes.c_int32),
        ("w0", ctypes.c_double),
        ("law", ctypes.c_double * 3),
        ("axis_scale", ctypes.c_double * 3),
        ("eps", ctypes.c_double),
        ("vi_kind", ctypes.c_int32),
        ("vi_k", ctypes.c_double),
        ("sigma", ctypes.c_double),
    ]


class HfsError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {hfs_error_string(code)} (status {code})")


_lib = None


def lib():
    """Load libhfs.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1007_3470_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        sig = {
            "hfs_create": [ctypes.POINTER(vp), i32, i32, ctypes.POINTER(hfs_instance), i64],
            "hfs_destroy": [vp],
            "hfs_set_stream": [vp, vp],
            "hfs_state_size": [vp, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_size_t)],
            "hfs_instance_offset": [vp, i64, ctypes.POINTER(i64)],
            "hfs_workspace_size": [vp, i64, ctypes.POINTER(ctypes.c_size_t)],
            "hfs_bind": [vp, vp, vp, ctypes.c_size_t, i64],
            "hfs_set_schedule": [vp, i32, i32, i32, ctypes.POINTER(dbl), i32, ctypes.POINTER(dbl), i32, dbl],
            "hfs_set_mode": [vp, i32, i32],
            "hfs_set_norm_projection": [vp, i32],
            "hfs_set_dft_engine": [vp, i32],
            "hfs_set_schedule_reuse": [vp, i32],
            "hfs_set_graphs": [vp, i32],
            "hfs_set_time": [vp, dbl],
            "hfs_get_time": [vp, ctypes.POINTER(dbl)],
            "hfs_set_psi": [vp, vp, i32],
            "hfs_get_psi": [vp, vp, i32],
            "hfs_step": [vp, i64],
            "hfs_norm": [vp, ctypes.POINTER(dbl)],
            "hfs_energy": [vp, ctypes.POINTER(dbl)],
            "hfs_sync_status": [vp],
            "hfs_set_plan": [vp, i32, i32],
            "hfs_autotune": [vp, i32, ctypes.POINTER(ctypes.c_int32)],
            "hfs_set_occupancy": [vp, i32],
            "hfs_autotune_cache": [vp, ctypes.c_char_p, i32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(i32)],
            "hfs_set_profiling": [vp, i32],
            "hfs_last_step_kernel_ms": [vp, ctypes.POINTER(ctypes.c_float)],
            "hfs_step1d_noalloc": [vp, i32, ctypes.POINTER(hfs_instance), i64, i32, i32, i32, dbl, dbl, i64, vp, i32],
            "hfs_error_string": [i32],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = i32
        L.hfs_destroy.restype = None
        L.hfs_error_string.restype = ctypes.c_char_p
        _lib = L
    return _lib


def hfs_error_string(code: int) -> str:
    try:
        return lib().hfs_error_string(int(code)).decode()
    except RuntimeError:
        return f"status {code}"


def _check(code: int, where: str):
    if code != HFS_OK:
        raise HfsError(code, where)


# --- one-to-one wrappers -----------------------------------------------------

def make_instances(instances: Iterable) -> ctypes.Array:
    """Marshal workload instances (objects or dicts with the hfs_instance
    field names of workloads.Instance) into a ctypes array."""
    items = list(instances)
    arr = (hfs_instance * len(items))()
    for k, it in enumerate(items):
        d = it if isinstance(it, dict) else it.as_dict()
        c = arr[k]
        n = list(d["n"])
        for a in range(3):
            c.n[a] = int(n[a]) if a < len(n) else 1
            c.lo[a] = float(d["a"][a]) if a < len(n) else 0.0
            c.hi[a] = float(d["b"][a]) if a < len(n) else 1.0
            c.law[a] = float(d.get("law", (0, 0, 0))[a])
            c.axis_scale[a] = float(d.get("axis_scale", (1, 1, 1))[a])
        c.mu = float(d.get("mu", 1.0))
        c.omega_law = int(d.get("omega_law", 0))
        c.w0 = float(d.get("w0", 1.0))
        c.eps = float(d.get("eps", 0.0))
        c.vi_kind = int(d.get("vi_kind", 0))
        c.vi_k = float(d.get("vi_k", 0.0))
        c.sigma = float(d.get("sigma", 0.0))
    return arr


def hfs_create(dim: int, precision: int, instances: ctypes.Array) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().hfs_create(ctypes.byref(h), dim, precision, instances, len(instances)), "hfs_create")
    return h


def hfs_destroy(h):
    lib().hfs_destroy(h)


def hfs_set_stream(h, stream_ptr: int):
    _check(lib().hfs_set_stream(h, ctypes.c_void_p(stream_ptr)), "hfs_set_stream")


def hfs_state_size(h) -> tuple[int, int]:
    e, b = ctypes.c_int64(), ctypes.c_size_t()
    _check(lib().hfs_state_size(h, ctypes.byref(e), ctypes.byref(b)), "hfs_state_size")
    return e.value, b.value


def hfs_instance_offset(h, i: int) -> int:
    o = ctypes.c_int64()
    _check(lib().hfs_instance_offset(h, i, ctypes.byref(o)), "hfs_instance_offset")
    return o.value


def hfs_workspace_size(h, chunk_steps: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().hfs_workspace_size(h, chunk_steps, ctypes.byref(b)), "hfs_workspace_size")
    return b.value


def hfs_bind(h, psi_ptr: int, work_ptr: int, work_bytes: int, chunk_steps: int):
    _check(lib().hfs_bind(h, ctypes.c_void_p(psi_ptr), ctypes.c_void_p(work_ptr), work_bytes, chunk_steps),
           "hfs_bind")


def hfs_set_schedule(h, split: int, flow: int, composition: int, dt: float,
                     a: Optional[Sequence[float]] = None, b: Optional[Sequence[float]] = None):
    if composition == HFS_COMP_CUSTOM:
        av = (ctypes.c_double * len(a))(*a)
        bv = (ctypes.c_double * len(b))(*b)
        _check(lib().hfs_set_schedule(h, split, flow, composition, av, len(a), bv, len(b), dt), "hfs_set_schedule")
    else:
        _check(lib().hfs_set_schedule(h, split, flow, composition, None, 0, None, 0, dt), "hfs_set_schedule")


def hfs_set_mode(h, mode: int, steps_per_launch: int = 1):
    _check(lib().hfs_set_mode(h, mode, steps_per_launch), "hfs_set_mode")


def hfs_set_norm_projection(h, enable: bool):
    _check(lib().hfs_set_norm_projection(h, 1 if enable else 0), "hfs_set_norm_projection")


def hfs_set_dft_engine(h, engine: int):
    _check(lib().hfs_set_dft_engine(h, int(engine)), "hfs_set_dft_engine")


def hfs_set_schedule_reuse(h, enable: bool) -> int:
    """Returns the status: HFS_OK, or HFS_ERR_WORKSPACE when the context was
    left unbound for a larger workspace (other errors raise)."""
    st = lib().hfs_set_schedule_reuse(h, 1 if enable else 0)
    if st not in (0, HFS_ERR_WORKSPACE):
        _check(st, "hfs_set_schedule_reuse")
    return st


def hfs_set_graphs(h, enable: bool):
    _check(lib().hfs_set_graphs(h, 1 if enable else 0), "hfs_set_graphs")


def hfs_set_time(h, t: float):
    _check(lib().hfs_set_time(h, t), "hfs_set_time")


def hfs_get_time(h) -> float:
    t = ctypes.c_double()
    _check(lib().hfs_get_time(h, ctypes.byref(t)), "hfs_get_time")
    return t.value


def hfs_set_psi(h, src_ptr: int, on_device: bool):
    _check(lib().hfs_set_psi(h, ctypes.c_void_p(src_ptr), 1 if on_device else 0), "hfs_set_psi")


def hfs_get_psi(h, dst_ptr: int, on_device: bool):
    _check(lib().hfs_get_psi(h, ctypes.c_void_p(dst_ptr), 1 if on_device else 0), "hfs_get_psi")


def hfs_step(h, nsteps: int):
    _check(lib().hfs_step(h, nsteps), "hfs_step")


def hfs_norm(h, count: int) -> np.ndarray:
    out = np.zeros(count, dtype=np.float64)
    _check(lib().hfs_norm(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "hfs_norm")
    return out


def hfs_energy(h, count: int) -> np.ndarray:
    out = np.zeros(count, dtype=np.float64)
    _check(lib().hfs_energy(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "hfs_energy")
    return out


def hfs_sync_status(h) -> int:
    return lib().hfs_sync_status(h)


def hfs_set_plan(h, n: int, plan: int):
    """plan: elements per thread (4, 8, 16), | HFS_PLAN_ALT_ORDER for the
    alternative radix order of 16."""
    _check(lib().hfs_set_plan(h, n, plan), "hfs_set_plan")


def hfs_set_occupancy(h, ctas_per_sm: int):
    _check(lib().hfs_set_occupancy(h, ctas_per_sm), "hfs_set_occupancy")


def hfs_autotune(h, trial_steps: int) -> list[int]:
    best = (ctypes.c_int32 * 6)()
    _check(lib().hfs_autotune(h, trial_steps, best), "hfs_autotune")
    return list(best)


def hfs_autotune_cache(h, path: str, trial_steps: int) -> tuple[list[int], bool]:
    """(plans per grid size 128 ... 4096, whether they came from the cache)."""
    best = (ctypes.c_int32 * 6)()
    hit = ctypes.c_int()
    _check(lib().hfs_autotune_cache(h, os.fsencode(path), trial_steps, best, ctypes.byref(hit)),
           "hfs_autotune_cache")
    return list(best), bool(hit.value)


def hfs_set_profiling(h, enable: bool):
    _check(lib().hfs_set_profiling(h, 1 if enable else 0), "hfs_set_profiling")


def hfs_last_step_kernel_ms(h) -> float:
    ms = ctypes.c_float()
    _check(lib().hfs_last_step_kernel_ms(h, ctypes.byref(ms)), "hfs_last_step_kernel_ms")
    return ms.value


NOALLOC_MAX_INSTANCES = 512


def hfs_step1d_noalloc(psi_ptr: int, precision: int, instances: ctypes.Array, split: int, flow: int,
                       composition: int, dt: float, t0: float, nsteps: int, stream_ptr: int = 0, wait: bool = True):
    """Allocation-free batched 1D step on a caller-owned device state (see include/hfs.h)."""
    _check(lib().hfs_step1d_noalloc(ctypes.c_void_p(psi_ptr), precision, instances, len(instances), split, flow,
                                    composition, dt, t0, nsteps, ctypes.c_void_p(stream_ptr), 1 if wait else 0),
           "hfs_step1d_noalloc")


# --- convenience owner of the caller-side buffers ------------------------------

class Solver:
    """Owns a context plus its state and workspace buffers (torch tensors on
    the current CUDA device) and enqueues on a torch stream."""

    def __init__(self, instances, dim: int = 1, precision: str = "c64", chunk_steps: int = 512,
                 stream=None, device=None):
        import torch
        self._torch = torch
        self.instances = list(instances)
        self.count = len(self.instances)
        self.dim = dim
        self.precision = HFS_C128 if precision == "c128" else HFS_C64
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        # a dedicated stream (capturable into CUDA graphs, unlike the legacy default stream)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self._cinst = make_instances(self.instances)
        with torch.cuda.device(self.device):
            self.h = hfs_create(dim, self.precision, self._cinst)
            hfs_set_stream(self.h, self.stream.cuda_stream)
            self.elems, self.state_bytes = hfs_state_size(self.h)
            self.chunk_steps = chunk_steps
            self.work_bytes = hfs_workspace_size(self.h, chunk_steps)
            cdt = torch.complex128 if self.precision == HFS_C128 else torch.complex64
            self.psi = torch.zeros(self.elems, dtype=cdt, device=self.device)
            self.work = torch.empty(self.work_bytes, dtype=torch.uint8, device=self.device)
            hfs_bind(self.h, self.psi.data_ptr(), self.work.data_ptr(), self.work_bytes, chunk_steps)
        self.offsets = [hfs_instance_offset(self.h, i) for i in range(self.count)]

    def close(self):
        if getattr(self, "h", None) is not None:
            self.stream.synchronize()
            hfs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_schedule(self, dt: float, composition: str = "strang", flow: int = HFS_FLOW_CF4,
                     split: int = HFS_SPLIT_HO, a=None, b=None):
        hfs_set_schedule(self.h, split, flow, COMPOSITIONS[composition], dt, a, b)

    def set_mode(self, mode: int, steps_per_launch: int = 1):
        hfs_set_mode(self.h, mode, steps_per_launch)

    def set_graphs(self, enable: bool):
        hfs_set_graphs(self.h, enable)

    def set_norm_projection(self, enable: bool):
        hfs_set_norm_projection(self.h, enable)

    def set_dft_engine(self, engine: int):
        hfs_set_dft_engine(self.h, engine)

    def set_schedule_reuse(self, enable: bool):
        """Keep the phase records of the last calls and compute the next
        call's in parallel with the step kernel (1D); re-binds with a larger
        workspace when the current one has no room for the second buffer."""
        torch = self._torch
        with torch.cuda.device(self.device):
            if hfs_set_schedule_reuse(self.h, enable) == HFS_ERR_WORKSPACE:
                self.work_bytes = hfs_workspace_size(self.h, self.chunk_steps)
                self.work = torch.empty(self.work_bytes, dtype=torch.uint8, device=self.device)
                hfs_bind(self.h, self.psi.data_ptr(), self.work.data_ptr(), self.work_bytes, self.chunk_steps)

    def set_time(self, t: float):
        hfs_set_time(self.h, t)

    @property
    def time(self) -> float:
        return hfs_get_time(self.h)

    def set_psi(self, psi):
        """psi: numpy array (host, complex) of the concatenated state, a list of
        per-instance arrays, or a torch complex tensor on the device."""
        torch = self._torch
        if isinstance(psi, torch.Tensor) and psi.is_cuda:
            src = psi.to(self.psi.dtype).contiguous()
            hfs_set_psi(self.h, src.data_ptr(), True)
            self.stream.synchronize()
            return
        if isinstance(psi, (list, tuple)):
            psi = np.concatenate([np.asarray(p).ravel() for p in psi])
        npdt = np.complex128 if self.precision == HFS_C128 else np.complex64
        host = np.ascontiguousarray(np.asarray(psi).ravel(), dtype=npdt)
        if host.size != self.elems:
            raise ValueError(f"state has {self.elems} elements, got {host.size}")
        hfs_set_psi(self.h, host.ctypes.data, False)

    def get_psi(self) -> np.ndarray:
        npdt = np.complex128 if self.precision == HFS_C128 else np.complex64
        out = np.empty(self.elems, dtype=npdt)
        hfs_get_psi(self.h, out.ctypes.data, False)
        return out

    def split(self, flat: np.ndarray) -> list[np.ndarray]:
        """Per-instance views of a concatenated state (3D: shaped (nz, ny, nx))."""
        out = []
        for i, inst in enumerate(self.instances):
            n = list(inst.n if not isinstance(inst, dict) else inst["n"])
            npts = int(np.prod(n))
            v = flat[self.offsets[i]:self.offsets[i] + npts]
            out.append(v.reshape(tuple(reversed(n))) if len(n) > 1 else v)
        return out

    def step(self, nsteps: int):
        hfs_step(self.h, nsteps)

    def norm(self) -> np.ndarray:
        return hfs_norm(self.h, self.count)

    def energy(self) -> np.ndarray:
        return hfs_energy(self.h, self.count)

    def status(self) -> int:
        return hfs_sync_status(self.h)

    def autotune(self, trial_steps: int = 20, cache: Optional[str] = None) -> list[int]:
        """Tune the 1D plans; with `cache`, reuse (or record) them in that JSON file."""
        if cache is None:
            return hfs_autotune(self.h, trial_steps)
        plans, self.tune_cache_hit = hfs_autotune_cache(self.h, cache, trial_steps)
        return plans

    def set_plan(self, n: int, ept: int):
        hfs_set_plan(self.h, n, ept)
