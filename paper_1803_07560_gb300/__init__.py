"""GB300 (sm_103a) Monte Carlo evaluation of the lattice Burgers functional
integral of Honkonen & Honkonen (arXiv:1803.07560).

Thin ctypes binding of the C ABI in ``include/bfi.h``: argument marshalling
only; every step of the computation runs in the CUDA library
``_build/libbfi.so``.  There is no CPU fallback: importing this package fails
if the library has not been built (``paper_1803_07560_gb300._build.build()``).
Device arrays are torch CUDA tensors (torch supplies device memory and
streams); host arrays are numpy arrays.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

FP64 = 0
FP32 = 1
FP32_COMPENSATED = 2   # evaluate() only

_P = ctypes.POINTER
_vp = ctypes.c_void_p


class BfiError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"bfi status {status}: {message}")
        self.status = status


class Lattice(ctypes.Structure):
    """Lattice of Eq. (Gen2): nx spatial sites (M), nt time slices (L)."""

    _fields_ = [("nx", ctypes.c_int32), ("nt", ctypes.c_int32), ("nu", ctypes.c_double),
                ("D", ctypes.c_double), ("a", ctypes.c_double), ("tau", ctypes.c_double),
                ("nonlinear", ctypes.c_double), ("mass2", ctypes.c_double)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("nsub", ctypes.c_int64), ("chunks", ctypes.c_int64),
                ("chunk_samples", ctypes.c_int64), ("total_samples", ctypes.c_int64),
                ("grid", ctypes.c_int32), ("block", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("slot_len", ctypes.c_int32), ("totals_len", ctypes.c_int32),
                ("scratch_bytes", ctypes.c_size_t), ("ctas_per_sm_max", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("tail_subvolume", ctypes.c_int64),
                ("tail_chunk_samples", ctypes.c_int64)]


class Chunking(ctypes.Structure):
    """How a job's budgets are cut into chunks (bfi_chunking)."""
    _fields_ = [("chunk_samples", ctypes.c_int64), ("tail_subvolume", ctypes.c_int64),
                ("tail_chunk_samples", ctypes.c_int64), ("chunks", ctypes.c_int64)]


class Work(ctypes.Structure):
    """Work of the last execution, sample by sample (bfi_work)."""
    _fields_ = [("samples", ctypes.c_uint64), ("stage1", ctypes.c_uint64), ("survivors", ctypes.c_uint64),
                ("full_screen", ctypes.c_uint64), ("evaluated", ctypes.c_uint64),
                ("two_stage_shape", ctypes.c_int32), ("rest_screen", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


class ServerConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("slots", ctypes.c_int32), ("memory_budget", ctypes.c_uint64),
                ("precision", ctypes.c_int), ("split_rel_var", ctypes.c_double),
                ("max_split_rounds", ctypes.c_int32)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int), ("nsub_final", ctypes.c_int64),
                ("passes", ctypes.c_int32), ("samples", ctypes.c_uint64), ("queued_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("cancelled", ctypes.c_uint64), ("samples", ctypes.c_uint64), ("bytes_in_use", ctypes.c_uint64),
                ("bytes_peak", ctypes.c_uint64), ("running", ctypes.c_int32), ("queued", ctypes.c_int32)]


class Job(ctypes.Structure):
    """One job of a batch (device arrays; host budgets)."""

    _fields_ = [("lattice", Lattice), ("nsub", ctypes.c_int64), ("samples", ctypes.POINTER(ctypes.c_uint64)),
                ("lo", ctypes.c_void_p), ("hi", ctypes.c_void_p), ("sub_id", ctypes.c_void_p),
                ("seed", ctypes.c_uint32), ("job_id", ctypes.c_uint32), ("slots", ctypes.c_void_p),
                ("totals", ctypes.c_void_p)]


SAMPLE_BOX, SAMPLE_TRANSFORM, SAMPLE_GAUSSIAN = 0, 1, 2
FAULT_NONE, FAULT_POOL_ALLOC, FAULT_LAUNCH, FAULT_COMPLETION, FAULT_SCHEDULER = 0, 1, 2, 3, 4


class Sampler(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("mean", ctypes.c_void_p), ("factor", ctypes.c_void_p)]


def _sampler(kind: int, d: int, mean=None, factor=None):
    """A bfi_sampler and the host arrays it points to (kept alive by the caller)."""
    keep = []
    mp = fp = None
    if kind == SAMPLE_GAUSSIAN:
        f, fp = _host(np.reshape(factor, (d, d)), np.float64)
        keep.append(f)
        if mean is not None:
            m, mp = _host(np.reshape(mean, (d,)), np.float64)
            keep.append(m)
    return Sampler(kind, mp, fp), keep


def gaussian_proposal(lat: Lattice, zero_mode_sigma: float = float("inf")) -> np.ndarray:
    """Factor F with F F^T = (A + I/sigma0^2)^-1 for the linear-limit action (see bfi.h)."""
    d = lat.nx * lat.nt
    out = np.empty((d, d))
    _check(_lib.bfi_gaussian_proposal(ctypes.byref(lat), float(zero_mode_sigma), ctypes.c_void_p(out.ctypes.data)))
    return out


class Convergence(ctypes.Structure):
    """The convergence test of Sec. 3 (see bfi_convergence in bfi.h)."""

    _fields_ = [("factor", ctypes.c_double), ("rel_tol", ctypes.c_double), ("abs_tol", ctypes.c_double),
                ("small", ctypes.c_double), ("max_depth", ctypes.c_int32), ("max_leaves", ctypes.c_int64)]


class AdaptiveStats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int64), ("evaluated", ctypes.c_int64), ("converged", ctypes.c_int64),
                ("kept_depth", ctypes.c_int64), ("kept_budget", ctypes.c_int64), ("leaves", ctypes.c_int64),
                ("samples", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def convergence(factor=2.0, rel_tol=0.0, abs_tol=0.0, small=0.0, max_depth=12, max_leaves=1 << 16) -> Convergence:
    return Convergence(factor, rel_tol, abs_tol, small, max_depth, max_leaves)


def lattice(nx, nt, nu=1.0, D=1.0, a=1.0, tau=1.0, nonlinear=1.0, mass2=0.0) -> Lattice:
    return Lattice(nx, nt, nu, D, a, tau, nonlinear, mass2)


# Every symbol the header declares, with its ctypes signature.
_SIGNATURES = {
    "bfi_num_r": (ctypes.c_int32, [ctypes.c_int32]),
    "bfi_slot_len": (ctypes.c_int32, [ctypes.c_int32]),
    "bfi_totals_len": (ctypes.c_int32, [ctypes.c_int32]),
    "bfi_last_error": (ctypes.c_char_p, []),
    "bfi_plan_create": (ctypes.c_int, [_P(_vp), _P(Lattice), ctypes.c_int64, _P(ctypes.c_uint64),
                                       ctypes.c_int, ctypes.c_int]),
    "bfi_plan_destroy": (ctypes.c_int, [_vp]),
    "bfi_plan_get_info": (ctypes.c_int, [_vp, _P(PlanInfo)]),
    "bfi_chunking_of": (ctypes.c_int, [ctypes.c_int64, _P(ctypes.c_uint64), _P(Chunking)]),
    "bfi_plan_execute": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_uint32, ctypes.c_uint32,
                                        _vp, _vp, _vp]),
    "bfi_plan_set_grid": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "bfi_plan_set_timing": (ctypes.c_int, [_vp, ctypes.c_int]),
    "bfi_batch_create": (ctypes.c_int, [_P(_vp), _vp, ctypes.c_int32, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int32, ctypes.c_int32]),
    "bfi_batch_launch": (ctypes.c_int, [_vp, _vp]),
    "bfi_batch_destroy": (ctypes.c_int, [_vp]),
    "bfi_autotune_grid": (ctypes.c_int, [_P(Lattice), ctypes.c_int, ctypes.c_int, _P(ctypes.c_int32)]),
    "bfi_plan_get_timing": (ctypes.c_int, [_vp, _P(ctypes.c_float)]),
    "bfi_plan_get_stats": (ctypes.c_int, [_vp, _P(ctypes.c_uint64), _P(ctypes.c_float)]),
    "bfi_plan_get_screen_stats": (ctypes.c_int, [_vp, _P(ctypes.c_uint64), _P(ctypes.c_int32)]),
    "bfi_plan_get_work": (ctypes.c_int, [_vp, _P(Work)]),
    "bfi_batch_get_work": (ctypes.c_int, [_vp, ctypes.c_int32, _P(Work)]),
    "bfi_integrate_static_scratch": (ctypes.c_int, [_P(Lattice), ctypes.c_int64, _P(ctypes.c_uint64), _vp,
                                                    _vp, _vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int,
                                                    _vp, _vp, _vp]),
    "bfi_server_create": (ctypes.c_int, [_P(_vp), _P(ServerConfig)]),
    "bfi_server_destroy": (ctypes.c_int, [_vp]),
    "bfi_server_shutdown": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "bfi_server_inject_fault": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int64]),
    "bfi_server_get_stats": (ctypes.c_int, [_vp, _P(ServerStats)]),
    "bfi_submit": (ctypes.c_int, [_vp, _P(Lattice), ctypes.c_int64, _vp, _vp, _vp, ctypes.c_uint32,
                                  ctypes.c_uint32, _P(_vp)]),
    "bfi_poll": (ctypes.c_int, [_vp, _P(ctypes.c_int32)]),
    "bfi_wait": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "bfi_cancel": (ctypes.c_int, [_vp]),
    "bfi_request_get_info": (ctypes.c_int, [_vp, _P(RequestInfo)]),
    "bfi_request_get_result": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "bfi_request_release": (ctypes.c_int, [_vp]),
    "bfi_request_get_work": (ctypes.c_int, [_vp, _P(Work)]),
    "bfi_nsphere": (ctypes.c_int, [ctypes.c_int32, _vp, _vp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                   ctypes.c_uint32, _P(ctypes.c_double), _P(ctypes.c_double),
                                   _P(ctypes.c_int32), ctypes.c_int]),
    "bfi_adaptive_nsphere": (ctypes.c_int, [ctypes.c_int32, _vp, _vp, ctypes.c_uint64, ctypes.c_uint32,
                                            ctypes.c_uint32, _P(Convergence), _P(ctypes.c_double),
                                            _P(ctypes.c_double), _P(AdaptiveStats), ctypes.c_int]),
    "bfi_adaptive_integrate": (ctypes.c_int, [_vp, _P(Lattice), _vp, _vp, ctypes.c_uint64, ctypes.c_uint32,
                                              ctypes.c_uint32, ctypes.c_int, _P(Convergence), _vp,
                                              _P(AdaptiveStats), ctypes.c_int64, _vp, _vp, _vp]),
    "bfi_plan_set_sampler": (ctypes.c_int, [_vp, _P(Sampler)]),
    "bfi_gaussian_proposal": (ctypes.c_int, [_P(Lattice), ctypes.c_double, _vp]),
    "bfi_ctx_set_sampler": (ctypes.c_int, [_vp, _P(Sampler), ctypes.c_int32]),
    "bfi_ctx_create": (ctypes.c_int, [_P(_vp), ctypes.c_int]),
    "bfi_ctx_destroy": (ctypes.c_int, [_vp]),
    "bfi_integrate": (ctypes.c_int, [_vp, _P(Lattice), ctypes.c_int64, _vp, _vp, _vp, _vp,
                                     ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, _vp, _vp]),
    "bfi_merge_host": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, _vp, _vp]),
    "bfi_error_bound": (ctypes.c_int, [_P(Lattice), ctypes.c_int, ctypes.c_int64, _vp, ctypes.c_double, _vp]),
    "bfi_points": (ctypes.c_int, [ctypes.c_int32, _vp, _vp, ctypes.c_uint32, ctypes.c_uint32,
                                  ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int,
                                  _vp, _vp]),
    "bfi_eval": (ctypes.c_int, [_P(Lattice), ctypes.c_int64, _vp, ctypes.c_int, _vp, _vp, _vp]),
}


def _load_library():
    if not os.path.exists(_build.LIB):
        raise ImportError(
            f"CUDA library not built: {_build.LIB} is missing "
            "(build it with paper_1803_07560_gb300._build.build())")
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load_library()
LIBRARY_PATH = _build.LIB
CLI_PATH = _build.CLI  # the line-protocol integrand program (Sec. 3), built beside the library


def _check(status: int):
    if status != 0:
        raise BfiError(status, _lib.bfi_last_error().decode())


def num_r(nx: int) -> int:
    return _lib.bfi_num_r(nx)


def slot_len(nx: int) -> int:
    return _lib.bfi_slot_len(nx)


def totals_len(nx: int) -> int:
    return _lib.bfi_totals_len(nx)


def _dev_ptr(t, dtype=None, numel=None, what="tensor"):
    """Device address of a contiguous CUDA tensor.  With numel, the tensor must
    hold exactly that many elements: the library reads and writes device
    arrays by the sizes the plan or call fixes, and cannot check them there."""
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise TypeError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected dtype {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{what} has {t.numel()} elements, the call needs {numel}")
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, ctypes.c_void_p(a.ctypes.data)


class Plan:
    """A planned job (lattice, precision, per-subvolume budgets) on one device."""

    def __init__(self, lat: Lattice, samples, precision: int = FP64, device: int = 0):
        smp = np.ascontiguousarray(np.atleast_1d(samples), dtype=np.uint64)
        self.lattice = lat
        self.precision = precision
        self.device = device
        self.nsub = int(smp.size)
        self.d = lat.nx * lat.nt
        handle = ctypes.c_void_p()
        _check(_lib.bfi_plan_create(ctypes.byref(handle), ctypes.byref(lat), smp.size,
                                    smp.ctypes.data_as(_P(ctypes.c_uint64)), precision, device))
        self._h = handle

    def info(self) -> PlanInfo:
        info = PlanInfo()
        _check(_lib.bfi_plan_get_info(self._h, ctypes.byref(info)))
        return info

    def execute(self, lo, hi, seed: int, job_id: int = 0, sub_id=None, slots=None, totals=None,
                stream=None):
        """Enqueue the whole path on 'stream'; lo/hi [nsub, d] float64 CUDA tensors."""
        import torch
        nx = self.lattice.nx
        if slots is None:
            slots = torch.empty((self.nsub, slot_len(nx)), dtype=torch.float64, device=lo.device)
        if totals is None:
            totals = torch.empty(totals_len(nx), dtype=torch.float64, device=lo.device)
        n, d = self.nsub, self.d
        _check(_lib.bfi_plan_execute(self._h, _dev_ptr(lo, torch.float64, n * d, "lo"),
                                     _dev_ptr(hi, torch.float64, n * d, "hi"),
                                     _dev_ptr(sub_id, torch.int32, n, "sub_id") if sub_id is not None else None,
                                     seed & 0xFFFFFFFF, job_id & 0xFFFFFFFF,
                                     _dev_ptr(slots, torch.float64, n * slot_len(nx), "slots"),
                                     _dev_ptr(totals, torch.float64, totals_len(nx), "totals"),
                                     _stream_ptr(stream)))
        return slots, totals

    def set_sampler(self, kind: int, mean=None, factor=None):
        smp, keep = _sampler(kind, self.d, mean, factor)
        _check(_lib.bfi_plan_set_sampler(self._h, ctypes.byref(smp)))

    def set_grid(self, ctas_per_sm: int):
        """Persistent grid: CTAs per SM (0 = occupancy limit); never changes results."""
        _check(_lib.bfi_plan_set_grid(self._h, ctas_per_sm))

    def set_timing(self, enable: bool = True):
        _check(_lib.bfi_plan_set_timing(self._h, int(enable)))

    def timing(self):
        """(integrand ms, merge ms) of the last timed execution (waits for it)."""
        ms = (ctypes.c_float * 2)()
        _check(_lib.bfi_plan_get_timing(self._h, ms))
        return float(ms[0]), float(ms[1])

    def stats(self):
        """(samples fully evaluated by the last execution, negligible-weight window)."""
        n = ctypes.c_uint64()
        w = ctypes.c_float()
        _check(_lib.bfi_plan_get_stats(self._h, ctypes.byref(n), ctypes.byref(w)))
        return int(n.value), float(w.value)

    def screen_stats(self):
        """(samples the full FP32 screen or stage 2 examined in the last
        execution, whether stage 1 of the two-stage screen ran on any chunk);
        see bfi_plan_get_screen_stats."""
        n = ctypes.c_uint64()
        two = ctypes.c_int32()
        _check(_lib.bfi_plan_get_screen_stats(self._h, ctypes.byref(n), ctypes.byref(two)))
        return int(n.value), bool(two.value)

    def work(self) -> Work:
        """Work of the last execution, sample by sample (bfi_plan_get_work)."""
        w = Work()
        _check(_lib.bfi_plan_get_work(self._h, ctypes.byref(w)))
        return w

    def close(self):
        if getattr(self, "_h", None):
            _lib.bfi_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """One device and stream; integrate() takes and returns host arrays."""

    def __init__(self, device: int = 0):
        handle = ctypes.c_void_p()
        _check(_lib.bfi_ctx_create(ctypes.byref(handle), device))
        self._h = handle
        self.device = device

    def integrate(self, lat: Lattice, lo, hi, samples, seed: int, job_id: int = 0, sub_id=None,
                  precision: int = FP64, want_slots: bool = True, out_slots=None, out_totals=None):
        d = lat.nx * lat.nt
        lo_a, lo_p = _host(np.reshape(lo, (-1, d)), np.float64)
        hi_a, hi_p = _host(np.reshape(hi, (-1, d)), np.float64)
        nsub = lo_a.shape[0]
        smp_a, smp_p = _host(np.broadcast_to(np.asarray(samples, dtype=np.uint64), (nsub,)), np.uint64)
        sid_a, sid_p = (None, None) if sub_id is None else _host(sub_id, np.uint32)
        if hi_a.shape != lo_a.shape or (sid_a is not None and sid_a.size != nsub):
            raise ValueError("lo, hi and sub_id must describe the same subvolumes")
        slots = out_slots if out_slots is not None else (
            np.empty((nsub, slot_len(lat.nx))) if want_slots else None)
        totals = out_totals if out_totals is not None else np.empty(totals_len(lat.nx))
        for a, n in ((slots, nsub * slot_len(lat.nx)), (totals, totals_len(lat.nx))):
            if a is not None and (a.dtype != np.float64 or not a.flags.c_contiguous or a.size != n):
                raise ValueError(f"an output array needs {n} contiguous float64 elements")
        _check(_lib.bfi_integrate(self._h, ctypes.byref(lat), nsub, lo_p, hi_p, smp_p, sid_p,
                                  seed & 0xFFFFFFFF, job_id & 0xFFFFFFFF, precision,
                                  None if slots is None else ctypes.c_void_p(slots.ctypes.data),
                                  ctypes.c_void_p(totals.ctypes.data)))
        return slots, totals

    def set_sampler(self, kind: int, d: int = 0, mean=None, factor=None):
        """Sampler of the next integrations (d: the dimension of a Gaussian factor)."""
        if kind == SAMPLE_GAUSSIAN and not d:
            d = int(round(np.sqrt(np.size(factor))))
        smp, keep = _sampler(kind, d, mean, factor)
        _check(_lib.bfi_ctx_set_sampler(self._h, ctypes.byref(smp), d))

    def adaptive_integrate(self, lat: Lattice, lo, hi, n: int, seed: int, conv: Convergence, job_id: int = 0,
                           precision: int = FP64, leaf_capacity: int = 0):
        """Adaptive subdivision of the box [lo, hi] (Sec. 3): (totals, stats)
        or, with leaf_capacity > 0, (totals, stats, leaf_lo, leaf_hi,
        leaf_slots) holding the first min(leaves, leaf_capacity) kept leaves."""
        d = lat.nx * lat.nt
        lo_a, lo_p = _host(np.broadcast_to(np.asarray(lo, dtype=np.float64), (d,)), np.float64)
        hi_a, hi_p = _host(np.broadcast_to(np.asarray(hi, dtype=np.float64), (d,)), np.float64)
        totals = np.empty(totals_len(lat.nx))
        stats = AdaptiveStats()
        cap = int(leaf_capacity)
        llo = np.empty((cap, d)) if cap else None
        lhi = np.empty((cap, d)) if cap else None
        lsl = np.empty((cap, slot_len(lat.nx))) if cap else None
        ptr = (lambda a: None if a is None else ctypes.c_void_p(a.ctypes.data))
        _check(_lib.bfi_adaptive_integrate(self._h, ctypes.byref(lat), lo_p, hi_p, int(n), seed & 0xFFFFFFFF,
                                           job_id & 0xFFFFFFFF, precision, ctypes.byref(conv),
                                           ctypes.c_void_p(totals.ctypes.data), ctypes.byref(stats), cap,
                                           ptr(llo), ptr(lhi), ptr(lsl)))
        if not cap:
            return totals, stats
        m = min(cap, stats.leaves)
        return totals, stats, llo[:m], lhi[:m], lsl[:m]

    def close(self):
        if getattr(self, "_h", None):
            _lib.bfi_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def integrate_static_scratch(lat: Lattice, samples, lo, hi, seed: int, job_id: int = 0, sub_id=None,
                             precision: int = FP64, slots=None, totals=None, stream=None):
    """The whole integration without any allocation by the library: its
    scratch is a fixed 16 MiB device array, for callers that cannot allocate
    device memory.  Inputs and outputs are the caller's CUDA tensors (allocated
    here only if not given).  Calls that overlap on the GPU race on the
    shared scratch; the first call on a device should precede stream capture."""
    import torch
    smp = np.ascontiguousarray(np.atleast_1d(samples), dtype=np.uint64)
    nsub = int(smp.size)
    if slots is None:
        slots = torch.empty((nsub, slot_len(lat.nx)), dtype=torch.float64, device=lo.device)
    if totals is None:
        totals = torch.empty(totals_len(lat.nx), dtype=torch.float64, device=lo.device)
    d = lat.nx * lat.nt
    _check(_lib.bfi_integrate_static_scratch(
        ctypes.byref(lat), nsub, smp.ctypes.data_as(_P(ctypes.c_uint64)), _dev_ptr(lo, torch.float64, nsub * d, "lo"),
        _dev_ptr(hi, torch.float64, nsub * d, "hi"),
        _dev_ptr(sub_id, torch.int32, nsub, "sub_id") if sub_id is not None else None,
        seed & 0xFFFFFFFF, job_id & 0xFFFFFFFF, precision,
        _dev_ptr(slots, torch.float64, nsub * slot_len(lat.nx), "slots"),
        _dev_ptr(totals, torch.float64, totals_len(lat.nx), "totals"), _stream_ptr(stream)))
    return slots, totals


def autotune_grid(lat: Lattice, precision: int = FP64, device: int = 0) -> int:
    """CTAs per SM chosen by timing for this lattice shape (cached per process)."""
    c = ctypes.c_int32()
    _check(_lib.bfi_autotune_grid(ctypes.byref(lat), precision, device, ctypes.byref(c)))
    return int(c.value)


class Batch:
    """Many jobs captured into one CUDA graph (one plan per job).

    jobs: list of dicts with keys lattice, samples (host), lo, hi (CUDA float64
    [nsub, d]), optional sub_id (CUDA int32), seed, job_id; outputs are
    allocated here (self.slots[i], self.totals[i]) unless given."""

    def __init__(self, jobs, precision: int = FP32, device: int = 0, nstreams: int = 8,
                 autotune: bool = True):
        import torch
        arr = (Job * len(jobs))()
        self._keep = []
        self.slots, self.totals = [], []
        for i, j in enumerate(jobs):
            lat = j["lattice"]
            smp = np.ascontiguousarray(np.atleast_1d(j["samples"]), dtype=np.uint64)
            lo, hi = j["lo"], j["hi"]
            slots = j.get("slots")
            if slots is None:
                slots = torch.empty((smp.size, slot_len(lat.nx)), dtype=torch.float64, device=lo.device)
            totals = j.get("totals")
            if totals is None:
                totals = torch.empty(totals_len(lat.nx), dtype=torch.float64, device=lo.device)
            sid = j.get("sub_id")
            arr[i].lattice = lat
            arr[i].nsub = smp.size
            arr[i].samples = smp.ctypes.data_as(_P(ctypes.c_uint64))
            n, d = int(smp.size), lat.nx * lat.nt
            arr[i].lo = _dev_ptr(lo, torch.float64, n * d, f"job {i} lo")
            arr[i].hi = _dev_ptr(hi, torch.float64, n * d, f"job {i} hi")
            arr[i].sub_id = None if sid is None else _dev_ptr(sid, torch.int32, n, f"job {i} sub_id")
            arr[i].seed = j.get("seed", 0) & 0xFFFFFFFF
            arr[i].job_id = j.get("job_id", i) & 0xFFFFFFFF
            arr[i].slots = _dev_ptr(slots, torch.float64, n * slot_len(lat.nx), f"job {i} slots")
            arr[i].totals = _dev_ptr(totals, torch.float64, totals_len(lat.nx), f"job {i} totals")
            self._keep += [smp, lo, hi, sid]
            self.slots.append(slots)
            self.totals.append(totals)
        handle = ctypes.c_void_p()
        _check(_lib.bfi_batch_create(ctypes.byref(handle), ctypes.cast(arr, ctypes.c_void_p), len(jobs),
                                     precision, device, nstreams, int(autotune)))
        self._h = handle

    def launch(self, stream=None):
        _check(_lib.bfi_batch_launch(self._h, _stream_ptr(stream)))

    def work(self, job: int) -> Work:
        """Work of job 'job' in the last replay (bfi_batch_get_work)."""
        w = Work()
        _check(_lib.bfi_batch_get_work(self._h, job, ctypes.byref(w)))
        return w

    def close(self):
        if getattr(self, "_h", None):
            _lib.bfi_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Request:
    """A job submitted to a Server."""

    def __init__(self, handle, server, lat: Lattice):
        self._h = handle
        self._server = server
        self.lattice = lat

    def poll(self) -> bool:
        done = ctypes.c_int32()
        _check(_lib.bfi_poll(self._h, ctypes.byref(done)))
        return bool(done.value)

    def wait(self, timeout_ms: int = -1):
        """Returns when done; raises BfiError (status 4 on timeout, 5 if cancelled)."""
        _check(_lib.bfi_wait(self._h, int(timeout_ms)))

    def cancel(self):
        _check(_lib.bfi_cancel(self._h))

    def work(self) -> Work:
        """Counted work of the request's completed passes (bfi_request_get_work)."""
        w = Work()
        _check(_lib.bfi_request_get_work(self._h, ctypes.byref(w)))
        return w

    def info(self) -> RequestInfo:
        info = RequestInfo()
        _check(_lib.bfi_request_get_info(self._h, ctypes.byref(info)))
        return info

    def result(self, leaves: bool = False):
        """totals, or (totals, slots, lo, hi, sub_id) of the leaf subvolumes."""
        lat = self.lattice
        totals = np.empty(totals_len(lat.nx))
        if not leaves:
            _check(_lib.bfi_request_get_result(self._h, ctypes.c_void_p(totals.ctypes.data), None, None, None,
                                               None))
            return totals
        n = self.info().nsub_final
        d = lat.nx * lat.nt
        slots = np.empty((n, slot_len(lat.nx)))
        lo = np.empty((n, d))
        hi = np.empty((n, d))
        sid = np.empty(n, dtype=np.uint32)
        _check(_lib.bfi_request_get_result(self._h, ctypes.c_void_p(totals.ctypes.data),
                                           ctypes.c_void_p(slots.ctypes.data), ctypes.c_void_p(lo.ctypes.data),
                                           ctypes.c_void_p(hi.ctypes.data), ctypes.c_void_p(sid.ctypes.data)))
        return totals, slots, lo, hi, sid

    def release(self):
        if getattr(self, "_h", None):
            _lib.bfi_request_release(self._h)
            self._h = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class Server:
    """Jobs admitted as they arrive (streams x memory budget), adaptive splitting."""

    def __init__(self, device: int = 0, slots: int = 8, memory_budget: int = 40 << 30,
                 precision: int = FP32, split_rel_var: float = 0.0, max_split_rounds: int = 0):
        cfg = ServerConfig(device, slots, memory_budget, precision, split_rel_var, max_split_rounds)
        handle = ctypes.c_void_p()
        _check(_lib.bfi_server_create(ctypes.byref(handle), ctypes.byref(cfg)))
        self._h = handle
        self._requests = []

    def submit(self, lat: Lattice, lo, hi, samples, seed: int, job_id: int = 0) -> Request:
        d = lat.nx * lat.nt
        lo_a, lo_p = _host(np.reshape(lo, (-1, d)), np.float64)
        hi_a, hi_p = _host(np.reshape(hi, (-1, d)), np.float64)
        nsub = lo_a.shape[0]
        smp_a, smp_p = _host(np.broadcast_to(np.asarray(samples, dtype=np.uint64), (nsub,)), np.uint64)
        if hi_a.shape != lo_a.shape:
            raise ValueError("lo and hi must describe the same subvolumes")
        h = ctypes.c_void_p()
        _check(_lib.bfi_submit(self._h, ctypes.byref(lat), nsub, lo_p, hi_p, smp_p, seed & 0xFFFFFFFF,
                               job_id & 0xFFFFFFFF, ctypes.byref(h)))
        req = Request(h, self, lat)
        self._requests.append(req)
        return req

    def stats(self) -> ServerStats:
        st = ServerStats()
        _check(_lib.bfi_server_get_stats(self._h, ctypes.byref(st)))
        return st

    def shutdown(self, timeout_ms: int = -1):
        """Stop admitting, cancel queued jobs, wait at most timeout_ms for
        running passes (raises BfiError with BFI_E_TIMEOUT if they run on)."""
        _check(_lib.bfi_server_shutdown(self._h, int(timeout_ms)))

    def inject_fault(self, point: int, nth: int = 0):
        """Host-side fault for tests of the failure path (bfi_server_inject_fault)."""
        _check(_lib.bfi_server_inject_fault(self._h, int(point), int(nth)))

    def close(self):
        if getattr(self, "_h", None):
            for r in self._requests:
                r.release()
            self._requests = []
            _lib.bfi_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nsphere(dims: int, n: int, seed: int, job_id: int = 0, lo=-1.0, hi=1.0, sub_id: int = 0, device: int = 0):
    """(result, abs_err, split_dim) of the N-sphere integrand of Sec. 3 on the GPU."""
    lo_a, lo_p = _host(np.broadcast_to(np.asarray(lo, dtype=np.float64), (dims,)), np.float64)
    hi_a, hi_p = _host(np.broadcast_to(np.asarray(hi, dtype=np.float64), (dims,)), np.float64)
    res, err, sd = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    _check(_lib.bfi_nsphere(dims, lo_p, hi_p, int(n), seed, job_id, sub_id, ctypes.byref(res), ctypes.byref(err),
                            ctypes.byref(sd), device))
    return res.value, err.value, sd.value


def adaptive_nsphere(dims: int, n: int, seed: int, conv: Convergence, job_id: int = 0, lo=-1.0, hi=1.0,
                     device: int = 0):
    """(result, abs_err, stats) of the N-sphere integrand with adaptive subdivision (Sec. 3)."""
    lo_a, lo_p = _host(np.broadcast_to(np.asarray(lo, dtype=np.float64), (dims,)), np.float64)
    hi_a, hi_p = _host(np.broadcast_to(np.asarray(hi, dtype=np.float64), (dims,)), np.float64)
    res, err, stats = ctypes.c_double(), ctypes.c_double(), AdaptiveStats()
    _check(_lib.bfi_adaptive_nsphere(dims, lo_p, hi_p, int(n), seed, job_id, ctypes.byref(conv), ctypes.byref(res),
                                     ctypes.byref(err), ctypes.byref(stats), device))
    return res.value, err.value, stats


def merge_host(nx: int, slots) -> np.ndarray:
    """FP64 merge of subvolume records on the host (the library's own merge)."""
    s_a, s_p = _host(np.reshape(slots, (-1, slot_len(nx))), np.float64)
    out = np.empty(totals_len(nx))
    _check(_lib.bfi_merge_host(nx, s_a.shape[0], s_p, ctypes.c_void_p(out.ctypes.data)))
    return out


def chunking(samples) -> Chunking:
    """How a job with these per-subvolume budgets is cut into chunks
    (bfi_chunking_of; host only)."""
    smp = np.ascontiguousarray(np.atleast_1d(samples), dtype=np.uint64)
    out = Chunking()
    _check(_lib.bfi_chunking_of(smp.size, smp.ctypes.data_as(_P(ctypes.c_uint64)), ctypes.byref(out)))
    return out


def error_bound(lat: Lattice, precision: int, slots, vmax: float) -> np.ndarray:
    """Stated arithmetic error of a result from its subvolume records (host
    array or CUDA tensor [nsub, slot_len]): [bound on |dZ|/Z, bound on
    |dC(r)|/C(0) for r = 0..R-1]; see bfi_error_bound."""
    if hasattr(slots, "cpu"):
        slots = slots.cpu().numpy()
    s_a, s_p = _host(np.reshape(slots, (-1, slot_len(lat.nx))), np.float64)
    out = np.empty(1 + num_r(lat.nx))
    _check(_lib.bfi_error_bound(ctypes.byref(lat), precision, s_a.shape[0], s_p, float(vmax),
                                ctypes.c_void_p(out.ctypes.data)))
    return out


def points(d, lo, hi, sub_id, seed, job_id, first, count, precision=FP64, stream=None):
    """Coordinates of samples [first, first+count) of one subvolume (CUDA tensors)."""
    import torch
    y = torch.empty((count, d), dtype=torch.float64, device=lo.device)
    _check(_lib.bfi_points(d, _dev_ptr(lo, torch.float64, d, "lo"), _dev_ptr(hi, torch.float64, d, "hi"), sub_id,
                           seed, job_id, first, count, precision, _dev_ptr(y), _stream_ptr(stream)))
    return y


def evaluate(lat: Lattice, y, precision=FP64, stream=None):
    """Action S and products P_r at points y [npts, d] (CUDA float64 tensor)."""
    import torch
    n = y.shape[0]
    S = torch.empty(n, dtype=torch.float64, device=y.device)
    P = torch.empty((n, num_r(lat.nx)), dtype=torch.float64, device=y.device)
    _check(_lib.bfi_eval(ctypes.byref(lat), n, _dev_ptr(y, torch.float64, n * lat.nx * lat.nt, "y"), precision, _dev_ptr(S),
                         _dev_ptr(P), _stream_ptr(stream)))
    return S, P
