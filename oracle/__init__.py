"""Plain FP64 CPU oracle for the lattice Burgers functional integral.

TEST INFRASTRUCTURE ONLY: this package may be imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``, never
by the product package.  It wraps ``oracle.c`` (built here with gcc, OpenMP
over subvolumes) through ctypes.  See ``oracle.c`` for the definitions it
follows (Eq. (Gen2), Sec. 3 and Sec. 4 of Honkonen & Honkonen,
arXiv:1803.07560) and for the record layouts.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_build", platform.machine(), "liboracle.so")  # per host architecture
_lib = None


class Lattice(ctypes.Structure):
    """Lattice of Eq. (Gen2): Nx spatial sites (M), Nt time slices (L)."""

    _fields_ = [
        ("nx", ctypes.c_int32),
        ("nt", ctypes.c_int32),
        ("nu", ctypes.c_double),
        ("D", ctypes.c_double),
        ("a", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("nonlinear", ctypes.c_double),
        ("mass2", ctypes.c_double),
    ]


def lattice(nx, nt, nu=1.0, D=1.0, a=1.0, tau=1.0, nonlinear=1.0, mass2=0.0) -> Lattice:
    return Lattice(nx, nt, nu, D, a, tau, nonlinear, mass2)


def build(force: bool = False) -> str:
    """Compile liboracle.so (plain C, -ffp-contract=off, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.POINTER
    u32p, u64p, dp = P(ctypes.c_uint32), P(ctypes.c_uint64), P(ctypes.c_double)
    lib.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
    lib.oracle_sample_words.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_uint64, ctypes.c_int, u32p]
    lib.oracle_action.argtypes = [P(Lattice), dp]
    lib.oracle_action.restype = ctypes.c_double
    lib.oracle_correlations.argtypes = [P(Lattice), dp, dp]
    lib.oracle_merge.argtypes = [ctypes.c_int, ctypes.c_int64, dp, dp]
    lib.oracle_integrate.argtypes = [P(Lattice), ctypes.c_int64, dp, dp, u64p, u32p,
                                     ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int,
                                     ctypes.c_int, dp, dp]
    lib.oracle_integrate.restype = ctypes.c_int
    lib.oracle_eval_points.argtypes = [P(Lattice), ctypes.c_int64, dp, dp, dp]
    lib.oracle_points.argtypes = [ctypes.c_int, dp, dp, ctypes.c_uint32, ctypes.c_uint32,
                                  ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64,
                                  ctypes.c_int, dp]
    lib.oracle_nsphere.argtypes = [ctypes.c_int, dp, dp, ctypes.c_uint64, ctypes.c_uint32,
                                   ctypes.c_uint32, ctypes.c_uint32, dp, dp, P(ctypes.c_int)]
    _lib = lib
    return lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def num_r(nx: int) -> int:
    return nx // 2 + 1


def slot_len(nx: int) -> int:
    return 5 + 3 * num_r(nx)


def totals_len(nx: int) -> int:
    return 4 + 2 * num_r(nx)


def philox4x32_10(ctr, key) -> np.ndarray:
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.oracle_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                             _ptr(out, ctypes.c_uint32))
    return out


def sample_words(seed: int, job_id: int, sid: int, i: int, d: int) -> np.ndarray:
    lib = _load()
    out = np.zeros(d, dtype=np.uint32)
    lib.oracle_sample_words(seed, job_id, sid, i, d, _ptr(out, ctypes.c_uint32))
    return out


def action(lat: Lattice, u) -> float:
    lib = _load()
    u = np.ascontiguousarray(u, dtype=np.float64)
    assert u.size == lat.nx * lat.nt
    return lib.oracle_action(ctypes.byref(lat), _ptr(u, ctypes.c_double))


def correlations(lat: Lattice, u) -> np.ndarray:
    lib = _load()
    u = np.ascontiguousarray(u, dtype=np.float64)
    P = np.zeros(num_r(lat.nx))
    lib.oracle_correlations(ctypes.byref(lat), _ptr(u, ctypes.c_double), _ptr(P, ctypes.c_double))
    return P


def eval_points(lat: Lattice, y) -> tuple[np.ndarray, np.ndarray]:
    lib = _load()
    d = lat.nx * lat.nt
    y = np.ascontiguousarray(y, dtype=np.float64).reshape(-1, d)
    S = np.zeros(y.shape[0])
    P = np.zeros((y.shape[0], num_r(lat.nx)))
    lib.oracle_eval_points(ctypes.byref(lat), y.shape[0], _ptr(y, ctypes.c_double),
                           _ptr(S, ctypes.c_double), _ptr(P, ctypes.c_double))
    return S, P


def points(d, lo, hi, sid, seed, job_id, first, count, fp32_points=False) -> np.ndarray:
    lib = _load()
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    y = np.zeros((count, d))
    lib.oracle_points(d, _ptr(lo, ctypes.c_double), _ptr(hi, ctypes.c_double), sid, seed,
                      job_id, first, count, int(fp32_points), _ptr(y, ctypes.c_double))
    return y


def merge(nx: int, slots) -> np.ndarray:
    lib = _load()
    slots = np.ascontiguousarray(slots, dtype=np.float64).reshape(-1, slot_len(nx))
    totals = np.zeros(totals_len(nx))
    lib.oracle_merge(nx, slots.shape[0], _ptr(slots, ctypes.c_double),
                     _ptr(totals, ctypes.c_double))
    return totals


def integrate(lat: Lattice, lo, hi, samples, seed: int, job_id: int = 0, sub_id=None,
              fp32_points: bool = False, nthreads: int | None = None):
    """Per-subvolume slots [nsub, 5+3R] and totals [4+2R] (layouts in oracle.c)."""
    lib = _load()
    d = lat.nx * lat.nt
    lo = np.ascontiguousarray(lo, dtype=np.float64).reshape(-1, d)
    hi = np.ascontiguousarray(hi, dtype=np.float64).reshape(-1, d)
    nsub = lo.shape[0]
    samples = np.ascontiguousarray(np.broadcast_to(np.asarray(samples, dtype=np.uint64), (nsub,)))
    sid = None if sub_id is None else np.ascontiguousarray(sub_id, dtype=np.uint32)
    slots = np.zeros((nsub, slot_len(lat.nx)))
    totals = np.zeros(totals_len(lat.nx))
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    rc = lib.oracle_integrate(ctypes.byref(lat), nsub, _ptr(lo, ctypes.c_double),
                              _ptr(hi, ctypes.c_double), _ptr(samples, ctypes.c_uint64),
                              None if sid is None else _ptr(sid, ctypes.c_uint32),
                              seed, job_id, int(fp32_points), nthreads,
                              _ptr(slots, ctypes.c_double), _ptr(totals, ctypes.c_double))
    if rc != 0:
        raise ValueError("oracle_integrate: invalid arguments")
    return slots, totals


def nsphere(dims: int, n: int, seed: int, job_id: int = 0, lo=-1.0, hi=1.0, split: bool = False, sub_id: int = 0):
    """Plain MC of sqrt(max(0, 1-|x|^2)) over a box (the integrand of Sec. 3):
    (result, abs_err), or (result, abs_err, split_dim) with split=True."""
    lib = _load()
    lo_a = np.ascontiguousarray(np.broadcast_to(np.asarray(lo, dtype=np.float64), (dims,)))
    hi_a = np.ascontiguousarray(np.broadcast_to(np.asarray(hi, dtype=np.float64), (dims,)))
    res, err, sd = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    lib.oracle_nsphere(dims, _ptr(lo_a, ctypes.c_double), _ptr(hi_a, ctypes.c_double), n,
                       seed, job_id, sub_id, ctypes.byref(res), ctypes.byref(err), ctypes.byref(sd))
    return (res.value, err.value, sd.value) if split else (res.value, err.value)
