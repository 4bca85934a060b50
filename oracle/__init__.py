"""CPU oracle for the stencil sweeps (ctypes wrapper around an5d_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the benchmark's CPU-baseline leg.  The CUDA product path never imports it.

The C source is compiled on first use with the host C compiler, without
fast-math and without FMA contraction, into ``oracle/_build``.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "an5d_oracle.c")
_BUILD = os.path.join(_HERE, "_build")

STAR = 0
BOX = 1

_lib = None


def _lib_path() -> str:
    with open(_SRC, "rb") as f:
        tag = hashlib.sha1(f.read()).hexdigest()[:12]
    return os.path.join(_BUILD, f"liban5d_oracle_{tag}.so")


def build(verbose: bool = False) -> str:
    """Compile the oracle library if it is missing or stale; return its path."""
    path = _lib_path()
    if os.path.exists(path):
        return path
    os.makedirs(_BUILD, exist_ok=True)
    cc = os.environ.get("CC", "gcc")
    tmp = path + f".tmp{os.getpid()}"
    cmd = [cc, "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(tmp, path)
    return path


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64 = ctypes.c_int, ctypes.c_int64
        for name in ("oracle_run_f32", "oracle_run_f64", "oracle_run_f16s",
                     "oracle_run_dot2", "oracle_run_periodic_f64"):
            fn = getattr(L, name)
            fn.argtypes = [i32, i32, i32, P, P, P, P, i64]
            fn.restype = i32
        L.oracle_run_div_f32.argtypes = [i32, i32, i32, P, ctypes.c_float, i32, P, P, P, i64]
        L.oracle_run_div_f32.restype = i32
        L.oracle_run_div_f64.argtypes = [i32, i32, i32, P, ctypes.c_double, i32, P, P, P, i64]
        L.oracle_run_div_f64.restype = i32
        L.oracle_adjoint_f64.argtypes = [i32, i32, i32, P, P, P, P, i64, P, P, P]
        L.oracle_adjoint_f64.restype = i32
        L.oracle_offsets.argtypes = [i32, i32, i32, P]
        L.oracle_offsets.restype = i32
        L.oracle_set_threads.argtypes = [i32]
        L.oracle_set_threads.restype = None
        L.oracle_get_threads.argtypes = []
        L.oracle_get_threads.restype = i32
        L.oracle_f32_to_f16.argtypes = [ctypes.c_float]
        L.oracle_f32_to_f16.restype = ctypes.c_uint16
        L.oracle_f16_to_f32.argtypes = [ctypes.c_uint16]
        L.oracle_f16_to_f32.restype = ctypes.c_float
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dims(dims) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(dims, dtype=np.int64))


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"{what} failed with status {rc}")


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(lib().oracle_get_threads())


def offsets(ndim: int, shape: int, radius: int) -> np.ndarray:
    """Canonical offsets as an (n, 3) int array of (dz, dy, dx)."""
    buf = np.zeros(3 * 1024, dtype=np.int32)
    n = lib().oracle_offsets(ndim, shape, radius, _ptr(buf))
    if n < 0:
        raise ValueError("unsupported stencil")
    return buf[: 3 * n].reshape(n, 3).copy()


def _run(fn, ndim, shape, radius, coeffs, dims, u, T, cdtype, udtype):
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=cdtype))
    u = np.ascontiguousarray(u, dtype=udtype)
    out = np.empty_like(u)
    d = _dims(dims)
    _check(fn(ndim, shape, radius, _ptr(c), _ptr(d), _ptr(u), _ptr(out), int(T)), fn.__name__)
    return out


def run_f32(ndim, shape, radius, coeffs, dims, u, T):
    """Plain method in FP32 (coefficients must already be FP32 values)."""
    return _run(lib().oracle_run_f32, ndim, shape, radius, coeffs, dims, u, T,
                np.float32, np.float32)


def run_f64(ndim, shape, radius, coeffs, dims, u, T):
    """Plain method in FP64."""
    return _run(lib().oracle_run_f64, ndim, shape, radius, coeffs, dims, u, T,
                np.float64, np.float64)


def run_f16s(ndim, shape, radius, coeffs, dims, u_f16, T):
    """FP16 storage / FP32 compute; u_f16 is a float16 array."""
    bits = np.ascontiguousarray(u_f16, dtype=np.float16).view(np.uint16)
    out = _run(lib().oracle_run_f16s, ndim, shape, radius, coeffs, dims, bits, T,
               np.float32, np.uint16)
    return out.view(np.float16)


def run_dot2(ndim, shape, radius, coeffs, dims, u, T):
    """Compensated (Dot2) FP32 method."""
    return _run(lib().oracle_run_dot2, ndim, shape, radius, coeffs, dims, u, T,
                np.float32, np.float32)


POST_DIV, POST_MUL_RCP = 1, 2


def run_div(dtype, ndim, shape, radius, coeffs, divisor, post, dims, u, T):
    """Division-type stencil (Table 4's j* rows): the plain chain, then per
    step a division by `divisor` (post=POST_DIV) or a multiplication by its
    reciprocal rounded to the dtype (post=POST_MUL_RCP).  dtype: "f32" or
    "f64"; `divisor` is rounded to the dtype first."""
    if dtype == "f32":
        fn, t = lib().oracle_run_div_f32, np.float32
    elif dtype == "f64":
        fn, t = lib().oracle_run_div_f64, np.float64
    else:
        raise ValueError(dtype)
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=t))
    u = np.ascontiguousarray(u, dtype=t)
    out = np.empty_like(u)
    d = _dims(dims)
    _check(fn(ndim, shape, radius, _ptr(c), float(t(divisor)), int(post), _ptr(d), _ptr(u),
              _ptr(out), int(T)), fn.__name__)
    return out


def run_periodic_f64(ndim, shape, radius, coeffs, dims, u, T):
    """Periodic FP64 variant on an unpadded grid of extents `dims`."""
    return _run(lib().oracle_run_periodic_f64, ndim, shape, radius, coeffs, dims, u, T,
                np.float64, np.float64)


def adjoint_f64(ndim, shape, radius, coeffs, dims, u0, target, T):
    """FP64 adjoint: returns (loss, grad_u0 (padded, zero halo), grad_c)."""
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    tg = np.ascontiguousarray(target, dtype=np.float64)
    gu = np.zeros_like(u0)
    gc = np.zeros(c.size, dtype=np.float64)
    loss = np.zeros(1, dtype=np.float64)
    d = _dims(dims)
    _check(lib().oracle_adjoint_f64(ndim, shape, radius, _ptr(c), _ptr(d), _ptr(u0), _ptr(tg),
                                    int(T), _ptr(gu), _ptr(gc), _ptr(loss)), "oracle_adjoint_f64")
    return float(loss[0]), gu, gc


def f32_to_f16_bits(x: float) -> int:
    return int(lib().oracle_f32_to_f16(float(x)))


def f16_bits_to_f32(h: int) -> float:
    return float(lib().oracle_f16_to_f32(int(h)))
