"""Python binding of the C ABI in include/an5d.h (ctypes; argument marshalling only).

Every function here has the name of the C entry point it calls.  Torch
tensors are passed as device pointers (``tensor.data_ptr()``) and streams
as ``torch.cuda.Stream.cuda_stream``; no computation happens in Python.
The library is the in-tree ``_build/liban5d.so``: if it is missing this
module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .inputs import STAR, BOX  # noqa: F401  (re-exported shape codes)

F32, F64, F16S_F32C, F32_COMPENSATED = 0, 1, 2, 3
DTYPES = {"f32": F32, "f64": F64, "f16": F16S_F32C, "f32c": F32_COMPENSATED}

AN5D_OK = 0
AN5D_ERR_INVALID_ARG = -1
AN5D_ERR_UNSUPPORTED = -2
AN5D_ERR_ALIAS = -3
AN5D_ERR_CUDA = -4
AN5D_ERR_OOM = -5
AN5D_ERR_TIMEOUT = -6

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "liban5d.so")

_lib = None


class An5dError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"an5d status {status}: {msg}")
        self.status = status


class an5d_paper_stencil(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("shape", ctypes.c_int), ("radius", ctypes.c_int),
                ("word_bytes", ctypes.c_int), ("op_fma", ctypes.c_int), ("op_mul", ctypes.c_int),
                ("op_add", ctypes.c_int), ("op_other", ctypes.c_int)]


class an5d_paper_device(ctypes.Structure):
    _fields_ = [("peak_comp_gflops", ctypes.c_double), ("peak_gm_gbs", ctypes.c_double),
                ("peak_sm_gbs", ctypes.c_double), ("sm_count", ctypes.c_int),
                ("max_threads_per_sm", ctypes.c_int)]


class an5d_paper_model_result(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "th_comp", "th_sm_read", "th_sm_write", "th_gm_read", "th_gm_write",
        "total_comp", "total_gm", "total_sm", "eff_alu", "eff_sm",
        "time_comp", "time_gm", "time_sm", "time_model", "gcells", "gflops")] + [
        ("n_tb", ctypes.c_int64), ("bound", ctypes.c_int)]


class an5d_config(ctypes.Structure):
    _fields_ = [("bT", ctypes.c_int), ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int),
                ("stream_axis", ctypes.c_int), ("hsn", ctypes.c_int),
                ("warps_per_cta", ctypes.c_int), ("ctas", ctypes.c_int),
                ("launches_per_pass", ctypes.c_int), ("model_gcells", ctypes.c_double),
                ("measured_gcells", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class an5d_grid_desc(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_int), ("radius", ctypes.c_int),
                ("coeffs", ctypes.c_void_p), ("ny", ctypes.c_int64), ("nx", ctypes.c_int64),
                ("T", ctypes.c_int64)]


class an5d_batch_info_t(ctypes.Structure):
    _fields_ = [("grids", ctypes.c_int), ("ctas", ctypes.c_int), ("items", ctypes.c_int64),
                ("cell_updates", ctypes.c_double), ("class_bt", ctypes.c_int * 4),
                ("class_tile_x", ctypes.c_int * 4)]

    def as_dict(self) -> dict:
        return {"grids": self.grids, "ctas": self.ctas, "items": self.items,
                "cell_updates": self.cell_updates, "class_bt": list(self.class_bt),
                "class_tile_x": list(self.class_tile_x)}


class an5d_adjoint_batch_info_t(ctypes.Structure):
    _fields_ = [("grids", ctypes.c_int), ("waves", ctypes.c_int), ("ctas", ctypes.c_int),
                ("items", ctypes.c_int64), ("cell_updates", ctypes.c_double),
                ("work_bytes", ctypes.c_size_t), ("class_nb", ctypes.c_int * 4)]

    def as_dict(self) -> dict:
        return {"grids": self.grids, "waves": self.waves, "ctas": self.ctas, "items": self.items,
                "cell_updates": self.cell_updates, "work_bytes": self.work_bytes,
                "class_nb": list(self.class_nb)}


class an5d_peaks(ctypes.Structure):
    _fields_ = [("hbm_gbs", ctypes.c_double), ("fp32_gflops", ctypes.c_double),
                ("fp64_gflops", ctypes.c_double), ("smem_gbs", ctypes.c_double),
                ("sm_clock_mhz", ctypes.c_double), ("sms", ctypes.c_int),
                ("measured", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


def load(path: str = LIB_PATH):
    """Load liban5d.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build the CUDA extension first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(path)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    L.an5d_coeff_count.argtypes = [I, I, I]
    L.an5d_coeff_count.restype = I
    L.an5d_plan_create.argtypes = [I, I, I, P, I, P]
    L.an5d_plan_create.restype = P
    L.an5d_plan_create_div.argtypes = [I, I, I, P, ctypes.c_double, I, I, P]
    L.an5d_plan_create_div.restype = P
    L.an5d_paper_model.argtypes = [ctypes.POINTER(an5d_paper_stencil), P, I, P, I,
                                   ctypes.POINTER(an5d_paper_device),
                                   ctypes.POINTER(an5d_paper_model_result)]
    L.an5d_paper_model.restype = I
    L.an5d_run.argtypes = [P, P, P, I64, P]
    L.an5d_run.restype = I
    L.an5d_run_host.argtypes = [P, P, P, I64, P]
    L.an5d_run_host.restype = I
    L.an5d_plan_destroy.argtypes = [P]
    L.an5d_plan_destroy.restype = None
    L.an5d_plan_config.argtypes = [P, ctypes.POINTER(an5d_config)]
    L.an5d_plan_config.restype = I
    L.an5d_plan_set_config.argtypes = [P, I, I]
    L.an5d_plan_set_config.restype = I
    L.an5d_plan_set_tile.argtypes = [P, I]
    L.an5d_plan_set_tile.restype = I
    L.an5d_plan_set_coeffs.argtypes = [P, P]
    L.an5d_plan_set_coeffs.restype = I
    L.an5d_plan_launches.argtypes = [P, I64]
    L.an5d_plan_launches.restype = I64
    L.an5d_plan_tune.argtypes = [P, I, I64, P]
    L.an5d_plan_tune.restype = I
    L.an5d_plan_status.argtypes = [P]
    L.an5d_plan_status.restype = I
    L.an5d_run_noalloc.argtypes = [I, I, I, P, I, P, P, P, I64, P]
    L.an5d_run_noalloc.restype = I
    L.an5d_error_norms.argtypes = [I, I, P, I, P, P, P, P]
    L.an5d_error_norms.restype = I
    L.an5d_plan_inject_stall.argtypes = [P, I]
    L.an5d_plan_inject_stall.restype = I
    L.an5d_batch_inject_stall.argtypes = [P, I]
    L.an5d_batch_inject_stall.restype = I
    L.an5d_run_adjoint.argtypes = [P, P, P, P, P, I64, P]
    L.an5d_run_adjoint.restype = I
    L.an5d_split_geometry.argtypes = [I, P, I, I, I, I, P]
    L.an5d_split_geometry.restype = I
    L.an5d_run_split.argtypes = [P, I, P, P, I64, P]
    L.an5d_run_split.restype = I
    L.an5d_batch_plan_create.argtypes = [I, P]
    L.an5d_batch_plan_create.restype = P
    L.an5d_batch_tune.argtypes = [P, P]
    L.an5d_batch_tune.restype = I
    L.an5d_batch_tune_run.argtypes = [P, P, P, P]
    L.an5d_batch_tune_run.restype = I
    L.an5d_batch_set_degrees.argtypes = [P, P]
    L.an5d_batch_set_degrees.restype = I
    L.an5d_batch_set_tiles.argtypes = [P, P]
    L.an5d_batch_set_tiles.restype = I
    L.an5d_batch_run.argtypes = [P, P, P, P]
    L.an5d_batch_run.restype = I
    L.an5d_batch_status.argtypes = [P]
    L.an5d_batch_status.restype = I
    L.an5d_batch_info.argtypes = [P, ctypes.POINTER(an5d_batch_info_t)]
    L.an5d_batch_info.restype = I
    L.an5d_batch_last_error.argtypes = []
    L.an5d_batch_last_error.restype = ctypes.c_char_p
    L.an5d_batch_plan_destroy.argtypes = [P]
    L.an5d_batch_plan_destroy.restype = None
    L.an5d_adjoint_batch_create.argtypes = [I, P, ctypes.c_size_t]
    L.an5d_adjoint_batch_create.restype = P
    L.an5d_adjoint_batch_run.argtypes = [P, P, P, P, P, P]
    L.an5d_adjoint_batch_run.restype = I
    L.an5d_adjoint_batch_info.argtypes = [P, ctypes.POINTER(an5d_adjoint_batch_info_t)]
    L.an5d_adjoint_batch_info.restype = I
    L.an5d_adjoint_batch_destroy.argtypes = [P]
    L.an5d_adjoint_batch_destroy.restype = None
    L.an5d_adjoint_batch_last_error.argtypes = []
    L.an5d_adjoint_batch_last_error.restype = ctypes.c_char_p
    L.an5d_measure_peaks.argtypes = [ctypes.POINTER(an5d_peaks), P]
    L.an5d_measure_peaks.restype = I
    L.an5d_get_peaks.argtypes = [ctypes.POINTER(an5d_peaks)]
    L.an5d_get_peaks.restype = I
    L.an5d_last_error.argtypes = []
    L.an5d_last_error.restype = ctypes.c_char_p
    L.an5d_last_status.argtypes = []
    L.an5d_last_status.restype = I
    L.an5d_version.argtypes = []
    L.an5d_version.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(rc: int) -> int:
    if rc != AN5D_OK:
        raise An5dError(rc, an5d_last_error())
    return rc


def _ptr(x) -> int | None:
    """Device or host address of a torch tensor, numpy array or int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------------------
# C entry points, same names.

def an5d_version() -> str:
    return load().an5d_version().decode()


def an5d_last_error() -> str:
    return load().an5d_last_error().decode()


def an5d_last_status() -> int:
    return load().an5d_last_status()


def an5d_coeff_count(ndim: int, shape: int, radius: int) -> int:
    n = load().an5d_coeff_count(ndim, shape, radius)
    if n < 0:
        raise An5dError(n, an5d_last_error())
    return n


def an5d_plan_create(ndim: int, shape: int, radius: int, coeffs, dtype, dims) -> int:
    """Returns an opaque plan handle (int)."""
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
    d = np.ascontiguousarray(np.asarray(dims, dtype=np.int64))
    h = load().an5d_plan_create(ndim, shape, radius, c.ctypes.data, dt, d.ctypes.data)
    if not h:
        raise An5dError(an5d_last_status(), an5d_last_error())
    return h


def an5d_run(plan: int, inp, out, T: int, stream=None) -> int:
    return _check(load().an5d_run(plan, _ptr(inp), _ptr(out), int(T), _stream(stream)))


def an5d_run_host(plan: int, inp: np.ndarray, out: np.ndarray, T: int, stream=None) -> int:
    return _check(load().an5d_run_host(plan, _ptr(inp), _ptr(out), int(T), _stream(stream)))


def an5d_run_noalloc(ndim: int, shape: int, radius: int, coeffs, dtype, dims, inp, out,
                     T: int, stream=None) -> int:
    """Allocation-free run (see an5d.h): same arguments as plan creation plus
    the buffers of an5d_run; synchronous."""
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
    d = np.ascontiguousarray(np.asarray(dims, dtype=np.int64))
    return _check(load().an5d_run_noalloc(ndim, shape, radius, c.ctypes.data, dt, d.ctypes.data,
                                          _ptr(inp), _ptr(out), int(T), _stream(stream)))


def an5d_error_norms(ndim: int, radius: int, dims, dtype, u, ref, stream=None) -> dict:
    """FP64 error norms of device array u against device FP64 array ref."""
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    d = np.ascontiguousarray(np.asarray(dims, dtype=np.int64))
    out = np.zeros(3, dtype=np.float64)
    _check(load().an5d_error_norms(ndim, radius, d.ctypes.data, dt, _ptr(u), _ptr(ref),
                                   out.ctypes.data, _stream(stream)))
    return {"max_abs": float(out[0]), "l2_diff": float(np.sqrt(out[1])),
            "l2_ref": float(np.sqrt(out[2])),
            "rel_l2": float(np.sqrt(out[1] / out[2])) if out[2] > 0 else float("nan")}


def an5d_run_adjoint(plan: int, u0, gT, grad_u0, T: int, stream=None) -> np.ndarray:
    """Adjoint run (see an5d.h); returns dL/dc as a float64 array."""
    gc = np.zeros(729, dtype=np.float64)  # room for the largest stencil
    _check(load().an5d_run_adjoint(plan, _ptr(u0), _ptr(gT), _ptr(grad_u0), gc.ctypes.data,
                                   int(T), _stream(stream)))
    return gc


def an5d_split_geometry(ndim: int, dims, radius: int, bT: int, nsub: int, k: int) -> dict:
    """Slab k of an nsub-way split along the slowest axis (see an5d.h):
    owned interior planes [a, b) and the padded planes [lo, hi) it holds."""
    d = np.ascontiguousarray(np.asarray(dims, dtype=np.int64))
    out = np.zeros(4, dtype=np.int64)
    _check(load().an5d_split_geometry(ndim, d.ctypes.data, radius, bT, nsub, k, out.ctypes.data))
    return {"a": int(out[0]), "b": int(out[1]), "lo": int(out[2]), "hi": int(out[3])}


def an5d_run_split(plan: int, nsub: int, inp, out, T: int, stream=None) -> int:
    """The plan's sweep as nsub slabs with deepened halos (see an5d.h)."""
    return _check(load().an5d_run_split(plan, int(nsub), _ptr(inp), _ptr(out), int(T),
                                        _stream(stream)))


def an5d_plan_inject_stall(plan: int, enable: bool) -> int:
    return _check(load().an5d_plan_inject_stall(plan, int(bool(enable))))


def an5d_batch_inject_stall(bp: int, enable: bool) -> int:
    return _bcheck(load().an5d_batch_inject_stall(bp, int(bool(enable))))


def an5d_plan_destroy(plan: int) -> None:
    load().an5d_plan_destroy(plan)


def an5d_plan_config(plan: int) -> dict:
    cfg = an5d_config()
    _check(load().an5d_plan_config(plan, ctypes.byref(cfg)))
    return cfg.as_dict()


def an5d_plan_set_config(plan: int, bT: int = 0, hsn: int = 0) -> int:
    return _check(load().an5d_plan_set_config(plan, int(bT), int(hsn)))


def an5d_plan_launches(plan: int, T: int) -> int:
    n = load().an5d_plan_launches(plan, int(T))
    if n < 0:
        _check(int(n))
    return int(n)


def an5d_plan_set_tile(plan: int, tile_x: int = 0) -> int:
    return _check(load().an5d_plan_set_tile(plan, int(tile_x)))


def an5d_plan_set_coeffs(plan: int, coeffs) -> int:
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
    return _check(load().an5d_plan_set_coeffs(plan, c.ctypes.data))


def an5d_plan_tune(plan: int, topk: int = 5, T_probe: int = 20, stream=None) -> int:
    return _check(load().an5d_plan_tune(plan, int(topk), int(T_probe), _stream(stream)))


def an5d_plan_status(plan: int) -> int:
    return load().an5d_plan_status(plan)


def an5d_measure_peaks(stream=None) -> dict:
    pk = an5d_peaks()
    _check(load().an5d_measure_peaks(ctypes.byref(pk), _stream(stream)))
    return pk.as_dict()


def an5d_get_peaks() -> dict:
    pk = an5d_peaks()
    _check(load().an5d_get_peaks(ctypes.byref(pk)))
    return pk.as_dict()


def an5d_paper_model(ndim: int, shape: int, radius: int, word_bytes: int, ops, dims, bT: int,
                     bS, hSN: int, device: dict) -> dict:
    """The paper's analytic model (see an5d.h).  ops = (fma, mul, add, other)
    per cell-update; bS: block sizes, x first; device: peak_comp_gflops,
    peak_gm_gbs, peak_sm_gbs, sm_count, max_threads_per_sm."""
    st = an5d_paper_stencil(ndim, shape, radius, word_bytes, *[int(v) for v in ops])
    dv = an5d_paper_device(float(device["peak_comp_gflops"]), float(device["peak_gm_gbs"]),
                           float(device["peak_sm_gbs"]), int(device["sm_count"]),
                           int(device.get("max_threads_per_sm", 2048)))
    d = np.ascontiguousarray(np.asarray(dims, dtype=np.int64))
    b = np.ascontiguousarray(np.asarray(bS, dtype=np.int32))
    out = an5d_paper_model_result()
    _check(load().an5d_paper_model(ctypes.byref(st), d.ctypes.data, int(bT), b.ctypes.data,
                                   int(hSN), ctypes.byref(dv), ctypes.byref(out)))
    r = {n: getattr(out, n) for n, _ in an5d_paper_model_result._fields_}
    r["bound"] = ("compute", "global", "shared")[out.bound]
    return r


POST_DIV, POST_MUL_RCP = 1, 2
POSTS = {"div": POST_DIV, "rcp": POST_MUL_RCP}


def an5d_plan_create_div(ndim: int, shape: int, radius: int, coeffs, divisor: float, post,
                         dtype, dims) -> int:
    """Plan of a division-type stencil (see an5d.h); post: "div"/"rcp" or the enum value."""
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    pv = POSTS[post] if isinstance(post, str) else int(post)
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
    d = np.ascontiguousarray(np.asarray(dims, dtype=np.int64))
    h = load().an5d_plan_create_div(ndim, shape, radius, c.ctypes.data, float(divisor), pv, dt,
                                    d.ctypes.data)
    if not h:
        raise An5dError(an5d_last_status(), an5d_last_error())
    return h


# ---------------------------------------------------------------------------
# Convenience wrapper.

class Plan:
    """RAII wrapper of an an5d plan."""

    def __init__(self, ndim: int, shape: int, radius: int, coeffs, dtype, dims,
                 divisor=None, post=None):
        """With `divisor` and `post` ("div" or "rcp") the plan is a
        division-type stencil (an5d_plan_create_div)."""
        self.ndim, self.shape, self.radius = ndim, shape, radius
        self.dtype = dtype
        self.dims = tuple(int(d) for d in dims)
        if divisor is None:
            self.handle = an5d_plan_create(ndim, shape, radius, coeffs, dtype, dims)
        else:
            self.handle = an5d_plan_create_div(ndim, shape, radius, coeffs, divisor,
                                               post or "div", dtype, dims)

    def run(self, inp, out, T: int, stream=None) -> None:
        an5d_run(self.handle, inp, out, T, stream)

    def run_host(self, inp: np.ndarray, out: np.ndarray, T: int, stream=None) -> None:
        an5d_run_host(self.handle, inp, out, T, stream)

    def config(self) -> dict:
        return an5d_plan_config(self.handle)

    def set_config(self, bT: int = 0, hsn: int = 0) -> None:
        an5d_plan_set_config(self.handle, bT, hsn)

    def launches(self, T: int) -> int:
        """Kernel launches one run of T steps enqueues."""
        return an5d_plan_launches(self.handle, T)

    def set_tile(self, tile_x: int = 0) -> None:
        """Select the sweep kernel's tile variant (0 = default width)."""
        an5d_plan_set_tile(self.handle, tile_x)

    def set_coeffs(self, coeffs) -> None:
        """Replace the coefficients; configuration and buffers are kept."""
        an5d_plan_set_coeffs(self.handle, coeffs)

    def tune(self, topk: int = 5, T_probe: int = 20, stream=None) -> dict:
        an5d_plan_tune(self.handle, topk, T_probe, stream)
        return self.config()

    def status(self) -> int:
        return an5d_plan_status(self.handle)

    def close(self) -> None:
        if self.handle:
            an5d_plan_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Batched form.

def an5d_batch_last_error() -> str:
    return load().an5d_batch_last_error().decode()


def _bcheck(rc: int) -> int:
    if rc != AN5D_OK:
        raise An5dError(rc, an5d_batch_last_error())
    return rc


def an5d_batch_plan_create(grids) -> tuple:
    """grids: list of (shape, radius, coeffs, ny, nx, T).  Returns (handle, keepalive)."""
    keep = [np.ascontiguousarray(np.asarray(g[2], dtype=np.float64)) for g in grids]
    arr = (an5d_grid_desc * len(grids))()
    for i, g in enumerate(grids):
        arr[i] = an5d_grid_desc(int(g[0]), int(g[1]), keep[i].ctypes.data, int(g[3]), int(g[4]),
                                int(g[5]))
    h = load().an5d_batch_plan_create(len(grids), ctypes.cast(arr, ctypes.c_void_p))
    if not h:
        raise An5dError(AN5D_ERR_INVALID_ARG, an5d_batch_last_error())
    return h, (keep, arr)


def an5d_batch_tune(bp: int, stream=None) -> int:
    return _bcheck(load().an5d_batch_tune(bp, _stream(stream)))


def an5d_batch_tune_run(bp: int, ins, outs, stream=None) -> int:
    n = len(ins)
    pi = (ctypes.c_void_p * n)(*[_ptr(x) for x in ins])
    po = (ctypes.c_void_p * n)(*[_ptr(x) for x in outs])
    return _bcheck(load().an5d_batch_tune_run(bp, ctypes.cast(pi, ctypes.c_void_p),
                                              ctypes.cast(po, ctypes.c_void_p), _stream(stream)))


def an5d_batch_set_degrees(bp: int, class_bt) -> int:
    a = (ctypes.c_int * 4)(*[int(x) for x in class_bt])
    return _bcheck(load().an5d_batch_set_degrees(bp, ctypes.cast(a, ctypes.c_void_p)))


def an5d_batch_set_tiles(bp: int, class_tile_x) -> int:
    a = (ctypes.c_int * 4)(*[int(x) for x in class_tile_x])
    return _bcheck(load().an5d_batch_set_tiles(bp, ctypes.cast(a, ctypes.c_void_p)))


def an5d_batch_run(bp: int, ins, outs, stream=None) -> int:
    n = len(ins)
    pi = (ctypes.c_void_p * n)(*[_ptr(x) for x in ins])
    po = (ctypes.c_void_p * n)(*[_ptr(x) for x in outs])
    return _bcheck(load().an5d_batch_run(bp, ctypes.cast(pi, ctypes.c_void_p),
                                         ctypes.cast(po, ctypes.c_void_p), _stream(stream)))


def an5d_batch_status(bp: int) -> int:
    return load().an5d_batch_status(bp)


def an5d_batch_info(bp: int) -> dict:
    info = an5d_batch_info_t()
    _bcheck(load().an5d_batch_info(bp, ctypes.byref(info)))
    return info.as_dict()


def an5d_batch_plan_destroy(bp: int) -> None:
    load().an5d_batch_plan_destroy(bp)


class Batch:
    """RAII wrapper of a batch plan; grids = [(shape, radius, coeffs, ny, nx, T), ...]."""

    def __init__(self, grids):
        self.grids = list(grids)
        self.handle, self._keep = an5d_batch_plan_create(self.grids)

    def tune(self, stream=None, ins=None, outs=None) -> dict:
        """Tune the degrees by timing whole runs; on (ins, outs) when given
        (outs are overwritten), else on temporary buffers."""
        if ins is not None:
            an5d_batch_tune_run(self.handle, ins, outs, stream)
        else:
            an5d_batch_tune(self.handle, stream)
        return self.info()

    def set_degrees(self, class_bt) -> None:
        an5d_batch_set_degrees(self.handle, class_bt)

    def set_tiles(self, class_tile_x) -> None:
        an5d_batch_set_tiles(self.handle, class_tile_x)

    def run(self, ins, outs, stream=None) -> None:
        an5d_batch_run(self.handle, ins, outs, stream)

    def status(self) -> int:
        return an5d_batch_status(self.handle)

    def info(self) -> dict:
        return an5d_batch_info(self.handle)

    def close(self) -> None:
        if self.handle:
            an5d_batch_plan_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Batched adjoint.

def an5d_adjoint_batch_last_error() -> str:
    return load().an5d_adjoint_batch_last_error().decode()


def _acheck(rc: int) -> int:
    if rc != AN5D_OK:
        raise An5dError(rc, an5d_adjoint_batch_last_error())
    return rc


def an5d_adjoint_batch_create(grids, budget_bytes: int = 0) -> tuple:
    """grids: list of (shape, radius, coeffs, ny, nx, T).  Returns (handle, keepalive)."""
    keep = [np.ascontiguousarray(np.asarray(g[2], dtype=np.float64)) for g in grids]
    arr = (an5d_grid_desc * len(grids))()
    for i, g in enumerate(grids):
        arr[i] = an5d_grid_desc(int(g[0]), int(g[1]), keep[i].ctypes.data, int(g[3]), int(g[4]),
                                int(g[5]))
    h = load().an5d_adjoint_batch_create(len(grids), ctypes.cast(arr, ctypes.c_void_p), int(budget_bytes))
    if not h:
        raise An5dError(AN5D_ERR_INVALID_ARG, an5d_adjoint_batch_last_error())
    return h, (keep, arr)


def an5d_adjoint_batch_run(ab: int, u0s, gTs, grad_u0s, stream=None) -> np.ndarray:
    """Returns dL/dc as an (n, 25) float64 array (row i: grid i, canonical order)."""
    n = len(u0s)
    pu = (ctypes.c_void_p * n)(*[_ptr(x) for x in u0s])
    pg = (ctypes.c_void_p * n)(*[_ptr(x) for x in gTs])
    po = (ctypes.c_void_p * n)(*[_ptr(x) for x in grad_u0s])
    dc = np.zeros((n, 25), dtype=np.float64)
    _acheck(load().an5d_adjoint_batch_run(ab, ctypes.cast(pu, ctypes.c_void_p), ctypes.cast(pg, ctypes.c_void_p),
                                          ctypes.cast(po, ctypes.c_void_p), dc.ctypes.data, _stream(stream)))
    return dc


def an5d_adjoint_batch_info(ab: int) -> dict:
    info = an5d_adjoint_batch_info_t()
    _acheck(load().an5d_adjoint_batch_info(ab, ctypes.byref(info)))
    return info.as_dict()


def an5d_adjoint_batch_destroy(ab: int) -> None:
    load().an5d_adjoint_batch_destroy(ab)


class AdjointBatch:
    """RAII wrapper of a batched adjoint; grids = [(shape, radius, coeffs, ny, nx, T), ...]."""

    def __init__(self, grids, budget_bytes: int = 0):
        self.grids = list(grids)
        self.handle, self._keep = an5d_adjoint_batch_create(self.grids, budget_bytes)

    def run(self, u0s, gTs, grad_u0s, stream=None) -> np.ndarray:
        return an5d_adjoint_batch_run(self.handle, u0s, gTs, grad_u0s, stream)

    def info(self) -> dict:
        return an5d_adjoint_batch_info(self.handle)

    def close(self) -> None:
        if self.handle:
            an5d_adjoint_batch_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
