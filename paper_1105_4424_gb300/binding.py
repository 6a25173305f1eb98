"""ctypes binding of libarol.so: the C entry points under the same names.

Argument marshalling only — every step of a task runs in the library's CUDA
kernels.  Device buffers are torch tensors (or raw integer addresses); the
stream defaults to torch's current CUDA stream.  A missing library is an
ImportError, never a silent fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# AROL_LIB selects another build of the library (e.g. libarol_debug.so)
LIB_PATH = os.environ.get("AROL_LIB") or os.path.join(_PKG, "libarol.so")

c_i32, c_i64, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p

AROL_F32, AROL_BF16, AROL_F16 = 0, 1, 2
ELEM = {"copy": 0, "fir": 1, "matmul": 2}
DTYPE = {"f32": AROL_F32, "bf16": AROL_BF16, "f16": AROL_F16}
STATUS = {0: "AROL_OK", 1: "AROL_ERR_INVALID", 2: "AROL_ERR_NOT_PARTITION", 3: "AROL_ERR_UNSUPPORTED",
          4: "AROL_ERR_CUDA", 5: "AROL_ERR_TIMEOUT", 6: "AROL_ERR_OOB"}


class ArrayDesc(ctypes.Structure):
    _fields_ = [("rank", c_i32), ("dtype", c_i32), ("shape", c_i64 * 4)]


class Tiler(ctypes.Structure):
    _fields_ = [("origin", c_i64 * 4), ("paving", (c_i64 * 4) * 4), ("fitting", (c_i64 * 2) * 4),
                ("pattern_rank", c_i32), ("reserved_", c_i32), ("pattern", c_i64 * 2)]


class TaskDesc(ctypes.Structure):
    _fields_ = [("rep_rank", c_i32), ("elem", c_i32), ("rep", c_i64 * 4), ("n_in", c_i32), ("n_out", c_i32),
                ("in_", ArrayDesc * 2), ("out", ArrayDesc * 1), ("in_tiler", Tiler * 2), ("out_tiler", Tiler * 1),
                ("fir_T", c_i32), ("fir_m", c_i32), ("fir_taps_host", c_vp)]


class TaskInfo(ctypes.Structure):
    _fields_ = [("kind", c_i32), ("kernel", c_i32), ("reps", c_i64), ("gathered_elems", c_i64),
                ("scattered_elems", c_i64), ("unique_bytes", c_i64), ("flops", ctypes.c_double),
                ("path", c_i32), ("reserved_", c_i32)]


class ArolError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built: run paper_1105_4424_gb300.build.build() "
                          "(nvcc, sm_103a); there is no fallback path")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    sig = {
        "arol_task_create": [P(TaskDesc), P(c_vp)],
        "arol_chain_create": [P(c_vp), ctypes.c_int, P(c_vp)],
        "arol_task_set_taps": [c_vp, c_vp, ctypes.c_int],
        "arol_task_run": [c_vp, P(c_vp), P(c_vp), c_vp],
        "arol_task_run_host": [c_vp, P(c_vp), P(c_vp), c_vp],
        "arol_task_backward": [c_vp, c_vp, P(c_vp), c_vp, c_vp, c_vp],
        "arol_task_fwd_bwd": [c_vp, P(c_vp), c_vp, c_vp, c_vp, c_vp, c_vp],
        "arol_task_info": [c_vp, P(TaskInfo)],
        "arol_task_sync_status": [c_vp, c_vp],
        "arol_tiler_cover": [P(ArrayDesc), P(Tiler), ctypes.c_int, P(c_i64), P(c_i64), P(c_i64)],
        "arol_selftest_wait_timeout": [c_vp],
        "arol_batch_create": [P(c_vp), ctypes.c_int, P(c_vp)],
        "arol_batch_run": [c_vp, P(c_vp), P(c_vp), c_vp],
        "arol_batch_run_per_task": [c_vp, P(c_vp), P(c_vp), c_vp],
        "arol_batch_tune": [c_vp, P(c_vp), P(c_vp), c_vp, ctypes.c_int],
        "arol_batch_config": [c_vp, P(c_i64), P(c_i32), P(c_i32)],
        "arol_task_shard_frames": [P(TaskDesc), ctypes.c_int, ctypes.c_int, P(TaskDesc), P(c_i64)],
        "arol_batch_sync_status": [c_vp, c_vp],
        "arol_last_error": [ctypes.c_char_p, ctypes.c_size_t],
        "arol_downscale_backward_noalloc": [c_vp, c_vp, c_vp, c_i64, c_i32, c_i32, c_vp, c_vp, c_vp],
        "arol_downscale_backward_noalloc_status": [c_vp],
        "arol_csr_spmv": [c_i64, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp],
        "arol_cg_create": [c_i64, c_i64, c_vp, c_vp, c_vp, P(c_vp)],
        "arol_csr_check": [c_i64, c_i64, c_vp, c_vp, c_vp],
        "arol_cg_solve": [c_vp, c_vp, c_vp, ctypes.c_double, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_double), c_vp],
        "arol_cg_last_error": [ctypes.c_char_p, ctypes.c_size_t],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.arol_task_destroy.argtypes = [c_vp]
    L.arol_task_destroy.restype = None
    L.arol_batch_destroy.argtypes = [c_vp]
    L.arol_batch_destroy.restype = None
    L.arol_cg_destroy.argtypes = [c_vp]
    L.arol_cg_destroy.restype = None
    L.arol_version.restype = ctypes.c_int
    L.arol_abi_struct_size.argtypes = [ctypes.c_int]
    L.arol_abi_struct_size.restype = c_i64
    for i, cls in enumerate((ArrayDesc, Tiler, TaskDesc, TaskInfo)):
        if L.arol_abi_struct_size(i) != ctypes.sizeof(cls):
            raise ImportError(f"ABI mismatch: {cls.__name__} is {ctypes.sizeof(cls)} bytes here, "
                              f"{L.arol_abi_struct_size(i)} in the library")
    return L


lib = _load()


def arol_last_error() -> str:
    buf = ctypes.create_string_buffer(1024)
    lib.arol_last_error(buf, len(buf))
    return buf.value.decode(errors="replace")


def _check(st):
    if st != 0:
        raise ArolError(st, arol_last_error())


def arol_version() -> int:
    return lib.arol_version()


# ------------------------------------------------------------- marshalling

def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _ptrs(xs):
    return (c_vp * max(1, len(xs)))(*[_ptr(x) for x in xs])


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def array_desc(shape, dtype="f32") -> ArrayDesc:
    a = ArrayDesc()
    a.rank = len(shape)
    a.dtype = DTYPE[dtype] if isinstance(dtype, str) else int(dtype)
    for k, v in enumerate(shape):
        a.shape[k] = int(v)
    return a


def tiler(origin, paving, fitting, pattern) -> Tiler:
    t = Tiler()
    for k, v in enumerate(origin):
        t.origin[k] = int(v)
    for k, row in enumerate(paving):
        for q, v in enumerate(row):
            t.paving[k][q] = int(v)
    for k, row in enumerate(fitting):
        for p, v in enumerate(row):
            t.fitting[k][p] = int(v)
    t.pattern_rank = len(pattern)
    for p, v in enumerate(pattern):
        t.pattern[p] = int(v)
    return t


def task_desc(spec) -> tuple:
    """TaskDesc from a task dict {"rep", "elem", "inputs", "outputs", "taps"}
    (ports {"shape", "dtype", "origin", "paving", "fitting", "pattern"}).
    Returns (desc, keepalive) — keep the second alive until the create call."""
    d = TaskDesc()
    d.rep_rank = len(spec["rep"])
    for q, v in enumerate(spec["rep"]):
        d.rep[q] = int(v)
    d.elem = ELEM[spec["elem"]]
    d.n_in = len(spec["inputs"])
    d.n_out = len(spec["outputs"])
    for i, p in enumerate(spec["inputs"]):
        d.in_[i] = array_desc(p["shape"], p["dtype"])
        d.in_tiler[i] = tiler(p["origin"], p["paving"], p["fitting"], p["pattern"])
    for i, p in enumerate(spec["outputs"]):
        d.out[i] = array_desc(p["shape"], p["dtype"])
        d.out_tiler[i] = tiler(p["origin"], p["paving"], p["fitting"], p["pattern"])
    keep = None
    taps = spec.get("taps")
    if taps is not None:
        keep = np.ascontiguousarray(taps, dtype=np.float32)
        d.fir_m, d.fir_T = keep.shape
        d.fir_taps_host = keep.ctypes.data
    return d, keep


def spec_of_desc(d, taps=None) -> dict:
    """The task dict of a TaskDesc (the inverse of task_desc; taps given
    separately, since a descriptor only points at them)."""
    inv = {v: k for k, v in DTYPE.items()}

    def port_of(a, t):
        r = a.rank
        return {"shape": tuple(int(a.shape[k]) for k in range(r)), "dtype": inv[a.dtype],
                "origin": tuple(int(t.origin[k]) for k in range(r)),
                "paving": tuple(tuple(int(t.paving[k][q]) for q in range(d.rep_rank)) for k in range(r)),
                "fitting": tuple(tuple(int(t.fitting[k][i]) for i in range(t.pattern_rank)) for k in range(r)),
                "pattern": tuple(int(t.pattern[i]) for i in range(t.pattern_rank))}
    return {"rep": tuple(int(d.rep[q]) for q in range(d.rep_rank)),
            "elem": {v: k for k, v in ELEM.items()}[d.elem],
            "inputs": [port_of(d.in_[i], d.in_tiler[i]) for i in range(d.n_in)],
            "outputs": [port_of(d.out[0], d.out_tiler[0])],
            "taps": taps}


def arol_task_shard_frames(spec: dict, parts: int, part: int):
    """(spec of part `part` of `parts`, its first frame): see include/arol.h."""
    d, keep = task_desc(spec)
    out = TaskDesc()
    first = c_i64()
    _check(lib.arol_task_shard_frames(ctypes.byref(d), int(parts), int(part), ctypes.byref(out), ctypes.byref(first)))
    del keep
    return spec_of_desc(out, spec.get("taps")), first.value


# ------------------------------------------------------------ entry points

def arol_task_create(desc) -> int:
    keep = None
    if isinstance(desc, dict):
        desc, keep = task_desc(desc)
    h = c_vp()
    _check(lib.arol_task_create(ctypes.byref(desc), ctypes.byref(h)))
    del keep
    return h.value


def arol_chain_create(tasks) -> int:
    h = c_vp()
    arr = (c_vp * len(tasks))(*tasks)
    _check(lib.arol_chain_create(arr, len(tasks), ctypes.byref(h)))
    return h.value


def arol_task_set_taps(t, taps, on_device: bool):
    if on_device:
        _check(lib.arol_task_set_taps(t, _ptr(taps), 1))
    else:
        a = np.ascontiguousarray(taps, dtype=np.float32)
        _check(lib.arol_task_set_taps(t, a.ctypes.data, 0))


def arol_task_run(t, ins, outs, stream=None):
    _check(lib.arol_task_run(t, _ptrs(ins), _ptrs(outs), _stream(stream)))


def arol_task_run_host(t, ins, outs, stream=None):
    _check(lib.arol_task_run_host(t, _ptrs(ins), _ptrs(outs), _stream(stream)))


def arol_task_backward(t, grad_out, saved_in, grad_in=None, grad_taps=None, stream=None):
    _check(lib.arol_task_backward(t, _ptr(grad_out), _ptrs(saved_in), _ptr(grad_in), _ptr(grad_taps),
                                  _stream(stream)))


def arol_task_fwd_bwd(t, ins, grad_out, out, grad_in=None, grad_taps=None, stream=None):
    _check(lib.arol_task_fwd_bwd(t, _ptrs(ins), _ptr(grad_out), _ptr(out), _ptr(grad_in), _ptr(grad_taps),
                                 _stream(stream)))


def arol_task_info(t) -> dict:
    info = TaskInfo()
    _check(lib.arol_task_info(t, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in TaskInfo._fields_ if not f.endswith("_")}


def arol_task_sync_status(t, stream=None):
    _check(lib.arol_task_sync_status(t, _stream(stream)))


def arol_task_destroy(t):
    if t:
        lib.arol_task_destroy(t)


def arol_tiler_cover(shape, port, rep) -> tuple:
    a = array_desc(shape)
    tl = tiler(port["origin"], port["paving"], port["fitting"], port["pattern"])
    r = (c_i64 * 4)(*(list(rep) + [0] * (4 - len(rep))))
    lo, hi = c_i64(), c_i64()
    _check(lib.arol_tiler_cover(ctypes.byref(a), ctypes.byref(tl), len(rep), r, ctypes.byref(lo), ctypes.byref(hi)))
    return lo.value, hi.value


def arol_selftest_wait_timeout(stream=None):
    _check(lib.arol_selftest_wait_timeout(_stream(stream)))


def arol_batch_create(tasks) -> int:
    h = c_vp()
    arr = (c_vp * len(tasks))(*tasks)
    _check(lib.arol_batch_create(arr, len(tasks), ctypes.byref(h)))
    return h.value


def arol_batch_run(b, ins, outs, stream=None):
    _check(lib.arol_batch_run(b, _ptrs(ins), _ptrs(outs), _stream(stream)))


def arol_batch_run_per_task(b, ins, outs, stream=None):
    _check(lib.arol_batch_run_per_task(b, _ptrs(ins), _ptrs(outs), _stream(stream)))


def arol_batch_tune(b, ins, outs, stream=None, force=False):
    _check(lib.arol_batch_tune(b, _ptrs(ins), _ptrs(outs), _stream(stream), 1 if force else 0))


def arol_batch_config(b) -> dict:
    tile, ctas, thr = c_i64(), c_i32(), c_i32()
    _check(lib.arol_batch_config(b, ctypes.byref(tile), ctypes.byref(ctas), ctypes.byref(thr)))
    return {"tile_reps": tile.value, "ctas_per_sm": ctas.value, "threads": thr.value}


def arol_batch_sync_status(b, stream=None):
    _check(lib.arol_batch_sync_status(b, _stream(stream)))


def arol_batch_destroy(b):
    if b:
        lib.arol_batch_destroy(b)


def arol_downscale_backward_noalloc(x, grad_out, taps, frames, height, width, grad_in=None, grad_taps=None,
                                    stream=None):
    """Backward of the fused downscaler chain with no device allocation (see
    include/arol.h); raises ArolError with the status code on failure."""
    st = lib.arol_downscale_backward_noalloc(_ptr(x), _ptr(grad_out), _ptr(taps), int(frames), int(height),
                                             int(width), _ptr(grad_in), _ptr(grad_taps), _stream(stream))
    if st != 0:
        raise ArolError(st, "arol_downscale_backward_noalloc rejected the call")


def arol_downscale_backward_noalloc_status(stream=None):
    """Synchronizes the stream; raises ArolError (AROL_ERR_TIMEOUT) if a bounded
    wait of the no-allocation backward gave up since the last query."""
    st = lib.arol_downscale_backward_noalloc_status(_stream(stream))
    if st != 0:
        raise ArolError(st, "arol_downscale_backward_noalloc: a device-side wait gave up")


def _check_cg(st):
    if st != 0:
        buf = ctypes.create_string_buffer(1024)
        lib.arol_cg_last_error(buf, len(buf))
        raise ArolError(st, buf.value.decode(errors="replace"))


def arol_csr_spmv(n_rows, nnz, row_ptr, col_idx, vals, x, y, stream=None):
    _check_cg(lib.arol_csr_spmv(int(n_rows), int(nnz), _ptr(row_ptr), _ptr(col_idx), _ptr(vals), _ptr(x), _ptr(y),
                                _stream(stream)))


def arol_csr_check(n_rows, nnz, row_ptr, col_idx, stream=None):
    _check_cg(lib.arol_csr_check(int(n_rows), int(nnz), _ptr(row_ptr), _ptr(col_idx), _stream(stream)))


def arol_cg_create(n_rows, nnz, row_ptr, col_idx, vals) -> int:
    h = c_vp()
    _check_cg(lib.arol_cg_create(int(n_rows), int(nnz), _ptr(row_ptr), _ptr(col_idx), _ptr(vals), ctypes.byref(h)))
    return h.value


def arol_cg_solve(h, b, x, tol, max_iter, stream=None):
    it, rel = ctypes.c_int(), ctypes.c_double()
    _check_cg(lib.arol_cg_solve(h, _ptr(b), _ptr(x), float(tol), int(max_iter), ctypes.byref(it), ctypes.byref(rel),
                                _stream(stream)))
    return it.value, rel.value


def arol_cg_destroy(h):
    if h:
        lib.arol_cg_destroy(h)
