"""ctypes wrapper of ``oracle/cpu_ref.c`` — TEST INFRASTRUCTURE ONLY.

The C file is the task definition written out in plain C (OpenMP over the
repetition space, float64 accumulation).  It is used for parity at sizes the
Python loops cannot reach and as the timed CPU baseline.  ``build()`` compiles
it with gcc; it never touches the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpu_ref.c")
_LIB = os.path.join(_HERE, "_cpu_ref.so")
_DT = {"f32": 0, "bf16": 1, "f64": 2, "f16": 1}   # f16 ports: 16-bit words moved by a copy, never decoded in C
_ELEM = {"copy": 0, "fir": 1, "matmul": 2}


class OrefPort(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("shape", ctypes.c_int64 * 4), ("origin", ctypes.c_int64 * 4),
                ("paving", (ctypes.c_int64 * 4) * 4), ("fitting", (ctypes.c_int64 * 2) * 4),
                ("pattern_rank", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("pattern", ctypes.c_int64 * 2)]


def build(force: bool = False) -> str:
    """Compile cpu_ref.c into oracle/_cpu_ref.so (gcc, OpenMP, -O2)."""
    stamp = _LIB + ".arch"
    if not os.path.exists(stamp) or open(stamp).read().strip() != platform.machine():
        force = True   # a library of another host architecture
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
        with open(stamp, "w") as f:
            f.write(platform.machine() + "\n")
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        L.oref_run_task.argtypes = [ctypes.c_int, P(ctypes.c_int64), ctypes.c_int, ctypes.c_int,
                                    P(OrefPort), P(ctypes.c_void_p), P(OrefPort), ctypes.c_void_p,
                                    P(ctypes.c_double), ctypes.c_int, ctypes.c_int]
        L.oref_cover_check.argtypes = [ctypes.c_int, P(ctypes.c_int64), P(OrefPort)]
        L.oref_fir_vjp.argtypes = [ctypes.c_int, P(ctypes.c_int64), P(OrefPort), ctypes.c_void_p,
                                   P(OrefPort), P(ctypes.c_double), P(ctypes.c_double),
                                   ctypes.c_int, ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double)]
        L.oref_matmul_sample.argtypes = [P(OrefPort), ctypes.c_void_p, P(OrefPort), ctypes.c_void_p,
                                         P(OrefPort), ctypes.c_int64, P(ctypes.c_int64),
                                         P(ctypes.c_int64), P(ctypes.c_double), P(ctypes.c_double)]
        L.oref_threads.restype = ctypes.c_int
        L.oref_set_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def threads() -> int:
    return lib().oref_threads()


def set_threads(n: int) -> None:
    lib().oref_set_threads(int(n))


def _port(p, dtype=None):
    s = OrefPort()
    s.rank = len(p["shape"])
    s.dtype = _DT[dtype or p["dtype"]]
    for k in range(s.rank):
        s.shape[k] = p["shape"][k]
        s.origin[k] = p["origin"][k]
        for q, v in enumerate(p["paving"][k]):
            s.paving[k][q] = v
        for q, v in enumerate(p["fitting"][k]):
            s.fitting[k][q] = v
    s.pattern_rank = len(p["pattern"])
    for q, v in enumerate(p["pattern"]):
        s.pattern[q] = v
    return s


def _rep(R):
    return (ctypes.c_int64 * 4)(*(list(R) + [0] * (4 - len(R))))


def _dtype_of(x, declared):
    if x.dtype == np.float64:
        return "f64"
    if x.dtype == np.uint16:
        return "bf16"
    if x.dtype == np.float32:
        return "f32"
    return declared


def _half_input(x, p, elem):
    """IEEE half inputs (float16 arrays, or uint16 words on an f16 port): a
    copy moves their 16-bit words; arithmetic reads their values, which
    float64 holds exactly, so the C code never decodes binary16 itself."""
    if x.dtype == np.float16 or (x.dtype == np.uint16 and p["dtype"] == "f16"):
        return x.view(np.uint16) if elem == "copy" else x.view(np.float16).astype(np.float64)
    return x


def run_task(tk, inputs):
    """One task.  Returns [Y]: float64 for fir/matmul, raw bits for copy."""
    L = lib()
    ins = [_half_input(np.ascontiguousarray(x), p, tk["elem"]) for x, p in zip(inputs, tk["inputs"])]
    ports = (OrefPort * 2)(*[_port(p, _dtype_of(x, p["dtype"])) for p, x in zip(tk["inputs"], ins)])
    ptrs = (ctypes.c_void_p * 2)(*[x.ctypes.data for x in ins])
    op = tk["outputs"][0]
    if tk["elem"] == "copy":
        Y = np.zeros(op["shape"], dtype=ins[0].dtype)
    else:
        Y = np.zeros(op["shape"], dtype=np.float64)
    taps = tk["taps"]
    if taps is not None:
        H = np.ascontiguousarray(taps, dtype=np.float64)
        m, T = H.shape
        hp = H.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    else:
        m = T = 0
        hp = None
    rc = L.oref_run_task(len(tk["rep"]), _rep(tk["rep"]), _ELEM[tk["elem"]], len(ins),
                         ports, ptrs, ctypes.byref(_port(op)), Y.ctypes.data, hp, m, T)
    if rc == 1:
        raise ValueError("output tiler does not partition its array")
    if rc:
        raise RuntimeError(f"oref_run_task failed ({rc})")
    return [Y]


def run_chain(tasks, inputs):
    cur = inputs
    for tk in tasks:
        cur = run_task(tk, cur)
    return cur


def cover_ok(tk) -> bool:
    return lib().oref_cover_check(len(tk["rep"]), _rep(tk["rep"]), ctypes.byref(_port(tk["outputs"][0]))) == 0


def fir_vjp(tk, x, g):
    """(dX float64, dH float64) of sum(g * Y) for one fir task."""
    L = lib()
    x = np.ascontiguousarray(x)
    g = np.ascontiguousarray(g, dtype=np.float64)
    H = np.ascontiguousarray(tk["taps"], dtype=np.float64)
    m, T = H.shape
    ip = _port(tk["inputs"][0], _dtype_of(x, tk["inputs"][0]["dtype"]))
    dX = np.zeros(tk["inputs"][0]["shape"], dtype=np.float64)
    dH = np.zeros((m, T), dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    rc = L.oref_fir_vjp(len(tk["rep"]), _rep(tk["rep"]), ctypes.byref(ip), x.ctypes.data,
                        ctypes.byref(_port(tk["outputs"][0])), g.ctypes.data_as(dp),
                        H.ctypes.data_as(dp), m, T, dX.ctypes.data_as(dp), dH.ctypes.data_as(dp))
    if rc:
        raise RuntimeError(f"oref_fir_vjp failed ({rc})")
    return dX, dH


def chain_vjp(tasks, inputs, g):
    acts = [inputs]
    for tk in tasks[:-1]:
        acts.append(run_task(tk, acts[-1]))
    dHs = [None] * len(tasks)
    for n in range(len(tasks) - 1, -1, -1):
        g, dHs[n] = fir_vjp(tasks[n], acts[n][0], g)
    return g, dHs


def matmul_sample(tk, a_bits, b_bits, rows, cols):
    """(values, sum of |a||b| terms) of C at the sampled (row, col) pairs."""
    L = lib()
    pa, pb, pc = (_port(p) for p in (tk["inputs"][0], tk["inputs"][1], tk["outputs"][0]))
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int64)
    vals = np.zeros(len(rows), dtype=np.float64)
    absv = np.zeros(len(rows), dtype=np.float64)
    ip = ctypes.POINTER(ctypes.c_int64)
    dp = ctypes.POINTER(ctypes.c_double)
    a_bits = np.ascontiguousarray(a_bits)
    b_bits = np.ascontiguousarray(b_bits)
    L.oref_matmul_sample(ctypes.byref(pa), a_bits.ctypes.data, ctypes.byref(pb), b_bits.ctypes.data,
                         ctypes.byref(pc), len(rows), rows.ctypes.data_as(ip), cols.ctypes.data_as(ip),
                         vals.ctypes.data_as(dp), absv.ctypes.data_as(dp))
    return vals, absv
