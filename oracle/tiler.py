"""The Array-OL repetitive task, written out as its definition (float64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): nothing in the product
path imports this module.

Definition followed (MARTE Repetitive Structure Modeling, named in Sec. 3;
repetitive tasks on the GPU, Sec. 7; ports with shape, type and direction,
Sec. 5 and Sec. 6.3).  An array port has shape ``s`` (rank d, row-major).  A
tiler has origin ``o`` (d), paving ``P`` (d x q), fitting ``F`` (d x p) and a
pattern shape ``S`` (p).  For every repetition index ``r`` in the repetition
space ``R`` (q) and every pattern index ``i`` in ``S``, the tiler names the
array element

    e(r, i) = (o + P r + F i) mod s          (componentwise, Euclidean mod)

An input tiler *gathers* the pattern ``p_r[i] = X[e(r, i)]``; the elementary
task maps the input patterns to the output pattern ``y_r``; the output tiler
*scatters* ``Y[e_out(r, j)] = y_r[j]``.  An output tiler must write every
element of its array exactly once (single assignment); anything else is an
error here, as it is in the library.

Elementary tasks (patterns flattened row-major when their rank is 2):

* copy:    y[j] = p[j]          (raw bits: no arithmetic, NaN payloads kept)
* fir:     y[j] = sum_k H[j, k] p[k]        for j < m, k < T  (a bank of m
           tap rows; H is m x T)
* matmul:  y = p_A . p_B        (pattern shapes (a, K) and (K, b))

Readings of points the paper leaves open: ``mod`` is Euclidean (result in
[0, s) also for negative sums); the FIR is a bank of m tap rows over one
T-element pattern; a frame dimension is one more array dimension and one more
repetition dimension (paving 1, fitting 0); an output tiler that is not a
partition of its array is rejected, never accumulated.
"""
from __future__ import annotations

import itertools

import numpy as np


class NotAPartition(ValueError):
    """An output tiler that does not write each array element exactly once."""


# --------------------------------------------------------------------------
# Address generation: e(r, i) = (o + P r + F i) mod s
# --------------------------------------------------------------------------

def emod(a: int, s: int) -> int:
    """Euclidean remainder: the unique value in [0, s) congruent to a mod s."""
    assert s > 0
    q = a // s           # floor division
    rem = a - q * s
    assert 0 <= rem < s
    return rem


def tiler_element(t: dict, r, i):
    """The array index (tuple) that tiler ``t`` names for repetition ``r`` and
    pattern index ``i``: (o + P r + F i) mod s, one array dimension at a time."""
    s, o, P, F = t["shape"], t["origin"], t["paving"], t["fitting"]
    idx = []
    for k in range(len(s)):
        v = o[k]
        for qd in range(len(r)):
            v += P[k][qd] * r[qd]
        for pd in range(len(i)):
            v += F[k][pd] * i[pd]
        idx.append(emod(v, s[k]))
    return tuple(idx)


def pattern_indices(t: dict):
    """All pattern indices i of tiler ``t`` in row-major order."""
    return list(itertools.product(*[range(n) for n in t["pattern"]]))


def repetition_indices(R):
    return list(itertools.product(*[range(n) for n in R]))


# --------------------------------------------------------------------------
# Elementary tasks
# --------------------------------------------------------------------------

def elem_fir(p, H):
    """y[j] = sum_k H[j, k] * p[k], accumulated in float64."""
    m, T = H.shape
    assert len(p) == T
    y = []
    for j in range(m):
        acc = 0.0
        for k in range(T):
            acc += float(H[j, k]) * float(p[k])
        y.append(acc)
    return y


def elem_matmul(pa, pb, a_shape, b_shape):
    """y = A . B for patterns A (a x K) and B (K x b), float64, flattened."""
    a, K = a_shape
    K2, b = b_shape
    assert K == K2
    A = np.asarray(pa, dtype=np.float64).reshape(a, K)
    B = np.asarray(pb, dtype=np.float64).reshape(K, b)
    return list(np.matmul(A, B).reshape(-1))


# --------------------------------------------------------------------------
# One task: gather -> elementary task -> scatter
# --------------------------------------------------------------------------

def _as_values(x, dtype):
    """Element values the task reads (Sec. 5 typeAllocation).  bf16 arrays
    are given as uint16 bit patterns: a bfloat16 is the upper half of a
    binary32, so shifting the bits up 16 places gives its value exactly.  f16
    arrays are IEEE binary16 (numpy float16, or its uint16 bit patterns);
    every binary16 value is exact in float64."""
    if dtype == "bf16":
        return (np.asarray(x, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    if dtype == "f16":
        x = np.asarray(x)
        return (x.view(np.float16) if x.dtype == np.uint16 else x.astype(np.float16)).astype(np.float64)
    return np.asarray(x, dtype=np.float64)


def _raw(x):
    x = np.ascontiguousarray(x)
    return x.view({2: np.uint16, 4: np.uint32, 8: np.uint64}[x.dtype.itemsize])


def run_task(tk: dict, inputs):
    """Run one task by its definition.

    ``inputs`` are numpy arrays (float32/float64, or uint16 bf16 bit patterns).
    Returns ``[Y]``: float64 for fir/matmul; for copy, the input's raw bit
    patterns (same itemsize), so the copy is bit-exact by construction.
    Raises ``NotAPartition`` unless every output element is written once.
    """
    R = tk["rep"]
    ins, outs = tk["inputs"], tk["outputs"]
    assert len(outs) == 1
    out = outs[0]
    elem = tk["elem"]
    if elem == "copy":
        assert len(ins) == 1
        X = _raw(inputs[0])
        Y = np.zeros(out["shape"], dtype=X.dtype)
    else:
        Xs = [_as_values(x, p["dtype"]) for x, p in zip(inputs, ins)]
        Y = np.zeros(out["shape"], dtype=np.float64)
    count = np.zeros(out["shape"], dtype=np.int64)
    in_pat = [pattern_indices(p) for p in ins]
    out_pat = pattern_indices(out)
    for r in repetition_indices(R):
        if elem == "copy":
            pat = [X[tiler_element(ins[0], r, i)] for i in in_pat[0]]
            y = pat
        elif elem == "fir":
            pat = [Xs[0][tiler_element(ins[0], r, i)] for i in in_pat[0]]
            y = elem_fir(pat, tk["taps"])
        elif elem == "matmul":
            pa = [Xs[0][tiler_element(ins[0], r, i)] for i in in_pat[0]]
            pb = [Xs[1][tiler_element(ins[1], r, i)] for i in in_pat[1]]
            y = elem_matmul(pa, pb, ins[0]["pattern"], ins[1]["pattern"])
        else:
            raise ValueError(elem)
        assert len(y) == len(out_pat), "output pattern size must match the elementary task"
        for j, jj in enumerate(out_pat):
            e = tiler_element(out, r, jj)
            Y[e] = y[j]
            count[e] += 1
    if not np.all(count == 1):
        raise NotAPartition("output tiler does not write each element exactly once")
    return [Y]


def cover_count(out_port: dict, R):
    """How many (r, j) pairs the output tiler maps onto each array element."""
    count = np.zeros(out_port["shape"], dtype=np.int64)
    for r in repetition_indices(R):
        for j in pattern_indices(out_port):
            count[tiler_element(out_port, r, j)] += 1
    return count


def run_chain(tasks, inputs):
    """Tasks chained through shared arrays (Sec. 5, ``associatedParts``): the
    output array of task k is the input array of task k+1.  The intermediate
    stays float64."""
    cur = inputs
    for tk in tasks:
        cur = run_task(tk, cur)
    return cur


# --------------------------------------------------------------------------
# Adjoint (reverse mode) of one task and of a chain
# --------------------------------------------------------------------------

def task_vjp(tk: dict, inputs, grad_out):
    """Gradients of sum(grad_out * Y) for a copy or fir task.

    The adjoint of a gather that visits an element several times (overlapping
    fittings, modulo wrap) is a scatter-ADD over every (r, i) that maps to it:

        dX[e]     = sum over (r, k) with e_in(r, k) = e of  sum_j H[j, k] dY[e_out(r, j)]
        dH[j, k]  = sum_r dY[e_out(r, j)] * X[e_in(r, k)]

    Returns (dX float64 with the input shape, dH float64 m x T or None).
    """
    R = tk["rep"]
    ip, op = tk["inputs"][0], tk["outputs"][0]
    X = _as_values(inputs[0], ip["dtype"])
    G = np.asarray(grad_out, dtype=np.float64)
    dX = np.zeros(ip["shape"], dtype=np.float64)
    in_pat = pattern_indices(ip)
    out_pat = pattern_indices(op)
    if tk["elem"] == "copy":
        for r in repetition_indices(R):
            for i, j in zip(in_pat, out_pat):
                dX[tiler_element(ip, r, i)] += G[tiler_element(op, r, j)]
        return dX, None
    assert tk["elem"] == "fir"
    H = np.asarray(tk["taps"], dtype=np.float64)
    m, T = H.shape
    dH = np.zeros((m, T), dtype=np.float64)
    for r in repetition_indices(R):
        e_in = [tiler_element(ip, r, i) for i in in_pat]
        g = [G[tiler_element(op, r, j)] for j in out_pat]
        for k in range(T):
            s = 0.0
            for j in range(m):
                s += H[j, k] * g[j]
                dH[j, k] += g[j] * X[e_in[k]]
            dX[e_in[k]] += s
    return dX, dH


def chain_vjp(tasks, inputs, grad_out):
    """Reverse mode through a chain: recompute every intermediate forward in
    float64, then apply ``task_vjp`` from the last task back to the first.
    Returns (dX of the chain input, [dH of each task, in task order])."""
    acts = [inputs]
    for tk in tasks[:-1]:
        acts.append(run_task(tk, acts[-1]))
    g = grad_out
    dHs = [None] * len(tasks)
    for n in range(len(tasks) - 1, -1, -1):
        g, dHs[n] = task_vjp(tasks[n], acts[n], g)
    return g, dHs
