"""Seeded synthetic workloads for Array-OL repetitive tasks.

This module only *describes* tasks and *draws* their inputs.  It holds none of
the method's arithmetic (no tiler address generation, no filtering, no
products): both the CPU oracle (``oracle/``) and the CUDA binding
(``paper_1105_4424_gb300``) consume the plain dictionaries built here, each in
its own code.

A task is a dict::

    {"rep":      (R_0, ..., R_{q-1}),               # repetition space
     "elem":     "copy" | "fir" | "matmul",         # elementary task
     "inputs":   [port, ...],                       # 1 (copy, fir) or 2 (matmul)
     "outputs":  [port],                            # exactly 1
     "taps":     float32 ndarray (m, T) or None}    # FIR tap bank

and a port is ``{"shape", "dtype", "origin", "paving", "fitting", "pattern"}``
with ``paving`` a d x q and ``fitting`` a d x p nested tuple (d = array rank,
p = pattern rank).  Arrays are dense and row-major.

All random draws use ``numpy.random.Generator(PCG64(seed))`` in the fixed
order stated in each builder's docstring.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "rng", "port", "task", "fir_row_task", "downscale_chain",
    "config0", "config1", "config1_bf16", "config1_f16", "config1_5to2", "config2", "config3", "config4",
    "config0_scaled", "diagonal_fir", "separable_pass", "random_separable_chain",
    "bf16_round", "bf16_bits_to_f32", "f16_round", "random_tiler_task", "stencil27_csr",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def port(shape, origin, paving, fitting, pattern, dtype="f32"):
    d = len(shape)
    paving = tuple(tuple(int(v) for v in row) for row in paving)
    fitting = tuple(tuple(int(v) for v in row) for row in fitting)
    assert len(origin) == d and len(paving) == d and len(fitting) == d
    return {"shape": tuple(int(v) for v in shape), "dtype": dtype,
            "origin": tuple(int(v) for v in origin), "paving": paving,
            "fitting": fitting, "pattern": tuple(int(v) for v in pattern)}


def task(rep, elem, inputs, outputs, taps=None):
    return {"rep": tuple(int(v) for v in rep), "elem": elem,
            "inputs": list(inputs), "outputs": list(outputs),
            "taps": None if taps is None else np.ascontiguousarray(taps, dtype=np.float32)}


def fir_row_task(height, width, T, m, step, taps):
    """Row FIR downscaler on an (height, width) array.

    Input tiler: origin 0, paving [[1,0],[0,step]], fitting [[0],[1]],
    pattern (T,), repetition space (height, ceil(width/step)); the last
    pattern of a row wraps around the right edge (modulo the array shape).
    Output tiler: (height, m*ceil(width/step)), paving [[1,0],[0,m]],
    fitting [[0],[1]], pattern (m,), which partitions the output array.
    """
    reps = -(-width // step)
    inp = port((height, width), (0, 0), ((1, 0), (0, step)), ((0,), (1,)), (T,))
    out = port((height, m * reps), (0, 0), ((1, 0), (0, m)), ((0,), (1,)), (m,))
    return task((height, reps), "fir", [inp], [out], taps)


def downscale_chain(frames, height, width, taps_h, taps_v, step_h=8, step_v=8, dtypes=("f32", "f32", "f32")):
    """Horizontal then vertical FIR downscaler on rank-3 (frames, height, width).

    The frame dimension enters every tiler as an extra array dimension and an
    extra repetition dimension with paving 1 and fitting 0.  The horizontal
    pass tiles along the last dimension, the vertical pass is the same form
    transposed onto the middle dimension.  The horizontal output array is the
    vertical input array (one shared allocation between the two tasks).
    """
    mh, th = taps_h.shape
    mv, tv = taps_v.shape
    assert width % step_h == 0 and height % step_v == 0
    wr = width // step_h
    mid_w = wr * mh
    hr = height // step_v
    out_h = hr * mv
    d_in, d_mid, d_out = dtypes
    t_h = task(
        (frames, height, wr), "fir",
        [port((frames, height, width), (0, 0, 0),
              ((1, 0, 0), (0, 1, 0), (0, 0, step_h)), ((0,), (0,), (1,)), (th,), d_in)],
        [port((frames, height, mid_w), (0, 0, 0),
              ((1, 0, 0), (0, 1, 0), (0, 0, mh)), ((0,), (0,), (1,)), (mh,), d_mid)],
        taps_h)
    t_v = task(
        (frames, hr, mid_w), "fir",
        [port((frames, height, mid_w), (0, 0, 0),
              ((1, 0, 0), (0, step_v, 0), (0, 0, 1)), ((0,), (1,), (0,)), (tv,), d_mid)],
        [port((frames, out_h, mid_w), (0, 0, 0),
              ((1, 0, 0), (0, mv, 0), (0, 0, 1)), ((0,), (1,), (0,)), (mv,), d_out)],
        taps_v)
    return [t_h, t_v]


def config1_bf16(seed=0, frames=64, height=1080, width=1920, mid="f32", out="bf16"):
    """The chained downscaler with bfloat16 frames: X drawn as in config1
    (U[0,1) float32), then rounded to bfloat16 (RNE); returns bit patterns."""
    g = rng(seed)
    x = bf16_round(g.random((frames, height, width), dtype=np.float32))
    Hh = _taps(g, 3, 8)
    Hv = _taps(g, 3, 8)
    return downscale_chain(frames, height, width, Hh, Hv, dtypes=("bf16", mid, out)), [x]


def config1_f16(seed=0, frames=64, height=1080, width=1920, mid="f32", out="f16"):
    """The chained downscaler with IEEE half frames: X drawn as in config1
    (U[0,1) float32), then rounded to float16 (RNE); returns float16 arrays."""
    g = rng(seed)
    x = f16_round(g.random((frames, height, width), dtype=np.float32))
    Hh = _taps(g, 3, 8)
    Hv = _taps(g, 3, 8)
    return downscale_chain(frames, height, width, Hh, Hv, dtypes=("f16", mid, out)), [x]


def _taps(g, m, T):
    return (g.standard_normal((m, T), dtype=np.float64) / T).astype(np.float32)


def config0(seed=0):
    """64x64 float32 U[0,1) -> 8-tap/3-output FIR, step 4, wrap -> 64x48.

    Draw order: X (64x64), then taps H (3x8) ~ N(0,1)/8, j-major.
    """
    g = rng(seed)
    x = g.random((64, 64), dtype=np.float32)
    H = _taps(g, 3, 8)
    inp = port((64, 64), (0, 0), ((1, 0), (0, 4)), ((0,), (1,)), (8,))
    out = port((64, 48), (0, 0), ((1, 0), (0, 3)), ((0,), (1,)), (3,))
    return task((64, 16), "fir", [inp], [out], H), [x]


def config1(seed=0, frames=64, height=1080, width=1920):
    """Two chained 8->3 FIR downscalers on frames x height x width float32.

    Draw order: X (frames, height, width) U[0,1), taps_h (3x8), taps_v (3x8).
    """
    g = rng(seed)
    x = g.random((frames, height, width), dtype=np.float32)
    Hh = _taps(g, 3, 8)
    Hv = _taps(g, 3, 8)
    return downscale_chain(frames, height, width, Hh, Hv), [x]


def bf16_round(x: np.ndarray) -> np.ndarray:
    """float32 -> bfloat16 bit patterns (uint16), round to nearest even."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    nan = np.isnan(x)
    bias = ((u >> 16) & 1) + 0x7FFF
    b = ((u + bias) >> 16).astype(np.uint16)
    b[nan] = 0x7FC0
    return b


def f16_round(x: np.ndarray) -> np.ndarray:
    """float32 -> IEEE half (numpy float16), round to nearest even; values
    from 65520 (halfway between the largest half, 65504, and 2^16) up round
    to infinity."""
    return np.ascontiguousarray(x, dtype=np.float32).astype(np.float16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.ascontiguousarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def matmul_task(M, N, K, tile_m=128, tile_n=128):
    """C (M,N) f32 = A (M,K) bf16 . B (K,N) bf16 as a repetitive task.

    Repetition space (M/tile_m, N/tile_n); A's tiler fetches the tile_m x K row
    panel (paving [[tile_m,0],[0,0]], fitting identity), B's tiler the
    K x tile_n column panel (paving [[0,0],[0,tile_n]]), C's tiler the
    tile_m x tile_n tile (paving diag(tile_m, tile_n)), a partition of C.
    """
    assert M % tile_m == 0 and N % tile_n == 0
    eye = ((1, 0), (0, 1))
    a = port((M, K), (0, 0), ((tile_m, 0), (0, 0)), eye, (tile_m, K), "bf16")
    b = port((K, N), (0, 0), ((0, 0), (0, tile_n)), eye, (K, tile_n), "bf16")
    c = port((M, N), (0, 0), ((tile_m, 0), (0, tile_n)), eye, (tile_m, tile_n), "f32")
    return task((M // tile_m, N // tile_n), "matmul", [a, b], [c])


def config2(seed=0, M=4096, N=4096, K=4096):
    """Matmul task; A then B drawn N(0,1) as float32, rounded to bf16 (RNE).

    Returns (task, [A_bits, B_bits]) with uint16 bfloat16 bit patterns.
    """
    g = rng(seed)
    a = bf16_round(g.standard_normal((M, K), dtype=np.float32))
    b = bf16_round(g.standard_normal((K, N), dtype=np.float32))
    return matmul_task(M, N, K), [a, b]


def config3_params(seed=0, n=512, lo=32, hi=2048):
    """Per-instance parameters of the uneven batch, drawn in this order for
    each instance: height, width ~ round(exp(U(ln lo, ln hi))); T ~ U{3..32};
    m ~ U{1..floor(T/2)}; step ~ U{m..T}."""
    g = rng(seed)
    params = []
    for _ in range(n):
        h = int(round(math.exp(g.uniform(math.log(lo), math.log(hi)))))
        w = int(round(math.exp(g.uniform(math.log(lo), math.log(hi)))))
        T = int(g.integers(3, 33))
        m = int(g.integers(1, T // 2 + 1))
        step = int(g.integers(m, T + 1))
        params.append((h, w, T, m, step))
    return params, g


def config3(seed=0, n=512, lo=32, hi=2048):
    """512 independent row-FIR instances of uneven size (see config3_params).

    After all parameters, for each instance in order: taps (m x T) ~ N(0,1)/T,
    then X (height x width) U[0,1).
    """
    params, g = config3_params(seed, n, lo, hi)
    tasks, xs = [], []
    for (h, w, T, m, step) in params:
        H = _taps(g, m, T)
        x = g.random((h, w), dtype=np.float32)
        tasks.append(fir_row_task(h, w, T, m, step, H))
        xs.append(x)
    return tasks, xs


def config4(seed=0, frames=16, height=1080, width=1920):
    """Forward + backward of the downscaler chain; loss = sum(W * out).

    Draw order: X, taps_h, taps_v, then W ~ N(0,1) with the output shape.
    """
    g = rng(seed)
    x = g.random((frames, height, width), dtype=np.float32)
    Hh = _taps(g, 3, 8)
    Hv = _taps(g, 3, 8)
    chain = downscale_chain(frames, height, width, Hh, Hv)
    out_shape = chain[1]["outputs"][0]["shape"]
    w = g.standard_normal(out_shape, dtype=np.float32)
    return chain, [x], w


def random_tiler_task(g: np.random.Generator, elem="copy", max_side=12,
                      max_rank=3, max_abs=6, fir_pattern_rank=1, max_rep=5):
    """A random small task: random input tiler (negative origin, paving and
    fitting entries allowed, overlaps and wrap-around allowed) and an output
    tiler that partitions its array by construction.  Repetition extents are
    drawn in 1..max_rep.

    The output array's dimensions are a random permutation of the repetition
    dimensions and the output pattern dimensions; with probability 1/2 the
    last repetition dimension is merged with the (rank-1) output pattern into
    one array dimension of size R*m (paving m, fitting 1), as in a downscaler.
    """
    q = int(g.integers(1, 3))
    R = tuple(int(v) for v in g.integers(1, max_rep + 1, size=q))
    d = int(g.integers(1, max_rank + 1))
    shape = tuple(int(v) for v in g.integers(1, max_side + 1, size=d))
    p = fir_pattern_rank if elem == "fir" else int(g.integers(1, 3))
    S = tuple(int(v) for v in g.integers(1, 5, size=p))
    origin = tuple(int(v) for v in g.integers(-3 * max_abs, 3 * max_abs + 1, size=d))
    paving = tuple(tuple(int(v) for v in g.integers(-max_abs, max_abs + 1, size=q)) for _ in range(d))
    fitting = tuple(tuple(int(v) for v in g.integers(-max_abs, max_abs + 1, size=p)) for _ in range(d))
    inp = port(shape, origin, paving, fitting, S)
    T = int(np.prod(S))
    if elem == "fir":
        m = int(g.integers(1, T + 1))
        if fir_pattern_rank == 2 and m > 1 and m % 2 == 0:
            S_out = (2, m // 2)          # a 2-D output pattern (m flattened row-major)
        else:
            S_out = (m,)
        taps = _taps(g, m, T)
    else:
        S_out = S
        taps = None
    p_out = len(S_out)
    merge = (p_out == 1) and bool(g.integers(0, 2))
    if merge:
        dims = [("r", k) for k in range(q - 1)] + [("m", 0)]
    else:
        dims = [("r", k) for k in range(q)] + [("s", k) for k in range(p_out)]
    perm = g.permutation(len(dims))
    dims = [dims[i] for i in perm]
    oshape, opav, ofit = [], [], []
    for kind, k in dims:
        prow, frow = [0] * q, [0] * p_out
        if kind == "r":
            oshape.append(R[k]); prow[k] = 1
        elif kind == "s":
            oshape.append(S_out[k]); frow[k] = 1
        else:
            oshape.append(R[q - 1] * S_out[0]); prow[q - 1] = S_out[0]; frow[0] = 1
        opav.append(tuple(prow)); ofit.append(tuple(frow))
    oorigin = tuple(int(v) for v in g.integers(-max_abs, max_abs + 1, size=len(oshape)))
    out = port(tuple(oshape), oorigin, tuple(opav), tuple(ofit), S_out)
    return task(R, elem, [inp], [out], taps)


def stencil27_csr(side=51, seed=0, shift=0.012):
    """A symmetric positive definite CSR matrix with the sparsity of a 27-point
    stencil on a side^3 grid (side = 51 gives N = 132651 rows and
    NNZ = 151^3 = 3442951 nonzeros) and a right-hand side.

    Off-diagonal weights w_ij = w_ji ~ U(0.5, 1.5) are drawn once per
    neighbour pair (i < j), in row-major order of i, then neighbour offset
    order; a_ij = -w_ij and a_ii = (1 + shift) * sum_j w_ij (strictly
    diagonally dominant, hence SPD).  Then b ~ N(0, 1).
    Returns (row_ptr int64, col_idx int32, vals float64, b float64).
    """
    g = rng(seed)
    n = side ** 3
    idx = np.arange(n, dtype=np.int64)
    iz, iy, ix = idx // (side * side), (idx // side) % side, idx % side
    offs = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    upper = [o for o in offs if (o[0], o[1], o[2]) > (0, 0, 0)]     # j > i in row-major order
    rows, cols, ws = [], [], []
    for (dz, dy, dx) in upper:
        ok = (iz + dz >= 0) & (iz + dz < side) & (iy + dy >= 0) & (iy + dy < side) & (ix + dx >= 0) & (ix + dx < side)
        i = idx[ok]
        j = i + dz * side * side + dy * side + dx
        rows.append(i)
        cols.append(j)
        ws.append(g.uniform(0.5, 1.5, size=i.size))
    i = np.concatenate(rows)
    j = np.concatenate(cols)
    w = np.concatenate(ws)
    diag = np.zeros(n)
    np.add.at(diag, i, w)
    np.add.at(diag, j, w)
    r = np.concatenate([i, j, idx])
    c = np.concatenate([j, i, idx])
    v = np.concatenate([-w, -w, (1.0 + shift) * diag])
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, r + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    b = g.standard_normal(n)
    return row_ptr, c.astype(np.int32), v, b


def ragged_csr(n=3000, seed=0, max_row=70):
    """A general (unsymmetric) CSR matrix with ragged rows for SpMV edge cases:
    row lengths uniform in [0, max_row] with every tenth row empty and every
    seventh row a single entry; columns distinct, sorted, uniform in [0, n);
    values ~ N(0, 1).  Returns (row_ptr int64, col_idx int32, vals float64).
    """
    g = rng(seed)
    lens = g.integers(0, max_row + 1, size=n)
    lens[::10] = 0
    lens[3::7] = 1
    lens = np.minimum(lens, n)
    cols = [np.sort(g.choice(n, size=int(k), replace=False)) for k in lens]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(lens)
    col = np.concatenate(cols).astype(np.int32) if n else np.zeros(0, np.int32)
    vals = g.standard_normal(int(row_ptr[-1]))
    return row_ptr, col, vals


def config1_5to2(seed=0, frames=64, height=1080, width=1920):
    """The chained downscaler with 5-tap -> 2-output banks at step 4 on both
    axes (overlapping windows that wrap at the right and bottom edges):
    (frames, height, width) -> (frames, height / 2, width / 2).  Draw order:
    X U[0,1), taps_h (2 x 5) N(0,1)/5, taps_v (2 x 5) N(0,1)/5."""
    g = rng(seed)
    x = g.random((frames, height, width), dtype=np.float32)
    Hh = _taps(g, 2, 5)
    Hv = _taps(g, 2, 5)
    return downscale_chain(frames, height, width, Hh, Hv, step_h=4, step_v=4), [x]


def config0_scaled(seed=0, frames=64, height=1080, width=1920):
    """The 64 x 64 task's tiler (8-tap -> 3-output bank, step 4 along the row,
    windows overlapping two-fold and wrapping at the row end) on frames x
    height x width float32.  Draw order: X U[0,1), taps (3 x 8) N(0,1)/8."""
    g = rng(seed)
    x = g.random((frames, height, width), dtype=np.float32)
    H = _taps(g, 3, 8)
    reps = width // 4
    t = task((frames, height, reps), "fir",
             [port((frames, height, width), (0, 0, 0), ((1, 0, 0), (0, 1, 0), (0, 0, 4)), ((0,), (0,), (1,)), (8,))],
             [port((frames, height, 3 * reps), (0, 0, 0), ((1, 0, 0), (0, 1, 0), (0, 0, 3)), ((0,), (0,), (1,)), (3,))],
             H)
    return t, [x]


def diagonal_fir(seed=0, frames=64, height=1080, width=1920):
    """A tiler that none of the specialised kernels takes: repetition (f, r0,
    r1) reads the 8-element diagonal X[f, r0 + i, 8 r1 + i] (i < 8, rows mod
    height), so every element is read exactly once but a pattern advances
    along both array dimensions; an 8-tap -> 3-output bank writes 3
    consecutive outputs per repetition: (frames, height, width) ->
    (frames, height, 3 width / 8).  Draw order: X U[0,1), taps (3 x 8)."""
    g = rng(seed)
    x = g.random((frames, height, width), dtype=np.float32)
    H = _taps(g, 3, 8)
    reps = width // 8
    t = task((frames, height, reps), "fir",
             [port((frames, height, width), (0, 0, 0), ((1, 0, 0), (0, 1, 0), (0, 0, 8)), ((0,), (1,), (1,)), (8,))],
             [port((frames, height, 3 * reps), (0, 0, 0), ((1, 0, 0), (0, 1, 0), (0, 0, 3)), ((0,), (0,), (1,)), (3,))],
             H)
    return t, [x]


def separable_pass(in_shape, axis, T, m, step, origin, reps, taps):
    """One pass of a separable chain on rank-2 (rows, cols) or rank-3
    (frames, rows, cols) arrays: a fir along the columns of every row (axis
    1) or down the rows of every column (axis 0), input paving `step` and
    origin `origin` along that axis, `reps` repetitions there (windows wrap
    modulo the extent), m outputs per repetition; identity on the other axis
    and on the frames."""
    d = len(in_shape)
    ax = d - 1 if axis == 1 else d - 2
    rep = tuple(reps if k == ax else in_shape[k] for k in range(d))
    out_shape = tuple(m * reps if k == ax else in_shape[k] for k in range(d))
    pin = tuple(tuple((step if k == ax else 1) if q == k else 0 for q in range(d)) for k in range(d))
    pout = tuple(tuple((m if k == ax else 1) if q == k else 0 for q in range(d)) for k in range(d))
    fit = tuple((1,) if k == ax else (0,) for k in range(d))
    org = tuple(origin if k == ax else 0 for k in range(d))
    return task(rep, "fir", [port(in_shape, org, pin, fit, (T,))],
                [port(out_shape, (0,) * d, pout, fit, (m,))], taps)


def random_separable_chain(g: np.random.Generator, max_side=40, frames=None):
    """2 to 4 passes of random axis, taps T in 1..12, outputs m in 1..5,
    step 1..9, origin, and repetitions (ceil(n / step), or up to three times
    the extent: windows that wrap several times), on frames x rows x cols
    (rank 2 when frames is 1).  Draw order: frames, rows, cols, then per pass
    axis, T, m, step, the repetition rule, reps, origin, taps N(0,1)/T.
    Returns (chain, input shape)."""
    F = int(g.integers(1, 4)) if frames is None else frames
    shape = (int(g.integers(1, max_side + 1)), int(g.integers(1, max_side + 1)))
    if F > 1:
        shape = (F,) + shape
    chain, cur = [], shape
    for _ in range(int(g.integers(2, 5))):
        axis = int(g.integers(0, 2))
        n = cur[-1] if axis == 1 else cur[-2]
        T, m, step = int(g.integers(1, 13)), int(g.integers(1, 6)), int(g.integers(1, 10))
        reps = -(-n // step) if g.random() < 0.6 else int(g.integers(1, 3 * n + 3))
        origin = int(g.integers(0, n))
        t = separable_pass(cur, axis, T, m, step, origin, reps, _taps(g, m, T))
        chain.append(t)
        cur = t["outputs"][0]["shape"]
    return chain, shape


def chain_batch(seed=0, n=128):
    """n independent two-task 8->3 downscaler chains on single float32 frames
    of uneven sizes: per chain, in a fixed draw order, height = 8 * U{8..128},
    width = 8 * U{8..256}, X ~ U[0,1), taps_h and taps_v ~ N(0,1)/8 (3 x 8).
    Returns (list of chains, list of inputs)."""
    g = rng(seed)
    chains, xs = [], []
    for _ in range(n):
        h = 8 * int(g.integers(8, 129))
        w = 8 * int(g.integers(8, 257))
        x = g.random((1, h, w), dtype=np.float32)
        chains.append(downscale_chain(1, h, w, _taps(g, 3, 8), _taps(g, 3, 8)))
        xs.append(x)
    return chains, xs


def random_row_column_chain(g: np.random.Generator, max_rows=300, max_cols=1500, frames=None):
    """A row pass then a column pass (the streaming kernel's case) of random
    taps (T_h in 1..24, T_v in 1..32), outputs (m in 1..4), steps (S_h in
    1..8, S_v in 1..24), origins and repetitions (ceil(n /
    step), or up to twice the extent: windows that wrap), on frames x rows x
    cols.  Draw order: frames, rows, cols, then per pass T, m, step, the
    repetition rule, reps, origin, taps N(0,1)/T.  Returns (chain, input
    shape)."""
    F = int(g.integers(1, 4)) if frames is None else frames
    shape = (F, int(g.integers(1, max_rows + 1)), int(g.integers(1, max_cols + 1)))
    chain, cur = [], shape
    for axis, tmax, smax in ((1, 24, 8), (0, 32, 24)):
        n = cur[-1] if axis == 1 else cur[-2]
        T, m = int(g.integers(1, tmax + 1)), int(g.integers(1, 5))
        step = int(g.integers(1, smax + 1))
        reps = -(-n // step) if g.random() < 0.7 else int(g.integers(1, 2 * n + 2))
        origin = int(g.integers(0, n))
        t = separable_pass(cur, axis, T, m, step, origin, reps, _taps(g, m, T))
        chain.append(t)
        cur = t["outputs"][0]["shape"]
    return chain, shape
