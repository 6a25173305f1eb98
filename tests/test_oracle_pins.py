"""Pins of the CPU oracle to things other than itself (no GPU needed).

Every pin here is a hand-worked value, a closed form, a library routine on a
special case, an invariant or brute force.  The mutation tests at the end
plant plausible mistakes in the oracle (on the CPU) and check that some pin
catches each one.
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import tiler as O

HERE = os.path.dirname(os.path.abspath(__file__))


def _ints(s):
    return tuple(int(v) for v in s.split(",")) if s.strip() else ()


def _rows(s):
    return tuple(_ints(r) for r in s.split("|"))


def golden_addresses():
    cases = []
    with open(os.path.join(HERE, "golden", "tiler_addresses.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            shape, origin, pav, fit, r, i, e = [c.strip() for c in line.split(";")]
            t = {"shape": _ints(shape), "origin": _ints(origin), "paving": _rows(pav),
                 "fitting": _rows(fit)}
            cases.append((t, _ints(r), _ints(i), _ints(e)))
    return cases


# ---------------------------------------------------------------- addresses

def check_golden_addresses():
    for t, r, i, e in golden_addresses():
        assert O.tiler_element(t, r, i) == e, (t, r, i, e)


def test_golden_addresses():
    assert len(golden_addresses()) >= 10
    check_golden_addresses()


def test_emod_is_euclidean():
    for a in range(-50, 50):
        for s in (1, 2, 3, 7, 64):
            v = O.emod(a, s)
            assert 0 <= v < s and (a - v) % s == 0 and int(np.mod(a, s)) == v


# ---------------------------------------------- gather/scatter special cases

def check_row_tiler_vs_take(seed=1):
    """Row tiler (paving [[1,0],[0,S]], fitting [[0],[1]], origin (a,b)) with a
    copy task: pattern r is numpy.take of row (a+r0) mod H over columns
    b+S*r1 .. b+S*r1+T-1 in 'wrap' mode."""
    g = W.rng(seed)
    for (H, Wd, T, S, a, b) in [(5, 16, 8, 4, 0, 0), (3, 10, 4, 3, -2, 7), (4, 9, 5, 2, 1, -4)]:
        x = g.random((H, Wd), dtype=np.float32)
        reps = (H, -(-Wd // S))
        inp = W.port((H, Wd), (a, b), ((1, 0), (0, S)), ((0,), (1,)), (T,))
        out = W.port((H, reps[1] * T), (0, 0), ((1, 0), (0, T)), ((0,), (1,)), (T,))
        y = O.run_task(W.task(reps, "copy", [inp], [out]), [x])[0].view(np.float32)
        for r0 in range(reps[0]):
            for r1 in range(reps[1]):
                ref = np.take(x[(a + r0) % H], np.arange(b + S * r1, b + S * r1 + T), mode="wrap")
                np.testing.assert_array_equal(y[r0, r1 * T:(r1 + 1) * T], ref)


def test_row_tiler_vs_numpy_take():
    check_row_tiler_vs_take()


def check_shift_is_roll(seed=2):
    """Repetition space = the array shape, paving I, pattern (1,), fitting 0,
    origin (a, b): the copy task is numpy.roll by (-a, -b)."""
    g = W.rng(seed)
    x = g.random((6, 7), dtype=np.float32)
    for (a, b) in [(0, 0), (2, -3), (-5, 9), (13, 1)]:
        inp = W.port((6, 7), (a, b), ((1, 0), (0, 1)), ((0,), (0,)), (1,))
        out = W.port((6, 7), (0, 0), ((1, 0), (0, 1)), ((0,), (0,)), (1,))
        y = O.run_task(W.task((6, 7), "copy", [inp], [out]), [x])[0].view(np.float32)
        np.testing.assert_array_equal(y, np.roll(x, (-a, -b), axis=(0, 1)))
    # shear paving [[1,0],[1,1]]: repetition r reads X[r0, r0 + r1], so row r0
    # of the result is row r0 of X rolled left by r0
    inp = W.port((6, 7), (0, 0), ((1, 0), (1, 1)), ((0,), (0,)), (1,))
    out = W.port((6, 7), (0, 0), ((1, 0), (0, 1)), ((0,), (0,)), (1,))
    y = O.run_task(W.task((6, 7), "copy", [inp], [out]), [x])[0].view(np.float32)
    for r0 in range(6):
        np.testing.assert_array_equal(y[r0], np.roll(x[r0], -r0))


def test_shift_tiler_is_numpy_roll():
    check_shift_is_roll()


def check_transpose_tilers(seed=3):
    """Paving [[0,1],[1,0]] (repetition r reads X[r1, r0]) and, separately,
    fitting [[0,1],[1,0]] within one pattern, both give numpy's transpose."""
    g = W.rng(seed)
    x = g.random((4, 6), dtype=np.float32)
    inp = W.port((4, 6), (0, 0), ((0, 1), (1, 0)), ((0,), (0,)), (1,))
    out = W.port((6, 4), (0, 0), ((1, 0), (0, 1)), ((0,), (0,)), (1,))
    y = O.run_task(W.task((6, 4), "copy", [inp], [out]), [x])[0].view(np.float32)
    np.testing.assert_array_equal(y, x.T)
    inp = W.port((4, 6), (0, 0), ((0,), (0,)), ((0, 1), (1, 0)), (6, 4))
    out = W.port((6, 4), (0, 0), ((0,), (0,)), ((1, 0), (0, 1)), (6, 4))
    y = O.run_task(W.task((1,), "copy", [inp], [out]), [x])[0].view(np.float32)
    np.testing.assert_array_equal(y, x.T)


def test_transpose_tilers():
    check_transpose_tilers()


def test_identity_round_trip_and_nan_payload():
    """A bijective tiler used for input and output returns X bit for bit,
    including a signalling-NaN payload and negative zero."""
    g = W.rng(4)
    x = g.random((5, 8), dtype=np.float32)
    raw = x.view(np.uint32)
    raw[1, 2] = 0x7F800123   # NaN with payload
    raw[3, 5] = 0x80000000   # -0.0
    t = W.port((5, 8), (3, -11), ((1, 0), (0, 4)), ((0,), (1,)), (4,))
    y = O.run_task(W.task((5, 2), "copy", [t], [t]), [x])[0]
    np.testing.assert_array_equal(y.view(np.uint32), raw)


def test_partition_invariant():
    tk, _ = W.config0()
    assert np.all(O.cover_count(tk["outputs"][0], tk["rep"]) == 1)
    for t in W.downscale_chain(2, 16, 24, np.ones((3, 8), np.float32), np.ones((3, 8), np.float32)):
        assert np.all(O.cover_count(t["outputs"][0], t["rep"]) == 1)
    g = W.rng(5)
    for _ in range(30):
        t = W.random_tiler_task(g, "copy")
        assert np.all(O.cover_count(t["outputs"][0], t["rep"]) == 1)
    # overlapping output tiler (step 2 with 3 outputs): not a partition
    bad = W.port((4, 6), (0, 0), ((1, 0), (0, 2)), ((0,), (1,)), (3,))
    assert O.cover_count(bad, (4, 3)).max() == 2
    with pytest.raises(O.NotAPartition):
        O.run_task(W.task((4, 3), "copy", [bad], [bad]), [np.zeros((4, 6), np.float32)])


# ---------------------------------------------------------------------- FIR

def check_fir_vs_correlate(seed=6):
    """Row FIR without wrap: y_r[j] = numpy.correlate(row, H[j], 'valid')[S*r1]."""
    g = W.rng(seed)
    H_, Wd, T, m, S = 3, 40, 8, 3, 4
    x = g.random((H_, Wd), dtype=np.float32)
    Hk = g.standard_normal((m, T)).astype(np.float32)
    reps = (H_, (Wd - T) // S + 1)
    inp = W.port((H_, Wd), (0, 0), ((1, 0), (0, S)), ((0,), (1,)), (T,))
    out = W.port((H_, reps[1] * m), (0, 0), ((1, 0), (0, m)), ((0,), (1,)), (m,))
    y = O.run_task(W.task(reps, "fir", [inp], [out], Hk), [x])[0]
    for r0 in range(H_):
        for j in range(m):
            c = np.correlate(x[r0].astype(np.float64), Hk[j].astype(np.float64), "valid")
            np.testing.assert_allclose(y[r0, j::m], c[::S][:reps[1]], rtol=1e-13, atol=1e-15)


def test_fir_vs_numpy_correlate():
    check_fir_vs_correlate()


def test_fir_linear_in_x_and_taps():
    tk, (x,) = W.config0(7)
    g = W.rng(8)
    x2 = g.random(x.shape, dtype=np.float32).astype(np.float64)
    a, b = 0.75, -1.25
    f = lambda xx: O.run_task(tk, [xx])[0]
    np.testing.assert_allclose(f(a * x.astype(np.float64) + b * x2), a * f(x) + b * f(x2), rtol=1e-12, atol=1e-12)
    H2 = g.standard_normal(tk["taps"].shape).astype(np.float32)
    t2 = dict(tk, taps=H2)
    t3 = dict(tk, taps=(tk["taps"].astype(np.float64) + H2))
    np.testing.assert_allclose(O.run_task(t3, [x])[0], f(x) + O.run_task(t2, [x])[0], rtol=1e-12, atol=1e-12)


def check_chain_block_closed_form(seed=9):
    """Separable 8x8 -> 3x3 downscaler chain: every output 3x3 block equals
    Hv . Xblock . Hh^T (numpy einsum on the reshaped frames)."""
    g = W.rng(seed)
    F, Hh_, Ww = 2, 16, 24
    x = g.random((F, Hh_, Ww), dtype=np.float32)
    Hh = g.standard_normal((3, 8)).astype(np.float32)
    Hv = g.standard_normal((3, 8)).astype(np.float32)
    chain = W.downscale_chain(F, Hh_, Ww, Hh, Hv)
    y = O.run_chain(chain, [x])[0]
    xb = x.astype(np.float64).reshape(F, Hh_ // 8, 8, Ww // 8, 8)
    ref = np.einsum("jk,fbkcl,il->fbjci", Hv.astype(np.float64), xb, Hh.astype(np.float64))
    np.testing.assert_allclose(y, ref.reshape(F, Hh_ // 8 * 3, Ww // 8 * 3), rtol=1e-12, atol=1e-12)


def test_chain_block_closed_form():
    check_chain_block_closed_form()


# ------------------------------------------------------------------- matmul

def test_matmul_task_is_block_matmul():
    """The tiled matmul task (panels x panels -> tiles) equals numpy.matmul of
    the whole matrices, and a naive triple loop on one entry."""
    g = W.rng(10)
    M, N, K, tm, tn = 8, 12, 5, 4, 6
    a = W.bf16_round(g.standard_normal((M, K), dtype=np.float32))
    b = W.bf16_round(g.standard_normal((K, N), dtype=np.float32))
    tk = W.matmul_task(M, N, K, tm, tn)
    y = O.run_task(tk, [a, b])[0]
    A = W.bf16_bits_to_f32(a).astype(np.float64)
    B = W.bf16_bits_to_f32(b).astype(np.float64)
    np.testing.assert_allclose(y, A @ B, rtol=1e-14, atol=1e-14)
    s = 0.0
    for k in range(K):
        s += A[5, k] * B[k, 7]
    assert abs(y[5, 7] - s) < 1e-12


def test_bf16_round_known_values():
    # 1.0 -> 0x3F80; 1 + 2^-8 (tie) -> even 0x3F80; 1 + 3*2^-8 (tie) -> 0x3F82; -2.0 -> 0xC000
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.0, 1.0 + 2 ** -7], dtype=np.float32)
    np.testing.assert_array_equal(W.bf16_round(v), np.array([0x3F80, 0x3F80, 0x3F82, 0xC000, 0x3F81], np.uint16))


def test_f16_round_known_values():
    """IEEE binary16 rounding of the input generator, values worked by hand:
    ties go to the even significand, 65520 (halfway to 2^16) overflows, and
    the subnormal step is 2^-24."""
    v = np.array([1.0, 1.0 + 2 ** -11, 1.0 + 3 * 2 ** -11, -2.0, 65504.0, 65520.0,
                  2 ** -24, 2 ** -25, 3 * 2 ** -26], dtype=np.float32)
    want = np.array([0x3C00, 0x3C00, 0x3C02, 0xC000, 0x7BFF, 0x7C00, 0x0001, 0x0000, 0x0001], np.uint16)
    np.testing.assert_array_equal(W.f16_round(v).view(np.uint16), want)


def test_oracle_reads_bf16_values():
    """The oracle's bf16 reads against values decoded by hand from bfloat16
    fields (sign, 8-bit exponent with bias 127, 7-bit fraction):
    0x4049 = +2^(128-127) * (1 + 73/128), 0xC2F7 = -2^6 * (1 + 119/128),
    0x3EAB = 2^-2 * (1 + 43/128), 0x0001 and 0x007F the smallest and largest
    subnormals (fraction/128 * 2^-126), 0x7F7F the largest finite value."""
    bits = np.array([0x3F80, 0x4049, 0xC2F7, 0x3EAB, 0x0001, 0x007F, 0x7F7F, 0x8000], np.uint16)
    want = [1.0, 3.140625, -123.5, 0.333984375, 2.0 ** -133, 127 * 2.0 ** -133, 255 * 2.0 ** 120, 0.0]
    got = O._as_values(bits, "bf16")
    assert got.dtype == np.float64 and list(got) == want
    assert np.signbit(got[-1]) and not np.signbit(got[0])   # 0x8000 is -0


def test_oracle_reads_f16_values():
    """The oracle's f16 reads against values decoded by hand from binary16
    fields (sign, 5-bit exponent with bias 15, 10-bit fraction)."""
    bits = np.array([0x3C00, 0x3555, 0x0001, 0x8400, 0x7BFF, 0x03FF], np.uint16)
    want = [1.0, 1365 / 4096, 2.0 ** -24, -(2.0 ** -14), 65504.0, 1023 * 2.0 ** -24]
    got = O._as_values(bits, "f16")
    assert got.dtype == np.float64 and list(got) == want
    assert list(O._as_values(bits.view(np.float16), "f16")) == want


def test_f16_fir_and_copy_through_both_oracles():
    """An f16 FIR reads the exact half values (the same as an f32 task on the
    widened values); an f16 copy moves the 16-bit words unchanged."""
    from oracle import cpu_ref as C
    g = W.rng(41)
    tk = W.random_tiler_task(g, "fir", max_side=8)
    x = W.f16_round(g.standard_normal(tk["inputs"][0]["shape"]).astype(np.float32))
    t16 = dict(tk, inputs=[dict(tk["inputs"][0], dtype="f16")])
    ref = O.run_task(tk, [x.astype(np.float64)])[0]
    np.testing.assert_array_equal(O.run_task(t16, [x])[0], ref)
    np.testing.assert_allclose(C.run_task(t16, [x])[0], ref, rtol=1e-13, atol=1e-300)
    tc = W.random_tiler_task(g, "copy", max_side=8)
    tc = dict(tc, inputs=[dict(tc["inputs"][0], dtype="f16")], outputs=[dict(tc["outputs"][0], dtype="f16")])
    xc = W.f16_round(g.standard_normal(tc["inputs"][0]["shape"]).astype(np.float32))
    yo = O.run_task(tc, [xc])[0]
    yc = C.run_task(tc, [xc])[0]
    np.testing.assert_array_equal(yo.view(np.uint16), yc.view(np.uint16))
    assert set(yo.view(np.uint16).ravel()) <= set(xc.view(np.uint16).ravel())


# ----------------------------------------------------------------- adjoints

def _inner(a, b):
    return float(np.sum(np.asarray(a, np.float64) * np.asarray(b, np.float64)))


def check_adjoint_identity(seed=11):
    """<T(X), G> = <X, T^T(G)> for random overlapping, wrapping fir tasks
    (T linear in X), and <dH, D> = <T_D(X), G> (T linear in the taps)."""
    g = W.rng(seed)
    for _ in range(12):
        tk = W.random_tiler_task(g, "fir")
        x = g.standard_normal(tk["inputs"][0]["shape"])
        G = g.standard_normal(tk["outputs"][0]["shape"])
        y = O.run_task(tk, [x])[0]
        dX, dH = O.task_vjp(tk, [x], G)
        assert abs(_inner(y, G) - _inner(x, dX)) <= 1e-10 * (1 + abs(_inner(y, G)))
        D = g.standard_normal(tk["taps"].shape)
        yD = O.run_task(dict(tk, taps=D), [x])[0]
        assert abs(_inner(dH, D) - _inner(yD, G)) <= 1e-10 * (1 + abs(_inner(yD, G)))


def test_adjoint_identity():
    check_adjoint_identity()


def test_copy_adjoint_identity():
    g = W.rng(12)
    for _ in range(12):
        tk = W.random_tiler_task(g, "copy")
        x = g.standard_normal(tk["inputs"][0]["shape"])
        G = g.standard_normal(tk["outputs"][0]["shape"])
        y = O.run_task(tk, [x])[0].view(np.float64)
        dX, _ = O.task_vjp(tk, [x], G)
        assert abs(_inner(y, G) - _inner(x, dX)) <= 1e-10 * (1 + abs(_inner(y, G)))


def check_chain_finite_differences(seed=13):
    """Central finite differences on a 32x32 frame of the downscaler chain,
    loss = sum(W * out).  The loss is linear in X and in each tap entry, so
    the central difference is exact up to rounding."""
    g = W.rng(seed)
    x = g.random((1, 32, 32))
    Hh = g.standard_normal((3, 8)) / 8
    Hv = g.standard_normal((3, 8)) / 8
    chain = W.downscale_chain(1, 32, 32, Hh, Hv)
    chain = [dict(t, taps=np.asarray(h, np.float64)) for t, h in zip(chain, (Hh, Hv))]
    Wt = g.standard_normal((1, 12, 12))
    loss = lambda c, xx: _inner(O.run_chain(c, [xx])[0], Wt)
    dX, (dHh, dHv) = O.chain_vjp(chain, [x], Wt)
    h = 1e-3
    for idx in [(0, 0, 0), (0, 5, 17), (0, 31, 31), (0, 8, 8), (0, 20, 3)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (loss(chain, xp) - loss(chain, xm)) / (2 * h)
        assert abs(fd - dX[idx]) < 1e-9, (idx, fd, dX[idx])
    for n, dH in ((0, dHh), (1, dHv)):
        for (j, k) in [(0, 0), (1, 3), (2, 7)]:
            cp = [dict(t, taps=t["taps"].copy()) for t in chain]
            cm = [dict(t, taps=t["taps"].copy()) for t in chain]
            cp[n]["taps"][j, k] += h
            cm[n]["taps"][j, k] -= h
            fd = (loss(cp, x) - loss(cm, x)) / (2 * h)
            assert abs(fd - dH[j, k]) < 1e-9, (n, j, k, fd, dH[j, k])


def test_chain_finite_differences_32x32():
    check_chain_finite_differences()


def test_chain_vjp_block_closed_form():
    """Gradient of the separable chain in closed form: dX block = Hv^T G Hh,
    dHv = sum G (Xb Hh^T)^T, dHh = sum (Hv^T G)^T Xb."""
    g = W.rng(14)
    F, Hh_, Ww = 2, 16, 24
    x = g.random((F, Hh_, Ww))
    Hh = g.standard_normal((3, 8))
    Hv = g.standard_normal((3, 8))
    chain = W.downscale_chain(F, Hh_, Ww, Hh, Hv)
    chain = [dict(t, taps=np.asarray(h)) for t, h in zip(chain, (Hh, Hv))]
    G = g.standard_normal((F, Hh_ // 8 * 3, Ww // 8 * 3))
    dX, (dHh, dHv) = O.chain_vjp(chain, [x], G)
    xb = x.reshape(F, Hh_ // 8, 8, Ww // 8, 8)
    gb = G.reshape(F, Hh_ // 8, 3, Ww // 8, 3)
    np.testing.assert_allclose(dX.reshape(xb.shape), np.einsum("jk,fbjci,il->fbkcl", Hv, gb, Hh), atol=1e-12)
    mid = np.einsum("fbkcl,il->fbkci", xb, Hh)      # horizontal pass, 8 rows x 3 cols per block
    np.testing.assert_allclose(dHv, np.einsum("fbjci,fbkci->jk", gb, mid), atol=1e-11)
    dmid = np.einsum("jk,fbjci->fbkci", Hv, gb)
    np.testing.assert_allclose(dHh, np.einsum("fbkci,fbkcl->il", dmid, xb), atol=1e-11)


# ------------------------------------------------------ C oracle agreement

def test_c_oracle_agrees_with_python_oracle():
    from oracle import cpu_ref as C
    g = W.rng(15)
    for elem in ("copy", "fir"):
        for _ in range(25):
            tk = W.random_tiler_task(g, elem)
            x = g.random(tk["inputs"][0]["shape"], dtype=np.float32)
            yp = O.run_task(tk, [x])[0]
            yc = C.run_task(tk, [x])[0]
            if elem == "copy":
                np.testing.assert_array_equal(yp.view(np.uint32), yc.view(np.uint32))
            else:
                np.testing.assert_allclose(yc, yp, rtol=1e-13, atol=1e-15)
                G = g.standard_normal(tk["outputs"][0]["shape"])
                dXp, dHp = O.task_vjp(tk, [x], G)
                dXc, dHc = C.fir_vjp(tk, x, G)
                np.testing.assert_allclose(dXc, dXp, rtol=1e-12, atol=1e-13)
                np.testing.assert_allclose(dHc, dHp, rtol=1e-12, atol=1e-13)
    tk, (x,) = W.config0()
    np.testing.assert_allclose(C.run_task(tk, [x])[0], O.run_task(tk, [x])[0], rtol=1e-13, atol=1e-15)
    a = W.bf16_round(g.standard_normal((8, 6), dtype=np.float32))
    b = W.bf16_round(g.standard_normal((6, 12), dtype=np.float32))
    mt = W.matmul_task(8, 12, 6, 4, 6)
    yp = O.run_task(mt, [a, b])[0]
    np.testing.assert_allclose(C.run_task(mt, [a, b])[0], yp, rtol=1e-13, atol=1e-14)
    rows, cols = np.array([0, 7, 3]), np.array([0, 11, 6])
    vals, _ = C.matmul_sample(mt, a, b, rows, cols)
    np.testing.assert_allclose(vals, yp[rows, cols], rtol=1e-13, atol=1e-14)
    bad = W.port((4, 6), (0, 0), ((1, 0), (0, 2)), ((0,), (1,)), (3,))
    assert not C.cover_ok(W.task((4, 3), "copy", [bad], [bad]))
    with pytest.raises(ValueError):
        C.run_task(W.task((4, 3), "copy", [bad], [bad]), [np.zeros((4, 6), np.float32)])


# ------------------------------------------- planted mistakes must be caught

def _trunc_mod(a, s):                      # C-style remainder: wrong for a < 0
    return int(np.fmod(a, s))


def _element_no_origin(t, r, i):
    return _REAL_ELEMENT(dict(t, origin=tuple(0 for _ in t["origin"])), r, i)


def _element_transposed_paving(t, r, i):
    P = t["paving"]
    if len(P) == len(r) and all(len(row) == len(r) for row in P):
        P = tuple(tuple(P[q][k] for q in range(len(P))) for k in range(len(P)))
    return _REAL_ELEMENT(dict(t, paving=P), r, i)


def _element_swapped_ri(t, r, i):
    if len(r) == len(i):
        r, i = i, r
    return _REAL_ELEMENT(t, r, i)


def _elem_fir_dropped_tap(p, H):
    return _REAL_FIR(p[:-1] + [0.0], H)


def _elem_fir_transposed(p, H):
    return _REAL_FIR(p, H[:, ::-1])


_REAL_ELEMENT = O.tiler_element
_REAL_FIR = O.elem_fir

_ADDRESS_PINS = [check_golden_addresses, check_row_tiler_vs_take, check_shift_is_roll,
                 check_transpose_tilers, check_chain_block_closed_form]
_FIR_PINS = [check_fir_vs_correlate, check_chain_block_closed_form, check_chain_finite_differences]


def _some_pin_fails(pins):
    for pin in pins:
        try:
            pin()
        except (AssertionError, IndexError, ValueError):
            return True
    return False


@pytest.mark.parametrize("attr,bad", [
    ("emod", _trunc_mod),
    ("tiler_element", _element_no_origin),
    ("tiler_element", _element_transposed_paving),
    ("tiler_element", _element_swapped_ri),
])
def test_planted_address_mistake_is_caught(monkeypatch, attr, bad):
    monkeypatch.setattr(O, attr, bad)
    assert _some_pin_fails(_ADDRESS_PINS)


@pytest.mark.parametrize("bad", [_elem_fir_dropped_tap, _elem_fir_transposed])
def test_planted_fir_mistake_is_caught(monkeypatch, bad):
    monkeypatch.setattr(O, "elem_fir", bad)
    assert _some_pin_fails(_FIR_PINS)


def test_2d_fir_patterns_c_oracle_and_adjoint():
    from oracle import cpu_ref as C
    g = W.rng(16)
    for _ in range(20):
        tk = W.random_tiler_task(g, "fir", fir_pattern_rank=2)
        x = g.standard_normal(tk["inputs"][0]["shape"])
        y = O.run_task(tk, [x])[0]
        np.testing.assert_allclose(C.run_task(tk, [x])[0], y, rtol=1e-13, atol=1e-14)
        G = g.standard_normal(tk["outputs"][0]["shape"])
        dX, dH = O.task_vjp(tk, [x], G)
        assert abs(_inner(y, G) - _inner(x, dX)) <= 1e-10 * (1 + abs(_inner(y, G)))


def test_2d_fir_is_a_sum_of_rolled_arrays():
    """A FIR on a 2-D pattern (fitting identity, diagonal paving (s0, s1),
    m outputs along the output row) against its closed form as a sum of
    shifted arrays: y[r0, m r1 + j] = sum_{a,b} H[j, a p1 + b] x[(s0 r0 + a + o0)
    mod H, (s1 r1 + b + o1) mod W], i.e. numpy.roll then a strided slice."""
    g = W.rng(17)
    cases = [(12, 10, 3, 3, 1, 1, 1, (-1, -1)),    # 3x3 stencil with wrap
             (9, 14, 2, 5, 3, 2, 2, (4, -7)),      # strided, overlapping, 2 outputs
             (7, 7, 5, 5, 1, 1, 3, (-2, 30))]      # pattern as wide as the array, origin past the edge
    for (Hh, Ww, p0, p1, s0, s1, m, o) in cases:
        R0, R1 = -(-Hh // s0), -(-Ww // s1)
        inp = W.port((Hh, Ww), o, ((s0, 0), (0, s1)), ((1, 0), (0, 1)), (p0, p1))
        out = W.port((R0, m * R1), (0, 0), ((1, 0), (0, m)), ((0,), (1,)), (m,))
        tk = W.task((R0, R1), "fir", [inp], [out], g.standard_normal((m, p0 * p1)))
        taps = tk["taps"].astype(np.float64)
        x = g.standard_normal((Hh, Ww))
        want = np.zeros((R0, m * R1))
        for j in range(m):
            acc = np.zeros((Hh, Ww))
            for a in range(p0):
                for b in range(p1):
                    acc += taps[j, a * p1 + b] * np.roll(x, (-(a + o[0]), -(b + o[1])), axis=(0, 1))
            want[:, j::m] = acc[::s0, ::s1]
        np.testing.assert_allclose(O.run_task(tk, [x])[0], want, rtol=1e-12, atol=1e-12)
