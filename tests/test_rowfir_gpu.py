"""Parity of the row-FIR batch kernel (staged row tiles) with the C oracle
on the cases its tiling has to get right: rows that wrap at the array's end
(row origin), output columns that wrap (output origin), windows that wrap
past a row's end once or several times (T > W), rows of 1..5 words, every
step 1..32 and output count 1..16, and input/output views that are not
16-byte aligned.  FIR outputs within 1e-5 of the summed absolute terms."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cpu_ref as C
from tests.gpu_helpers import assert_fir_close, dev, fir_scale, host

pytestmark = pytest.mark.gpu


def row_task(g, H, Wd, T, m, S, R0=None, R1=None, o=(0, 0), oo=(0, 0)):
    """A row FIR with origins: input rows (o0 + r0) mod H, columns
    (o1 + S r1 + k) mod W; output (oo0 + r0, oo1 + m r1 + j) on an
    (R0, m R1) array (a partition for any output origin)."""
    R0 = H if R0 is None else R0
    R1 = -(-Wd // S) if R1 is None else R1
    taps = (g.standard_normal((m, T)) / T).astype(np.float32)
    inp = W.port((H, Wd), o, ((1, 0), (0, S)), ((0,), (1,)), (T,))
    out = W.port((R0, m * R1), oo, ((1, 0), (0, m)), ((0,), (1,)), (m,))
    return W.task((R0, R1), "fir", [inp], [out], taps)


def cases():
    g = W.rng(301)
    out = []
    for S in range(1, 33):
        T = int(g.integers(max(3, S // 2), 33))
        m = int(g.integers(1, 17))
        out.append(row_task(g, int(g.integers(1, 70)), int(g.integers(S, 700)), T, m, S))
    # rows that wrap at H, output columns and rows that wrap
    out.append(row_task(g, 50, 301, 9, 4, 5, R0=50, o=(37, 11), oo=(13, 7)))
    out.append(row_task(g, 40, 96, 16, 3, 8, R0=33, o=(39, 95), oo=(32, 35)))
    # windows longer than a row (T > W) and tiny rows
    for Wd in (1, 2, 3, 4, 5, 7):
        out.append(row_task(g, 37, Wd, 19, 2, 1 + Wd % 3))
    # many repetitions past one row's width (the window wraps several times)
    out.append(row_task(g, 9, 13, 6, 2, 3, R1=40))
    # long rows split into pieces, and a 1 x 1 array
    out.append(row_task(g, 3, 4099, 32, 16, 31))
    out.append(row_task(g, 1, 1, 3, 1, 1))
    return out


def test_rowfir_cases_batched_and_single(arol):
    tasks = cases()
    g = W.rng(302)
    xs = [g.standard_normal(t["inputs"][0]["shape"]).astype(np.float32) for t in tasks]
    b = arol.Batch(tasks)
    outs = b.empty_outputs()
    b.run([dev(x) for x in xs], outs)
    b.sync_status()
    for i, (tk, x) in enumerate(zip(tasks, xs)):
        ref = C.run_task(tk, [x])[0]
        assert_fir_close(host(outs[i]), ref, fir_scale(tk, x, C.run_chain), what=f"batched case {i}")
    # the same tasks one by one (one-member batches of the same kernel)
    for i in (0, 7, 31, 32, 33, 40, 41):
        t = arol.Task(tasks[i])
        y = t.run([dev(xs[i])])
        t.sync_status()
        assert t.info["path"] == 1
        assert_fir_close(host(y), C.run_task(tasks[i], [xs[i]])[0], fir_scale(tasks[i], xs[i], C.run_chain),
                         what=f"single case {i}")


def test_rowfir_unaligned_views(arol):
    """Inputs and outputs that start 1, 2 or 3 floats past a 16-byte
    boundary: the row copies take their ragged ends word by word."""
    g = W.rng(303)
    tasks = [row_task(g, 23, 517, 11, 3, 4), row_task(g, 5, 64, 8, 5, 8), row_task(g, 31, 33, 7, 1, 2)]
    xs = [g.standard_normal(t["inputs"][0]["shape"]).astype(np.float32) for t in tasks]
    for shift in (1, 2, 3):
        ins, outs, keep = [], [], []
        for t, x in zip(tasks, xs):
            xb = torch.zeros(x.size + shift, device="cuda")
            xb[shift:] = dev(x).reshape(-1)
            ins.append(xb[shift:].view(x.shape))
            shp = t["outputs"][0]["shape"]
            yb = torch.full((int(np.prod(shp)) + shift,), float("nan"), device="cuda")
            outs.append(yb[shift:].view(shp))
            keep += [xb, yb]
        b = arol.Batch(tasks)
        b.run(ins, outs)
        b.sync_status()
        for i, (tk, x) in enumerate(zip(tasks, xs)):
            assert_fir_close(host(outs[i]), C.run_task(tk, [x])[0], fir_scale(tk, x, C.run_chain),
                             what=f"shift {shift} case {i}")


def test_rowfir_results_do_not_depend_on_the_launch_shape(arol, monkeypatch):
    """Autotuning changes the tile budget and grid, not one bit of the result."""
    tasks, xs = W.config3(seed=9, n=40, lo=32, hi=700)
    b = arol.Batch(tasks)
    ins = [dev(x) for x in xs]
    o1 = b.empty_outputs()
    b.run(ins, o1)
    monkeypatch.setenv("AROL_TUNE", "force")
    b.tune(ins, b.empty_outputs())
    o2 = b.empty_outputs()
    b.run(ins, o2)
    b.sync_status()
    for a, c in zip(o1, o2):
        assert torch.equal(a, c)


@pytest.mark.parametrize("S", [2, 4, 8])
def test_rowfir_regions(arol, S):
    """Single row-FIR tasks in 16-word regions: every output count the form
    takes, 1 to 8 taps, origin 0 or a multiple of 16 (windows that wrap at
    the row's end), against the C oracle.  The same task on views one float
    past a 16-byte boundary takes the row-FIR tiles, within the same bound."""
    g = W.rng(310 + S)
    for M in range(1, (2 if S == 2 else 4) + 1):
        for T in sorted({1, S, 8, int(g.integers(1, 9))}):
            Wd = 16 * int(g.integers(1, 40))
            H = int(g.integers(1, 50))
            o1 = 16 * int(g.integers(0, Wd // 16))
            tk = row_task(g, H, Wd, T, M, S, R1=Wd // S, o=(0, o1))
            x = g.standard_normal((H, Wd)).astype(np.float32)
            ref = C.run_task(tk, [x])[0]
            scale = fir_scale(tk, x, C.run_chain)
            t = arol.Task(tk)
            assert t.info["path"] == 5
            y = t.run([dev(x)])
            xb = torch.zeros(x.size + 1, device="cuda")
            xb[1:] = dev(x).reshape(-1)
            y1 = t.run([xb[1:].view(x.shape)])
            t.sync_status()
            assert_fir_close(host(y), ref, scale, what=f"S {S} M {M} T {T} W {Wd} o {o1}")
            assert_fir_close(host(y1), ref, scale, what=f"S {S} M {M} T {T} W {Wd} o {o1}, unaligned")


def test_rowfir_regions_config0_scaled_full_size(arol):
    """The 64 x 64 task's tiler (8 taps, 3 outputs, step 4, windows wrapping
    at the row end) on 64 x 1080 x 1920 float32, as the bench runs it,
    against the C oracle element by element."""
    tk, (x,) = W.config0_scaled()
    t = arol.Task(tk)
    assert t.info["path"] == 5
    y = t.run([dev(x)])
    t.sync_status()
    assert_fir_close(host(y), C.run_task(tk, [x])[0], fir_scale(tk, x, C.run_chain), what="config0 scaled")
