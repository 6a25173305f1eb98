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
