"""Column-FIR tasks over frames whose windows overlap or wrap within a frame
(T > step, or an origin): they keep the column-FIR path with the frame as
an outer repetition, alone and inside batches, and match the C oracle.  A
batch with an output count above 16 runs them on the per-repetition walk,
also matching."""
import numpy as np
import pytest

import workloads as W
from oracle import cpu_ref as C
from tests.gpu_helpers import assert_fir_close, dev, fir_scale, host

pytestmark = pytest.mark.gpu


def col_task(g, F, H, Wd, T, m, S, origin=0, reps=None):
    reps = -(-H // S) if reps is None else reps
    return W.separable_pass((F, H, Wd), 0, T, m, S, origin, reps, (g.standard_normal((m, T)) / T).astype(np.float32))


def cases(g):
    return [col_task(g, 4, 64, 96, 5, 2, 4),            # the 5 -> 2 step-4 column stage
            col_task(g, 3, 37, 50, 9, 3, 2, origin=30),  # overlap 4.5x, windows wrap at the bottom
            col_task(g, 2, 8, 33, 12, 4, 3, reps=7),     # windows longer than the frame
            col_task(g, 5, 120, 17, 32, 16, 32)]         # the largest T and m


def test_framed_column_fir_tasks(arol):
    g = W.rng(501)
    for n, tk in enumerate(cases(g)):
        x = g.standard_normal(tk["inputs"][0]["shape"]).astype(np.float32)
        t = arol.Task(tk)
        assert t.info["path"] == 2
        y = t.run([dev(x)])
        t.sync_status()
        assert_fir_close(host(y), C.run_task(tk, [x])[0], fir_scale(tk, x, C.run_chain), what=f"column case {n}")


@pytest.mark.parametrize("with_wide_m", [False, True])
def test_framed_column_fir_in_batches(arol, with_wide_m):
    g = W.rng(502)
    tasks = cases(g)
    if with_wide_m:
        # a 40-tap, 20-output row task: m > 16 sends the batch's other tiles to the per-repetition walk
        tasks.append(W.fir_row_task(9, 200, 40, 20, 20, (g.standard_normal((20, 40)) / 40).astype(np.float32)))
    xs = [g.standard_normal(t["inputs"][0]["shape"]).astype(np.float32) for t in tasks]
    b = arol.Batch(tasks)
    outs = b.empty_outputs()
    b.run([dev(x) for x in xs], outs)
    b.sync_status()
    for n, (tk, x) in enumerate(zip(tasks, xs)):
        assert_fir_close(host(outs[n]), C.run_task(tk, [x])[0], fir_scale(tk, x, C.run_chain), what=f"batched {n}")
