"""Batches whose members are chains (Sec. 5: tasks linked through shared
arrays) mixed with single tasks: one graph launch, one persistent launch per
chain stage.  Every member against the oracle's chain; the graph path equals
the one-launch-per-task path and a second run bit for bit."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cpu_ref as C
from oracle import tiler as O
from tests.gpu_helpers import FIR_RTOL, assert_fir_close, dev, fir_scale, host
from tests.test_parity_gpu import _three_task_chain

pytestmark = pytest.mark.gpu


def _members(g):
    """(member spec, input) pairs: single tasks, 2- and 3-stage chains."""
    out = []
    tk, (x,) = W.config0(seed=21)
    out.append((tk, x))
    chain, (x,) = W.config1(seed=22, frames=2, height=16, width=64)
    out.append((chain, x))
    out.append((_three_task_chain(g), g.standard_normal((24, 32)).astype(np.float32)))
    for i in range(6):
        tk = W.random_tiler_task(g, "fir" if i % 2 else "copy")
        out.append((tk, g.random(tk["inputs"][0]["shape"], dtype=np.float32)))
    chain, (x,) = W.config1(seed=23, frames=3, height=24, width=1928)
    out.append((chain, x))
    out.append((_three_task_chain(g), g.standard_normal((24, 32)).astype(np.float32)))
    return out


def _check(spec, x, y):
    chain = spec if isinstance(spec, list) else [spec]
    ref = O.run_chain(chain, [x])[0]
    if len(chain) == 1 and chain[0]["elem"] == "copy":
        np.testing.assert_array_equal(y.view(np.uint32), ref.view(np.uint32))
    else:
        assert_fir_close(y, ref, fir_scale(chain, x), what=f"batch member of {len(chain)} stage(s)")


def test_batch_of_chains_and_tasks(arol):
    g = W.rng(120)
    members = _members(g)
    b = arol.Batch([m for m, _ in members])
    ins = [dev(x) for _, x in members]
    outs = b.empty_outputs()
    b.run(ins, outs)
    outs2 = b.empty_outputs()
    b.run_per_task(ins, outs2)
    outs3 = b.empty_outputs()
    b.run(ins, outs3)
    torch.cuda.synchronize()
    for (spec, x), y, y2, y3 in zip(members, outs, outs2, outs3):
        y = host(y)
        _check(spec, x, y)
        np.testing.assert_array_equal(y, host(y2))
        np.testing.assert_array_equal(y, host(y3))


def test_batch_chain_with_bf16_intermediate(arol):
    """bfloat16 frames and intermediate inside a batch: the intermediate is
    rounded to nearest even by the first stage, as in a standalone chain."""
    chain, (x,) = W.config1_bf16(seed=24, frames=2, height=16, width=64, mid="bf16", out="f32")
    g = W.rng(121)
    tk = W.random_tiler_task(g, "fir")
    xt = g.random(tk["inputs"][0]["shape"], dtype=np.float32)
    b = arol.Batch([chain, tk])
    outs = b.empty_outputs()
    b.run([dev(x), dev(xt)], outs)
    torch.cuda.synchronize()
    xv = W.bf16_bits_to_f32(x).astype(np.float64)
    f32_chain = [dict(chain[0], inputs=[dict(chain[0]["inputs"][0], dtype="f32")],
                      outputs=[dict(chain[0]["outputs"][0], dtype="f32")]),
                 dict(chain[1], inputs=[dict(chain[1]["inputs"][0], dtype="f32")])]
    ref = O.run_chain(f32_chain, [xv])[0]
    scale = fir_scale(f32_chain, xv)
    err = np.abs(host(outs[0]).astype(np.float64) - ref)
    assert np.all(err <= (FIR_RTOL + 2.0 ** -8) * scale + 1e-38)
    assert_fir_close(host(outs[1]), O.run_task(tk, [xt])[0], fir_scale(tk, xt), what="batch fir next to a chain")


def test_batch_rejects_matmul_members(arol):
    spec = W.matmul_task(128, 128, 128)
    with pytest.raises(arol.ArolError):
        arol.Batch([spec])


def _row_cases():
    """Row-FIR tasks that reach every exact-m template and both tile layouts
    at their capacity edges (4096-float windows, 2048 repetitions; whole
    rows up to 2048 words), with origins that wrap."""
    g = W.rng(122)
    cases = []
    for m in range(1, 17):                          # every output count, T up to 32
        T = max(m, int(g.integers(m, 33)))
        S = int(g.integers(1, T + 1))
        cases.append((int(g.integers(1, 6)), int(g.integers(40, 700)), T, m, S))
    # a long row: step 32, T 32 -> at most (4096 - 32) / 32 + 1 = 128 repetitions per tile
    for w in (32 * 127, 32 * 128, 32 * 128 + 5, 32 * 129):
        cases.append((2, w, 32, 3, 32))
    for w in (2047, 2048, 2049):                    # whole rows: two per tile, then one
        cases.append((5, w, 9, 2, 5))
    # step 1: pieces capped at 2048 repetitions; whole rows capped at 2048
    # repetitions per tile (two rows of 1024, then one row of 1025)
    for w in (2048, 2049, 4100):
        cases.append((3, w, 4, 1, 1))
    for w in (1024, 1025):
        cases.append((5, w, 4, 1, 1))
    cases.append((3, 2, 7, 1, 1))                   # a row shorter than its pattern
    tasks, xs = [], []
    for (h, w, T, m, S) in cases:
        taps = (g.standard_normal((m, T)) / T).astype(np.float32)
        tk = W.fir_row_task(h, w, T, m, S, taps)
        tasks.append(tk)
        xs.append(g.standard_normal((h, w)).astype(np.float32))
    return tasks, xs


def test_batch_row_fir_edges(arol):
    tasks, xs = _row_cases()
    b = arol.Batch(tasks)
    ins = [dev(x) for x in xs]
    outs, outs2 = b.empty_outputs(), b.empty_outputs()
    b.run(ins, outs)
    b.run_per_task(ins, outs2)
    torch.cuda.synchronize()
    for tk, x, y, y2 in zip(tasks, xs, outs, outs2):
        y = host(y)
        assert_fir_close(y, C.run_task(tk, [x])[0], fir_scale(tk, x, C.run_chain),
                         what=f"row fir {x.shape} m={tk['outputs'][0]['pattern'][0]}")
        np.testing.assert_array_equal(y, host(y2))
    # other launch shapes give the same bits
    b.tune(ins, outs, force=True)
    outs3 = b.empty_outputs()
    b.run(ins, outs3)
    torch.cuda.synchronize()
    for y2, y3 in zip(outs2, outs3):
        np.testing.assert_array_equal(host(y2), host(y3))


def test_batch_mixes_bf16_and_row_tasks(arol):
    """A bf16 task (generic path) among row-FIR tasks (staged path)."""
    g = W.rng(123)
    tasks, xs = _row_cases()
    tasks, xs = tasks[:4], xs[:4]
    tk = W.random_tiler_task(g, "fir")
    tk = dict(tk, inputs=[dict(tk["inputs"][0], dtype="bf16")], outputs=[dict(tk["outputs"][0], dtype="bf16")])
    xb = W.bf16_round(g.standard_normal(tk["inputs"][0]["shape"]).astype(np.float32))
    b = arol.Batch(tasks + [tk])
    outs = b.empty_outputs()
    b.run([dev(x) for x in xs] + [dev(xb)], outs)
    torch.cuda.synchronize()
    for t, x, y in zip(tasks, xs, outs[:4]):
        assert_fir_close(host(y), C.run_task(t, [x])[0], fir_scale(t, x, C.run_chain), what="row fir next to bf16")
    xv = W.bf16_bits_to_f32(xb).astype(np.float64)
    tk_v = dict(tk, inputs=[dict(tk["inputs"][0], dtype="f32")], outputs=[dict(tk["outputs"][0], dtype="f32")])
    ref = O.run_task(tk_v, [xv])[0]
    got = W.bf16_bits_to_f32(host(outs[4])).astype(np.float64)
    assert np.all(np.abs(got - ref) <= FIR_RTOL * fir_scale(tk_v, xv) + 2.0 ** -8 * np.abs(ref) + 1e-38)


def _col_task(g, h, w, T, m, S, origin=(0, 0), out_origin=(0, 0)):
    """Column FIR: repetition (r0, c) reads rows origin0 + S*r0 + k (mod h) of
    column origin1 + c (mod w); m consecutive output rows per repetition."""
    R0 = -(-h // S)
    taps = (g.standard_normal((m, T)) / T).astype(np.float32)
    inp = W.port((h, w), origin, ((S, 0), (0, 1)), ((1,), (0,)), (T,))
    out = W.port((m * R0, w), out_origin, ((m, 0), (0, 1)), ((1,), (0,)), (m,))
    return W.task((R0, w), "fir", [inp], [out], taps)


def test_batch_column_fir(arol):
    """Column FIRs for every output count, with wrapping origins, steps below
    and above T, and a framed column task whose windows overlap the next
    frame (so it must not be merged into one tall array)."""
    g = W.rng(124)
    tasks, xs = [], []
    for m in range(1, 17):
        T = int(g.integers(m, 33))
        S = int(g.integers(1, T + 3))
        h, w = int(g.integers(8, 90)), int(g.integers(3, 300))
        tk = _col_task(g, h, w, T, m, S, origin=(int(g.integers(-40, 40)), int(g.integers(-40, 40))),
                       out_origin=(int(g.integers(0, 5)), int(g.integers(0, 7))))
        tasks.append(tk)
        xs.append(g.standard_normal((h, w)).astype(np.float32))
    # frames with overlapping windows (T > S): rows wrap within each frame
    F, h, w, T, m, S = 3, 24, 40, 6, 2, 4
    taps = (g.standard_normal((m, T)) / T).astype(np.float32)
    inp = W.port((F, h, w), (0, 0, 0), ((1, 0, 0), (0, S, 0), (0, 0, 1)), ((0,), (1,), (0,)), (T,))
    out = W.port((F, m * h // S, w), (0, 0, 0), ((1, 0, 0), (0, m, 0), (0, 0, 1)), ((0,), (1,), (0,)), (m,))
    tasks.append(W.task((F, h // S, w), "fir", [inp], [out], taps))
    xs.append(g.standard_normal((F, h, w)).astype(np.float32))
    b = arol.Batch(tasks)
    ins = [dev(x) for x in xs]
    outs, outs2 = b.empty_outputs(), b.empty_outputs()
    b.run(ins, outs)
    b.run_per_task(ins, outs2)
    torch.cuda.synchronize()
    for tk, x, y, y2 in zip(tasks, xs, outs, outs2):
        y = host(y)
        assert_fir_close(y, O.run_task(tk, [x])[0], fir_scale(tk, x), what=f"column fir {x.shape}")
        np.testing.assert_array_equal(y, host(y2))
        # the single-task path agrees
        np.testing.assert_allclose(host(arol.Task(tk).run([dev(x)])), y, rtol=1e-6, atol=1e-6)


def test_task_handle_takes_the_staged_paths(arol):
    """A single row-FIR task, a column-FIR task and an unfused chain run on
    the batch engine through their own handles: results match the oracle,
    host taps set between runs take effect, device taps fall back to the
    per-repetition path with the same results."""
    g = W.rng(125)
    H = (g.standard_normal((3, 11)) / 11).astype(np.float32)
    row = W.fir_row_task(37, 300, 11, 3, 4, H)
    col = _col_task(g, 90, 70, 7, 2, 5, origin=(-3, 4))
    x_row = g.standard_normal((37, 300)).astype(np.float32)
    x_col = g.standard_normal((90, 70)).astype(np.float32)
    for tk, x in ((row, x_row), (col, x_col)):
        t = arol.Task(tk)
        y = host(t.run([dev(x)]))
        assert_fir_close(y, O.run_task(tk, [x])[0], fir_scale(tk, x), what="task handle")
        H2 = (g.standard_normal(tk["taps"].shape) / tk["taps"].shape[1]).astype(np.float32)
        t.set_taps(H2)
        tk2 = dict(tk, taps=H2)
        y2 = host(t.run([dev(x)]))
        assert_fir_close(y2, O.run_task(tk2, [x])[0], fir_scale(tk2, x), what="task handle, new taps")
        H2d = torch.from_numpy(H2).cuda()                 # device taps (borrowed: kept alive here)
        t.set_taps(H2d)                                   # per-repetition path
        np.testing.assert_allclose(host(t.run([dev(x)])), y2, rtol=1e-6, atol=1e-6)
        del H2d
    chain = _three_task_chain(g)
    x = g.standard_normal((24, 32)).astype(np.float32)
    c = arol.Chain(chain)
    assert_fir_close(host(c.run([dev(x)])), O.run_chain(chain, [x])[0], fir_scale(chain, x), what="unfused chain handle")


def test_task_handle_on_two_streams(arol):
    """The same handle on two streams with different buffers, interleaved:
    a new buffer table is ordered after the other stream's launches."""
    g = W.rng(126)
    H = (g.standard_normal((2, 9)) / 9).astype(np.float32)
    tk = W.fir_row_task(64, 2000, 9, 2, 3, H)
    t = arol.Task(tk)
    xs = [g.standard_normal((64, 2000)).astype(np.float32) for _ in range(2)]
    xd = [dev(x) for x in xs]
    ys = [t.empty_output("cuda") for _ in range(2)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for rep in range(20):
        for k in range(2):
            with torch.cuda.stream(streams[k]):
                t.run([xd[k]], ys[k])
    torch.cuda.synchronize()
    for x, y in zip(xs, ys):
        assert_fir_close(host(y), C.run_task(tk, [x])[0], fir_scale(tk, x, C.run_chain), what="two streams")


def test_batched_chains_full_size(arol):
    """The bench's 128 two-stage chains of uneven frames, in the bench's
    launch configuration (one graph, default tiles): every eighth member
    against the C oracle's chain, all members against one fused launch each."""
    chains, xs = W.chain_batch()
    b = arol.Batch(chains)
    ins = [dev(x) for x in xs]
    outs = b.empty_outputs()
    b.run(ins, outs)
    torch.cuda.synchronize()
    for i, (chain, x, y) in enumerate(zip(chains, xs, outs)):
        y = host(y)
        if i % 8 == 0:
            assert_fir_close(y, C.run_chain(chain, [x])[0], fir_scale(chain, x, C.run_chain), what=f"chain {i}")
        yf = host(arol.Chain(chain).run([ins[i]]))
        np.testing.assert_allclose(y, yf, rtol=1e-5, atol=1e-6)
