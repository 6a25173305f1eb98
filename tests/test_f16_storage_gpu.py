"""IEEE half storage (Sec. 5 typeAllocation) for copy and FIR tasks, batches
and the fused chain.

The arithmetic stays f32.  Half inputs are widened exactly (the oracle reads
the same values); every store into a half array rounds to nearest even.  A
half keeps 11 significant bits, so a rounded normal value errs by at most
2^-11 of its magnitude, and a rounded subnormal by at most 2^-25.  Tolerance
per element: 1e-5 of the summed absolute terms (the f32 bound of the other
tests); plus, for a rounded intermediate, 2^-11 of that sum and 2^-25 times
the sum of the absolute taps that read it; plus, for a rounded output,
2^-11 |y| + 2^-25.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cpu_ref as C
from oracle import tiler as O
from tests.gpu_helpers import FIR_RTOL, assert_fir_close, dev, fir_scale, host

pytestmark = pytest.mark.gpu

U16 = 2.0 ** -11      # relative rounding bound of a normal half
SUB16 = 2.0 ** -25    # absolute rounding bound of a subnormal half
UB16 = 2.0 ** -8      # relative rounding bound of a bfloat16


def to_f64(y):
    if y.dtype == np.uint16:
        return W.bf16_bits_to_f32(y).astype(np.float64)
    return y.astype(np.float64)


def check(y, y64, scale, out_half, what, mid_abs_taps=None):
    tol = FIR_RTOL * scale
    if mid_abs_taps is not None:
        tol = tol + U16 * scale + SUB16 * mid_abs_taps
    if out_half:
        tol = tol + U16 * np.abs(y64) + SUB16
    err = np.abs(to_f64(y) - y64)
    bad = err > tol + 1e-38
    assert not bad.any(), f"{what}: {int(bad.sum())} of {bad.size} out of tolerance, worst {err.max():.3e}"


def values_task(tk):
    """The same task on f32 arrays: the oracle then reads widened values."""
    return dict(tk, inputs=[dict(p, dtype="f32") for p in tk["inputs"]],
                outputs=[dict(p, dtype="f32") for p in tk["outputs"]])


@pytest.mark.parametrize("dt_in,dt_out", [("f16", "f16"), ("f16", "f32"), ("f32", "f16")])
def test_generic_fir_f16_storage(arol, dt_in, dt_out):
    g = W.rng(311)
    for _ in range(25):
        tk = W.random_tiler_task(g, "fir", fir_pattern_rank=int(g.integers(1, 3)))
        tk = dict(tk, inputs=[dict(tk["inputs"][0], dtype=dt_in)], outputs=[dict(tk["outputs"][0], dtype=dt_out)])
        xf = g.standard_normal(tk["inputs"][0]["shape"]).astype(np.float32)
        x = W.f16_round(xf) if dt_in == "f16" else xf
        t = arol.Task(tk)
        y = host(t.run([dev(x)]))
        torch.cuda.synchronize()
        assert y.dtype == (np.float16 if dt_out == "f16" else np.float32)
        xv = to_f64(x)
        tv = values_task(tk)
        check(y, O.run_task(tv, [xv])[0], fir_scale(tv, xv), dt_out == "f16", f"{dt_in}->{dt_out}")


def test_random_f16_copy_tilers_bit_exact(arol):
    """Copies move half words untouched, NaN payloads and subnormals included."""
    g = W.rng(312)
    for _ in range(30):
        tk = W.random_tiler_task(g, "copy")
        tk = dict(tk, inputs=[dict(tk["inputs"][0], dtype="f16")], outputs=[dict(tk["outputs"][0], dtype="f16")])
        bits = g.integers(0, 65536, size=tk["inputs"][0]["shape"], dtype=np.uint16)
        t = arol.Task(tk)
        y = host(t.run([dev(bits.view(np.float16))]))
        torch.cuda.synchronize()
        np.testing.assert_array_equal(y.view(np.uint16), O.run_task(tk, [bits.view(np.float16)])[0].view(np.uint16))


@pytest.mark.parametrize("mid,out", [("f32", "f16"), ("f16", "f16"), ("f32", "f32"), ("f16", "f32")])
@pytest.mark.parametrize("shape", [(1, 8, 64), (2, 24, 136), (3, 16, 1928)])
def test_fused_f16_chain(arol, mid, out, shape):
    chain, (x,) = W.config1_f16(seed=27, frames=shape[0], height=shape[1], width=shape[2], mid=mid, out=out)
    c = arol.Chain(chain)
    assert c.info["kernel"] == 1
    y = host(c.run([dev(x)]))
    xv = to_f64(x)
    ref = C.run_chain(chain, [xv])[0]
    hv = float(np.abs(chain[1]["taps"]).sum(axis=1).max())
    check(y, ref, fir_scale(chain, xv, C.run_chain), out == "f16", f"f16 chain {mid}/{out} {shape}",
          mid_abs_taps=hv if mid == "f16" else None)


def test_f16_chain_full_size(arol):
    chain, (x,) = W.config1_f16(seed=29)
    c = arol.Chain(chain)
    y = host(c.run([dev(x)]))
    xv = to_f64(x)
    check(y, C.run_chain(chain, [xv])[0], fir_scale(chain, xv, C.run_chain), True, "f16 chain 64x1080x1920")


def test_mixed_16bit_chain_runs_unfused(arol):
    """bfloat16 frames with a half output: two 16-bit types in one chain run
    task by task through the library's intermediate, and stay correct."""
    chain, (x,) = W.config1_bf16(seed=30, frames=2, height=16, width=64, mid="f32", out="f16")
    c = arol.Chain(chain)
    assert c.info["kernel"] == 3
    y = host(c.run([dev(x)]))
    assert y.dtype == np.float16
    xv = to_f64(x)
    tv = [values_task(t) for t in chain]
    check(y, O.run_chain(tv, [xv])[0], fir_scale(tv, xv), True, "bf16 frames, f16 output")


def test_batch_with_f16_member(arol):
    """A half task (generic path) among f32 row-FIR tasks (staged path)."""
    g = W.rng(313)
    params = [(5, 300, 9, 2, 5), (3, 1000, 16, 4, 8), (7, 64, 4, 1, 1)]
    tasks, xs = [], []
    for (h, w, T, m, S) in params:
        tasks.append(W.fir_row_task(h, w, T, m, S, (g.standard_normal((m, T)) / T).astype(np.float32)))
        xs.append(g.standard_normal((h, w)).astype(np.float32))
    tk = W.random_tiler_task(g, "fir")
    tk = dict(tk, inputs=[dict(tk["inputs"][0], dtype="f16")], outputs=[dict(tk["outputs"][0], dtype="f16")])
    xh = W.f16_round(g.standard_normal(tk["inputs"][0]["shape"]).astype(np.float32))
    b = arol.Batch(tasks + [tk])
    outs = b.empty_outputs()
    assert outs[-1].dtype == torch.float16
    b.run([dev(x) for x in xs] + [dev(xh)], outs)
    torch.cuda.synchronize()
    for t, x, y in zip(tasks, xs, outs[:-1]):
        check(host(y), C.run_task(t, [x])[0], fir_scale(t, x, C.run_chain), False, "row fir next to f16")
    xv = to_f64(xh)
    tv = values_task(tk)
    check(host(outs[-1]), O.run_task(tv, [xv])[0], fir_scale(tv, xv), True, "f16 member of a batch")


def test_f16_backward_against_oracle(arol):
    """IEEE half frames and output with a float32 intermediate: dX and the
    tap gradients in float32 against the oracle's adjoint on the widened
    values (the backward reads X in its storage)."""
    chain, (x,) = W.config1_f16(seed=31, frames=2, height=16, width=128, mid="f32", out="f16")
    c = arol.Chain(chain)
    xv = x.astype(np.float64)
    f32_chain = [dict(t, inputs=[dict(t["inputs"][0], dtype="f32")], outputs=[dict(t["outputs"][0], dtype="f32")])
                 for t in chain]
    G = W.rng(131).standard_normal(chain[-1]["outputs"][0]["shape"]).astype(np.float32)
    gx = torch.empty(x.shape, device="cuda")
    gt = torch.empty(48, device="cuda")
    c.backward(dev(G), [dev(x)], gx, gt)
    c.sync_status()
    g64 = G.astype(np.float64)
    dX, (dHh, dHv) = C.chain_vjp(f32_chain, [xv], g64)
    absc = [dict(t, taps=np.abs(np.asarray(t["taps"], np.float64))) for t in f32_chain]
    sX, (sHh, sHv) = C.chain_vjp(absc, [np.abs(xv)], np.abs(g64))
    assert_fir_close(host(gx), dX, sX, 1e-5, "f16 dX")
    got = host(gt)
    assert_fir_close(got[:24].reshape(3, 8), dHh, sHh, 1e-5, "f16 dHh")
    assert_fir_close(got[24:].reshape(3, 8), dHv, sHv, 1e-5, "f16 dHv")
