"""bfloat16 storage (Sec. 5 typeAllocation) for FIR tasks and the fused chain.

The arithmetic stays f32.  Inputs stored as bfloat16 are widened exactly (the
oracle reads the same values); every store into a bfloat16 array rounds to
nearest even.  bfloat16 keeps 8 significant bits, so rounding to nearest
errs by at most 2^-8 of the stored magnitude.  Tolerance per element: 1e-5 of
the summed absolute terms (the f32 bound of the other tests), plus 2^-8 of
that sum for a rounded intermediate, plus 2^-8 |y| for the rounded output.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cpu_ref as C
from oracle import tiler as O
from tests.gpu_helpers import FIR_RTOL, assert_fir_close, dev, fir_scale, host

pytestmark = pytest.mark.gpu


def to_f64(y):
    return W.bf16_bits_to_f32(y).astype(np.float64) if y.dtype == np.uint16 else y.astype(np.float64)


def check(y, y64, scale, mid_rounded, out_bf16, what):
    tol = (FIR_RTOL + (2.0 ** -8 if mid_rounded else 0.0)) * scale + (2.0 ** -8 * np.abs(y64) if out_bf16 else 0.0)
    err = np.abs(to_f64(y) - y64)
    bad = err > tol + 1e-38
    assert not bad.any(), f"{what}: {int(bad.sum())} of {bad.size} out of tolerance"


@pytest.mark.parametrize("dt_in,dt_out", [("bf16", "bf16"), ("bf16", "f32"), ("f32", "bf16")])
def test_generic_fir_bf16_storage(arol, dt_in, dt_out):
    g = W.rng(301)
    for _ in range(25):
        tk = W.random_tiler_task(g, "fir", fir_pattern_rank=int(g.integers(1, 3)))
        tk = dict(tk, inputs=[dict(tk["inputs"][0], dtype=dt_in)], outputs=[dict(tk["outputs"][0], dtype=dt_out)])
        xf = g.standard_normal(tk["inputs"][0]["shape"]).astype(np.float32)
        x = W.bf16_round(xf) if dt_in == "bf16" else xf
        t = arol.Task(tk)
        y = host(t.run([dev(x)]))
        torch.cuda.synchronize()
        # the oracle reads the same values: exact widening of the stored bits
        xv = to_f64(x)
        tk_v = dict(tk, inputs=[dict(tk["inputs"][0], dtype="f32")])
        check(y, O.run_task(tk_v, [xv])[0], fir_scale(tk_v, xv), False, dt_out == "bf16", f"{dt_in}->{dt_out}")


@pytest.mark.parametrize("mid,out", [("f32", "bf16"), ("bf16", "bf16"), ("f32", "f32"), ("bf16", "f32")])
@pytest.mark.parametrize("shape", [(1, 8, 64), (2, 24, 136), (3, 16, 1928)])
def test_fused_bf16_chain(arol, mid, out, shape):
    chain, (x,) = W.config1_bf16(seed=17, frames=shape[0], height=shape[1], width=shape[2], mid=mid, out=out)
    c = arol.Chain(chain)
    assert c.info["kernel"] == 1
    y = host(c.run([dev(x)]))
    xv = to_f64(x)
    ref = C.run_chain(chain, [xv])[0]
    check(y, ref, fir_scale(chain, xv, C.run_chain), mid == "bf16", out == "bf16", f"bf16 chain {mid}/{out} {shape}")


def test_f32_frames_with_bf16_output_run_unfused(arol):
    chain, (x,) = W.config1(seed=18, frames=2, height=16, width=64)
    chain = W.downscale_chain(2, 16, 64, chain[0]["taps"], chain[1]["taps"], dtypes=("f32", "f32", "bf16"))
    c = arol.Chain(chain)
    assert c.info["kernel"] == 3
    y = host(c.run([dev(x)]))
    check(y, O.run_chain(chain, [x])[0], fir_scale(chain, x), False, True, "unfused bf16 output")


def test_bf16_chain_full_size(arol):
    chain, (x,) = W.config1_bf16(seed=19)
    c = arol.Chain(chain)
    y = host(c.run([dev(x)]))
    xv = to_f64(x)
    check(y, C.run_chain(chain, [xv])[0], fir_scale(chain, xv, C.run_chain), False, True, "bf16 chain 64x1080x1920")


def test_bf16_backward_against_oracle(arol):
    """bfloat16 frames with a float32 intermediate: the backward reads X in
    its storage (widened exactly) and gives float32 dX and tap gradients,
    against the oracle's adjoint on the widened values."""
    chain, (x,) = W.config1_bf16(seed=20, frames=2, height=24, width=96, mid="f32", out="bf16")
    c = arol.Chain(chain)
    xv = to_f64(x)
    f32_chain = [dict(t, inputs=[dict(t["inputs"][0], dtype="f32")], outputs=[dict(t["outputs"][0], dtype="f32")])
                 for t in chain]
    G = W.rng(122).standard_normal(chain[-1]["outputs"][0]["shape"]).astype(np.float32)
    gx = torch.empty(x.shape, device="cuda")
    gt = torch.empty(48, device="cuda")
    c.backward(dev(G), [dev(x)], gx, gt)
    c.sync_status()
    g64 = G.astype(np.float64)
    dX, (dHh, dHv) = C.chain_vjp(f32_chain, [xv], g64)
    absc = [dict(t, taps=np.abs(np.asarray(t["taps"], np.float64))) for t in f32_chain]
    sX, (sHh, sHv) = C.chain_vjp(absc, [np.abs(xv)], np.abs(g64))
    assert_fir_close(host(gx), dX, sX, 1e-5, "bf16 dX")
    got = host(gt)
    assert_fir_close(got[:24].reshape(3, 8), dHh, sHh, 1e-5, "bf16 dHh")
    assert_fir_close(got[24:].reshape(3, 8), dHv, sHv, 1e-5, "bf16 dHv")


def test_bf16_intermediate_backward_is_rejected(arol):
    chain, (x,) = W.config1_bf16(seed=21, frames=1, height=8, width=64, mid="bf16", out="f32")
    c = arol.Chain(chain)
    with pytest.raises(arol.ArolError) as e:
        c.backward(torch.zeros(1, 3, 24, device="cuda"), [dev(x)], torch.empty(1, 8, 64, device="cuda"), None)
    assert e.value.status == 3
