"""Parity of the fused separable chain kernels (kernel 4: 2 to 4 row and
column passes fused through shared-memory tiles; kernel 5: a row pass then a
column pass streamed by rows) with the C oracle: random chains
(any taps, outputs, step, origin, windows that wrap once or several times,
frames), the 5-tap -> 2 step-4 downscaler at 64 x 1080 x 1920, a three-task
chain, and the forward + backward entry on a general chain.  FIR outputs
within 1e-5 of the summed absolute terms (accumulation order differs from
the oracle's)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cpu_ref as C
from tests.gpu_helpers import assert_fir_close, dev, fir_scale, host

pytestmark = pytest.mark.gpu
RTOL = 1e-5


def _abs_chain(tasks):
    return [dict(t, taps=np.abs(np.asarray(t["taps"], np.float64))) for t in tasks]


def test_random_separable_chains(arol):
    g = W.rng(401)
    fused = 0
    for n in range(60):
        chain, shape = W.random_separable_chain(g)
        x = g.standard_normal(shape).astype(np.float32)
        c = arol.Chain(chain)
        fused += c.info["kernel"] in (4, 5)
        y = c.run([dev(x)])
        c.sync_status()
        assert_fir_close(host(y), C.run_chain(chain, [x])[0], fir_scale(chain, x, C.run_chain),
                         what=f"chain {n} ({len(chain)} passes)")
    assert fused >= 45   # chains whose regions outgrow shared memory run stage by stage (checked all the same)


@pytest.mark.parametrize("stream", ["on", "off"])
def test_5to2_step4_downscaler_full_size(arol, monkeypatch, stream):
    """64 frames of 1080 x 1920 through the streaming kernel and, with it
    switched off, through the tile kernel."""
    monkeypatch.setenv("AROL_SEPSTREAM", stream)
    chain, (x,) = W.config1_5to2()
    c = arol.Chain(chain)
    assert c.info["kernel"] == (5 if stream == "on" else 4)
    y = c.run([dev(x)])
    c.sync_status()
    assert_fir_close(host(y), C.run_chain(chain, [x])[0], fir_scale(chain, x, C.run_chain), what="5->2 step 4")


def test_three_pass_chain_with_frames(arol):
    """Row 6-tap -> 3 step 4, column 5-tap -> 2 step 4, row 3-tap -> 1 step 2
    with origin 1 (its windows wrap at the row end) on 3 frames."""
    g = W.rng(402)
    F, Hh, Ww = 3, 96, 160
    t1 = W.separable_pass((F, Hh, Ww), 1, 6, 3, 4, 0, Ww // 4, (g.standard_normal((3, 6)) / 6).astype(np.float32))
    s1 = t1["outputs"][0]["shape"]
    t2 = W.separable_pass(s1, 0, 5, 2, 4, 0, Hh // 4, (g.standard_normal((2, 5)) / 5).astype(np.float32))
    s2 = t2["outputs"][0]["shape"]
    t3 = W.separable_pass(s2, 1, 3, 1, 2, 1, s2[2] // 2, (g.standard_normal((1, 3)) / 3).astype(np.float32))
    chain = [t1, t2, t3]
    x = g.random((F, Hh, Ww)).astype(np.float32)
    c = arol.Chain(chain)
    assert c.info["kernel"] == 4
    y = c.run([dev(x)])
    c.sync_status()
    assert_fir_close(host(y), C.run_chain(chain, [x])[0], fir_scale(chain, x, C.run_chain), what="3-pass chain")


def test_fwd_bwd_on_a_general_chain(arol):
    """The forward + backward entry accepts every fir chain: on the 5 -> 2
    step-4 downscaler it matches the oracle's output and adjoint."""
    chain, (x,) = W.config1_5to2(seed=3, frames=2, height=64, width=96)
    G = W.rng(403).standard_normal(chain[-1]["outputs"][0]["shape"]).astype(np.float32)
    c = arol.Chain(chain)
    y = torch.empty(chain[-1]["outputs"][0]["shape"], device="cuda")
    gx = torch.empty(x.shape, device="cuda")
    gt = torch.empty(20, device="cuda")
    c.fwd_bwd([dev(x)], dev(G), y, gx, gt)
    c.sync_status()
    g64 = G.astype(np.float64)
    assert_fir_close(host(y), C.run_chain(chain, [x])[0], fir_scale(chain, x, C.run_chain), what="fwd_bwd y")
    dX, dHs = C.chain_vjp(chain, [x], g64)
    sX, sHs = C.chain_vjp(_abs_chain(chain), [np.abs(x)], np.abs(g64))
    assert_fir_close(host(gx), dX, sX, RTOL, "fwd_bwd dX")
    got = host(gt)
    assert_fir_close(got[:10].reshape(2, 5), dHs[0], sHs[0], RTOL, "fwd_bwd dHh")
    assert_fir_close(got[10:].reshape(2, 5), dHs[1], sHs[1], RTOL, "fwd_bwd dHv")


def test_backward_of_random_separable_chains(arol):
    """dX and every tap gradient of random separable chains (windows that
    wrap once or several times, any step, origin and frames) against the C
    oracle's adjoint: dX by each pass's transposed tiler as a gather."""
    g = W.rng(404)
    for n in range(25):
        chain, shape = W.random_separable_chain(g)
        x = g.standard_normal(shape).astype(np.float32)
        G = g.standard_normal(chain[-1]["outputs"][0]["shape"]).astype(np.float32)
        c = arol.Chain(chain)
        gx = torch.empty(x.shape, device="cuda")
        ntaps = sum(t["taps"].size for t in chain)
        gt = torch.empty(ntaps, device="cuda")
        c.backward(dev(G), [dev(x)], gx, gt)
        c.sync_status()
        g64 = G.astype(np.float64)
        dX, dHs = C.chain_vjp(chain, [x], g64)
        sX, sHs = C.chain_vjp(_abs_chain(chain), [np.abs(x)], np.abs(g64))
        assert_fir_close(host(gx), dX, sX, RTOL, f"chain {n} dX")
        got = host(gt)
        off = 0
        for dH, sH in zip(dHs, sHs):
            assert_fir_close(got[off:off + dH.size].reshape(dH.shape), dH, sH, RTOL, f"chain {n} dH")
            off += dH.size


@pytest.mark.parametrize("mh,Th,Sh,oh", [(1, 3, 2, 0), (2, 5, 4, 3), (4, 8, 4, 1), (2, 8, 3, 39)])
def test_row_column_chain_backward_partial_requests(arol, mh, Th, Sh, oh):
    """A row pass (1, 2 or 4 outputs per repetition, windows that wrap) then
    a column pass whose repetitions tile the rows, against the C oracle's
    adjoint.  dX alone (no tap gradients: the intermediate is not
    recomputed) and the tap gradients alone give the same bits as the call
    asking for both."""
    g = W.rng(420 + mh + Th)
    F, H, Wx, Rh = 2, 48, 40, 12
    row = W.separable_pass((F, H, Wx), 1, Th, mh, Sh, oh, Rh, (g.standard_normal((mh, Th)) / Th).astype(np.float32))
    col = W.separable_pass((F, H, mh * Rh), 0, 5, 2, 4, 4, H // 4, (g.standard_normal((2, 5)) / 5).astype(np.float32))
    chain = [row, col]
    x = g.standard_normal((F, H, Wx)).astype(np.float32)
    G = g.standard_normal(col["outputs"][0]["shape"]).astype(np.float32)
    c = arol.Chain(chain)
    ntaps = mh * Th + 10
    gx, gx1 = torch.empty(x.shape, device="cuda"), torch.empty(x.shape, device="cuda")
    gt, gt1 = torch.empty(ntaps, device="cuda"), torch.empty(ntaps, device="cuda")
    c.backward(dev(G), [dev(x)], gx, gt)
    c.backward(dev(G), [dev(x)], gx1, None)
    c.backward(dev(G), [dev(x)], None, gt1)
    c.sync_status()
    g64 = G.astype(np.float64)
    dX, dHs = C.chain_vjp(chain, [x], g64)
    sX, sHs = C.chain_vjp(_abs_chain(chain), [np.abs(x)], np.abs(g64))
    assert_fir_close(host(gx), dX, sX, RTOL, "dX")
    got = host(gt)
    assert_fir_close(got[:mh * Th].reshape(mh, Th), dHs[0], sHs[0], RTOL, "dH row pass")
    assert_fir_close(got[mh * Th:].reshape(2, 5), dHs[1], sHs[1], RTOL, "dH column pass")
    np.testing.assert_array_equal(host(gx1), host(gx))
    np.testing.assert_array_equal(host(gt1), got)
