"""Parity of the hand-written adjoint (through the C ABI) with the oracle
gradient and with FP64 finite differences.

Tolerance: every gradient element within 1e-5 of the sum of absolute terms
behind it (the FP64 oracle gradient on |H|, |X|, |G|).  The longest FP32
accumulation chain in a tap gradient is a per-thread sum of a few hundred
products followed by a log-depth tree, so its error stays below
~300 * 2^-24 < 2e-5 of that sum in the worst case and far below in practice.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cpu_ref as C
from oracle import tiler as O
from tests.gpu_helpers import assert_fir_close, dev, host

pytestmark = pytest.mark.gpu
RTOL = 1e-5


def _abs_chain(tasks):
    return [dict(t, taps=np.abs(np.asarray(t["taps"], np.float64))) for t in tasks]


def check_chain_grads(arol, tasks, x, g, vjp=O.chain_vjp):
    g = np.asarray(g, dtype=np.float32).astype(np.float64)   # the device gets float32
    c = arol.Chain(tasks) if len(tasks) > 1 else arol.Task(tasks[0])
    gx = torch.empty(x.shape, device="cuda")
    ntaps = sum(t["taps"].size for t in tasks)
    gt = torch.empty(ntaps, device="cuda")
    c.backward(dev(g.astype(np.float32)), [dev(x)], gx, gt)
    torch.cuda.synchronize()
    dX, dHs = vjp(tasks, [x], g) if len(tasks) > 1 else (lambda r: (r[0], [r[1]]))(O.task_vjp(tasks[0], [x], g))
    sX, sHs = (vjp(_abs_chain(tasks), [np.abs(x)], np.abs(g)) if len(tasks) > 1 else
               (lambda r: (r[0], [r[1]]))(O.task_vjp(_abs_chain(tasks)[0], [np.abs(x)], np.abs(g))))
    assert_fir_close(host(gx), dX, sX, RTOL, "dX")
    got = host(gt)
    off = 0
    for dH, sH in zip(dHs, sHs):
        n = dH.size
        assert_fir_close(got[off:off + n].reshape(dH.shape), dH, sH, RTOL, "dH")
        off += n
    return c, host(gx), got


def test_backward_config0_overlap_and_wrap(arol):
    tk, (x,) = W.config0()
    g = W.rng(201).standard_normal((64, 48))
    check_chain_grads(arol, [tk], x, g)


def test_backward_random_fir_tilers(arol):
    g = W.rng(202)
    for _ in range(25):
        tk = W.random_tiler_task(g, "fir")
        x = g.standard_normal(tk["inputs"][0]["shape"]).astype(np.float32)
        G = g.standard_normal(tk["outputs"][0]["shape"])
        check_chain_grads(arol, [tk], x, G)


@pytest.mark.parametrize("shape", [(1, 8, 8), (2, 16, 32), (3, 24, 40)])
def test_backward_fused_chain_small(arol, shape):
    chain, (x,) = W.config1(seed=11, frames=shape[0], height=shape[1], width=shape[2])
    G = W.rng(203).standard_normal(chain[-1]["outputs"][0]["shape"])
    c, _, _ = check_chain_grads(arol, chain, x, G)
    assert c.info["kernel"] == 1


def test_backward_overlapping_chain(arol):
    tk, (x,) = W.config0(seed=4)
    g = W.rng(204)
    nxt = W.task((64, 16), "fir", [W.port((64, 48), (0, 0), ((1, 0), (0, 3)), ((0,), (1,)), (3,))],
                 [W.port((64, 16), (0, 0), ((1, 0), (0, 1)), ((0,), (1,)), (1,))],
                 g.standard_normal((1, 3)).astype(np.float32))
    G = g.standard_normal((64, 16))
    c, _, _ = check_chain_grads(arol, [tk, nxt], x, G)
    assert c.info["kernel"] == 4


def test_backward_config4_full_size(arol):
    chain, (x,), w = W.config4()
    check_chain_grads(arol, chain, x, w.astype(np.float64), vjp=C.chain_vjp)


def test_fwd_bwd_config4_full_size_against_oracle(arol):
    """The fused forward+backward entry at the size it is timed at (16 frames
    of 1080 x 1920): output, dX and both tap gradients element by element
    against the C oracle's FP64 forward and adjoint."""
    chain, (x,), w = W.config4()
    c = arol.Chain(chain)
    xd, wd = dev(x), dev(w)
    y = torch.empty(chain[-1]["outputs"][0]["shape"], device="cuda")
    gx = torch.empty_like(xd)
    gt = torch.empty(48, device="cuda")
    c.fwd_bwd([xd], wd, y, gx, gt)
    c.sync_status()
    assert c.info["kernel"] == 1
    w64 = w.astype(np.float64)
    assert_fir_close(host(y), C.run_chain(chain, [x])[0],
                     C.run_chain(_abs_chain(chain), [np.abs(x).astype(np.float64)])[0], RTOL, "fwd_bwd y")
    dX, (dHh, dHv) = C.chain_vjp(chain, [x], w64)
    sX, (sHh, sHv) = C.chain_vjp(_abs_chain(chain), [np.abs(x)], np.abs(w64))
    assert_fir_close(host(gx), dX, sX, RTOL, "fwd_bwd dX")
    g = host(gt)
    assert_fir_close(g[:24].reshape(3, 8), dHh, sHh, RTOL, "fwd_bwd dHh")
    assert_fir_close(g[24:].reshape(3, 8), dHv, sHv, RTOL, "fwd_bwd dHv")


def test_fwd_bwd_equals_separate_calls_and_is_deterministic(arol):
    chain, (x,), w = W.config4(frames=2, height=64, width=128)
    c = arol.Chain(chain)
    xd, wd = dev(x), dev(w)
    y1 = c.run([xd])
    gx1 = torch.empty_like(xd)
    gt1 = torch.empty(48, device="cuda")
    c.backward(wd, [xd], gx1, gt1)
    y2 = torch.empty_like(y1)
    gx2 = torch.empty_like(xd)
    gt2 = torch.empty(48, device="cuda")
    c.fwd_bwd([xd], wd, y2, gx2, gt2)
    gx3 = torch.empty_like(xd)
    gt3 = torch.empty(48, device="cuda")
    c.backward(wd, [xd], gx3, gt3)
    torch.cuda.synchronize()
    # the fused kernel computes the forward exactly as the forward kernel does;
    # its gradients sum in another order (another thread layout): tolerance
    assert torch.equal(y1, y2)
    sX, (sHh, sHv) = O.chain_vjp(_abs_chain(chain), [np.abs(x)], np.abs(w.astype(np.float64)))
    assert_fir_close(host(gx2), host(gx1).astype(np.float64), sX, RTOL, "fwd_bwd dX")
    assert_fir_close(host(gt2), host(gt1).astype(np.float64),
                     np.concatenate([sHh.reshape(-1), sHv.reshape(-1)]), RTOL, "fwd_bwd dH")
    # the same call twice gives the same bits (no atomics in any sum)
    assert torch.equal(gx1, gx3) and torch.equal(gt1, gt3)


def test_backward_32x32_against_fp64_finite_differences(arol):
    """GPU gradient of loss = sum(W * out) on one 32x32 frame against FP64
    central differences of the oracle (exact up to rounding: the loss is
    linear in X and in every tap)."""
    g = W.rng(205)
    x = g.random((1, 32, 32)).astype(np.float32)
    Hh = (g.standard_normal((3, 8)) / 8).astype(np.float32)
    Hv = (g.standard_normal((3, 8)) / 8).astype(np.float32)
    chain = W.downscale_chain(1, 32, 32, Hh, Hv)
    Wt = g.standard_normal((1, 12, 12))
    c = arol.Chain(chain)
    gx = torch.empty((1, 32, 32), device="cuda")
    gt = torch.empty(48, device="cuda")
    c.backward(dev(Wt.astype(np.float32)), [dev(x)], gx, gt)
    torch.cuda.synchronize()
    gx, gt = host(gx), host(gt)
    x64 = x.astype(np.float64)
    c64 = [dict(t, taps=np.asarray(t["taps"], np.float64)) for t in chain]
    loss = lambda cc, xx: float(np.sum(O.run_chain(cc, [xx])[0] * Wt))
    h = 1e-3
    for idx in [(0, 0, 0), (0, 7, 30), (0, 31, 31), (0, 16, 9)]:
        xp, xm = x64.copy(), x64.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (loss(c64, xp) - loss(c64, xm)) / (2 * h)
        assert abs(gx[idx] - fd) <= 1e-5 * (1 + abs(fd)), (idx, gx[idx], fd)
    for n in range(2):
        for (j, k) in [(0, 0), (2, 7), (1, 4)]:
            cp = [dict(t, taps=t["taps"].copy()) for t in c64]
            cm = [dict(t, taps=t["taps"].copy()) for t in c64]
            cp[n]["taps"][j, k] += h
            cm[n]["taps"][j, k] -= h
            fd = (loss(cp, x64) - loss(cm, x64)) / (2 * h)
            assert abs(gt[24 * n + 8 * j + k] - fd) <= 1e-4 * (1 + abs(fd)), (n, j, k, gt[24 * n + 8 * j + k], fd)


def test_autograd_function(arol):
    chain, (x,), w = W.config4(seed=3, frames=2, height=32, width=64)
    c = arol.Chain(chain)
    xd = dev(x).requires_grad_(True)
    taps = torch.cat([dev(chain[0]["taps"]).reshape(-1), dev(chain[1]["taps"]).reshape(-1)]).requires_grad_(True)
    out = arol.apply_task(c, xd, taps)
    loss = (out * dev(w)).sum()
    loss.backward()
    dX, (dHh, dHv) = O.chain_vjp(chain, [x], w.astype(np.float64))
    sX, (sHh, sHv) = O.chain_vjp(_abs_chain(chain), [np.abs(x)], np.abs(w.astype(np.float64)))
    assert_fir_close(host(xd.grad), dX, sX, RTOL, "autograd dX")
    gt = host(taps.grad)
    assert_fir_close(gt[:24].reshape(3, 8), dHh, sHh, RTOL, "autograd dHh")
    assert_fir_close(gt[24:].reshape(3, 8), dHv, sHv, RTOL, "autograd dHv")


def test_misaligned_gradient_buffer_falls_back(arol):
    chain, (x,), w = W.config4(seed=6, frames=2, height=16, width=64)
    c = arol.Chain(chain)
    gbuf = torch.zeros(w.size + 1, device="cuda")
    gbuf[1:] = dev(w).reshape(-1)
    gx = torch.empty(x.shape, device="cuda")
    gt = torch.empty(48, device="cuda")
    c.backward(gbuf[1:].view(w.shape), [dev(x)], gx, gt)
    gx2 = torch.empty(x.shape, device="cuda")
    gt2 = torch.empty(48, device="cuda")
    c.backward(dev(w), [dev(x)], gx2, gt2)
    c.sync_status()
    sX, (sHh, sHv) = O.chain_vjp(_abs_chain(chain), [np.abs(x)], np.abs(w.astype(np.float64)))
    assert_fir_close(host(gx), host(gx2).astype(np.float64), sX, RTOL, "misaligned dL/dY")
    assert_fir_close(host(gt), host(gt2).astype(np.float64),
                     np.concatenate([sHh.reshape(-1), sHv.reshape(-1)]), RTOL, "misaligned dL/dY taps")


@pytest.mark.parametrize("axis,T,m,S,reps_mul", [(1, 5, 2, 4, 1), (0, 7, 3, 2, 3), (1, 20, 10, 6, 2), (0, 1, 1, 1, 1)])
def test_backward_separable_pass_tasks(arol, axis, T, m, S, reps_mul):
    """Single row or column FIR passes (the separable adjoint and tap-gradient
    kernels; m = 10 > 8 takes the owner-computes tap gradients), windows that
    wrap once or several times (reps_mul times the covering repetitions),
    against the C oracle's adjoint."""
    g = W.rng(206 + T)
    shape = (3, 37, 50)
    n = shape[2] if axis == 1 else shape[1]
    reps = reps_mul * -(-n // S)
    tk = W.separable_pass(shape, axis, T, m, S, 3 % n, reps, (g.standard_normal((m, T)) / T).astype(np.float32))
    x = g.standard_normal(shape).astype(np.float32)
    G = g.standard_normal(tk["outputs"][0]["shape"])
    check_chain_grads(arol, [tk], x, G)


@pytest.mark.parametrize("axis,T,m,S", [(1, 9, 2, 5), (0, 7, 3, 2), (0, 12, 4, 4), (1, 16, 8, 4)])
def test_backward_separable_pass_exact_tiling(arol, axis, T, m, S):
    """Repetitions that tile the axis exactly (S R = n): dX by the
    per-repetition adjoint, windows overlapping up to four repetitions and
    wrapping at the end, origin 5."""
    g = W.rng(230 + T)
    shape = (2, 36, 60)
    n = shape[2] if axis == 1 else shape[1]
    tk = W.separable_pass(shape, axis, T, m, S, 5, n // S, (g.standard_normal((m, T)) / T).astype(np.float32))
    x = g.standard_normal(shape).astype(np.float32)
    G = g.standard_normal(tk["outputs"][0]["shape"])
    check_chain_grads(arol, [tk], x, G)


@pytest.mark.parametrize("axis,T,m,S,width,dt", [
    (0, 5, 2, 4, 60, "f32"), (0, 8, 3, 4, 60, "f32"), (0, 5, 2, 4, 62, "f32"), (0, 6, 2, 3, 60, "bf16"),
    (1, 5, 2, 4, 60, "f32"), (1, 3, 1, 3, 60, "f16"), (1, 12, 4, 6, 60, "f32"), (1, 5, 2, 2, 62, "bf16"),
    (1, 4, 2, 2, 62, "f32"), (1, 8, 3, 8, 64, "f32")])
def test_backward_one_sweep_pass(arol, axis, T, m, S, width, dt):
    """Passes whose repetitions tile the axis (S R = n) with at most 4 outputs
    and 16 taps: dX and the tap gradients in one sweep over the data (column
    passes four columns at a time when the width is a multiple of 4, else the
    adjoint and tap-gradient kernels; row passes staged a row at a time, rows
    of 30 or 62 words alternating the 16-byte and the word-by-word staging;
    steps 2, 4 and 8 in their step-specialised forms), origin 5, inputs in
    f32, bfloat16 or IEEE half, against the oracle.  A
    call asking for dX alone or the tap gradients alone gives the same bits."""
    _one_sweep_case(arol, axis, T, m, S, width, dt, 5)


@pytest.mark.parametrize("T,m,S,width,origin,dt", [
    (5, 2, 4, 64, 16, "f32"), (8, 3, 8, 128, 0, "f32"), (6, 2, 2, 96, 32, "f32"), (7, 4, 4, 48, 0, "f32"),
    (5, 2, 4, 64, 0, "bf16")])
def test_backward_row_pass_regions(arol, T, m, S, width, origin, dt):
    """Row passes on rows of a multiple of 16 words, origin a multiple of 16,
    steps 2, 4 and 8: the 16-word-region form (swizzled 16-byte shared loads
    and stores, halos for the windows that wrap at either end of a row),
    against the oracle.  bfloat16 X: the tap gradients take the staged-row
    form and dX alone the region form, with the same dX bits."""
    _one_sweep_case(arol, 1, T, m, S, width, dt, origin)


def _one_sweep_case(arol, axis, T, m, S, width, dt, origin):
    g = W.rng(250 + T + width)
    shape = (2, 36, width)
    n = shape[2] if axis == 1 else shape[1]
    tk = W.separable_pass(shape, axis, T, m, S, origin, n // S, (g.standard_normal((m, T)) / T).astype(np.float32))
    xf = g.standard_normal(shape).astype(np.float32)
    if dt == "bf16":
        x = W.bf16_round(xf)
        xv = W.bf16_bits_to_f32(x)
    elif dt == "f16":
        x = xf.astype(np.float16)
        xv = x.astype(np.float32)
    else:
        x = xv = xf
    G = g.standard_normal(tk["outputs"][0]["shape"]).astype(np.float32)
    t = arol.Task(dict(tk, inputs=[dict(tk["inputs"][0], dtype=dt)]))
    gx, gx1 = torch.empty(shape, device="cuda"), torch.empty(shape, device="cuda")
    gt, gt1 = torch.empty(m * T, device="cuda"), torch.empty(m * T, device="cuda")
    t.backward(dev(G), [dev(x)], gx, gt)
    t.backward(dev(G), [dev(x)], gx1, None)
    t.backward(dev(G), [dev(x)], None, gt1)
    t.sync_status()
    g64 = G.astype(np.float64)
    dX, dH = O.task_vjp(tk, [xv], g64)
    sX, sH = O.task_vjp(_abs_chain([tk])[0], [np.abs(xv)], np.abs(g64))
    assert_fir_close(host(gx), dX, sX, RTOL, "dX")
    assert_fir_close(host(gt).reshape(m, T), dH, sH, RTOL, "dH")
    np.testing.assert_array_equal(host(gx1), host(gx))
    np.testing.assert_array_equal(host(gt1), host(gt))
