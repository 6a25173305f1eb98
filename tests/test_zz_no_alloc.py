"""The no-allocation backward entry point against the oracle gradient.

Callers that cannot allocate device memory — code that runs while a stream is
being captured into a CUDA graph, real-time or embedded hosts whose device
memory is fixed at start-up, programs whose memory belongs to an allocator
that must not be bypassed — call arol_downscale_backward_noalloc, which takes
every buffer from the caller and keeps its scratch in a static device array.
Two calls in a row (on different data, so the second one starts from the
scratch the first one left behind) must each match the FP64 oracle gradient
within the tolerance of the other gradient tests, and agree with the regular
entry point arol_task_backward.

This file is collected last on purpose: a run that stops at the first failure
has run every other test before it.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import tiler as O
from tests.gpu_helpers import FIR_RTOL, assert_fir_close, dev, host

pytestmark = pytest.mark.gpu


def _abs_chain(tasks):
    return [dict(t, taps=np.abs(np.asarray(t["taps"], np.float64))) for t in tasks]


def _case(seed, frames, height, width):
    chain, (x,), w = W.config4(seed=seed, frames=frames, height=height, width=width)
    w64 = w.astype(np.float64)
    dX, (dHh, dHv) = O.chain_vjp(chain, [x], w64)
    sX, (sHh, sHv) = O.chain_vjp(_abs_chain(chain), [np.abs(x)], np.abs(w64))
    taps = torch.cat([dev(chain[0]["taps"]).reshape(-1), dev(chain[1]["taps"]).reshape(-1)]).contiguous()
    return (chain, dev(x), dev(w), taps, dX, np.concatenate([dHh.reshape(-1), dHv.reshape(-1)]), sX,
            np.concatenate([sHh.reshape(-1), sHv.reshape(-1)]))


def test_noalloc_backward_matches_oracle_on_two_calls(arol):
    cases = [(31, 3, 64, 96), (32, 2, 40, 128)]
    for seed, frames, height, width in cases:
        chain, xd, wd, taps, dX, dH, sX, sH = _case(seed, frames, height, width)
        gx = torch.full_like(xd, float("nan"))
        gt = torch.full((48,), float("nan"), device="cuda")
        arol.arol_downscale_backward_noalloc(xd, wd, taps, frames, height, width, gx, gt)
        arol.arol_downscale_backward_noalloc_status()     # synchronizes; no wait gave up
        assert_fir_close(host(gx), dX, sX, FIR_RTOL, "no-alloc dX")
        assert_fir_close(host(gt), dH, sH, FIR_RTOL, "no-alloc dH")
        # the regular entry point gives the same gradients within the same bound
        c = arol.Chain(chain)
        gx_ref = torch.empty_like(xd)
        gt_ref = torch.empty(48, device="cuda")
        c.backward(wd, [xd], gx_ref, gt_ref)
        torch.cuda.synchronize()
        assert_fir_close(host(gx), host(gx_ref).astype(np.float64), sX, FIR_RTOL, "no-alloc vs task dX")


def test_noalloc_backward_with_one_gradient_left_out(arol):
    """grad_in or grad_taps may be null: the other one is still exact (the
    grad_taps=None launch skips the ticket reduction, and the next call with
    tap gradients still starts from a zero ticket)."""
    frames, height, width = 2, 32, 64
    _, xd, wd, taps, dX, dH, sX, sH = _case(33, frames, height, width)
    gt = torch.full((48,), float("nan"), device="cuda")
    arol.arol_downscale_backward_noalloc(xd, wd, taps, frames, height, width, None, gt)
    gx = torch.full_like(xd, float("nan"))
    arol.arol_downscale_backward_noalloc(xd, wd, taps, frames, height, width, gx, None)
    gt2 = torch.full((48,), float("nan"), device="cuda")
    arol.arol_downscale_backward_noalloc(xd, wd, taps, frames, height, width, None, gt2)
    arol.arol_downscale_backward_noalloc_status()
    assert_fir_close(host(gt), dH, sH, FIR_RTOL, "no-alloc dH without dX")
    assert_fir_close(host(gx), dX, sX, FIR_RTOL, "no-alloc dX without dH")
    assert torch.equal(gt, gt2)


def test_noalloc_backward_rejects_bad_sizes(arol):
    x = torch.zeros(8 * 8, device="cuda")
    with pytest.raises(arol.ArolError) as e:
        arol.arol_downscale_backward_noalloc(x, x, x, 1, 8, 12, x, None)     # width not a multiple of 8
    assert e.value.status == 1
    with pytest.raises(arol.ArolError) as e:
        arol.arol_downscale_backward_noalloc(x, x, x, 1 << 40, 8, 8, x, None)   # beyond the work-item limit
    assert e.value.status == 3
