"""Batches whose row-then-column chain members run together on the
streaming chain kernel (one launch over every such member, intermediates on
chip), mixed with single tasks and with chains that run stage by stage.
Every member against the C oracle; the one-launch path equals one launch per
member and a second run bit for bit; the same batch with the streaming
kernel switched off (stage by stage) agrees within the FIR tolerance."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cpu_ref as C
from tests.gpu_helpers import assert_fir_close, dev, fir_scale, host
from tests.test_parity_gpu import _three_task_chain

pytestmark = pytest.mark.gpu


def _members(g):
    out = []
    for _ in range(10):
        chain, shape = W.random_row_column_chain(g, max_rows=200, max_cols=900)
        out.append((chain, g.standard_normal(shape).astype(np.float32)))
    chain, (x,) = W.config1(seed=31, frames=2, height=48, width=256)   # 8 -> 3 step 8
    out.append((chain, x))
    chain, (x,) = W.config1_5to2(seed=32, frames=3, height=60, width=200)
    out.append((chain, x))
    tk, (x,) = W.config0(seed=33)
    out.append((tk, x))
    out.append((_three_task_chain(g), g.standard_normal((24, 32)).astype(np.float32)))
    return out


def _check(spec, x, y, what):
    chain = spec if isinstance(spec, list) else [spec]
    ref = C.run_chain(chain, [x])[0]
    assert_fir_close(y, ref, fir_scale(chain, x, C.run_chain), what=what)


def test_batch_of_streamed_chains(arol, monkeypatch):
    g = W.rng(130)
    members = _members(g)
    b = arol.Batch([m for m, _ in members])
    ins = [dev(x) for _, x in members]
    outs = b.empty_outputs()
    b.run(ins, outs)
    outs2 = b.empty_outputs()
    b.run_per_task(ins, outs2)
    outs3 = b.empty_outputs()
    b.run(ins, outs3)
    b.sync_status()
    monkeypatch.setenv("AROL_SEPSTREAM", "off")
    bs = arol.Batch([m for m, _ in members])
    outs4 = bs.empty_outputs()
    bs.run(ins, outs4)
    bs.sync_status()
    for n, ((spec, x), y, y2, y3, y4) in enumerate(zip(members, outs, outs2, outs3, outs4)):
        y = host(y)
        _check(spec, x, y, f"member {n}")
        np.testing.assert_array_equal(y, host(y2))
        np.testing.assert_array_equal(y, host(y3))
        _check(spec, x, host(y4), f"member {n}, stage by stage")


def test_chain_batch_small(arol):
    """The 128-chain workload's recipe, 24 members: uneven 8 -> 3 chains."""
    chains, xs = W.chain_batch(seed=3, n=24)
    b = arol.Batch(chains)
    outs = b.empty_outputs()
    b.run([dev(x) for x in xs], outs)
    b.sync_status()
    for n, (c, x, y) in enumerate(zip(chains, xs, outs)):
        _check(c, x, host(y), f"chain {n}")


def test_batched_downscaler_members_follow_alignment(arol):
    """8 -> 3 chain members run on the batched downscaler while their input
    is 16-byte aligned; a run with one member's input one float off a
    boundary takes that member stage by stage (tables and graph rebuilt),
    and a later aligned run returns to the batched kernel.  Every run
    against the C oracle."""
    g = W.rng(132)
    members = []
    for k in range(4):
        chain, (x,) = W.config1(seed=40 + k, frames=1 + k % 2, height=8 * (4 + 3 * k), width=8 * (16 + 11 * k))
        members.append((chain, x))
    tk = W.random_tiler_task(g, "fir")
    members.append((tk, g.standard_normal(tk["inputs"][0]["shape"]).astype(np.float32)))
    b = arol.Batch([m for m, _ in members])
    aligned = [dev(x) for _, x in members]
    for shift in (0, 1, 0):
        ins = list(aligned)
        if shift:
            x = members[2][1]
            buf = torch.zeros(x.size + shift, device="cuda")
            buf[shift:] = dev(x).reshape(-1)
            ins[2] = buf[shift:].view(x.shape)
        outs = b.empty_outputs()
        b.run(ins, outs)
        b.sync_status()
        for n, ((spec, x), y) in enumerate(zip(members, outs)):
            _check(spec, x, host(y), f"member {n}, shift {shift}")
