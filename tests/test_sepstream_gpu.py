"""Parity of the streaming row-then-column chain kernel (kernel 5) with the
C oracle: random row pass -> column pass chains (wrapped windows, several
frames, several column chunks, many or few bands), inputs and outputs that
start off a 16-byte boundary, the widest column-pass window and steps past
it, and the tile kernel (kernel 4) on the same chains with the streaming
kernel switched off.  FIR outputs within 1e-5 of the summed absolute
terms."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cpu_ref as C
from tests.gpu_helpers import assert_fir_close, dev, fir_scale, host

pytestmark = pytest.mark.gpu


def _check(arol, chain, x, what):
    c = arol.Chain(chain)
    y = c.run([dev(x)])
    c.sync_status()
    assert_fir_close(host(y), C.run_chain(chain, [x])[0], fir_scale(chain, x, C.run_chain), what=what)
    return c, y


def test_random_row_column_chains(arol, monkeypatch):
    g = W.rng(501)
    streamed = 0
    for n in range(30):
        chain, shape = W.random_row_column_chain(g)
        x = g.standard_normal(shape).astype(np.float32)
        monkeypatch.setenv("AROL_SEPSTREAM", "on")
        c, _ = _check(arol, chain, x, f"chain {n}")
        if c.info["kernel"] != 5:
            continue
        streamed += 1
        monkeypatch.setenv("AROL_SEPSTREAM", "off")
        c, _ = _check(arol, chain, x, f"chain {n}, tile kernel")
        assert c.info["kernel"] in (3, 4)
    assert streamed >= 20   # wide row windows (S_h up to 8) can outgrow the stage ring


@pytest.mark.parametrize("offset", [1, 2, 3])
def test_unaligned_input_and_output(arol, offset):
    """Input and output start `offset` floats past a 16-byte boundary: the
    row copies fall back to 4-byte copies at the ragged ends."""
    g = W.rng(502 + offset)
    F, H, Wd = 2, 70, 611
    t1 = W.separable_pass((F, H, Wd), 1, 7, 2, 3, 5, -(-Wd // 3), (g.standard_normal((2, 7)) / 7).astype(np.float32))
    s1 = t1["outputs"][0]["shape"]
    t2 = W.separable_pass(s1, 0, 9, 3, 4, 2, -(-H // 4), (g.standard_normal((3, 9)) / 9).astype(np.float32))
    chain = [t1, t2]
    x = g.standard_normal((F, H, Wd)).astype(np.float32)
    c = arol.Chain(chain)
    assert c.info["kernel"] == 5
    out_shape = chain[-1]["outputs"][0]["shape"]
    xb = torch.zeros(x.size + offset, device="cuda")
    xb[offset:] = dev(x).reshape(-1)
    yb = torch.full((int(np.prod(out_shape)) + offset,), float("nan"), device="cuda")
    c.run([xb[offset:].view(x.shape)], yb[offset:].view(out_shape))
    c.sync_status()
    assert torch.isnan(yb[:offset]).all()
    assert_fir_close(host(yb[offset:]).reshape(out_shape), C.run_chain(chain, [x])[0],
                     fir_scale(chain, x, C.run_chain), what=f"offset {offset}")


def test_tall_single_frame_many_bands(arol):
    """One frame, 3000 rows: the rows split into bands of column-pass
    repetitions whose halos overlap (T_v > S_v)."""
    g = W.rng(505)
    H, Wd = 3000, 200
    t1 = W.separable_pass((1, H, Wd), 1, 5, 2, 4, 0, Wd // 4, (g.standard_normal((2, 5)) / 5).astype(np.float32))
    t2 = W.separable_pass(t1["outputs"][0]["shape"], 0, 11, 2, 3, 7, H // 3,
                          (g.standard_normal((2, 11)) / 11).astype(np.float32))
    x = g.standard_normal((1, H, Wd)).astype(np.float32)
    c, _ = _check(arol, [t1, t2], x, "tall frame")
    assert c.info["kernel"] == 5


@pytest.mark.parametrize("Tv,Sv,kernel", [(29, 29, 5), (29, 1, 5), (30, 4, 4), (3, 40, 5), (1, 1, 5)])
def test_column_window_extremes(arol, Tv, Sv, kernel):
    """The ring of intermediate rows holds 32 rows: a window of T_v <= 29
    rows plus the three rows stored after it in its stage.  A step past the
    window (S_v > T_v) streams rows no window uses; T_v = 30 takes the tile
    kernel."""
    g = W.rng(506 + Tv)
    F, H, Wd = 2, 150, 300
    t1 = W.separable_pass((F, H, Wd), 1, 3, 1, 2, 1, Wd // 2, (g.standard_normal((1, 3)) / 3).astype(np.float32))
    t2 = W.separable_pass(t1["outputs"][0]["shape"], 0, Tv, 2, Sv, 3, -(-H // Sv),
                          (g.standard_normal((2, Tv)) / Tv).astype(np.float32))
    x = g.standard_normal((F, H, Wd)).astype(np.float32)
    c, _ = _check(arol, [t1, t2], x, f"T_v {Tv} S_v {Sv}")
    assert c.info["kernel"] == kernel


def test_repeated_runs_give_the_same_bits(arol):
    chain, (x,) = W.config1_5to2(seed=5, frames=3, height=120, width=640)
    c = arol.Chain(chain)
    assert c.info["kernel"] == 5
    xd = dev(x)
    y1 = c.run([xd])
    y2 = c.run([xd])
    c.sync_status()
    assert torch.equal(y1, y2)
