"""The seeded input recipes: sizes, ranges and types as stated for each
workload, the same draws for the same seed, and output tilers that partition
their arrays."""
import numpy as np

import workloads as W
from oracle import cpu_ref as C


def test_uneven_batch_recipe():
    params, _ = W.config3_params()
    assert len(params) == 512
    for (h, w, T, m, S) in params:
        assert 32 <= h <= 2048 and 32 <= w <= 2048
        assert 3 <= T <= 32 and 1 <= m <= T // 2 and m <= S <= T
    assert W.config3_params()[0] == params                       # same seed, same draws
    assert W.config3_params(seed=1)[0] != params
    tasks, xs = W.config3(n=24)
    for tk, x, (h, w, T, m, S) in zip(tasks, xs, params):
        assert x.shape == (h, w) and x.dtype == np.float32 and 0.0 <= x.min() and x.max() < 1.0
        assert tk["taps"].shape == (m, T)
        assert tk["rep"] == (h, -(-w // S))
        assert tk["outputs"][0]["shape"] == (h, m * -(-w // S))
        assert C.cover_ok(tk)


def test_chain_recipes():
    chain, (x,) = W.config1(frames=2, height=16, width=64)
    assert x.shape == (2, 16, 64) and x.dtype == np.float32
    assert chain[0]["outputs"][0]["shape"] == chain[1]["inputs"][0]["shape"] == (2, 16, 24)
    assert chain[1]["outputs"][0]["shape"] == (2, 6, 24)
    assert all(C.cover_ok(t) for t in chain)
    cb, (xb,) = W.config1_bf16(frames=1, height=8, width=64)
    assert xb.dtype == np.uint16 and cb[0]["inputs"][0]["dtype"] == "bf16"
    ch, (xh,) = W.config1_f16(frames=1, height=8, width=64)
    assert xh.dtype == np.float16 and ch[0]["inputs"][0]["dtype"] == "f16"
    # the 16-bit frames are the float32 draw rounded: the same seed gives the same values
    x32 = W.config1(frames=1, height=8, width=64)[1][0]
    np.testing.assert_array_equal(xh, x32.astype(np.float16))
    np.testing.assert_array_equal(xb, W.bf16_round(x32))


def test_batched_chain_recipe():
    chains, xs = W.chain_batch(n=16)
    assert len(chains) == 16
    for c, x in zip(chains, xs):
        _, h, w = x.shape
        assert h % 8 == 0 and w % 8 == 0 and 64 <= h <= 1024 and 64 <= w <= 2048
        assert c[1]["outputs"][0]["shape"] == (1, h // 8 * 3, w // 8 * 3)
        assert c[0]["taps"].shape == c[1]["taps"].shape == (3, 8)


def test_backward_and_matmul_recipes():
    chain, (x,), w = W.config4(frames=2, height=16, width=64)
    assert x.shape == (2, 16, 64) and w.shape == chain[1]["outputs"][0]["shape"] == (2, 6, 24)
    tk, (a, b) = W.config2(M=256, N=384, K=128)
    assert a.dtype == np.uint16 and a.shape == (256, 128) and b.shape == (128, 384)
    assert tk["rep"] == (2, 3) and tk["outputs"][0]["shape"] == (256, 384)
