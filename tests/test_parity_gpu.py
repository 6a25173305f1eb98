"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bit-exact for gather/scatter (copy tasks, NaN payloads included); FP32 FIR
within 1e-5 of the summed absolute terms per element (see gpu_helpers);
matmul within 2e-2 of the FP64 result (per element, scaled by (|A||B|)_ij, and
normwise) with an FP32-accumulation check of 1e-4 normwise on top.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cpu_ref as C
from oracle import tiler as O
from tests.gpu_helpers import assert_fir_close, dev, fir_scale, host

pytestmark = pytest.mark.gpu


def run1(A, spec, xs, out=None):
    t = A.Task(spec)
    ins = [dev(x) for x in xs]
    y = t.run(ins, out)
    torch.cuda.synchronize()
    return t, host(y)


# ------------------------------------------------------------ single tasks

def test_config0_fir(arol):
    tk, (x,) = W.config0()
    t, y = run1(arol, tk, [x])
    assert t.info["kernel"] == 0
    y64 = O.run_task(tk, [x])[0]
    assert_fir_close(y, y64, fir_scale(tk, x), what="config0")


def test_random_copy_tilers_bit_exact(arol):
    g = W.rng(101)
    for n in range(80):
        tk = W.random_tiler_task(g, "copy")
        x = g.random(tk["inputs"][0]["shape"], dtype=np.float32)
        raw = x.reshape(-1).view(np.uint32)
        raw[:: max(1, raw.size // 3)] = 0x7FA00001 + n     # NaN payloads must survive
        _, y = run1(arol, tk, [x])
        ref = O.run_task(tk, [x])[0]
        np.testing.assert_array_equal(y.view(np.uint32), ref.view(np.uint32))


def test_random_bf16_copy_tilers_bit_exact(arol):
    g = W.rng(102)
    for _ in range(30):
        tk = W.random_tiler_task(g, "copy")
        tk = dict(tk, inputs=[dict(tk["inputs"][0], dtype="bf16")], outputs=[dict(tk["outputs"][0], dtype="bf16")])
        bits = g.integers(0, 65536, size=tk["inputs"][0]["shape"], dtype=np.uint16)
        _, y = run1(arol, tk, [bits])
        np.testing.assert_array_equal(y, O.run_task(tk, [bits])[0])


def test_random_fir_tilers(arol):
    g = W.rng(103)
    for _ in range(60):
        tk = W.random_tiler_task(g, "fir")
        x = g.standard_normal(tk["inputs"][0]["shape"]).astype(np.float32)
        _, y = run1(arol, tk, [x])
        assert_fir_close(y, O.run_task(tk, [x])[0], fir_scale(tk, x), what="random fir")


def test_tiled_walk_long_repetition_rows(arol):
    """Repetition spaces up to 300 along their last dimension on arrays up to
    64 wide: the block-tiled walk gives each thread several repetitions 2^lb
    apart, some of whose patterns wrap and some not.  Copies bit-exact (f32
    and bf16 words), fir banks (m up to 16) against the C oracle."""
    g = W.rng(110)
    for n in range(40):
        elem = "copy" if n % 2 == 0 else "fir"
        tk = W.random_tiler_task(g, elem, max_side=64, max_rep=300)
        if elem == "copy" and n % 4 == 0:
            tk = dict(tk, inputs=[dict(tk["inputs"][0], dtype="bf16")], outputs=[dict(tk["outputs"][0], dtype="bf16")])
            x = g.integers(0, 65536, size=tk["inputs"][0]["shape"], dtype=np.uint16)
        elif elem == "copy":
            x = g.random(tk["inputs"][0]["shape"], dtype=np.float32)
        else:
            x = g.standard_normal(tk["inputs"][0]["shape"]).astype(np.float32)
        _, y = run1(arol, tk, [x])
        ref = C.run_task(tk, [x])[0]
        if elem == "copy":
            np.testing.assert_array_equal(y.view(np.uint16 if x.dtype == np.uint16 else np.uint32),
                                          ref.view(np.uint16 if x.dtype == np.uint16 else np.uint32))
        else:
            assert_fir_close(y, ref, fir_scale(tk, x, C.run_chain), what=f"long-row fir {n}")


def test_diagonal_tiler_with_wrapping_rows(arol):
    """The diagonal 8-element patterns of the generic bench case on 3 frames
    of 40 x 256: the last 7 rows' patterns wrap to the top (the wrapping
    walk), the rest take the linear walk."""
    tk, (x,) = W.diagonal_fir(seed=2, frames=3, height=40, width=256)
    _, y = run1(arol, tk, [x])
    assert_fir_close(y, C.run_task(tk, [x])[0], fir_scale(tk, x, C.run_chain), what="diagonal")


def test_fir_bank_sizes(arol):
    """m from 1 to 32 (every register-bank instantiation), T up to 64."""
    g = W.rng(104)
    for (T, m, S) in [(3, 1, 1), (8, 3, 4), (16, 5, 8), (17, 8, 9), (32, 16, 16), (40, 9, 12), (64, 32, 32)]:
        H = (g.standard_normal((m, T)) / T).astype(np.float32)
        tk = W.fir_row_task(7, 97, T, m, S, H)
        x = g.random((7, 97), dtype=np.float32)
        _, y = run1(arol, tk, [x])
        assert_fir_close(y, O.run_task(tk, [x])[0], fir_scale(tk, x), what=f"T={T} m={m}")


def test_empty_task_is_a_no_op(arol):
    p_in = W.port((4,), (0,), ((1,),), ((1,),), (1,))
    p_out = W.port((0,), (0,), ((1,),), ((1,),), (1,))
    t = arol.Task(W.task((0,), "copy", [p_in], [p_out]))
    y = t.run([torch.zeros(4, device="cuda")])
    torch.cuda.synchronize()
    assert y.numel() == 0


def test_identity_round_trip(arol):
    g = W.rng(105)
    x = g.random((33, 41), dtype=np.float32)
    p = W.port((33, 41), (-5, 17), ((1, 0), (0, 1)), ((0,), (0,)), (1,))
    _, y = run1(arol, W.task((33, 41), "copy", [p], [p]), [x])
    np.testing.assert_array_equal(y.view(np.uint32), x.view(np.uint32))


# ------------------------------------------------------------------ chains

@pytest.mark.parametrize("shape", [(1, 8, 8), (2, 16, 32), (3, 24, 40), (1, 64, 136), (2, 8, 1928)])
def test_fused_chain_small(arol, shape):
    chain, (x,) = W.config1(seed=7, frames=shape[0], height=shape[1], width=shape[2])
    c = arol.Chain(chain)
    assert c.info["kernel"] == 1
    y = host(c.run([dev(x)]))
    ref = (C.run_chain if x.size > 50000 else O.run_chain)(chain, [x])[0]
    assert_fir_close(y, ref, fir_scale(chain, x, C.run_chain), what=f"chain {shape}")


def test_fused_chain_rank2_frame(arol):
    g = W.rng(106)
    x = g.random((24, 48), dtype=np.float32)
    Hh = (g.standard_normal((3, 8)) / 8).astype(np.float32)
    Hv = (g.standard_normal((3, 8)) / 8).astype(np.float32)
    h = W.task((24, 6), "fir", [W.port((24, 48), (0, 0), ((1, 0), (0, 8)), ((0,), (1,)), (8,))],
               [W.port((24, 18), (0, 0), ((1, 0), (0, 3)), ((0,), (1,)), (3,))], Hh)
    v = W.task((3, 18), "fir", [W.port((24, 18), (0, 0), ((8, 0), (0, 1)), ((1,), (0,)), (8,))],
               [W.port((9, 18), (0, 0), ((3, 0), (0, 1)), ((1,), (0,)), (3,))], Hv)
    c = arol.Chain([h, v])
    assert c.info["kernel"] == 1
    y = host(c.run([dev(x)]))
    assert_fir_close(y, O.run_chain([h, v], [x])[0], fir_scale([h, v], x), what="rank-2 chain")


def test_config1_full_size(arol):
    """64 frames of 1080x1920, the full workload, against the C oracle."""
    chain, (x,) = W.config1()
    c = arol.Chain(chain)
    y = host(c.run([dev(x)]))
    ref = C.run_chain(chain, [x])[0]
    assert_fir_close(y, ref, fir_scale(chain, x, C.run_chain), what="config1 full")


def test_fused_chain_with_overlap_and_wrap(arol):
    tk, (x,) = W.config0(seed=3)
    g = W.rng(107)
    nxt = W.task((64, 16), "fir", [W.port((64, 48), (0, 0), ((1, 0), (0, 3)), ((0,), (1,)), (3,))],
                 [W.port((64, 16), (0, 0), ((1, 0), (0, 1)), ((0,), (1,)), (1,))],
                 g.standard_normal((1, 3)).astype(np.float32))
    c = arol.Chain([tk, nxt])
    assert c.info["kernel"] == 4
    y = host(c.run([dev(x)]))
    assert_fir_close(y, O.run_chain([tk, nxt], [x])[0], fir_scale([tk, nxt], x), what="fused overlapping chain")


def test_unfused_chain(arol):
    from tests.test_abi_host import unfusable_chain
    chain = unfusable_chain()
    x = W.rng(108).standard_normal((16, 16)).astype(np.float32)
    c = arol.Chain(chain)
    assert c.info["kernel"] == 3
    y = host(c.run([dev(x)]))
    assert_fir_close(y, O.run_chain(chain, [x])[0], fir_scale(chain, x), what="unfused chain")


def test_misaligned_input_takes_the_unfused_path(arol):
    chain, (x,) = W.config1(seed=8, frames=2, height=16, width=32)
    c = arol.Chain(chain)
    buf = torch.zeros(x.size + 1, device="cuda")
    buf[1:] = dev(x).reshape(-1)
    y = host(c.run([buf[1:].view(x.shape)]))
    assert_fir_close(y, O.run_chain(chain, [x])[0], fir_scale(chain, x), what="misaligned")


def test_run_host_matches_run(arol):
    chain, (x,) = W.config1(seed=9, frames=3, height=32, width=64)
    c = arol.Chain(chain)
    y_dev = host(c.run([dev(x)]))
    out = np.empty(chain[-1]["outputs"][0]["shape"], dtype=np.float32)
    c.run_host([x], out)
    np.testing.assert_array_equal(out, y_dev)
    tk, (x0,) = W.config0()
    t = arol.Task(tk)
    out0 = np.empty((64, 48), np.float32)
    t.run_host([x0], out0)
    np.testing.assert_array_equal(out0, host(t.run([dev(x0)])))


# ------------------------------------------------------------------ matmul

def _check_matmul(A_bits, B_bits, Cg, rows=None, cols=None, tk=None):
    if rows is None:
        Af = W.bf16_bits_to_f32(A_bits).astype(np.float64)
        Bf = W.bf16_bits_to_f32(B_bits).astype(np.float64)
        ref = Af @ Bf
        scale = np.abs(Af) @ np.abs(Bf)
        got = Cg.astype(np.float64)
    else:
        ref, scale = C.matmul_sample(tk, A_bits, B_bits, rows, cols)
        got = Cg[rows, cols].astype(np.float64)
    err = np.abs(got - ref)
    assert np.all(err <= 2e-2 * scale + 1e-30), float(np.max(err / scale))
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= 2e-2
    assert rel <= 1e-4, rel      # FP32 accumulation of exact bf16 products
    return rel


@pytest.mark.parametrize("mnk", [(128, 128, 64), (256, 256, 64), (256, 384, 192), (512, 512, 512), (384, 768, 1024),
                                 (768, 2048, 320)])
def test_matmul_full(arol, mnk):
    M, N, K = mnk
    g = W.rng(108)
    a = W.bf16_round(g.standard_normal((M, K), dtype=np.float32))
    b = W.bf16_round(g.standard_normal((K, N), dtype=np.float32))
    tk = W.matmul_task(M, N, K)
    t = arol.Task(tk)
    assert t.info["kernel"] == 2
    c = t.run([dev(a), dev(b)])
    t.sync_status()
    _check_matmul(a, b, host(c))


def test_matmul_4096_sampled(arol):
    tk, (a, b) = W.config2()
    t = arol.Task(tk)
    c = t.run([dev(a), dev(b)])
    t.sync_status()
    Cg = host(c)
    g = W.rng(109)
    rows = g.integers(0, 4096, 1024)
    cols = g.integers(0, 4096, 1024)
    # four whole 128x128 tiles: corners and one interior tile
    for (r0, c0) in [(0, 0), (31, 31), (0, 31), (17, 9)]:
        rr, cc = np.meshgrid(np.arange(128) + 128 * r0, np.arange(128) + 128 * c0, indexing="ij")
        rows = np.concatenate([rows, rr.reshape(-1)])
        cols = np.concatenate([cols, cc.reshape(-1)])
    _check_matmul(a, b, Cg, rows, cols, tk)


_MATMUL_SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
import paper_1105_4424_gb300 as A, workloads as W
M, N, K = 768, 2048, 320
g = W.rng(111)
a = W.bf16_round(g.standard_normal((M, K), dtype=np.float32))
b = W.bf16_round(g.standard_normal((K, N), dtype=np.float32))
t = A.Task(W.matmul_task(M, N, K))
bf = lambda u: torch.from_numpy(u.view(np.int16)).cuda().view(torch.bfloat16)
c = t.run([bf(a), bf(b)])
t.sync_status()
np.savez(sys.argv[2], a=a, b=b, c=c.cpu().numpy())
"""


@pytest.mark.parametrize("env", [{"AROL_MATMUL_MAX_CLUSTERS": "7"}, {"AROL_MATMUL_MAX_CLUSTERS": "5"},
                                 {"AROL_MATMUL_PAIR": "0"}])
def test_matmul_schedules(arol, tmp_path, env):
    """24 tiles of 256 x 256 on 7 clusters: three rounds of whole tiles and a
    fourth of half-width tiles; on 5 clusters: five rounds, no split; and the
    one-SM kernel.  All against the FP64 product."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    f = str(tmp_path / "mm.npz")
    subprocess.run([sys.executable, "-c", _MATMUL_SCRIPT, root, f], check=True, env=dict(os.environ, **env), timeout=300)
    o = np.load(f)
    _check_matmul(o["a"], o["b"], o["c"])


# ------------------------------------------------------------------ batches

def test_batch_config3_matches_per_task_and_oracle(arol):
    tasks, xs = W.config3()
    b = arol.Batch(tasks)
    ins = [dev(x) for x in xs]
    outs = b.empty_outputs()
    b.run(ins, outs)
    outs2 = b.empty_outputs()
    b.run_per_task(ins, outs2)
    torch.cuda.synchronize()
    # every instance against the C oracle (the per-task launches run the same
    # kernel body, so equality with them alone would check the path against itself)
    for i, (tk, x) in enumerate(zip(tasks, xs)):
        y = host(outs[i])
        assert_fir_close(y, C.run_task(tk, [x])[0], fir_scale(tk, x, C.run_chain), what=f"instance {i}")
        np.testing.assert_array_equal(y, host(outs2[i]))
    # the autotuner changes the tiling, not the results; new buffers refresh the table
    b.tune(ins, outs, force=True)
    outs3 = b.empty_outputs()
    b.run(ins, outs3)
    torch.cuda.synchronize()
    for i in range(len(tasks)):
        np.testing.assert_array_equal(host(outs3[i]), host(outs2[i]))


def test_batch_of_random_tilers(arol):
    g = W.rng(110)
    tasks = [W.random_tiler_task(g, "fir" if i % 2 else "copy") for i in range(40)]
    xs = [g.random(t["inputs"][0]["shape"], dtype=np.float32) for t in tasks]
    b = arol.Batch(tasks)
    outs = b.empty_outputs()
    b.run([dev(x) for x in xs], outs)
    torch.cuda.synchronize()
    for tk, x, y in zip(tasks, xs, outs):
        ref = O.run_task(tk, [x])[0]
        if tk["elem"] == "copy":
            np.testing.assert_array_equal(host(y).view(np.uint32), ref.view(np.uint32))
        else:
            assert_fir_close(host(y), ref, fir_scale(tk, x), what="batch fir")


_VARIANT_SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
import paper_1105_4424_gb300 as A, workloads as W
chain, (x,), w = W.config4(seed=12, frames=2, height=24, width=64)
c = A.Chain(chain)
xd, wd = torch.from_numpy(x).cuda(), torch.from_numpy(w).cuda()
y = c.run([xd]); gx = torch.empty_like(xd); gt = torch.empty(48, device="cuda")
c.backward(wd, [xd], gx, gt); c.sync_status()
np.savez(sys.argv[2], y=y.cpu().numpy(), gx=gx.cpu().numpy(), gt=gt.cpu().numpy())
"""


def test_register_and_bulk_variants_agree(arol, tmp_path):
    """The fused chain has two kernel variants (bulk-copy pipeline, default;
    register-direct loads, AROL_FUSED_VARIANT=regs); both match the oracle."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = {}
    for variant in ("bulk", "regs"):
        env = dict(os.environ)
        if variant == "regs":
            env["AROL_FUSED_VARIANT"] = "regs"
        f = str(tmp_path / f"{variant}.npz")
        subprocess.run([sys.executable, "-c", _VARIANT_SCRIPT, root, f], check=True, env=env, timeout=300)
        outs[variant] = np.load(f)
    chain, (x,), w = W.config4(seed=12, frames=2, height=24, width=64)
    y64 = O.run_chain(chain, [x])[0]
    for variant, o in outs.items():
        assert_fir_close(o["y"], y64, fir_scale(chain, x), what=f"{variant} forward")
    np.testing.assert_allclose(outs["bulk"]["gx"], outs["regs"]["gx"], rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(outs["bulk"]["gt"], outs["regs"]["gt"], rtol=1e-4, atol=1e-5)


def test_large_indices_near_the_32bit_limit(arol):
    """Repetition indices up to 7e5 and base sums just under 2^31 (the 32-bit
    multiply-shift division path) with awkward extents, and a variant just
    over it (64-bit path), both bit-exact against the C oracle."""
    g = W.rng(111)
    x = g.random((7, 999983), dtype=np.float32)
    for pav in (3000, 3100):            # 3000 * 700000 < 2^31 <= 3100 * 700000
        inp = W.port((7, 999983), (5, 999980), ((3, 0), (0, pav)), ((0,), (1,)), (3,))
        out = W.port((3, 700001 * 3), (0, 0), ((1, 0), (0, 3)), ((0,), (1,)), (3,))
        tk = W.task((3, 700001), "copy", [inp], [out])
        _, y = run1(arol, tk, [x])
        np.testing.assert_array_equal(y.view(np.uint32), C.run_task(tk, [x])[0].view(np.uint32))


def test_batch_row_fir_tasks_with_shifted_origins(arol):
    """Row-FIR tasks (the row-tile path) whose input and output origins are
    shifted, negative or past the array (so reads and writes wrap), long rows
    split across tiles and short rows packed into one tile."""
    g = W.rng(112)
    tasks, xs = [], []
    for (h, w, T, m, S) in [(5, 3000, 7, 2, 3), (9, 40, 32, 16, 32), (3, 17, 5, 1, 1), (40, 64, 12, 5, 6),
                            (2, 999, 31, 4, 17), (1, 8, 3, 3, 3)]:
        base = W.fir_row_task(h, w, T, m, S, (g.standard_normal((m, T)) / T).astype(np.float32))
        inp = dict(base["inputs"][0], origin=(int(g.integers(-50, 50)), int(g.integers(-5000, 5000))))
        out = dict(base["outputs"][0], origin=(int(g.integers(-50, 50)), int(g.integers(-5000, 5000))))
        tasks.append(W.task(base["rep"], "fir", [inp], [out], base["taps"]))
        xs.append(g.random((h, w), dtype=np.float32))
    b = arol.Batch(tasks)
    outs = b.empty_outputs()
    b.run([dev(x) for x in xs], outs)
    outs2 = b.empty_outputs()
    b.run_per_task([dev(x) for x in xs], outs2)
    torch.cuda.synchronize()
    for tk, x, y, y2 in zip(tasks, xs, outs, outs2):
        ref = C.run_task(tk, [x])[0]
        assert_fir_close(host(y), ref, fir_scale(tk, x, C.run_chain), what="row fir batch")
        np.testing.assert_array_equal(host(y), host(y2))


def test_random_2d_fir_patterns(arol):
    """FIR banks on 2-D patterns (2-D fittings: stencils, oriented windows) and
    2-D output patterns, with wrap and overlap."""
    g = W.rng(113)
    for _ in range(40):
        tk = W.random_tiler_task(g, "fir", fir_pattern_rank=2)
        x = g.standard_normal(tk["inputs"][0]["shape"]).astype(np.float32)
        _, y = run1(arol, tk, [x])
        assert_fir_close(y, O.run_task(tk, [x])[0], fir_scale(tk, x), what="2-D fir")


def test_3x3_stencil_as_a_repetitive_task(arol):
    """A 3x3 stencil (pattern (3, 3), fitting identity) over a wrapped image:
    numpy.roll sums are the closed form."""
    g = W.rng(114)
    x = g.standard_normal((37, 53)).astype(np.float32)
    H = g.standard_normal((1, 9)).astype(np.float32)
    inp = W.port((37, 53), (-1, -1), ((1, 0), (0, 1)), ((1, 0), (0, 1)), (3, 3))
    out = W.port((37, 53), (0, 0), ((1, 0), (0, 1)), ((0,), (0,)), (1,))
    tk = W.task((37, 53), "fir", [inp], [out], H)
    _, y = run1(arol, tk, [x])
    ref = np.zeros((37, 53))
    for a in range(3):
        for b in range(3):
            ref += H[0, 3 * a + b] * np.roll(x.astype(np.float64), (1 - a, 1 - b), axis=(0, 1))
    assert_fir_close(y, ref, fir_scale(tk, x), what="3x3 stencil")


def _three_task_chain(g):
    """Horizontal 2:1, vertical 2:1, horizontal 4-tap/2-output: an unfused chain."""
    H1 = (g.standard_normal((1, 2)) / 2).astype(np.float32)
    H2 = (g.standard_normal((1, 2)) / 2).astype(np.float32)
    H3 = (g.standard_normal((2, 4)) / 4).astype(np.float32)
    t1 = W.task((24, 16), "fir", [W.port((24, 32), (0, 0), ((1, 0), (0, 2)), ((0,), (1,)), (2,))],
                [W.port((24, 16), (0, 0), ((1, 0), (0, 1)), ((0,), (1,)), (1,))], H1)
    t2 = W.task((12, 16), "fir", [W.port((24, 16), (0, 0), ((2, 0), (0, 1)), ((1,), (0,)), (2,))],
                [W.port((12, 16), (0, 0), ((1, 0), (0, 1)), ((1,), (0,)), (1,))], H2)
    t3 = W.task((12, 4), "fir", [W.port((12, 16), (0, 3), ((1, 0), (0, 4)), ((0,), (1,)), (4,))],
                [W.port((12, 8), (0, 0), ((1, 0), (0, 2)), ((0,), (1,)), (2,))], H3)
    return [t1, t2, t3]


def test_three_task_chain_forward_and_backward(arol):
    g = W.rng(115)
    chain = _three_task_chain(g)
    x = g.standard_normal((24, 32)).astype(np.float32)
    c = arol.Chain(chain)
    assert c.info["kernel"] == 4
    y = host(c.run([dev(x)]))
    assert_fir_close(y, O.run_chain(chain, [x])[0], fir_scale(chain, x), what="3-task chain")
    G = g.standard_normal((12, 8)).astype(np.float32)
    gx = torch.empty((24, 32), device="cuda")
    gt = torch.empty(2 + 2 + 8, device="cuda")
    c.backward(dev(G), [dev(x)], gx, gt)
    torch.cuda.synchronize()
    dX, dHs = O.chain_vjp(chain, [x], G.astype(np.float64))
    abs_chain = [dict(t, taps=np.abs(t["taps"].astype(np.float64))) for t in chain]
    sX, sHs = O.chain_vjp(abs_chain, [np.abs(x)], np.abs(G.astype(np.float64)))
    assert_fir_close(host(gx), dX, sX, what="3-task chain dX")
    got, off = host(gt), 0
    for dH, sH in zip(dHs, sHs):
        assert_fir_close(got[off:off + dH.size].reshape(dH.shape), dH, sH, what="3-task chain dH")
        off += dH.size


@pytest.mark.parametrize("case", [
    # (H, W, p0, p1, s0, s1, m, origin, out_origin)
    (37, 53, 3, 3, 1, 1, 1, (-1, -1), (0, 0)),      # 3x3 stencil with wrap (register-blocked kernel)
    (70, 130, 5, 5, 1, 1, 1, (-2, -2), (1, 3)),     # 5x5 stencil, shifted output (register-blocked kernel)
    (33, 65, 3, 3, 1, 1, 2, (-1, -1), (0, 0)),      # 3x3 pattern with two outputs (general kernel)
    (50, 256, 3, 3, 1, 1, 1, (-1, -1), (0, 0)),     # rows a multiple of 4: 16-byte window copies, wrap
    (40, 160, 5, 5, 1, 1, 1, (-2, 157), (2, 1)),    # 16-byte copies, window start near the row end
    (300, 700, 5, 7, 1, 1, 1, (-2, -3), (3, 5)),    # larger stencil, shifted output
    # more 32x128 stencil tiles (1152, 1024) than CTAs resident on a GB300
    # (152 SMs x 4), so CTAs take several tiles through both buffers
    (4096, 1030, 3, 3, 1, 1, 1, (-1, -1), (5, 7)),  # element window copies, ragged last tile column
    (2048, 2048, 5, 5, 1, 1, 1, (-2, -2), (0, 0)),  # 16-byte window copies
    (1000, 520, 3, 3, 1, 1, 1, (-1, -1), (998, 0)), # output strips that wrap and a ragged last tile row
    (64, 96, 4, 4, 4, 4, 2, (0, 0), (0, 0)),        # non-overlapping 4x4 blocks, 2 outputs
    (90, 200, 3, 8, 2, 3, 5, (7, -11), (1, 2)),     # strided, overlapping, 5 outputs
    (9, 5, 6, 6, 1, 1, 3, (4, 1), (0, 0)),          # pattern wider than the array
    (40, 4000, 2, 2, 1, 40, 16, (0, 0), (0, 0)),    # window too wide for a tile: per-repetition path
])
def test_fir_2d_pattern_tiles(arol, case):
    """FIR on 2-D patterns (the 2-D window path, or the per-repetition path
    when the window does not fit): every output element against the oracle."""
    H, W_, p0, p1, s0, s1, m, origin, oo = case
    g = W.rng(hash(case) % 1000)
    R0, R1 = -(-H // s0), -(-W_ // s1)
    taps = (g.standard_normal((m, p0 * p1)) / (p0 * p1)).astype(np.float32)
    inp = W.port((H, W_), origin, ((s0, 0), (0, s1)), ((1, 0), (0, 1)), (p0, p1))
    out = W.port((R0, m * R1), oo, ((1, 0), (0, m)), ((0,), (1,)), (m,))
    tk = W.task((R0, R1), "fir", [inp], [out], taps)
    x = g.standard_normal((H, W_)).astype(np.float32)
    t, y = run1(arol, tk, [x])
    ref = (C.run_task if H * W_ > 20000 else O.run_task)(tk, [x])[0]
    assert_fir_close(y, ref, fir_scale(tk, x, C.run_chain if H * W_ > 20000 else O.run_chain), what=f"2-D FIR {case}")


def test_stencil_8192_full_size(arol):
    """The bench's 3x3 stencil on 8192x8192 with wrap, every element against
    the numpy.roll closed form (sum over a, b of H[a, b] x[i + a - 1, j + b - 1])."""
    n = 8192
    g = W.rng(5)
    x = g.random((n, n), dtype=np.float32)
    H = (g.standard_normal((1, 9)) / 9).astype(np.float32)
    inp = W.port((n, n), (-1, -1), ((1, 0), (0, 1)), ((1, 0), (0, 1)), (3, 3))
    out = W.port((n, n), (0, 0), ((1, 0), (0, 1)), ((0,), (0,)), (1,))
    _, y = run1(arol, W.task((n, n), "fir", [inp], [out], H), [x])
    x64 = x.astype(np.float64)
    ref = np.zeros((n, n))
    scale = np.zeros((n, n))
    for a in range(3):
        for b in range(3):
            sh = np.roll(x64, (1 - a, 1 - b), axis=(0, 1))
            ref += float(H[0, 3 * a + b]) * sh
            scale += abs(float(H[0, 3 * a + b])) * np.abs(sh)
    assert_fir_close(y, ref, scale, what="8192^2 stencil")
