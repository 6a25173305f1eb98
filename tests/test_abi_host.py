"""The C-ABI library on the host (no GPU): it loads, exports every symbol the
header declares, agrees on struct layout, and its host-only logic (descriptor
validation, partition check, work accounting) matches the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle import tiler as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    import __graft_entry__
    __graft_entry__._build_module().build()
    from paper_1105_4424_gb300 import binding
    return binding


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(arol_\w+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol(B):
    names = declared_symbols()
    assert "arol_task_create" in names and "arol_batch_run" in names and len(names) >= 20
    lib = ctypes.CDLL(B.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layout_matches(B):
    for i, cls in enumerate((B.ArrayDesc, B.Tiler, B.TaskDesc, B.TaskInfo)):
        assert B.lib.arol_abi_struct_size(i) == ctypes.sizeof(cls)
    assert B.arol_version() == 101


def _err(B, spec):
    with pytest.raises(B.ArolError) as e:
        B.arol_task_create(spec)
    return e.value.status


def test_validation_errors(B):
    tk, _ = W.config0()
    assert _err(B, W.task(tk["rep"], "fir", tk["inputs"], tk["outputs"], np.zeros((2, 8), np.float32))) == 1
    bad = W.port((4, 6), (0, 0), ((1, 0), (0, 2)), ((0,), (1,)), (3,))
    assert _err(B, W.task((4, 3), "copy", [bad], [bad])) == 2            # overlapping output tiler
    short = W.port((64, 47), (0, 0), ((1, 0), (0, 3)), ((0,), (1,)), (3,))
    assert _err(B, W.task(tk["rep"], "fir", tk["inputs"], [short], tk["taps"])) == 2
    mism = dict(tk["inputs"][0], dtype="bf16")
    assert _err(B, W.task(tk["rep"], "copy", [mism], [tk["outputs"][0]])) == 1   # dtype differs
    big = W.task(tk["rep"], "fir", tk["inputs"], tk["outputs"], np.zeros((3, 8), np.float32))
    d, keep = B.task_desc(big)
    d.rep_rank = 5
    with pytest.raises(B.ArolError):
        B.arol_task_create(d)
    mm = W.matmul_task(256, 256, 96)                                     # K not a multiple of 64
    assert _err(B, mm) == 3
    mm = W.matmul_task(256, 256, 128, 64, 128)                           # tiles other than 128 x 128
    assert _err(B, mm) == 3
    assert _err(B, W.task((0,), "copy", [W.port((4,), (0,), ((1,),), ((1,),), (1,))],
                          [W.port((4,), (0,), ((1,),), ((1,),), (1,))])) == 2   # empty rep, non-empty output


def test_empty_task_is_accepted(B):
    p_in = W.port((4,), (0,), ((1,),), ((1,),), (1,))
    p_out = W.port((0,), (0,), ((1,),), ((1,),), (1,))
    h = B.arol_task_create(W.task((0,), "copy", [p_in], [p_out]))
    info = B.arol_task_info(h)
    assert info["reps"] == 0 and info["scattered_elems"] == 0
    B.arol_task_destroy(h)


def test_partition_check_matches_oracle(B):
    g = W.rng(21)
    for _ in range(200):
        tk = W.random_tiler_task(g, "copy")
        R = tk["rep"]
        for port in (tk["inputs"][0], tk["outputs"][0]):
            counts = O.cover_count(port, R)
            lo, hi = B.arol_tiler_cover(port["shape"], port, R)
            assert (lo, hi) == (int(counts.min()), int(counts.max()))
            spec = W.task(R, "copy", [tk["inputs"][0]], [port])
            if port is tk["outputs"][0] or (lo == hi == 1):
                B.arol_task_destroy(B.arol_task_create(spec))
            else:
                with pytest.raises(B.ArolError) as e:
                    B.arol_task_create(spec)
                assert e.value.status == 2


def test_16bit_storage_descriptors(B):
    """IEEE half storage (arol_dtype 2) is accepted next to f32 and bfloat16;
    an unknown dtype is a malformed descriptor; matmul takes bfloat16 only;
    the fused chain needs its 16-bit arrays to share one type."""
    tk, _ = W.config0()
    f16 = W.task(tk["rep"], "fir", [dict(tk["inputs"][0], dtype="f16")], [dict(tk["outputs"][0], dtype="f16")],
                 tk["taps"])
    h = B.arol_task_create(f16)
    assert B.arol_task_info(h)["unique_bytes"] == 2 * (64 * 64 + 64 * 48)
    B.arol_task_destroy(h)
    d, keep = B.task_desc(f16)
    d.in_[0].dtype = 3
    with pytest.raises(B.ArolError) as e:
        B.arol_task_create(d)
    assert e.value.status == 1
    mm = W.matmul_task(256, 256, 128)
    mm = dict(mm, inputs=[dict(p, dtype="f16") for p in mm["inputs"]])
    assert _err(B, mm) == 3
    Hh = np.ones((3, 8), np.float32)
    for dts, kernel in [(("f16", "f16", "f16"), 1), (("f16", "f32", "f16"), 1), (("f16", "f16", "f32"), 1),
                        (("bf16", "bf16", "bf16"), 1), (("f16", "bf16", "f32"), 3), (("bf16", "f32", "f16"), 3),
                        (("f32", "f16", "f32"), 3)]:
        chain = W.downscale_chain(2, 16, 64, Hh, Hh, dtypes=dts)
        subs = [B.arol_task_create(s) for s in chain]
        h = B.arol_chain_create(subs)
        assert B.arol_task_info(h)["kernel"] == kernel, dts
        for x in subs + [h]:
            B.arol_task_destroy(x)


def test_info_counts_the_downscaler_chain(B):
    Hh = np.ones((3, 8), np.float32)
    chain = W.downscale_chain(64, 1080, 1920, Hh, Hh)
    subs = [B.arol_task_create(s) for s in chain]
    h = B.arol_chain_create(subs)
    info = B.arol_task_info(h)
    assert info["kernel"] == 1                       # fused separable downscaler
    assert info["unique_bytes"] == 4 * (64 * 1080 * 1920 + 64 * 405 * 720)
    assert info["gathered_elems"] == 64 * 1080 * 240 * 8 + 64 * 135 * 720 * 8
    assert info["scattered_elems"] == 64 * 1080 * 720 + 64 * 405 * 720
    for x in subs + [h]:
        B.arol_task_destroy(x)
    # row passes with overlap (step 4 < T = 8) and wrap: the general fused chain
    tk, _ = W.config0()
    nxt = W.task((64, 16), "fir", [W.port((64, 48), (0, 0), ((1, 0), (0, 3)), ((0,), (1,)), (3,))],
                 [W.port((64, 16), (0, 0), ((1, 0), (0, 1)), ((0,), (1,)), (1,))], np.ones((1, 3), np.float32))
    subs = [B.arol_task_create(tk), B.arol_task_create(nxt)]
    h = B.arol_chain_create(subs)
    assert B.arol_task_info(h)["kernel"] == 4
    for x in subs + [h]:
        B.arol_task_destroy(x)
    # a task on a 2-D pattern is no row or column pass: stage by stage
    subs = [B.arol_task_create(t) for t in unfusable_chain()]
    h = B.arol_chain_create(subs)
    assert B.arol_task_info(h)["kernel"] == 3
    for x in subs + [h]:
        B.arol_task_destroy(x)


def unfusable_chain():
    """A 3 x 3 pattern FIR (one output per repetition), then a row pass."""
    t1 = W.task((16, 16), "fir", [W.port((16, 16), (-1, -1), ((1, 0), (0, 1)), ((1, 0), (0, 1)), (3, 3))],
                [W.port((16, 16), (0, 0), ((1, 0), (0, 1)), ((0,), (1,)), (1,))], np.ones((1, 9), np.float32))
    t2 = W.task((16, 8), "fir", [W.port((16, 16), (0, 0), ((1, 0), (0, 2)), ((0,), (1,)), (2,))],
                [W.port((16, 8), (0, 0), ((1, 0), (0, 1)), ((0,), (1,)), (1,))], np.ones((1, 2), np.float32))
    return [t1, t2]


def test_chain_rejects_mismatched_arrays(B):
    tk, _ = W.config0()
    subs = [B.arol_task_create(tk), B.arol_task_create(tk)]
    with pytest.raises(B.ArolError) as e:
        B.arol_chain_create(subs)
    assert e.value.status == 1
    for x in subs:
        B.arol_task_destroy(x)


def test_null_arguments_are_rejected(B):
    with pytest.raises(B.ArolError):
        B.arol_task_run(None, [0], [0], 0)
    tk, _ = W.config0()
    h = B.arol_task_create(tk)
    with pytest.raises(B.ArolError) as e:
        B.arol_task_run(h, [None], [None], 0)
    assert e.value.status == 1
    B.arol_task_destroy(h)


def test_batch_accepts_chain_members_and_rejects_matmul(B):
    """Batch creation is host-only: chains enter as their stages, matmul
    tasks are refused with AROL_ERR_UNSUPPORTED."""
    chain, _ = W.config1(seed=1, frames=1, height=16, width=64)
    single, _ = W.config0()
    parts = [B.arol_task_create(t) for t in chain]
    ch = B.arol_chain_create(parts)
    one = B.arol_task_create(single)
    b = B.arol_batch_create([ch, one, ch])
    B.arol_batch_destroy(b)
    mm = B.arol_task_create(W.matmul_task(128, 128, 128))
    with pytest.raises(B.ArolError) as e:
        B.arol_batch_create([one, mm])
    assert e.value.status == 3
    for h in parts + [ch, one, mm]:
        B.arol_task_destroy(h)


def test_batch_rejects_members_with_device_taps(B):
    """Taps borrowed from device memory cannot be copied into a batch: the
    creation fails with AROL_ERR_INVALID (the pointer is never read here)."""
    single, _ = W.config0()
    t = B.arol_task_create(single)
    B.lib.arol_task_set_taps(t, ctypes.c_void_p(0x1000), 1)
    with pytest.raises(B.ArolError) as e:
        B.arol_batch_create([t])
    assert e.value.status == 1
    # host taps again: accepted
    B.arol_task_set_taps(t, np.zeros((3, 8), np.float32), False)
    b = B.arol_batch_create([t])
    B.arol_batch_destroy(b)
    B.arol_task_destroy(t)


def test_tune_off_keeps_the_launch_shape_without_device_work(B):
    """AROL_TUNE=off: arol_batch_tune returns at once with the launch shape
    unchanged and touches no buffer (the pointers here are not device memory,
    and no GPU is needed)."""
    import subprocess
    import sys
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from paper_1105_4424_gb300 import binding as B\n"
        "import workloads as W\n"
        "tk, _ = W.config0()\n"
        "h = B.arol_task_create(tk)\n"
        "b = B.arol_batch_create([h])\n"
        "before = B.arol_batch_config(b)\n"
        "B.arol_batch_tune(b, [16], [32], stream=0)\n"
        "assert B.arol_batch_config(b) == before, (before, B.arol_batch_config(b))\n"
        "print('ok')\n" % ROOT)
    env = dict(os.environ, AROL_TUNE="off")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stderr


def _path(B, spec):
    h = B.arol_task_create(spec)
    try:
        return B.arol_task_info(h)["path"]
    finally:
        B.arol_task_destroy(h)


def _row(g, Wd, T, m, S, R1, o=(0, 0), oo=(0, 0), H=8):
    """A row FIR on an H x Wd array: R1 repetitions per row at step S from
    origin o, m outputs per repetition from output origin oo."""
    inp = W.port((H, Wd), o, ((1, 0), (0, S)), ((0,), (1,)), (T,))
    out = W.port((H, m * R1), oo, ((1, 0), (0, m)), ((0,), (1,)), (m,))
    return W.task((H, R1), "fir", [inp], [out], (g.standard_normal((m, T)) / T).astype(np.float32))


def _fir2d(n0, n1, p0, p1, s0=1, s1=1, m=1, dtype="f32"):
    R0, R1 = -(-n0 // s0), -(-n1 // s1)
    inp = W.port((n0, n1), (-(p0 // 2), -(p1 // 2)), ((s0, 0), (0, s1)), ((1, 0), (0, 1)), (p0, p1), dtype)
    out = W.port((R0, m * R1), (0, 0), ((1, 0), (0, m)), ((0,), (1,)), (m,), dtype)
    return W.task((R0, R1), "fir", [inp], [out], np.ones((m, p0 * p1), np.float32))


def test_info_reports_the_kernel_path(B):
    """Which kernel a single task takes, decided on the host: the row FIR in
    16-word regions, the staged row and column FIR tiles, the 2-D window
    tiles and the register-blocked stencil are f32-only paths; 16-bit
    storage, copies and anything else take the per-repetition walk."""
    tk, _ = W.config0()
    assert _path(B, tk) == 5                                              # row FIR, step 4, wrap: regions
    shifted = dict(tk, inputs=[dict(tk["inputs"][0], origin=(0, 8))])
    assert _path(B, shifted) == 1                                         # origin not a multiple of 16: tiles
    wide = W.config0_scaled(frames=2, height=8, width=1920)[0]
    assert _path(B, wide) == 5
    assert _path(B, W.config0_scaled(frames=2, height=8, width=1928)[0]) == 1   # rows not a multiple of 16
    g = W.rng(1)
    assert _path(B, _row(g, 64, 5, 2, 4, 16, o=(0, 16))) == 5              # origin a multiple of 16
    assert _path(B, _row(g, 64, 8, 4, 8, 8)) == 5                          # step 8, 4 outputs
    assert _path(B, _row(g, 64, 5, 3, 2, 32)) == 1                         # step 2 takes at most 2 outputs
    assert _path(B, _row(g, 64, 9, 2, 4, 16)) == 1                         # more than 8 taps
    assert _path(B, _row(g, 64, 5, 2, 4, 16, oo=(0, 4))) == 1              # output columns not from 0
    assert _path(B, _row(g, 64, 5, 2, 4, 16, o=(3, 0))) == 1               # rows shifted
    assert _path(B, _row(g, 64, 5, 2, 4, 15)) == 1                         # repetitions short of the row
    assert _path(B, dict(tk, inputs=[dict(tk["inputs"][0], dtype="f16")])) == 0
    assert _path(B, dict(tk, outputs=[dict(tk["outputs"][0], dtype="bf16")])) == 0
    col = W.task((16, 64), "fir", [W.port((64, 64), (0, 0), ((4, 0), (0, 1)), ((1,), (0,)), (8,))],
                 [W.port((48, 64), (0, 0), ((3, 0), (0, 1)), ((1,), (0,)), (3,))], np.ones((3, 8), np.float32))
    assert _path(B, col) == 2                                             # column FIR
    assert _path(B, _fir2d(8192, 8192, 3, 3)) == 4                        # the bench's 3x3 stencil
    assert _path(B, _fir2d(70, 130, 5, 5)) == 4
    assert _path(B, _fir2d(64, 96, 3, 3, m=2)) == 3                       # two outputs: 2-D window tiles
    assert _path(B, _fir2d(300, 700, 5, 7)) == 3                          # not square
    assert _path(B, _fir2d(90, 200, 3, 3, s0=2)) == 3                     # strided
    assert _path(B, _fir2d(8192, 8192, 3, 3, dtype="f16")) == 0           # 16-bit storage
    cp = W.random_tiler_task(W.rng(3), "copy")
    assert _path(B, cp) == 0
    mm = B.arol_task_create(W.matmul_task(256, 256, 128))
    assert B.arol_task_info(mm)["kernel"] == 2 and B.arol_task_info(mm)["path"] == -1
    B.arol_task_destroy(mm)
    chain = W.downscale_chain(2, 16, 64, np.ones((3, 8), np.float32), np.ones((3, 8), np.float32))
    subs = [B.arol_task_create(s) for s in chain]
    h = B.arol_chain_create(subs)
    assert B.arol_task_info(h)["path"] == -1
    for x in subs + [h]:
        B.arol_task_destroy(x)


def _chain_kernel(B, chain):
    parts = [B.arol_task_create(t) for t in chain]
    ch = B.arol_chain_create(parts)
    k = B.arol_task_info(ch)["kernel"]
    for h in parts + [ch]:
        B.arol_task_destroy(h)
    return k


def test_row_then_column_chains_choose_the_streaming_kernel(B, monkeypatch):
    """Chain creation is host-only: a row pass then a column pass takes the
    streaming kernel (kernel 5) when the column window fits its ring (T_v <=
    29), the tile kernel (4) with AROL_SEPSTREAM=off or a longer window, and
    a column pass first always takes the tile kernel."""
    chain, _ = W.config1_5to2(frames=2, height=64, width=96)
    assert _chain_kernel(B, chain) == 5
    monkeypatch.setenv("AROL_SEPSTREAM", "off")
    assert _chain_kernel(B, chain) == 4
    monkeypatch.delenv("AROL_SEPSTREAM")
    g = W.rng(9)
    t1 = W.separable_pass((1, 64, 64), 1, 3, 1, 2, 0, 32, np.ones((1, 3), np.float32))
    t2 = W.separable_pass(t1["outputs"][0]["shape"], 0, 30, 1, 2, 0, 32, (g.standard_normal((1, 30)) / 30).astype(np.float32))
    assert _chain_kernel(B, [t1, t2]) == 4
    c1 = W.separable_pass((1, 64, 64), 0, 3, 1, 2, 0, 32, np.ones((1, 3), np.float32))
    c2 = W.separable_pass(c1["outputs"][0]["shape"], 1, 3, 1, 2, 0, 32, np.ones((1, 3), np.float32))
    assert _chain_kernel(B, [c1, c2]) == 4


def test_batch_with_streamed_and_fused_chain_members(B):
    """A batch mixing 8 -> 3 chains (the batched downscaler), row-then-column
    chains (the batched streaming kernel), a three-pass chain and single
    tasks is created on the host without device work."""
    members = []
    chain, _ = W.config1(seed=2, frames=1, height=16, width=64)
    members.append(chain)
    chain, _ = W.config1_5to2(seed=3, frames=1, height=32, width=96)
    members.append(chain)
    g = W.rng(10)
    for _ in range(3):
        c, _ = W.random_separable_chain(g)
        members.append(c)
    single, _ = W.config0()
    handles, made = [], []
    for m in members:
        parts = [B.arol_task_create(t) for t in m]
        made += parts
        handles.append(B.arol_chain_create(parts))
    handles.append(B.arol_task_create(single))
    b = B.arol_batch_create(handles)
    B.arol_batch_destroy(b)
    for h in made + handles:
        B.arol_task_destroy(h)
