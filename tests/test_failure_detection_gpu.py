"""Failure detection without a GPU fault: a bounded device wait that runs out
is reported as AROL_ERR_TIMEOUT through an error word, and an injected
allocation failure surfaces as AROL_ERR_CUDA; in both cases the context and
the handles stay usable."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import tiler as O
from tests.gpu_helpers import assert_fir_close, dev, fir_scale, host
from tests.test_parity_gpu import _three_task_chain

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives(arol):
    with pytest.raises(arol.ArolError) as e:
        arol.arol_selftest_wait_timeout()
    assert e.value.status == 5              # AROL_ERR_TIMEOUT
    tk, (x,) = W.config0(seed=4)            # the context still runs work
    y = host(arol.Task(tk).run([dev(x)]))
    assert_fir_close(y, O.run_task(tk, [x])[0], fir_scale(tk, x), what="after timeout")


def test_allocation_failure_is_reported_and_retried(arol, monkeypatch):
    g = W.rng(130)
    chain = _three_task_chain(g)
    x = g.standard_normal((24, 32)).astype(np.float32)
    c = arol.Chain(chain)
    monkeypatch.setenv("AROL_FAIL_ALLOC", "1")
    with pytest.raises(arol.ArolError) as e:
        c.run([dev(x)])
    assert e.value.status == 4               # AROL_ERR_CUDA (out of memory)
    monkeypatch.delenv("AROL_FAIL_ALLOC")
    y = host(c.run([dev(x)]))                # the same handle, retried
    assert_fir_close(y, O.run_chain(chain, [x])[0], fir_scale(chain, x), what="after allocation failure")
    torch.cuda.synchronize()


_DEBUG_SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
import paper_1105_4424_gb300 as A, workloads as W
g = W.rng(131)
outs = []
for i in range(30):
    tk = W.random_tiler_task(g, "fir" if i % 2 else "copy", fir_pattern_rank=1 + (i % 3 == 0))
    x = g.standard_normal(tk["inputs"][0]["shape"]).astype(np.float32)
    t = A.Task(tk)
    y = t.run([torch.from_numpy(x).cuda()])
    t.sync_status()                    # raises on a bounds-check hit
    outs.append(y.cpu().numpy())
np.savez(sys.argv[2], *outs)
"""


def test_debug_build_checks_every_index_without_false_alarms(arol, tmp_path):
    """The AROL_DEBUG build (bounds checks on every index the per-repetition
    walk computes, reported as AROL_ERR_OOB) runs random tilers without a
    single check firing and gives the release build's results bit for bit."""
    import os
    import subprocess
    import sys
    from paper_1105_4424_gb300 import build as BLD
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    lib = BLD.build_debug()
    files = {}
    for name, env in (("debug", dict(os.environ, AROL_LIB=lib)), ("release", dict(os.environ))):
        env.pop("AROL_LIB", None) if name == "release" else None
        f = str(tmp_path / f"{name}.npz")
        subprocess.run([sys.executable, "-c", _DEBUG_SCRIPT, root, f], check=True, env=env, timeout=600)
        files[name] = np.load(f)
    for k in files["release"].files:
        np.testing.assert_array_equal(files["debug"][k].view(np.uint32), files["release"][k].view(np.uint32))
