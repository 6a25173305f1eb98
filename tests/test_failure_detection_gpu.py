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
