"""The equal-partition path on one GPU: the parts of a sharded chain (run one
after the other here, each on its frame slice) put together give the
unsharded results, and their tap gradients add up to the full ones (what the
all-reduce of a multi-GPU run does)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cpu_ref as C
from tests.gpu_helpers import assert_fir_close, dev, fir_scale, host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("parts", [2, 3, 4])
def test_sharded_chain_parts_add_up(arol, parts):
    from paper_1105_4424_gb300 import shard
    chain, (x,), w = W.config4(seed=22, frames=7, height=64, width=128)
    ys, gxs, gt_sum = [], [], np.zeros(48)
    for p in range(parts):
        sc = shard.ShardedChain(chain, parts, p)
        sl = slice(sc.first, sc.first + sc.frames)
        xd = dev(np.ascontiguousarray(x[sl]))
        ys.append(host(sc.run([xd])))
        gx = torch.empty_like(xd)
        gt = torch.empty(48, device="cuda")
        sc.backward(dev(np.ascontiguousarray(w[sl])), [xd], gx, gt)   # no process group: the part's own sum
        torch.cuda.synchronize()
        gxs.append(host(gx))
        gt_sum += host(gt).astype(np.float64)
    y = np.concatenate(ys)
    assert_fir_close(y, C.run_chain(chain, [x])[0], fir_scale(chain, x, C.run_chain), what="sharded forward")
    dX, (dHh, dHv) = C.chain_vjp(chain, [x], w.astype(np.float64))
    abs_chain = [dict(t, taps=np.abs(t["taps"].astype(np.float64))) for t in chain]
    sX, (sHh, sHv) = C.chain_vjp(abs_chain, [np.abs(x)], np.abs(w.astype(np.float64)))
    assert_fir_close(np.concatenate(gxs), dX, sX, what="sharded dX")
    assert_fir_close(gt_sum, np.concatenate([dHh.reshape(-1), dHv.reshape(-1)]),
                     np.concatenate([sHh.reshape(-1), sHv.reshape(-1)]), what="sharded dH")
