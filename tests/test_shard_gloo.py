"""Equal partition over devices (Sec. 7), on CPU with two gloo ranks.

Each rank takes its part of the frames through the C ABI's
arol_task_shard_frames (host planning only), runs the oracle on its slice in
place of its GPU, and the parts are put together: the gathered forward must
equal a single-rank run bit for bit (frames are independent), the gathered
dL/dX likewise, and the all-reduced tap gradients (the one exchange of the
backward) must equal the single-rank tap gradients within the rounding of a
different summation order."""
import json
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, result_dir):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import workloads as W
    from oracle import cpu_ref as C
    from paper_1105_4424_gb300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    chain, (x,), w = W.config4(seed=21, frames=5, height=32, width=64)
    local, first = shard.shard_chain(chain, world, rank)
    n = local[0]["rep"][0]
    xl, wl = x[first:first + n], w[first:first + n]
    y = C.run_chain(local, [xl])[0]
    dX, dHs = C.chain_vjp(local, [xl], wl.astype(np.float64))
    dH = torch.from_numpy(np.concatenate([h.reshape(-1) for h in dHs]))
    shard.allreduce_taps(dH)
    # gather the frame slices (padded to the largest part)
    pad = -(-5 // world)
    def gather(a):
        t = torch.zeros((pad,) + a.shape[1:], dtype=torch.float64)
        t[:a.shape[0]] = torch.from_numpy(np.asarray(a, dtype=np.float64))
        out = [torch.zeros_like(t) for _ in range(world)]
        dist.all_gather(out, t)
        return out
    ys, dxs = gather(y), gather(dX)
    counts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(counts, torch.tensor([n]))
    if rank == 0:
        cs = [int(c.item()) for c in counts]
        np.save(os.path.join(result_dir, "y.npy"), np.concatenate([ys[r][:cs[r]].numpy() for r in range(world)]))
        np.save(os.path.join(result_dir, "dx.npy"), np.concatenate([dxs[r][:cs[r]].numpy() for r in range(world)]))
        np.save(os.path.join(result_dir, "dh.npy"), dH.numpy())
        with open(os.path.join(result_dir, "counts.json"), "w") as f:
            json.dump(cs, f)
    dist.destroy_process_group()


def test_two_part_forward_and_backward_equal_one_part(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    sys.path.insert(0, ROOT)
    import workloads as W
    from oracle import cpu_ref as C
    chain, (x,), w = W.config4(seed=21, frames=5, height=32, width=64)
    assert json.load(open(tmp_path / "counts.json")) == [3, 2]
    np.testing.assert_array_equal(np.load(tmp_path / "y.npy"), C.run_chain(chain, [x])[0])
    dX, dHs = C.chain_vjp(chain, [x], w.astype(np.float64))
    np.testing.assert_array_equal(np.load(tmp_path / "dx.npy"), dX)
    full = np.concatenate([h.reshape(-1) for h in dHs])
    scale = np.concatenate([h.reshape(-1) for h in C.chain_vjp(
        [dict(t, taps=np.abs(t["taps"].astype(np.float64))) for t in chain], [np.abs(x)],
        np.abs(w.astype(np.float64)))[1]])
    assert np.all(np.abs(np.load(tmp_path / "dh.npy") - full) <= 1e-12 * scale)


def test_shard_frames_parts_cover_the_task_once():
    sys.path.insert(0, ROOT)
    import workloads as W
    from paper_1105_4424_gb300 import shard
    chain, _ = W.config1(frames=7, height=16, width=32)
    for parts in (1, 2, 3, 4, 7):
        seen = []
        for p in range(parts):
            local, first = shard.shard_chain(chain, parts, p)
            n = local[0]["rep"][0]
            assert n in (7 // parts, 7 // parts + 1)
            for t, full in zip(local, chain):
                assert t["inputs"][0]["shape"][1:] == full["inputs"][0]["shape"][1:]
                assert t["outputs"][0]["shape"] == (n,) + tuple(full["outputs"][0]["shape"][1:])
                assert t["inputs"][0]["paving"] == full["inputs"][0]["paving"]
            seen += list(range(first, first + n))
        assert seen == list(range(7))


def test_shard_rejects_tasks_without_frames():
    sys.path.insert(0, ROOT)
    import workloads as W
    from paper_1105_4424_gb300 import ArolError, shard
    tk = W.matmul_task(256, 256, 128)        # repetition dim 0 walks 128-row panels: no frame dimension
    with pytest.raises(ArolError) as e:
        shard.shard_task(tk, 2, 0)
    assert e.value.status == 3
    with pytest.raises(ArolError) as e:
        shard.shard_task(W.config0()[0], 2, 2)   # part out of range
    assert e.value.status == 1


def test_members_partition_by_cost():
    sys.path.insert(0, ROOT)
    import workloads as W
    from paper_1105_4424_gb300 import shard
    tasks, _ = W.config3()
    costs = [shard.member_cost(t) for t in tasks]
    for parts in (2, 4, 8):
        own = shard.partition_members(costs, parts)
        assert sorted(i for o in own for i in o) == list(range(len(tasks)))
        loads = [sum(costs[i] for i in o) for o in own]
        assert max(loads) - min(loads) <= max(costs)     # greedy balance bound
