"""Equal partition of repetitive tasks over devices (Sec. 7: the generated
host code spreads the repetitive tasks of the conjugate-gradient loop equally
over 1, 2 or 4 GPUs).  One process per device; this module only plans and
reduces, the work of every part runs in the library's kernels on its device.

* Tasks and chains with a frame dimension split by frames
  (arol_task_shard_frames): every repetition is independent, so a forward
  needs no exchange between the parts.
* A backward's tap gradients are sums over the repetitions: each part's
  partial sum, added over the parts (one all-reduce of m x T floats per task),
  is the full gradient.  grad_in stays per part (each part owns its frames).
* A batch of independent members splits by members, balanced by cost.
"""
from __future__ import annotations

import numpy as np

from . import binding as B


def shard_task(spec: dict, parts: int, part: int):
    """(the part's task spec, its first frame) of a task with a frame dimension."""
    return B.arol_task_shard_frames(spec, parts, part)


def shard_chain(specs, parts: int, part: int):
    """Every task of a chain on the same frames: (part's specs, first frame)."""
    out, first = [], None
    for s in specs:
        t, f = shard_task(s, parts, part)
        if first is not None and f != first:
            raise ValueError("the chain's tasks do not share their frames")
        out.append(t)
        first = f
    return out, first


def partition_members(costs, parts: int):
    """Members split over `parts` devices by cost: longest first, each to the
    least loaded part (ties to the lower part), a deterministic greedy
    balance.  Returns one ascending index list per part."""
    load = [0.0] * parts
    own = [[] for _ in range(parts)]
    for i in sorted(range(len(costs)), key=lambda k: (-float(costs[k]), k)):
        p = min(range(parts), key=lambda q: (load[q], q))
        own[p].append(i)
        load[p] += float(costs[i])
    return [sorted(o) for o in own]


def member_cost(spec) -> float:
    """Bytes a member moves: its first input and its last output array."""
    first = spec[0] if isinstance(spec, (list, tuple)) else spec
    last = spec[-1] if isinstance(spec, (list, tuple)) else spec
    return float(np.prod(first["inputs"][0]["shape"]) + np.prod(last["outputs"][0]["shape"]))


def allreduce_taps(grad_taps, group=None):
    """Sums a part's tap gradients over every part (torch.distributed, any
    backend); a no-op in a single process.  In place; returns the tensor."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(grad_taps, op=dist.ReduceOp.SUM, group=group)
    return grad_taps


class ShardedChain:
    """A task or chain on this part's frames (`parts` parts, this one
    `part`): run() on the part's input slice gives the part's output slice;
    backward() gives the part's dL/dX slice and the full tap gradients (all
    parts' partial sums added by one all-reduce)."""

    def __init__(self, specs, parts: int, part: int):
        from .api import Chain, Task
        specs = list(specs) if isinstance(specs, (list, tuple)) else [specs]
        self.specs, self.first = shard_chain(specs, parts, part)
        self.frames = self.specs[0]["rep"][0]
        self.handle = Chain(self.specs) if len(self.specs) > 1 else Task(self.specs[0])

    def run(self, ins, out=None, stream=None):
        return self.handle.run(ins, out, stream=stream)

    def backward(self, grad_out, saved_in, grad_in=None, grad_taps=None, stream=None, group=None):
        self.handle.backward(grad_out, saved_in, grad_in, grad_taps, stream=stream)
        if grad_taps is not None:
            allreduce_taps(grad_taps, group)
        return grad_in, grad_taps
