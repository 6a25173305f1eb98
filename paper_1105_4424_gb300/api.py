"""Convenience wrappers over the C ABI: Task, Chain, Batch and the autograd
Function.  They only marshal arguments and allocate output tensors; the work
is done by the library's kernels."""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B

_TORCH_DTYPE = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}


def _out_port(spec):
    return spec["outputs"][0]


def _check_tensor(t, port, what):
    """The C ABI takes raw pointers: catch dtype/shape/layout mistakes here."""
    if not isinstance(t, torch.Tensor):
        return
    want = _TORCH_DTYPE[port["dtype"]]
    if t.dtype != want:
        raise TypeError(f"{what}: expected {want}, got {t.dtype}")
    if tuple(t.shape) != tuple(port["shape"]) and t.numel() != int(np.prod(port["shape"])):
        raise ValueError(f"{what}: expected shape {tuple(port['shape'])}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{what}: tensor must be contiguous")


class Task:
    """One repetitive task (copy, fir or matmul) built from a task dict."""

    def __init__(self, spec):
        self.spec = spec
        self.handle = B.arol_task_create(spec)

    @property
    def info(self):
        return B.arol_task_info(self.handle)

    @property
    def out_port(self):
        return _out_port(self.spec)

    def empty_output(self, device="cuda"):
        p = self.out_port
        return torch.empty(p["shape"], dtype=_TORCH_DTYPE[p["dtype"]], device=device)

    def set_taps(self, taps):
        if isinstance(taps, torch.Tensor) and taps.is_cuda:
            if taps.dtype != torch.float32 or not taps.is_contiguous():
                raise ValueError("device taps must be contiguous float32")
            B.arol_task_set_taps(self.handle, taps, True)
        else:
            B.arol_task_set_taps(self.handle, np.asarray(taps, dtype=np.float32), False)

    @property
    def in_ports(self):
        first = self.specs[0] if hasattr(self, "specs") else self.spec
        return first["inputs"]

    def run(self, ins, out=None, stream=None):
        if out is None:
            out = self.empty_output(ins[0].device)
        for t, p in zip(ins, self.in_ports):
            _check_tensor(t, p, "input")
        _check_tensor(out, self.out_port, "output")
        B.arol_task_run(self.handle, list(ins), [out], stream)
        return out

    def prepare(self, ins, out, stream=None):
        """Check and marshal the buffers once; returns a callable that runs
        the task on them (for timing loops)."""
        for t, p in zip(ins, self.in_ports):
            _check_tensor(t, p, "input")
        _check_tensor(out, self.out_port, "output")
        pin, pout, s = B._ptrs(list(ins)), B._ptrs([out]), B._stream(stream)
        keep = (list(ins), out)

        def run():
            B._check(B.lib.arol_task_run(self.handle, pin, pout, s))
            return keep[1]

        return run

    def run_host(self, ins, out, stream=None):
        B.arol_task_run_host(self.handle, list(ins), [out], stream)
        return out

    def backward(self, grad_out, saved_in, grad_in=None, grad_taps=None, stream=None):
        """Gradients are float32 whatever the arrays' storage: grad_out has
        the output's shape, grad_in the input's; saved_in keeps its storage."""
        _check_tensor(grad_out, dict(self.out_port, dtype="f32"), "grad_out")
        for t, p in zip(saved_in, self.in_ports):
            _check_tensor(t, p, "saved input")
        if grad_in is not None:
            _check_tensor(grad_in, dict(self.in_ports[0], dtype="f32"), "grad_in")
        if isinstance(grad_taps, torch.Tensor) and grad_taps.dtype != torch.float32:
            raise TypeError("grad_taps must be float32")
        B.arol_task_backward(self.handle, grad_out, list(saved_in), grad_in, grad_taps, stream)

    def fwd_bwd(self, ins, grad_out, out, grad_in=None, grad_taps=None, stream=None):
        B.arol_task_fwd_bwd(self.handle, list(ins), grad_out, out, grad_in, grad_taps, stream)

    def sync_status(self, stream=None):
        B.arol_task_sync_status(self.handle, stream)

    def close(self):
        if getattr(self, "handle", None):
            B.arol_task_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Chain(Task):
    """Tasks chained through shared arrays; the taps of a chain are the
    concatenation of each task's m x T block."""

    def __init__(self, specs):
        self.spec = specs[-1]
        self.specs = specs
        subs = [B.arol_task_create(s) for s in specs]
        try:
            self.handle = B.arol_chain_create(subs)
        finally:
            for h in subs:
                B.arol_task_destroy(h)


class Batch:
    """Independent copy/fir tasks and chains of them, run by one graph
    launch: the persistent launches of each chain stage over every member's
    tiles of that stage.  A member is a task spec or a list of specs (a chain,
    whose intermediates the batch allocates); its input is the first task's
    input, its output the last task's output."""

    def __init__(self, specs):
        self.specs = specs
        subs = []
        try:
            for s in specs:
                if isinstance(s, (list, tuple)):
                    parts = [B.arol_task_create(x) for x in s]
                    try:
                        subs.append(B.arol_chain_create(parts))
                    finally:
                        for h in parts:
                            B.arol_task_destroy(h)
                else:
                    subs.append(B.arol_task_create(s))
            self.handle = B.arol_batch_create(subs)
        finally:
            for h in subs:
                B.arol_task_destroy(h)

    def empty_outputs(self, device="cuda"):
        lasts = [s[-1] if isinstance(s, (list, tuple)) else s for s in self.specs]
        return [torch.empty(_out_port(s)["shape"], dtype=_TORCH_DTYPE[_out_port(s)["dtype"]], device=device)
                for s in lasts]

    def run(self, ins, outs, stream=None):
        B.arol_batch_run(self.handle, list(ins), list(outs), stream)
        return outs

    def prepare(self, ins, outs):
        """Marshal the pointer arrays once; returns (run, run_per_task)
        callables that reuse them (for timing loops)."""
        pin, pout = B._ptrs(list(ins)), B._ptrs(list(outs))
        keep = (list(ins), list(outs))

        def run(stream=None):
            B._check(B.lib.arol_batch_run(self.handle, pin, pout, B._stream(stream)))
            return keep[1]

        def run_per_task(stream=None):
            B._check(B.lib.arol_batch_run_per_task(self.handle, pin, pout, B._stream(stream)))
            return keep[1]

        return run, run_per_task

    def run_per_task(self, ins, outs, stream=None):
        B.arol_batch_run_per_task(self.handle, list(ins), list(outs), stream)
        return outs

    def tune(self, ins, outs, stream=None, force=False):
        B.arol_batch_tune(self.handle, list(ins), list(outs), stream, force)
        return self.config

    def sync_status(self, stream=None):
        """Synchronizes; raises ArolError if a bounded device wait gave up."""
        B.arol_batch_sync_status(self.handle, stream)

    @property
    def config(self):
        return B.arol_batch_config(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            B.arol_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class TaskFunction(torch.autograd.Function):
    """out = task(x; taps) with the library's hand-written adjoint:
    grad_x by the transposed-tiler scatter-add, grad_taps by the per-warp /
    per-CTA tap-gradient reduction.  `task` is a fir Task or Chain."""

    @staticmethod
    def forward(ctx, task, x, taps):
        x = x.contiguous()
        taps = taps.contiguous()
        task.set_taps(taps)
        out = task.run([x])
        ctx.task = task
        ctx.save_for_backward(x, taps)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        x, taps = ctx.saved_tensors
        task = ctx.task
        task.set_taps(taps)
        gx = torch.empty(x.shape, dtype=torch.float32, device=x.device) if ctx.needs_input_grad[1] else None
        gt = torch.empty_like(taps) if ctx.needs_input_grad[2] else None
        if gx is not None or gt is not None:
            task.backward(grad_out.float().contiguous(), [x], gx, gt)
        return None, (gx.to(x.dtype) if gx is not None else None), gt


def apply_task(task, x, taps):
    return TaskFunction.apply(task, x, taps)


class ConjugateGradient:
    """CG on a CSR matrix held in device tensors (row_ptr int64, col_idx
    int32, vals float64); the loop runs on the device."""

    def __init__(self, row_ptr, col_idx, vals):
        for t, dt in ((row_ptr, torch.int64), (col_idx, torch.int32), (vals, torch.float64)):
            if t.dtype != dt or not t.is_cuda or not t.is_contiguous():
                raise TypeError(f"expected a contiguous CUDA {dt} tensor")
        self.n = row_ptr.numel() - 1
        self.nnz = vals.numel()
        self._keep = (row_ptr, col_idx, vals)
        self.handle = B.arol_cg_create(self.n, self.nnz, row_ptr, col_idx, vals)

    def spmv(self, x, y=None, stream=None):
        y = torch.empty_like(x) if y is None else y
        row_ptr, col_idx, vals = self._keep
        B.arol_csr_spmv(self.n, self.nnz, row_ptr, col_idx, vals, x, y, stream)
        return y

    def solve(self, b, x=None, tol=1e-10, max_iter=1000, stream=None):
        x = torch.zeros_like(b) if x is None else x
        iters, rel = B.arol_cg_solve(self.handle, b, x, tol, max_iter, stream)
        return x, iters, rel

    def close(self):
        if getattr(self, "handle", None):
            B.arol_cg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
