"""Shared helpers of the GPU parity tests (host-side only)."""
import numpy as np
import torch

from oracle import tiler as O

# FP32 FIR tolerance: |y - y64| <= FIR_RTOL * sum_k |H[j,k]| |p[k]| per output
# element (the FP64 oracle run on absolute values gives that sum).  A T-term
# FP32 dot product in k order errs by at most ~T * 2^-24 of that sum
# (T <= 32: <= 1.9e-6), so 1e-5 holds with margin; a chain multiplies the
# absolute-value scales, which is what running the oracle on |H| and |X| does.
FIR_RTOL = 1e-5
FIR_ATOL = 1e-30


def dev(a: np.ndarray) -> torch.Tensor:
    """numpy -> CUDA tensor; uint16 arrays are bfloat16 bit patterns, float16
    arrays IEEE half."""
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint16:
        return torch.from_numpy(a.view(np.int16)).cuda().view(torch.bfloat16)
    return torch.from_numpy(a).cuda()


def host(t: torch.Tensor) -> np.ndarray:
    t = t.detach().cpu()
    if t.dtype == torch.bfloat16:
        return t.view(torch.int16).numpy().view(np.uint16)
    return t.numpy()


def abs_task(tk):
    return dict(tk, taps=np.abs(np.asarray(tk["taps"], dtype=np.float64)))


def fir_scale(tasks, x, run=O.run_chain):
    """sum of |terms| behind every output element of a fir task or chain."""
    tasks = tasks if isinstance(tasks, list) else [tasks]
    return run([abs_task(t) for t in tasks], [np.abs(np.asarray(x, dtype=np.float64))])[0]


def assert_fir_close(y, y64, scale, rtol=FIR_RTOL, what=""):
    y = np.asarray(y, dtype=np.float64)
    err = np.abs(y - y64)
    bound = rtol * scale + FIR_ATOL
    bad = err > bound
    assert not bad.any(), (f"{what}: {int(bad.sum())} of {bad.size} elements out of tolerance; "
                           f"worst err/scale = {float(np.max(err / np.maximum(scale, 1e-300))):.3e}")
    return float(np.max(err / np.maximum(scale, 1e-300))) if err.size else 0.0
