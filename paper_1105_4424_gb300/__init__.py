"""GB300-native Array-OL repetitive tasks (MARTE RSM) on one NVIDIA GB300.

The library ``libarol.so`` (CUDA for sm_103a, C ABI in ``include/arol.h``)
runs tasks whose input tilers gather pattern elements at
``(origin + paving . r + fitting . i) mod shape`` for every repetition index r,
apply an elementary task (FIR bank, copy, or a 128 x 128 matmul tile on the
tensor cores) and scatter through an output tiler.  This package is the thin
Python binding over that ABI; importing it fails when the library is not
built.
"""
from .binding import *  # noqa: F401,F403
from .binding import ArolError, lib  # noqa: F401
from .api import Batch, Chain, ConjugateGradient, Task, TaskFunction, apply_task  # noqa: F401

__all__ = [n for n in dir() if n.startswith("arol_")] + [
    "ArolError", "Task", "Chain", "Batch", "TaskFunction", "apply_task", "ConjugateGradient"]
