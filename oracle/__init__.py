"""CPU oracle for Array-OL repetitive tasks — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU
baseline and reference arm) may import, call, link or execute anything under
``oracle/``.  The product path (``paper_1105_4424_gb300``) never does.

Contents
--------
``tiler``    the definition itself, plain Python loops, float64 (``run_task``,
             ``run_chain``, ``task_vjp``, ``chain_vjp``, ``cover_count``).
``cpu_ref``  the same definition in plain C with OpenMP (``cpu_ref.c``), used
             for full-size parity and as the timed CPU baseline.

The repetitive-task semantics follow MARTE's Repetitive Structure Modeling
package (named in Sec. 3 of the paper; tasks "repetitive and thus potentially
parallel", Sec. 7).  The paper itself prints no tiler formula, FIR or matmul
value, so no function here is pinned to a printed number: every pin is a
closed form, an invariant, a textbook routine or brute force (see
``tests/test_oracle_pins.py``).
"""
