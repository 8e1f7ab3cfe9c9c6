"""CPU checker for the ASAGA solver: a plain, slow, float64 restatement of the
method in arXiv:1606.04809.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import, call or build anything here.
The solver (the CUDA library and its Python binding) never imports it, and it
shares no code with the solver: the only module both sides read is the seeded
data generator, which holds none of the method's arithmetic.
"""
