"""Plain, slow, FP64 CPU oracle of the nested-dissection + HSS preconditioner.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import,
call or execute anything under ``oracle/``.  The product (the CUDA library and
its Python binding) never does, and shares no code with it.
"""
