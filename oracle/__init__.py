"""CPU oracle for the Barnes-Hut AMR potential.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.  The library never does.
"""
