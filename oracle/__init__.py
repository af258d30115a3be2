"""ORACLE: plain, slow FP64 CPU restatement of the paper's method.

Test infrastructure only.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import, call, link or run anything here;
the library never does, and shares no code with it.
"""
