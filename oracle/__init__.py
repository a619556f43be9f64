"""CPU FP64 oracle for the randomized-multiplier GENP solve (arXiv:1406.5802).

Test infrastructure only: the test-suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  The
product path (the CUDA library and its Python binding) never imports it.
"""
