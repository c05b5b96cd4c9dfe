"""FP64 CPU oracle of the DSEM semi-Lagrangian step.  Test infrastructure only: imported by
tests/, by ``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``; never by
the library."""
