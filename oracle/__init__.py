"""FP64 CPU oracle of the OS-MPM hot path: test infrastructure only (see
``oracle.osmpm_oracle``).  Imported by the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the library."""
