"""GB300-native OS-MPM hot path: hand-written sm_103a CUDA behind the C ABI
declared in ``include/osmpm.h``, with a thin ctypes binding in
``paper_2605_09097_gb300.osmpm``.

Importing the package loads nothing; ``paper_2605_09097_gb300.osmpm`` loads
the compiled library and raises if it is missing."""
