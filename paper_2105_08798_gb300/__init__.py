"""GB300-native Green's-function pad update of the flexible boundary condition method.

The compute path is the C-ABI library ``libfbc.so`` (hand-written sm_103a CUDA
kernels, built by ``paper_2105_08798_gb300.build``); ``paper_2105_08798_gb300.fbc``
is the thin ctypes binding with the same entry-point names.  Importing this
package does not load the library; ``fbc.load()`` does, and fails loudly when
it is missing.
"""

__all__ = ["inputs", "fbc", "build"]
