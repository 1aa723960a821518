"""gx: GB300-native batched DC-OPF dispatch, implicit plan gradient and plan step.

The compute path is a C-ABI shared library of hand-written sm_103a CUDA kernels
(``csrc/``), reached through the thin ctypes binding in ``gx.py``.  Importing the
package does not load the library; ``paper_2410_13055_gb300.gx`` does, and raises
if it has not been built.
"""
__all__ = ["synth"]
