"""GB300-native (sm_103a) CGKS-5th / GKS-2nd hot path.

The compute path is the CUDA library ``libgks.so`` behind the C-ABI of
``include/gks.h``; :mod:`.gks` is its thin ctypes binding. There is no CPU
fallback: importing the binding without a built library raises.
"""
__all__ = ["workloads"]
