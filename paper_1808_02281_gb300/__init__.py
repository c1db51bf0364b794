"""GB300-native (sm_103a) molecular-dynamics hot path of the one-loop Symanzik
improved gauge action (D. Li, "The Calculation of Force in Lattice QCD",
Sec. II): action, force, and the MD momentum / link updates.

The compute runs in hand-written CUDA kernels behind the C-ABI library
``liblqcd.so``; ``lqcd`` is the thin ctypes binding that marshals torch
tensors (device memory, streams) into it.  Import ``synth`` for the seeded
synthetic inputs.
"""
__all__ = ["lqcd", "synth"]
