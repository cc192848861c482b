"""GB300-native batched Gaussian-splatting RGB-D renderer with LBS avatars.

The compute path is ``libgs.so`` (hand-written CUDA for sm_103a behind a C ABI,
``include/gs.h``); ``paper_2604_12626_gb300.api`` is the thin ctypes binding and
the ``torch.autograd.Function`` on top.  ``synth`` draws seeded synthetic inputs.
Importing the package does not load the CUDA library; ``api`` does, and raises
if it is missing.
"""
__all__ = ["api", "synth"]
