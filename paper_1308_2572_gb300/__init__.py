"""GB300-native aggregate risk analysis (Bahl et al., arXiv:1308.2572).

The compute path is the C-ABI library ``libart`` (hand-written sm_103a CUDA,
declared in ``include/art.h``); ``paper_1308_2572_gb300.art`` is its thin
ctypes binding and ``paper_1308_2572_gb300.autograd`` the
``torch.autograd.Function`` around the adjoint kernel. Importing this
package loads nothing; the binding loads the library on first use and
raises if it is missing.
"""
__all__ = ["art", "workloads"]
