"""GB300-native Hadamard-Babich integrator (arXiv 2210.02698).

The compute path is the C-ABI library ``libhb.so`` (CUDA, sm_103a) declared in
``include/hb.h``; ``binding`` marshals arguments to it and ``autograd`` wraps
the apply/adjoint pair as a ``torch.autograd.Function``.  Importing this
package loads nothing; ``binding.lib()`` loads the library and raises if it is
missing (there is no CPU fallback).
"""

__all__ = ["binding", "workloads"]
