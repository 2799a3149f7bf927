"""Batched Lagrangian-Decomposition bounds for ReLU networks on GB300.

The compute path is libld.so (hand-written sm_103a CUDA behind a C ABI,
declared in include/ld.h); `binding` is a thin ctypes layer over it and
`autograd` wraps the bound and its Danskin adjoint as a torch.autograd
Function.  `synth` holds the seeded synthetic inputs.  Importing this
package loads nothing; the library is loaded on first use and its absence
is an error (there is no CPU fallback).
"""

__all__ = ["binding", "autograd", "synth", "build"]
