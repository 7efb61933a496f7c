"""Exact inference on discrete graphical models by tensor-network contraction on
one GB300 GPU (arXiv 2405.14060): PR, MAR (adjoint contraction), MPE / MMAP
(max-plus contraction with argmax backtracking) and backward sampling.

Submodules: ``tn`` (ctypes binding of libtn), ``synth`` (seeded synthetic
models), ``autograd`` (log Z as a torch.autograd.Function), ``build``.
"""
