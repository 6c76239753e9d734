"""GB300-native lattice Boltzmann hot path (arXiv 2512.12213): fused BGK
collide-stream for D2Q9/D3Q19 with five body-force models, the low-Rm Lorentz
force and the Maxwell-stress equilibrium; stress and strain-rate tensors;
half-step momentum-exchange wall force; shifted 16-bit population storage;
and a hand-written adjoint.

Importing the package does not load the CUDA library; ``lbm`` does, on first
use, and raises if it has not been built.
"""
__all__ = ["lbm", "inputs", "workloads"]
