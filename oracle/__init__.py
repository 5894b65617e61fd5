"""FP64 CPU oracle for the NQS variational Monte Carlo hot path.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA path
shares no code with it: nothing here calls into the CUDA library and the CUDA
library never calls into this package.

Every function states the passage of "Neural Quantum States in Mixed
Precision" (arXiv 2601.20782) it follows; readings where the paper is silent
or garbled are stated where they are used.

Pins (tests/test_oracle_*.py) tie each part to something other than itself:
cuRAND's host Philox4x32-10, the free-fermion closed form of the 1D TFIM,
exact diagonalisation, exact MH transition matrices, product-state closed
forms, central finite differences and numerical quadrature.

``complex_rbm`` is the oracle of the complex-parameter RBM (App. G as written, with
complex a, b, W): its pins are the reduction to the real RBM, the sign map of a visible
phase i pi/2 between the TFIM with +h and -h, the Rayleigh quotient of the sparse
Hamiltonian, and finite differences of the exact energy in both directions of each
parameter.
"""
