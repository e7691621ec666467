"""CPU oracle for the geometric-sum polynomial filter eigensolver (Luitz, arXiv:2102.05054).

This package is TEST INFRASTRUCTURE. It is a plain, slow, complex128 numpy/scipy
restatement of what the GPU path computes, written from the paper:

* ``oracle.model``  -- the kicked-Ising Floquet operator U = D.K applied matrix-free
  (Sec. 2: local Floquet operators admit a cheap matrix-free product), its dense form by
  Kronecker products and matrix exponentials, and the special cases whose spectra
  are known in closed form.
* ``oracle.geosum`` -- the geometric sum g_k(U) (Eq. geo, k-term reading), in the
  accumulate and Horner forms, and its closed form on the unit circle (Eqs. geo2,
  gkmapping).
* ``oracle.krylov`` -- Arnoldi with classical Gram-Schmidt and one
  reorthogonalisation (Eq. arnoldi), Rayleigh quotients and residuals (Eq. residual),
  the selection of the eigenpairs closest to the target, dense diagonalisation and
  ARPACK on g_k(U) (Sec. 4).

* ``oracle.brickwork`` -- the paper's own two-layer brickwork circuit of two-qubit gates
  (Sec. 2, Eqs. U, unitary), applied gate by gate.
* ``oracle.entropy`` -- entanglement entropy of a state for a cut of the chain and the
  Page value for random states (Sec. 5, Eqs. ee, page).

It shares no code with the CUDA path and neither imports the other. Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline leg and its
``--impl reference`` arm) may import it; the product path never calls it.

Every function cites the passage of the paper it follows. Parity status of each
function is stated in its docstring; all are pinned by ``tests/test_oracle.py``
against quantities fixed independently of this code (dense matrix exponentials,
closed-form special cases, the paper's statements about g_k, brute force on tiny
inputs).
"""

from . import brickwork, entropy, geosum, krylov, model  # noqa: F401
