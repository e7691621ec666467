"""GB300-native geometric-sum polynomial filter eigensolver for Floquet unitaries
(Luitz, arXiv:2102.05054): kicked-Ising U, the filtered matvec g_k(U)|psi>, and
Krylov-Schur Arnoldi on g_k(U), all in hand-written sm_103a CUDA behind the C ABI of
``include/floquet.h``.

``paper_2102_05054_gb300.floquet`` is the ctypes binding to that library; it is imported
lazily so that ``paper_2102_05054_gb300.inputs`` can be used without a GPU.
"""

__all__ = ["inputs", "floquet"]
