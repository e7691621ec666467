"""Entanglement entropy of eigenstates and the Page value, CPU oracle (test infrastructure:
only tests/, __graft_entry__.smoke() and bench.py's CPU arms use it).

Sec. 5 of Luitz, arXiv:2102.05054 (Eq. ee): cut the chain into subsystem A of L_A qubits and
B of L - L_A qubits, S_A = -sum_i s_i^2 ln s_i^2 with s_i the singular values of the state
reshaped as a 2^{L_A} x 2^{L - L_A} matrix (rows indexed by A). Subsystem A is qubits
0 .. L_A - 1 here, i.e. the low L_A bits of the amplitude index (qubit i = bit i), so the
matrix element (a, b) is psi[a + 2^{L_A} b]. For random pure states the mean is Page's value
(Eq. page), for L_A <= L_B: S = sum_{k = 2^{L_B} + 1}^{2^L} 1/k - (2^{L_A} - 1) / 2^{L_B + 1}.
"""

import numpy as np


def schmidt_values(psi, L, LA):
    """Singular values of psi as a 2^LA x 2^(L-LA) matrix, rows = the low LA bits."""
    psi = np.asarray(psi, dtype=np.complex128)
    assert psi.shape == (1 << L,) and 0 <= LA <= L
    # row-major reshape: index b * 2^LA + a -> [b, a], the transpose of the (a, b) matrix
    mat = psi.reshape(1 << (L - LA), 1 << LA)
    return np.linalg.svd(mat, compute_uv=False)


def entanglement_entropy(psi, L, LA):
    """S_A of Eq. ee for a normalised state (natural logarithm)."""
    p = schmidt_values(psi, L, LA) ** 2
    p = p[p > 0]
    return float(-np.sum(p * np.log(p)))


def page_entropy(LA, LB):
    """Eq. page: mean S_A of random pure states, stated for LA <= LB (symmetric otherwise)."""
    if LA > LB:
        LA, LB = LB, LA
    m, n = 1 << LA, 1 << LB
    k = np.arange(n + 1, m * n + 1, dtype=np.float64)
    return float(np.sum(1.0 / k) - (m - 1) / (2.0 * n))
