"""Brickwork random-circuit Floquet operator, CPU oracle (test infrastructure; see
``oracle/__init__``).

Sec. 2 of Luitz, arXiv:2102.05054 (Eqs. U, unitary): one period is a two-layer brickwork of
two-qubit unitaries on neighbouring qubits, U = U_a U_b with (0-based qubits, L even)

    U_a = u_{0,1} u_{2,3} ... u_{L-2,L-1},
    U_b = u_0 u_{1,2} u_{3,4} ... u_{L-3,L-2} u_{L-1},

u_0 and u_{L-1} single-qubit boundary gates; U_b acts first. Qubit i is bit i of the
amplitude index; a bond gate's matrix indices are b_i + 2 b_{i+1} (row = output). The gates
are inputs (Haar-random in the paper, drawn by ``paper_2102_05054_gb300.inputs``).

The oracle applies U gate by gate, the plain definition; the paper's two-matrix product
(Eq. matvec) is what the GPU path implements, and the tests compare the two.
"""

import numpy as np


def apply_gate2(psi, L, i, u):
    """u (4 x 4) on qubits (i, i+1) of a state of L qubits."""
    t = np.asarray(psi).reshape(1 << (L - i - 2), 2, 2, 1 << i)  # axes: high, b_{i+1}, b_i, low
    u4 = np.asarray(u).reshape(2, 2, 2, 2)  # [b'_{i+1}, b'_i, b_{i+1}, b_i]
    return np.einsum("ABab,habl->hABl", u4, t).reshape(-1)


def apply_gate1(psi, L, q, u):
    """u (2 x 2) on qubit q."""
    t = np.asarray(psi).reshape(1 << (L - q - 1), 2, 1 << q)
    return np.einsum("Aa,hal->hAl", np.asarray(u), t).reshape(-1)


class Brickwork:
    """U = U_a U_b of Eq. unitary for given gates g2 ((L-1) x 4 x 4) and g1 (2 x 2 x 2)."""

    def __init__(self, L, g2, g1):
        assert L >= 4 and L % 2 == 0
        self.L, self.d = L, 1 << L
        self.g2 = np.asarray(g2, dtype=np.complex128)
        self.g1 = np.asarray(g1, dtype=np.complex128)
        assert self.g2.shape == (L - 1, 4, 4) and self.g1.shape == (2, 2, 2)

    def apply_u(self, psi):
        L = self.L
        x = np.asarray(psi, dtype=np.complex128)
        # U_b: boundary gates and the odd bonds (1,2), (3,4), ...
        x = apply_gate1(x, L, 0, self.g1[0])
        for i in range(1, L - 2, 2):
            x = apply_gate2(x, L, i, self.g2[i])
        x = apply_gate1(x, L, L - 1, self.g1[1])
        # U_a: the even bonds (0,1), (2,3), ...
        for i in range(0, L - 1, 2):
            x = apply_gate2(x, L, i, self.g2[i])
        return x

    def apply_u_block(self, X):
        return np.stack([self.apply_u(X[:, j]) for j in range(X.shape[1])], axis=1)

    def dense(self):
        return self.apply_u_block(np.eye(self.d, dtype=np.complex128))
