"""Kicked-Ising Floquet operator, CPU oracle (test infrastructure; see ``oracle/__init__``).

The paper (Sec. 2, Eqs. U/unitary) benchmarks a brickwork circuit; its method applies to
any local Floquet operator with a cheap matrix-free product (Sec. 1, the overview of the
method; Sec. 2, the paragraph after Eq. matvec).
The operator here is the periodically kicked Ising chain

    U = D . K,   K = exp(-i g sum_i X_i),   D = exp(-i sum_i (J Z_i Z_{i+1} + h_i Z_i)),

with periodic boundaries (bond (L-1, 0) included, L >= 3).

Conventions (fixed for the whole project):
  * amplitude index s = sum_i b_i 2^i, qubit i is bit i (little endian);
  * Z|0> = +|0>, so z_i(s) = 1 - 2 b_i(s);
  * exp(-i g X) = cos(g) I - i sin(g) X;
  * the kick acts first, then the diagonal phase layer (U = D K).

Parity: ``apply_u`` is pinned against ``dense_u_expm`` (dense matrix exponentials of the
Kronecker-product generators), brute-force phases on tiny L, unitarity, and the
closed-form spectra of the special cases g = 0, J = 0 and g = pi/2 (tests/test_oracle.py).
"""

import numpy as np


def bit_table(L):
    """b[s, i] = bit i of s, for all d = 2^L indices (qubit i = bit i)."""
    s = np.arange(1 << L, dtype=np.int64)
    return ((s[:, None] >> np.arange(L, dtype=np.int64)[None, :]) & 1).astype(np.int64)


def diagonal_phases(L, J, h):
    """theta_s = J sum_i z_i z_{(i+1) mod L} + sum_i h_i z_i, z_i = 1 - 2 b_i(s).

    The diagonal layer multiplies amplitude s by exp(-i theta_s).
    """
    h = np.asarray(h, dtype=np.float64)
    assert h.shape == (L,)
    z = 1 - 2 * bit_table(L)                      # (d, L), entries +-1
    zz = z * np.roll(z, -1, axis=1)               # z_i z_{i+1 mod L}
    return J * zz.sum(axis=1).astype(np.float64) + z.astype(np.float64) @ h


def apply_kick(psi, L, g):
    """psi <- prod_q (cos g I - i sin g X_q) psi, one qubit at a time.

    For qubit q the pair (s, s xor 2^q) is rotated: a' = c a - i sn b, b' = c b - i sn a.
    Implemented by viewing psi as (2^(L-q-1), 2, 2^q); axis 1 is bit q.
    """
    c, sn = np.cos(g), np.sin(g)
    out = np.array(psi, dtype=np.complex128, copy=True)
    for q in range(L):
        v = out.reshape(1 << (L - q - 1), 2, 1 << q)
        a = v[:, 0, :].copy()
        b = v[:, 1, :].copy()
        v[:, 0, :] = c * a - 1j * sn * b
        v[:, 1, :] = c * b - 1j * sn * a
    return out


class KickedIsing:
    """Matrix-free U = D K for one disorder realisation (J, g, h[0..L-1])."""

    def __init__(self, L, J, g, h):
        if L < 3:
            raise ValueError("periodic chain needs L >= 3")
        self.L, self.J, self.g = int(L), float(J), float(g)
        self.h = np.asarray(h, dtype=np.float64).copy()
        self.d = 1 << self.L
        self.phase = np.exp(-1j * diagonal_phases(self.L, self.J, self.h))

    def apply_u(self, psi):
        """U psi = D (K psi)."""
        return self.phase * apply_kick(psi, self.L, self.g)

    def apply_u_block(self, X):
        """U applied to each column of X (d x n)."""
        return np.stack([self.apply_u(X[:, i]) for i in range(X.shape[1])], axis=1)

    def dense(self):
        """Dense U built column by column from the matrix-free product (small L only)."""
        d = self.d
        U = np.empty((d, d), dtype=np.complex128)
        e = np.zeros(d, dtype=np.complex128)
        for s in range(d):
            e[:] = 0.0
            e[s] = 1.0
            U[:, s] = self.apply_u(e)
        return U


def single_site(op, i, L):
    """Kronecker embedding of a 2x2 operator on qubit i (bit i); np.kron puts its left
    factor on the high bits, so the order is I_{2^(L-1-i)} (x) op (x) I_{2^i}."""
    return np.kron(np.kron(np.eye(1 << (L - 1 - i)), op), np.eye(1 << i))


def dense_u_expm(L, J, g, h):
    """Dense U = expm(-i H_D) expm(-i g sum X_i) from Kronecker-product generators.

    An independent construction (no bit tricks, no closed-form rotations) used only to
    pin ``KickedIsing.apply_u``; practical for L <= 8.
    """
    from scipy.linalg import expm

    X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
    d = 1 << L
    HX = np.zeros((d, d), dtype=np.complex128)
    HD = np.zeros((d, d), dtype=np.complex128)
    for i in range(L):
        HX += single_site(X, i, L)
        Zi = single_site(Z, i, L)
        Zj = single_site(Z, (i + 1) % L, L)
        HD += J * (Zi @ Zj) + h[i] * Zi
    return expm(-1j * HD) @ expm(-1j * g * HX)


def spectrum_g0(L, J, h):
    """g = 0: U = D is diagonal; eigenpairs (exp(-i theta_s), |s>) at any L."""
    return np.exp(-1j * diagonal_phases(L, J, h))


def spectrum_j0(L, g, h):
    """J = 0: U = prod_i exp(-i h_i Z_i) exp(-i g X_i) is a product of 2x2 unitaries, so its
    eigenvalues are all products of one eigenvalue of each single-site factor."""
    X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    evs = np.ones(1, dtype=np.complex128)
    for i in range(L):
        u = np.diag([np.exp(-1j * h[i]), np.exp(1j * h[i])]) @ (
            np.cos(g) * np.eye(2) - 1j * np.sin(g) * X)
        lam = np.linalg.eigvals(u)
        evs = np.multiply.outer(lam, evs).ravel()
    return evs


def spectrum_g_half_pi(L, J, h):
    """g = pi/2: K = (-i)^L X^{(x)L} maps |s> to |s xor (2^L - 1)>, so U couples only the
    pair {s, sbar}; on that pair U = (-i)^L [[0, D_s], [D_sbar, 0]] with eigenvalues
    (-i)^L (+-) sqrt(D_s D_sbar)."""
    theta = diagonal_phases(L, J, h)
    d = 1 << L
    s = np.arange(d)
    sbar = s ^ (d - 1)
    keep = s < sbar
    root = np.exp(-0.5j * (theta[s[keep]] + theta[sbar[keep]]))
    pref = (-1j) ** L
    return np.concatenate([pref * root, -pref * root])
