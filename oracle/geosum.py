"""Geometric-sum polynomial filter g_k(U), CPU oracle (test infrastructure).

Sec. 3, Eq. geo defines the filter as a geometric series in exp(-i phi_tgt) U. This
project counts k as the NUMBER OF TERMS:

    g_k(U) = sum_{j=0}^{k-1} z^j U^j,    z = exp(-i phi),

so the paper's order-k filter (terms m = 0..k) is this g_{k+1}. With the k-term reading the
closed form (Eq. geo2) is [1 - z^k U^k][1 - z U]^{-1}, the peak of |g_k| on the unit circle
is k, and its zeros next to the target sit at phase offsets +-2 pi / k (Eq. gkmapping).

Parity: both forms are pinned by tests/test_oracle.py against the closed form on exact
eigenvectors of dense U, the telescoping identity (1 - z U) g_k(U) psi = psi - z^k U^k psi,
and commutation with U.
"""

import numpy as np


def zpow(phi, j):
    """z^j = exp(-i j phi), evaluated directly in float64 (no recurrence)."""
    return np.exp(-1j * float(phi) * float(j))


def filter_acc(op, psi, phi, k):
    """Accumulate form: acc = sum_{j<k} z^j psi_j with psi_0 = psi, psi_{j+1} = U psi_j."""
    acc = np.zeros_like(psi, dtype=np.complex128)
    v = np.array(psi, dtype=np.complex128, copy=True)
    for j in range(k):
        acc += zpow(phi, j) * v
        if j + 1 < k:
            v = op.apply_u(v)
    return acc


def filter_horner(op, psi, phi, k):
    """Horner form: acc <- psi + z U acc, k-1 times, starting from acc = psi."""
    z = zpow(phi, 1)
    psi = np.array(psi, dtype=np.complex128, copy=True)
    acc = psi.copy()
    for _ in range(k - 1):
        acc = psi + z * op.apply_u(acc)
    return acc


def filter_dense(U, phi, k):
    """g_k(U) as a dense matrix: the definition summed term by term (small d only)."""
    d = U.shape[0]
    G = np.zeros((d, d), dtype=np.complex128)
    P = np.eye(d, dtype=np.complex128)
    for j in range(k):
        G += zpow(phi, j) * P
        P = U @ P
    return G


def gk_closed(omega, phi, k):
    """g_k on an eigenvalue omega of U: (1 - w^k)/(1 - w), w = exp(-i phi) omega; k at w = 1."""
    w = np.atleast_1d(np.asarray(omega, dtype=np.complex128)) * zpow(phi, 1)
    out = np.empty_like(w)
    one = np.abs(1.0 - w) < 1e-14
    out[one] = k
    ww = w[~one]
    out[~one] = (1.0 - ww ** k) / (1.0 - ww)
    return out


def gk_on_circle(theta, phi, k):
    """|g_k(e^{i theta})| from the ratio of sines: |sin(k x/2) / sin(x/2)|, x = theta - phi."""
    x = np.atleast_1d(np.asarray(theta, dtype=np.float64)) - phi
    num = np.sin(0.5 * k * x)
    den = np.sin(0.5 * x)
    out = np.full_like(x, float(k))
    nz = np.abs(den) > 1e-300
    out[nz] = np.abs(num[nz] / den[nz])
    return out


def defect_coefficients(omega, phi, k):
    """Coefficients a_l (l = 0 .. k-2) of q(U) = sum_l a_l U^l with
    g_k(U) - g_k(omega) = q(U) (U - omega), z = exp(-i phi).

    Follows from Eq. geo term by term: z^j (U^j - omega^j) = z^j (U - omega) sum_{m<j}
    U^m omega^{j-1-m}; collecting the power U^l over j > l gives
    a_l = z^{l+1} sum_{j=0}^{k-2-l} (z omega)^j = z^{l+1} g_{k-1-l}(z omega) with g_n the
    n-term geometric sum at phase 0. Used by the FP64 polish of the FP32-filter form
    (g_k(U) x = g_k(omega) x + q(U) r, r = (U - omega) x)."""
    z = np.exp(-1j * phi)
    w = z * complex(omega)
    g = np.concatenate([[0.0 + 0j], np.cumsum(w ** np.arange(k))])  # g[n] = sum_{j<n} w^j
    return np.array([z ** (l + 1) * g[k - 1 - l] for l in range(k - 1)], dtype=np.complex128)
