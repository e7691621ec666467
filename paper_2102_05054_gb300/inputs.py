"""Seeded synthetic inputs shared by the CUDA path's callers and the CPU oracle.

This module holds no arithmetic of the method: it only draws the random numbers that a
caller passes in (disorder fields h_i, start vectors, test states) and names the
workloads. Both the oracle and the GPU path receive these values as plain arrays.

Disorder: h_i ~ U[-W, W] from ``numpy.random.default_rng(seed).uniform`` (the paper draws
its random circuits from a seeded generator; it names none, so numpy's PCG64 is used).
Start vector: complex Gaussian (independent real and imaginary parts), normalised
(Sec. 4 starts Arnoldi from a random vector).
"""

import math

import numpy as np

J_DEFAULT = 1.0
G_DEFAULT = 0.9045
START_SEED = 12345


def disorder(L, W, seed):
    """h_i ~ U[-W, W], i = 0..L-1, float64."""
    return np.random.default_rng(seed).uniform(-W, W, L).astype(np.float64)


def complex_gaussian(d, seed):
    """Normalised complex Gaussian vector of length d, complex128."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(d) + 1j * rng.standard_normal(d)
    return (v / np.linalg.norm(v)).astype(np.complex128)


def start_vector(L, seed=START_SEED):
    """Arnoldi start vector for a chain of L qubits."""
    return complex_gaussian(1 << L, seed)


def haar_unitary(n, rng):
    """n x n unitary from the uniform (Haar) measure: QR of a complex Gaussian matrix with
    the phases of R's diagonal moved into Q (the sampling the paper cites for its gates)."""
    z = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    dg = np.diag(r)
    return (q * (dg / np.abs(dg))).astype(np.complex128)


def brickwork_gates(L, seed):
    """Random gates of the two-layer brickwork circuit on L qubits (L even): bond gates
    g2[i] (4 x 4, acting on qubits i and i+1, i = 0..L-2) and the two boundary gates g1[0]
    on qubit 0 and g1[1] on qubit L-1 (2 x 2). Matrix indices of a bond gate are
    b_i + 2 b_{i+1} (row = output, column = input)."""
    rng = np.random.default_rng(seed)
    g2 = np.stack([haar_unitary(4, rng) for _ in range(L - 1)])
    g1 = np.stack([haar_unitary(2, rng) for _ in range(2)])
    return g2, g1


def random_states(d, n, seed):
    """n independent normalised complex Gaussian states as a d x n column-major block."""
    return np.stack([complex_gaussian(d, seed + i) for i in range(n)], axis=1)


# The five workloads of the kicked-Ising benchmark suite. Each lists the chain length L,
# disorder width W (h_i ~ U[-W, W]), target phase phi, filter length k (number of terms),
# Krylov dimension m, eigenpair count nev and the precision form.
WORKLOADS = {
    "kicked_ising_L10": dict(L=10, W=1.0, phi=0.0, k=64, m=64, nev=10, precision="fp64",
                             seed=1),
    "kicked_ising_L16": dict(L=16, W=2.0, phi=math.pi / 3, k=1024, m=160, nev=50,
                             precision="fp64", seed=1),
    "kicked_ising_L18_fp32filter": dict(L=18, W=1.0, phi=0.0, k=4096, m=200, nev=64,
                                        precision="filter_fp32", seed=1),
    "kicked_ising_L12_batched": dict(L=12, Ws=(0.5, 1.0, 2.0, 4.0), per_W=64,
                                     phis=(0.0, math.pi / 2, math.pi, 3 * math.pi / 2),
                                     k=256, m=64, nev=16, precision="fp64", seed=1),
    "kicked_ising_L20": dict(L=20, W=1.0, phi=0.0, k=16384, m=256, nev=100,
                             precision="filter_fp32", seed=1),
}


def batched_disorder(L, Ws, per_W, seed):
    """R = len(Ws) * per_W realisations; realisation r uses seed + r. Returns (R x L, W per r)."""
    hs, ws = [], []
    r = 0
    for W in Ws:
        for _ in range(per_W):
            hs.append(disorder(L, W, seed + r))
            ws.append(W)
            r += 1
    return np.stack(hs), np.array(ws)
