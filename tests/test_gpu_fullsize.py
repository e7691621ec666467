"""Parity at the full size of the L = 20 workload, in the launch configuration bench.py times
(L = 20, k = 16384, m = 256, nev = 100, phi = 0, double-float sweeps): the oracle cannot
diagonalise d = 2^20, so the returned pairs are checked one by one with the oracle's own
float64 U (Rayleigh quotient and residual of all nev pairs, one vector at a time), plus
properties that hold at any size, and completeness: a second solve with half the filter
length returns the same nev eigenvalues.
"""

import math

import numpy as np
import pytest

from oracle import krylov, model
from paper_2102_05054_gb300 import inputs

from gpu_util import from_dev, require_gpu, to_dev

pytestmark = pytest.mark.gpu


def test_L20_workload_full_size_sampled_residuals():
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    cfg = inputs.WORKLOADS["kicked_ising_L20"]
    L, k, m, nev, phi = cfg["L"], cfg["k"], cfg["m"], cfg["nev"], cfg["phi"]
    h = inputs.disorder(L, cfg["W"], cfg["seed"])
    fq = floquet.Floquet(L, inputs.J_DEFAULT, inputs.G_DEFAULT, h)
    v0 = to_dev(inputs.start_vector(L))
    ev = torch.empty((nev, 1 << L), dtype=torch.complex128, device="cuda")
    om, res, nconv, rc = fq.arnoldi_eigs(phi, k, nev, m, v0, precision=floquet.FILTER_DF,
                                         evecs=ev)
    assert rc == floquet.OK and nconv == nev
    assert res.max() <= 1e-10
    # eigenvalues of a unitary, sorted by closeness, all inside the main lobe of g_k
    assert np.abs(np.abs(om) - 1).max() < 1e-10
    ang = np.abs(np.angle(om * np.exp(-1j * phi)))
    assert np.all(np.diff(ang) >= 0) and ang.max() < 2 * math.pi / k
    # every pair by the oracle's float64 U: Rayleigh quotient and residual
    op = model.KickedIsing(L, inputs.J_DEFAULT, inputs.G_DEFAULT, h)
    X = from_dev(ev, 1 << L)
    om_cpu, r_cpu, Xn = krylov.rayleigh_residual(op, X)
    assert np.abs(om_cpu - om).max() < 1e-12
    assert r_cpu.max() <= 1e-10
    # distinct eigenvectors: an orthonormal set
    G = Xn.conj().T @ Xn
    assert np.abs(G - np.eye(nev)).max() < 1e-9
    del X, Xn, G, ev
    # completeness: a second solve with half the filter length (a lobe twice as wide, so a
    # different Krylov space) returns the same 100 eigenvalues
    om2, res2, nconv2, rc2 = fq.arnoldi_eigs(phi, k // 2, nev, m, v0, precision=floquet.FILTER_DF)
    assert rc2 == floquet.OK and nconv2 == nev and res2.max() <= 1e-10
    dev = np.abs(np.sort_complex(om)[:, None] - om2[None, :]).min(axis=1).max()
    assert dev <= 1e-10, dev
