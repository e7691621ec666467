"""The batched L = 12 workload at its full size, through the C ABI: 256 disorder realisations
(64 per W in {0.5, 1, 2, 4}) x 4 targets phi in {0, pi/2, pi, 3 pi/2} = 1024 problems in one
lockstep solve (k = 256, m = 64, nev = 16, FP64 sweeps). Every problem: n_conv = nev,
residuals <= 1e-10, eigenvalues on the unit circle and sorted by closeness. 32 problems (two realisations per W, all four targets) against the oracle's dense
spectrum: the nev closest eigenvalues to 1e-10.
"""

import numpy as np
import pytest

from oracle import krylov, model
from paper_2102_05054_gb300 import inputs

from gpu_util import require_gpu, to_dev

pytestmark = pytest.mark.gpu


def test_batched_L12_workload_1024_problems():
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    cfg = inputs.WORKLOADS["kicked_ising_L12_batched"]
    L, k, m, nev = cfg["L"], cfg["k"], cfg["m"], cfg["nev"]
    hs, ws = inputs.batched_disorder(L, cfg["Ws"], cfg["per_W"], cfg["seed"])
    phis = np.array(cfg["phis"])
    assert hs.shape[0] * phis.size == 1024
    v0 = to_dev(inputs.start_vector(L))
    om, res, nconv, rc = floquet.arnoldi_eigs_batched(L, inputs.J_DEFAULT, inputs.G_DEFAULT,
                                                      hs, phis, k, nev, m, v0,
                                                      precision=floquet.FP64)
    torch.cuda.synchronize()
    assert rc == floquet.OK
    assert np.all(nconv == nev)
    assert res.max() <= 1e-10
    assert np.abs(np.abs(om) - 1.0).max() < 1e-10
    for p, phi in enumerate(phis):
        ang = np.abs(np.angle(om[:, p, :] * np.exp(-1j * phi)))
        assert np.all(np.diff(ang, axis=1) >= -1e-12)
    # the oracle's dense spectrum for two realisations per W, all four targets
    per_w = cfg["per_W"]
    for wi in range(len(cfg["Ws"])):
        for r in (wi * per_w, wi * per_w + per_w - 1):
            op = model.KickedIsing(L, inputs.J_DEFAULT, inputs.G_DEFAULT, hs[r])
            lam = np.linalg.eigvals(op.dense())
            for p, phi in enumerate(phis):
                want = lam[krylov.select_closest(lam, phi, nev)]
                dev = np.abs(om[r, p][:, None] - want[None, :]).min(axis=1).max()
                assert dev <= 1e-10, (r, phi, dev)
