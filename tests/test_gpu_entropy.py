"""GPU entanglement entropy (Sec. 5, Eq. ee) against the CPU oracle, through the C ABI.

Bar: |S_gpu - S_oracle| <= 1e-10 (float64 throughout; the Gram matrix squares the singular
values, so eigenvalues near 0 lose relative accuracy, but they contribute -lambda ln lambda
-> 0; the bound is dominated by ~n eps ln(1/eps) of the tridiagonal eigenvalues).
"""

import numpy as np
import pytest

from oracle import entropy, krylov, model
from paper_2102_05054_gb300 import inputs

from gpu_util import from_dev, require_gpu, to_dev

pytestmark = pytest.mark.gpu


def _gpu_S(L, X, cuts):
    from paper_2102_05054_gb300 import floquet
    return floquet.entanglement_entropy(L, to_dev(X), cuts)


@pytest.mark.parametrize("L", [2, 5, 10, 13])
def test_entropy_random_states_every_cut(L):
    require_gpu()
    X = inputs.random_states(1 << L, 5, 30 + L)  # d x 5
    cuts = list(range(L + 1))
    S = _gpu_S(L, X, cuts)
    assert S.shape == (5, L + 1)
    for j in range(5):
        for c, LA in enumerate(cuts):
            want = entropy.entanglement_entropy(X[:, j], L, LA)
            assert abs(S[j, c] - want) < 1e-10, (j, LA, S[j, c], want)


def test_entropy_closed_forms():
    require_gpu()
    L = 10
    ghz = np.zeros(1 << L, dtype=np.complex128)
    ghz[0] = ghz[-1] = 1 / np.sqrt(2)
    one = np.zeros(1 << L, dtype=np.complex128)  # Bell pair on qubits (0, 1)
    one[0] = one[3] = 1 / np.sqrt(2)
    mx = np.zeros(1 << L, dtype=np.complex128)  # maximally entangled across the middle
    for a in range(1 << (L // 2)):
        mx[a + (a << (L // 2))] = 1
    mx /= np.linalg.norm(mx)
    X = np.stack([ghz, one, mx], axis=1)
    S = _gpu_S(L, X, list(range(L + 1)))
    for LA in range(L + 1):
        assert abs(S[0, LA] - (np.log(2) if 0 < LA < L else 0.0)) < 1e-12
        assert abs(S[1, LA] - (np.log(2) if LA == 1 else 0.0)) < 1e-12
    assert abs(S[2, L // 2] - (L // 2) * np.log(2)) < 1e-11


def test_entropy_of_eigenvectors_L12():
    # eigenvectors returned by the eigensolver (double-float form), every cut
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    L, nev = 12, 16
    h = inputs.disorder(L, 1.0, 3)
    fq = floquet.Floquet(L, 1.0, 0.9045, h)
    ev = torch.empty((nev, 1 << L), dtype=torch.complex128, device="cuda")
    v0 = to_dev(inputs.start_vector(L))
    om, res, nconv, rc = fq.arnoldi_eigs(0.0, 128, nev, 64, v0, precision=floquet.FILTER_DF,
                                         evecs=ev)
    assert rc == 0 and nconv == nev
    cuts = list(range(L + 1))
    S = floquet.entanglement_entropy(L, ev, cuts)
    V = from_dev(ev, 1 << L)
    for j in range(nev):
        v = V[:, j] / np.linalg.norm(V[:, j])
        for LA in cuts:
            assert abs(S[j, LA] - entropy.entanglement_entropy(v, L, LA)) < 1e-10


@pytest.mark.slow
def test_entropy_L20_middle_cut_and_page():
    # the full-size state, middle cut (reduced density matrix 1024 x 1024): against the
    # oracle's SVD, and a random state sits at the Page value to ~1e-3
    require_gpu()
    L = 20
    X = inputs.random_states(1 << L, 2, 44)
    S = _gpu_S(L, X, [1, 7, 10, 13])
    for j in range(2):
        for c, LA in enumerate([1, 7, 10, 13]):
            assert abs(S[j, c] - entropy.entanglement_entropy(X[:, j], L, LA)) < 1e-10
        assert abs(S[j, 2] - entropy.page_entropy(10, 10)) < 2e-3


def test_entropy_rejects_bad_arguments():
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    x = to_dev(inputs.complex_gaussian(1 << 6, 1))
    with pytest.raises(RuntimeError):
        floquet.entanglement_entropy(6, x, [7])
    with pytest.raises(RuntimeError):
        floquet.entanglement_entropy(24, torch.zeros(1, dtype=torch.complex128, device="cuda"),
                                     [12])
