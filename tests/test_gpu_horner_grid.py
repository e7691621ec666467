"""GPU parity of the persistent Horner filter (one cooperative launch for the whole k-step
loop, two alternating tile layouts; rows A1-A5) against the CPU oracle, element by element.

Every chain length with a persistent shape (13 <= L <= 22) is run in all three sweep
precisions, with several vectors per launch, a target phase off zero and filter lengths
whose last step lands in either layout (k even and odd). Tolerances, max |got - want| <=
tol * max |want| per vector, follow from the rounding per U application (about L + 3
roundings per amplitude): complex128 ~1e-15 and double-float ~1e-14 relative per step,
complex64 ~6e-8 per rounding with the errors of k steps adding like a random walk.
"""

import math

import numpy as np
import pytest

from oracle import geosum, model
from paper_2102_05054_gb300 import inputs

from gpu_util import from_dev, require_gpu, to_dev

pytestmark = pytest.mark.gpu


def _maxrel(got, want):
    return np.abs(got - want).max() / np.abs(want).max()


def _tol(sweep, L, k):
    from paper_2102_05054_gb300 import floquet
    if sweep == floquet.C64:
        return 1e-6 * math.sqrt(k) * (L + 3)
    if sweep == floquet.C128_DF:
        return 2e-13 * k * (L + 3)
    return 2e-15 * k * (L + 3)


# shapes per chain length that the autotuner can choose (the persistent kernel's shape table):
# every one is tested
_NSHAPES = {
    "C64": {13: 1, 14: 1, 15: 1, 16: 2, 17: 2, 18: 4, 19: 2, 20: 4, 21: 2, 22: 2},
    "C128_DF": {13: 1, 14: 1, 15: 1, 16: 2, 17: 1, 18: 3, 19: 1, 20: 4, 21: 1, 22: 1},
    "C128": {13: 1, 14: 1, 15: 1, 16: 1, 17: 1, 18: 1, 19: 1, 20: 2, 21: 1, 22: 1},
}
_CASES = [(s, L, i) for s, t in _NSHAPES.items() for L, n in t.items() for i in range(n)]


@pytest.mark.parametrize("sweep_name,L,shape", _CASES)
def test_persistent_horner_matches_oracle(sweep_name, L, shape, monkeypatch):
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    monkeypatch.setenv("FLOQUET_FILTER_KERNEL", "grid")
    monkeypatch.setenv("FLOQUET_GRID_SHAPE", str(shape))
    sweep = getattr(floquet, sweep_name)
    g = 0.9045 if L % 2 else 0.3          # cot form and tan form of the butterfly
    h = inputs.disorder(L, 1.0, 600 + L)
    fq = floquet.Floquet(L, 1.0, g, h)
    op = model.KickedIsing(L, 1.0, g, h)
    nvec = 3 if L <= 18 else 1
    k = 4 if L >= 21 else (5 if L % 2 else 6)
    phi = 0.7
    X = inputs.random_states(1 << L, nvec, 20 + L)
    dt = torch.complex64 if sweep == floquet.C64 else torch.complex128
    t_in = to_dev(X, dt)
    t_out = torch.empty_like(t_in)
    fq.filter_apply(phi, k, t_in, t_out, form=floquet.FORM_HORNER, sweep=sweep)
    torch.cuda.synchronize()
    got = from_dev(t_out).reshape(nvec, 1 << L).T
    for i in range(nvec):
        want = geosum.filter_horner(op, X[:, i], phi, k)
        assert _maxrel(got[:, i], want) < _tol(sweep, L, k), (L, sweep_name, i)


@pytest.mark.parametrize("sweep_name", ["C64", "C128_DF"])
def test_persistent_horner_long_filter_L16(sweep_name):
    # k = 257 (odd: the last step in layout A) and k = 256 against the oracle's Horner form
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    sweep = getattr(floquet, sweep_name)
    L = 16
    h = inputs.disorder(L, 2.0, 5)
    fq = floquet.Floquet(L, 1.0, 0.9045, h)
    op = model.KickedIsing(L, 1.0, 0.9045, h)
    x = inputs.complex_gaussian(1 << L, 77)
    dt = torch.complex64 if sweep == floquet.C64 else torch.complex128
    for k in (256, 257):
        t_in = to_dev(x, dt)
        t_out = torch.empty_like(t_in)
        fq.filter_apply(math.pi / 3, k, t_in, t_out, form=floquet.FORM_HORNER, sweep=sweep)
        torch.cuda.synchronize()
        want = geosum.filter_horner(op, x, math.pi / 3, k)
        assert _maxrel(from_dev(t_out), want) < _tol(sweep, L, k), (sweep_name, k)
