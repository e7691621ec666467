"""GPU parity of the brickwork random-circuit operator (Sec. 2, Eqs. U, unitary, matvec)
against the gate-by-gate CPU oracle, through the C ABI.

Tolerances: U applied as two float64 GEMMs (reductions of length d_L and d_R) agrees with
the gate-by-gate oracle to ~1e-15 relative; a k-term filter to ~k * 1e-15; eigenpairs to the
spec bars (|d omega| <= 1e-10, residual <= 1e-10).
"""

import numpy as np
import pytest

from oracle import brickwork, geosum, krylov
from paper_2102_05054_gb300 import inputs

from gpu_util import from_dev, require_gpu, to_dev

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _make(L, seed):
    from paper_2102_05054_gb300 import floquet
    g2, g1 = inputs.brickwork_gates(L, seed)
    return floquet.Floquet.brickwork(L, g2, g1), brickwork.Brickwork(L, g2, g1)


@pytest.mark.parametrize("L", [4, 6, 8, 10, 14, 16])
def test_brickwork_apply_u_matches_oracle(L):
    torch = require_gpu()
    fq, op = _make(L, 60 + L)
    X = inputs.random_states(1 << L, 3, 61)
    want = op.apply_u_block(X)
    t_in = to_dev(X)
    t_out = torch.empty_like(t_in)
    fq.apply_u(t_in, t_out)
    fq.apply_u(t_in, t_in)  # in place
    torch.cuda.synchronize()
    assert _rel(from_dev(t_out, 1 << L), want) < 1e-14
    assert _rel(from_dev(t_in, 1 << L), want) < 1e-14


@pytest.mark.parametrize("L,k", [(8, 17), (12, 64)])
def test_brickwork_filter_both_forms(L, k):
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    fq, op = _make(L, 70 + L)
    Y = inputs.random_states(1 << L, 2, 71)
    for form in (floquet.FORM_ACC, floquet.FORM_HORNER):
        t_in = to_dev(Y)
        t_out = torch.empty_like(t_in)
        fq.filter_apply(0.6, k, t_in, t_out, form=form)
        torch.cuda.synchronize()
        got = from_dev(t_out, 1 << L)
        for j in range(2):
            assert _rel(got[:, j], geosum.filter_acc(op, Y[:, j], 0.6, k)) < 1e-15 * k * 10


def test_brickwork_eigensolver_matches_dense_L10():
    # 50 pairs closest to 1 (the paper's benchmark task) with the paper's parameter rule
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    L, nev = 10, 50
    k, m = floquet.suggest_params(L, nev)
    fq, op = _make(L, 3)
    v0 = to_dev(inputs.start_vector(L))
    ev = torch.empty((nev, 1 << L), dtype=torch.complex128, device="cuda")
    om, res, nconv, rc = fq.arnoldi_eigs(0.0, k, nev, m, v0, evecs=ev)
    assert rc == 0 and nconv == nev
    om_d, X_d, _ = krylov.dense_eigs(op, 0.0, nev)
    assert np.abs(om - om_d).max() < 1e-10
    assert res.max() <= 1e-10
    _, r_cpu, _ = krylov.rayleigh_residual(op, from_dev(ev, 1 << L))
    assert r_cpu.max() <= 1e-10


def test_brickwork_eigensolver_L14_oracle_residuals():
    # a size past dense diagonalisation in a test: residuals recomputed by the oracle's U,
    # and every returned eigenvalue on the unit circle near the target
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    L, nev = 14, 50
    fq, op = _make(L, 4)
    v0 = to_dev(inputs.start_vector(L))
    ev = torch.empty((nev, 1 << L), dtype=torch.complex128, device="cuda")
    om, res, nconv, rc = fq.arnoldi_eigs(0.0, 256, nev, 128, v0, evecs=ev)
    assert rc == 0 and nconv == nev
    _, r_cpu, _ = krylov.rayleigh_residual(op, from_dev(ev, 1 << L))
    assert r_cpu.max() <= 1e-10
    assert np.abs(np.abs(om) - 1).max() < 1e-10


def test_brickwork_rejects_other_precisions():
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    fq, _ = _make(6, 5)
    x = to_dev(inputs.complex_gaussian(64, 1)).to(torch.complex64)
    with pytest.raises(RuntimeError):
        fq.apply_u(x, torch.empty_like(x))
    v0 = to_dev(inputs.start_vector(6))
    with pytest.raises(RuntimeError):
        fq.arnoldi_eigs(0.0, 16, 4, 16, v0, precision=floquet.FILTER_FP32)
    y = to_dev(inputs.complex_gaussian(64, 2))
    with pytest.raises(RuntimeError):  # the accumulate form has no double-float GEMM path
        fq.filter_apply(0.1, 4, y, torch.empty_like(y), form=floquet.FORM_ACC,
                        sweep=floquet.C128_DF)


def test_brickwork_cached_filter_graphs_survive_scratch_growth():
    # a cached one-vector filter graph must stay valid after a wider filter and after a plain
    # U application on many vectors have grown the operator's GEMM scratch
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    L, k = 8, 9
    fq, op = _make(L, 80)
    y = inputs.complex_gaussian(1 << L, 81)
    want = geosum.filter_acc(op, y, 0.3, k)

    def filt(vecs):
        t_in = to_dev(vecs)
        t_out = torch.empty_like(t_in)
        fq.filter_apply(0.3, k, t_in, t_out, form=floquet.FORM_HORNER)
        torch.cuda.synchronize()
        return from_dev(t_out, 1 << L)

    assert _rel(filt(y), want) < 1e-13
    wide = np.stack([y] * 5, axis=1)
    got = filt(wide)
    assert max(_rel(got[:, j], want) for j in range(5)) < 1e-13
    X = inputs.random_states(1 << L, 40, 82)
    t = to_dev(X)
    fq.apply_u(t, torch.empty_like(t))
    torch.cuda.synchronize()
    assert _rel(filt(y), want) < 1e-13


@pytest.mark.parametrize("L,k", [(4, 3), (8, 17), (12, 64), (16, 5)])
def test_brickwork_double_float_filter(L, k):
    # the double-float split-K GEMMs (FP32 pipes): Horner filter against the oracle; each
    # U application sums d_L + d_R products per amplitude with ~2^-48 relative rounding
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    fq, op = _make(L, 90 + L)
    Y = inputs.random_states(1 << L, 2, 91)
    t_in = to_dev(Y)
    t_out = torch.empty_like(t_in)
    fq.filter_apply(0.8, k, t_in, t_out, form=floquet.FORM_HORNER, sweep=floquet.C128_DF)
    torch.cuda.synchronize()
    got = from_dev(t_out, 1 << L)
    for j in range(2):
        assert _rel(got[:, j], geosum.filter_acc(op, Y[:, j], 0.8, k)) < 1e-13 * k


def test_brickwork_eigensolver_double_float_L10():
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    L, nev = 10, 50
    k, m = floquet.suggest_params(L, nev)
    fq, op = _make(L, 3)
    v0 = to_dev(inputs.start_vector(L))
    ev = torch.empty((nev, 1 << L), dtype=torch.complex128, device="cuda")
    om, res, nconv, rc = fq.arnoldi_eigs(0.0, k, nev, m, v0, evecs=ev,
                                         precision=floquet.FILTER_DF)
    assert rc == 0 and nconv == nev
    om_d, _, _ = krylov.dense_eigs(op, 0.0, nev)
    assert np.abs(om - om_d).max() < 1e-10
    _, r_cpu, _ = krylov.rayleigh_residual(op, from_dev(ev, 1 << L))
    assert r_cpu.max() <= 1e-10
