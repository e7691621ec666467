"""GPU parity of the Arnoldi pieces (rows A6-A9) against the CPU oracle, through the C ABI.

Bars (from the spec contract): eigenvalues |d lambda| <= 1e-10, eigenvector overlaps
|<v_ref|v>| >= 1 - 1e-9, residuals ||U v - omega v|| <= 1e-10. Gram-Schmidt and the small
eigensolver are pure float64 and are held to ~1e-13 relative (a few hundred ulps of the
problem's scale).
"""

import math

import numpy as np
import pytest

from oracle import geosum, krylov, model
from paper_2102_05054_gb300 import inputs

from gpu_util import from_dev, require_gpu, to_dev

pytestmark = pytest.mark.gpu


def _overlaps(A, B):
    return np.abs(np.sum(A.conj() * B, axis=0)) / (np.linalg.norm(A, axis=0) *
                                                 np.linalg.norm(B, axis=0))


@pytest.mark.parametrize("d,n", [(1024, 0), (1024, 1), (4096, 17), (65536, 64), (3000, 5)])
def test_gram_schmidt_matches_oracle(d, n):
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    rng = np.random.default_rng(d + n)
    if n:
        V, _ = np.linalg.qr(rng.standard_normal((d, n)) + 1j * rng.standard_normal((d, n)))
    else:
        V = np.zeros((d, 0), dtype=np.complex128)
    w = rng.standard_normal(d) + 1j * rng.standard_normal(d)
    h_ref, beta_ref, q_ref = krylov.cgs2(V, w) if n else (np.zeros(0), np.linalg.norm(w),
                                                           w / np.linalg.norm(w))
    tV = to_dev(V if n else np.zeros((d, 1), dtype=np.complex128))
    tw = to_dev(w)
    h = floquet.gram_schmidt(tV, n, tw)
    torch.cuda.synchronize()
    assert np.abs(h[:n] - h_ref).max(initial=0) < 1e-13 * np.linalg.norm(w)
    assert abs(h[n].real - beta_ref) < 1e-13 * np.linalg.norm(w)
    assert np.abs(from_dev(tw) - q_ref).max() < 1e-13
    if n:
        assert np.abs(V.conj().T @ from_dev(tw)).max() < 1e-14


@pytest.mark.parametrize("n", [1, 2, 3, 8, 37, 64, 100, 160, 256])
def test_small_eig_random(n):
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Af = np.asfortranarray(A)
    Y = torch.empty((n, n), dtype=torch.complex128, device="cuda")  # column-major n x n
    lam = floquet.small_eig(Af, Y)
    Yh = Y.cpu().numpy().T
    # A Y = Y diag(lam), unit columns, descending |lam|, same spectrum as LAPACK
    assert np.abs(A @ Yh - Yh * lam).max() < 1e-12 * np.linalg.norm(A)
    assert np.allclose(np.linalg.norm(Yh, axis=0), 1, atol=1e-13)
    assert np.all(np.diff(np.abs(lam)) <= 1e-12)
    ref = np.linalg.eigvals(A)
    for x in lam:
        assert np.min(np.abs(ref - x)) < 1e-10 * np.linalg.norm(A)


def test_small_eig_structured():
    # Hessenberg input (an Arnoldi projection) and a unitary with clustered spectrum
    require_gpu()
    from paper_2102_05054_gb300 import floquet
    L, k, m = 8, 16, 40
    op = model.KickedIsing(L, 1.0, 0.9045, inputs.disorder(L, 1.0, 3))
    from oracle import geosum
    _, H = krylov.arnoldi(lambda x: geosum.filter_acc(op, x, 0.0, k),
                          inputs.complex_gaussian(1 << L, 1), m)
    Hm = np.asfortranarray(H[:m])
    lam = floquet.small_eig(Hm)
    ref = np.linalg.eigvals(Hm)
    for x in lam:
        assert np.min(np.abs(ref - x)) < 1e-11 * np.abs(ref).max()
    U = model.KickedIsing(6, 1.0, 0.9045, inputs.disorder(6, 4.0, 5)).dense()
    lam = floquet.small_eig(np.asfortranarray(U))
    assert np.allclose(np.abs(lam), 1, atol=1e-12)
    _ = floquet


def test_ritz_residuals_matches_oracle():
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    L = 12
    h = inputs.disorder(L, 1.0, 8)
    fq = floquet.Floquet(L, 1.0, 0.9045, h)
    op = model.KickedIsing(L, 1.0, 0.9045, h)
    X = inputs.random_states(1 << L, 5, 3) * np.array([1, 2, 0.5, 3, 1])
    om, res = fq.ritz_residuals(to_dev(X))
    om_ref, res_ref, _ = krylov.rayleigh_residual(op, X)
    assert np.abs(om - om_ref).max() < 1e-14
    assert np.abs(res - res_ref).max() < 1e-13
    _ = torch


def _solve(L, J, g, W, seed, phi, k, nev, m, precision=0, **kw):
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    h = inputs.disorder(L, W, seed)
    fq = floquet.Floquet(L, J, g, h)
    op = model.KickedIsing(L, J, g, h)
    v0 = to_dev(inputs.start_vector(L))
    ev = torch.empty((nev, 1 << L), dtype=torch.complex128, device="cuda")
    om, res, nconv, rc = fq.arnoldi_eigs(phi, k, nev, m, v0, precision=precision, evecs=ev, **kw)
    return om, res, nconv, rc, from_dev(ev, 1 << L).reshape(1 << L, nev), op


def _check_against_dense(om, res, X, op, phi, nev, tol_l=1e-10, tol_ov=1e-9, tol_r=1e-10):
    om_d, X_d, _ = krylov.dense_eigs(op, phi, nev)
    assert np.abs(om - om_d).max() < tol_l, np.abs(om - om_d).max()
    assert _overlaps(X_d, X).min() > 1 - tol_ov
    assert res.max() <= tol_r
    # residuals recomputed by the oracle's own U
    _, r_cpu, _ = krylov.rayleigh_residual(op, X)
    assert r_cpu.max() <= tol_r


def test_arnoldi_eigs_L10_config_fp64():
    cfg = inputs.WORKLOADS["kicked_ising_L10"]
    om, res, nconv, rc, X, op = _solve(cfg["L"], 1.0, 0.9045, cfg["W"], cfg["seed"], cfg["phi"],
                                       cfg["k"], cfg["nev"], cfg["m"])
    assert rc == 0 and nconv == cfg["nev"]
    _check_against_dense(om, res, X, op, cfg["phi"], cfg["nev"])


@pytest.mark.parametrize("phi", [0.0, 1.3, -2.9])
def test_arnoldi_eigs_with_restarts(phi):
    # a Krylov space too small for one build: the Krylov-Schur restarts must be exercised
    om, res, nconv, rc, X, op = _solve(11, 1.0, 0.9045, 1.0, 4, phi, 128, 12, 30)
    assert rc == 0 and nconv == 12
    _check_against_dense(om, res, X, op, phi, 12)


def test_arnoldi_eigs_fp32_filter_form_L12():
    om, res, nconv, rc, X, op = _solve(12, 1.0, 0.9045, 1.0, 2, 0.0, 128, 24, 96, precision=1)
    assert rc == 0 and nconv == 24
    _check_against_dense(om, res, X, op, 0.0, 24)


def test_arnoldi_eigs_special_case_g0_L16():
    # g = 0: exact eigenvalues exp(-i theta_s) in closed form at L = 16 (the L16 workload size)
    L, phi, k, nev, m = 16, math.pi / 3, 1024, 50, 160
    om, res, nconv, rc, X, op = _solve(L, 1.0, 0.0, 2.0, 1, phi, k, nev, m)
    lam = model.spectrum_g0(L, 1.0, inputs.disorder(L, 2.0, 1))
    want = lam[krylov.select_closest(lam, phi, nev)]
    assert rc == 0 and nconv == nev
    assert np.abs(om - want).max() < 1e-10
    assert res.max() < 1e-10


@pytest.mark.parametrize("precision", [0, 2])
def test_arnoldi_eigs_batched_matches_dense(precision):
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    L, k, nev, m = 10, 64, 8, 48
    hs, _ = inputs.batched_disorder(L, (0.5, 2.0), 2, 10)
    phis = np.array([0.0, math.pi / 2, math.pi])
    v0 = to_dev(inputs.start_vector(L))
    om, res, nconv, rc = floquet.arnoldi_eigs_batched(L, 1.0, 0.9045, hs, phis, k, nev, m, v0,
                                                      precision=precision)
    assert rc == 0
    for r in range(hs.shape[0]):
        op = model.KickedIsing(L, 1.0, 0.9045, hs[r])
        for p, phi in enumerate(phis):
            om_d, _, _ = krylov.dense_eigs(op, phi, nev)
            assert np.abs(om[r, p] - om_d).max() < 1e-10
            assert res[r, p].max() < 1e-10
            assert nconv[r, p] == nev
    _ = torch


def test_arnoldi_eigs_double_float_form_L12():
    om, res, nconv, rc, X, op = _solve(12, 1.0, 0.9045, 1.0, 2, 0.0, 128, 24, 96, precision=2)
    assert rc == 0 and nconv == 24
    _check_against_dense(om, res, X, op, 0.0, 24)


def test_arnoldi_eigs_double_float_special_case_g0_L16():
    L, phi, k, nev, m = 16, math.pi / 3, 1024, 50, 160
    om, res, nconv, rc, X, op = _solve(L, 1.0, 0.0, 2.0, 1, phi, k, nev, m, precision=2)
    lam = model.spectrum_g0(L, 1.0, inputs.disorder(L, 2.0, 1))
    want = lam[krylov.select_closest(lam, phi, nev)]
    assert rc == 0 and nconv == nev
    assert np.abs(om - want).max() < 1e-10


@pytest.mark.parametrize("precision", [0, 2])
def test_arnoldi_eigs_with_paper_params_L12(precision):
    # filter length and Krylov dimension from the paper's rule (floquet_suggest_params):
    # L = 12, nev = 24 gives m = 128, k = 51 terms
    from paper_2102_05054_gb300 import floquet
    k, m = floquet.suggest_params(12, 24)
    assert (k, m) == (51, 128)
    om, res, nconv, rc, X, op = _solve(12, 1.0, 0.9045, 1.0, 6, 0.4, k, 24, m,
                                       precision=precision)
    assert rc == 0 and nconv == 24
    _check_against_dense(om, res, X, op, 0.4, 24)


@pytest.mark.parametrize("precision", [0, 2])
@pytest.mark.parametrize("L,nev,m,k,phi", [(3, 1, 7, 2, 0.0), (3, 2, 8, 4, 1.0),
                                           (4, 3, 8, 3, math.pi), (5, 2, 24, 4, -math.pi),
                                           (8, 1, 12, 16, 2.0)])
def test_arnoldi_eigs_degenerate_sizes(L, nev, m, k, phi, precision):
    # the smallest chain (d = 8), one pair, the shortest filter (k = 2 terms), the target
    # at +-pi, and Krylov dimensions up to the space dimension (m = d: the Krylov space is
    # the whole space, the last basis vector is zero). With a filter this weak and a tiny
    # Krylov space (say k = 2, m = 4 of d = 8) the |g_k| ratios are close to one and the
    # solve may end with FLOQUET_ENOCONV: that is the method's limit, not tested here.
    om, res, nconv, rc, X, op = _solve(L, 1.0, 0.9045, 1.0, 20 + L, phi, k, nev, m,
                                       precision=precision)
    assert rc == 0 and nconv == nev
    _check_against_dense(om, res, X, op, phi, nev)


def test_arnoldi_eigs_restart_limit_returns_partial():
    # max_restarts = 0 with a Krylov space too small to converge: FLOQUET_ENOCONV, the
    # converged count and the pairs found so far are reported, nothing is left running
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    L = 11
    fq = floquet.Floquet(L, 1.0, 0.9045, inputs.disorder(L, 1.0, 4))
    v0 = to_dev(inputs.start_vector(L))
    om, res, nconv, rc = fq.arnoldi_eigs(0.0, 16, 12, 20, v0, max_restarts=0)
    assert rc == floquet.ENOCONV
    assert 0 <= nconv < 12
    # the operator stays usable
    om2, res2, nconv2, rc2 = fq.arnoldi_eigs(0.0, 128, 12, 30, v0)
    assert rc2 == 0 and nconv2 == 12 and res2.max() <= 1e-10
    _ = torch


def test_arnoldi_eigs_invariant_start_vector():
    # g = 0: U is diagonal, and a start vector on one basis state spans an invariant Krylov
    # space of dimension 1 (exact breakdown, beta = 0). One pair is found exactly; asking for
    # two cannot succeed from this start: the call reports it without NaN or a fault
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    L = 6
    h = inputs.disorder(L, 1.0, 7)
    fq = floquet.Floquet(L, 1.0, 0.0, h)
    lam = model.spectrum_g0(L, 1.0, h)
    e0 = np.zeros(1 << L, dtype=np.complex128)
    e0[5] = 1
    v0 = to_dev(e0)
    # the target sits on that eigenvalue, so it is inside the filter's main lobe (a value
    # outside the lobe is never certified as the closest)
    phi = float(np.angle(lam[5]))
    om, res, nconv, rc = fq.arnoldi_eigs(phi, 8, 1, 10, v0, max_restarts=3, check=False)
    assert rc == 0 and nconv == 1
    assert abs(om[0] - lam[5]) < 1e-12 and res[0] < 1e-12
    om, res, nconv, rc = fq.arnoldi_eigs(phi, 8, 2, 10, v0, max_restarts=3, check=False)
    assert rc == floquet.ENOCONV and nconv <= 1
    # no NaN: a pair that was not found is marked by eigenvalue 0 and residual +inf
    assert not np.any(np.isnan(om)) and not np.any(np.isnan(res))
    for w, r in zip(om, res):
        assert (abs(abs(w) - 1) < 1e-12 and r < 1e-12) or (w == 0 and np.isinf(r))
    _ = torch


@pytest.mark.parametrize("sweep", ["c64", "df"])
@pytest.mark.parametrize("K", [2, 3, 64, 257])
def test_polish_correction_matches_oracle_defect_coefficients(K, sweep):
    # out_j = q_j(U) r_j with the oracle's defect coefficients a_l(omega_j) at target phi,
    # for Ritz values on the circle (at and away from the target) and inside / outside it
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    L, phi = 10, 0.4
    h = inputs.disorder(L, 1.0, 21)
    fq = floquet.Floquet(L, 1.0, 0.9045, h)
    op = model.KickedIsing(L, 1.0, 0.9045, h)
    omega = np.array([np.exp(0.4j), np.exp(-2.0j), 0.999 * np.exp(0.7j), 1.001 * np.exp(0.41j)])
    n = omega.size
    X = inputs.random_states(1 << L, n, 5)
    R = op.apply_u_block(X) - X * omega
    want = np.zeros_like(R)
    for j in range(n):
        a = geosum.defect_coefficients(omega[j], phi, K)
        p = R[:, j].copy()
        for l in range(K - 1):
            want[:, j] += a[l] * p
            p = op.apply_u(p)
    tR = to_dev(R)
    tout = torch.empty_like(tR)
    fq.polish_correction(phi, K, omega, tR, tout,
                         sweep=floquet.C64 if sweep == "c64" else floquet.C128_DF)
    torch.cuda.synchronize()
    got = from_dev(tout, 1 << L)
    # ~(L + 3) roundings per U application, accumulated over K - 1 terms
    u = 6e-8 if sweep == "c64" else 4e-15
    tol = 4 * u * (L + 3) * math.sqrt(K)
    for j in range(n):
        assert np.abs(got[:, j] - want[:, j]).max() <= tol * np.abs(want[:, j]).max(), j
    assert np.array_equal(from_dev(tR, 1 << L), R)  # the input is left untouched


def test_polish_correction_rejections():
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    fq = floquet.Floquet(9, 0.7, 0.4, inputs.disorder(9, 2.0, 3))
    omega = np.array([1.0, 1j])
    tR = to_dev(inputs.random_states(1 << 9, 2, 9))
    tout = torch.empty_like(tR)
    with pytest.raises(RuntimeError):
        fq.polish_correction(0.0, 1, omega, tR, tout)                      # K < 2
    with pytest.raises(RuntimeError):
        fq.polish_correction(0.0, 8, omega, tR, tout, sweep=floquet.C128)  # sweep type
    with pytest.raises(RuntimeError):
        fq.polish_correction(0.0, 8, np.array([np.nan, 1.0]), tR, tout)    # omega not finite
    with pytest.raises(RuntimeError):
        fq.polish_correction(0.0, 8, omega, tR, tR)                        # out overlaps R


def test_fp32_filter_form_with_double_float_corrections_L12(monkeypatch):
    # the polish with its correction sweeps fixed to double-float (by default it starts in
    # complex64 and switches once the worst residual stops halving)
    monkeypatch.setenv("FLOQUET_POLISH_SWEEP", "df")
    om, res, nconv, rc, X, op = _solve(12, 1.0, 0.9045, 1.0, 2, 0.0, 128, 24, 96, precision=1)
    assert rc == 0 and nconv == 24
    _check_against_dense(om, res, X, op, 0.0, 24)


def test_fp32_filter_form_switches_corrections_mid_polish_L12(monkeypatch, capfd):
    # complex64 corrections first, double-float from the polish's second iteration on: the
    # switch happens inside the loop (the library reports it on stderr when verbose)
    monkeypatch.setenv("FLOQUET_POLISH_DF_FROM", "1")
    monkeypatch.setenv("FLOQUET_VERBOSE", "1")
    om, res, nconv, rc, X, op = _solve(12, 1.0, 0.9045, 1.0, 2, 0.0, 128, 24, 96, precision=1)
    err = capfd.readouterr().err
    assert rc == 0 and nconv == 24
    _check_against_dense(om, res, X, op, 0.0, 24)
    if "floquet polish: iter 1 " in err:   # the polish ran past its first iteration
        assert "switching to double-float corrections at iteration 1" in err


@pytest.mark.parametrize("name,other", [("kicked_ising_L16", 0), ("kicked_ising_L18_fp32filter", 2)])
def test_fp32_filter_form_at_configs_L16_L18(name, other):
    # the FP32-filter form at the L = 16 and L = 18 configurations: every returned residual
    # <= 1e-10 by the oracle's U, eigenvalues equal to the FP64 (L = 16) or double-float
    # (L = 18) form's to 1e-10
    cfg = inputs.WORKLOADS[name]
    L, W, seed, phi = cfg["L"], cfg["W"], cfg["seed"], cfg["phi"]
    k, m, nev = cfg["k"], cfg["m"], cfg["nev"]
    om, res, nconv, rc, X, op = _solve(L, 1.0, 0.9045, W, seed, phi, k, nev, m, precision=1)
    assert rc == 0 and nconv == nev and res.max() <= 1e-10
    om_cpu, r_cpu, _ = krylov.rayleigh_residual(op, X)
    assert np.abs(om_cpu - om).max() < 1e-12
    assert r_cpu.max() <= 1e-10
    om2, res2, nconv2, rc2, _, _ = _solve(L, 1.0, 0.9045, W, seed, phi, k, nev, m,
                                          precision=other)
    assert rc2 == 0 and nconv2 == nev
    ok, dev = _same_set(om, om2, 1e-10)
    assert ok, dev


def _angles(om, phi):
    return np.abs(np.angle(om * np.exp(-1j * phi)))


def _same_set(a, b, tol):
    """Every eigenvalue of a matches one of b to tol (unit-circle values, so sort by angle)."""
    a = np.sort_complex(a)
    d = np.abs(a[:, None] - b[None, :]).min(axis=1)
    return d.max() <= tol, d.max()


def test_config_L16_oracle_residuals_and_completeness():
    # the physical L = 16 configuration (h ~ U[-2, 2], phi = pi/3, k = 1024, m = 160, nev = 50)
    cfg = inputs.WORKLOADS["kicked_ising_L16"]
    L, W, seed, phi = cfg["L"], cfg["W"], cfg["seed"], cfg["phi"]
    k, m, nev = cfg["k"], cfg["m"], cfg["nev"]
    om, res, nconv, rc, X, op = _solve(L, 1.0, 0.9045, W, seed, phi, k, nev, m)
    assert rc == 0 and nconv == nev and res.max() <= 1e-10
    # every pair, by the oracle's U: Rayleigh quotient and residual
    om_cpu, r_cpu, _ = krylov.rayleigh_residual(op, X)
    assert np.abs(om_cpu - om).max() < 1e-12
    assert r_cpu.max() <= 1e-10
    assert np.abs(X.conj().T @ X - np.eye(nev)).max() < 1e-9
    # completeness: a second solve with half the filter length returns the same 50 values
    om2, res2, nconv2, rc2, _, _ = _solve(L, 1.0, 0.9045, W, seed, phi, k // 2, nev, m)
    assert rc2 == 0 and nconv2 == nev
    ok, dev = _same_set(om, om2, 1e-10)
    assert ok, dev
    # ... and solves centred at phi -/+ delta agree with it on every value nearer to phi than
    # their own farthest one (a missed eigenvalue would show up in one set and not the other)
    delta = 0.25 * _angles(om, phi).max()
    for s in (-1.0, 1.0):
        ps = phi + s * delta
        om3, res3, nconv3, rc3, _, _ = _solve(L, 1.0, 0.9045, W, seed, ps, k, nev, m)
        assert rc3 == 0 and nconv3 == nev and res3.max() <= 1e-10
        a3 = _angles(om3, ps)
        reach = a3.max()
        inside = np.abs(np.angle(om * np.exp(-1j * ps))) < reach - 1e-9
        assert inside.sum() >= nev // 2
        ok, dev = _same_set(om[inside], om3, 1e-10)
        assert ok, dev
        back = _angles(om3, phi) < _angles(om, phi).max() - 1e-9
        ok, dev = _same_set(om3[back], om, 1e-10)
        assert ok, dev
