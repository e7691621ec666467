"""GPU parity of the U application (rows A1-A3) and the geometric-sum filter (A4-A5)
against the CPU oracle, through the C ABI.

Tolerances (derived from the arithmetic), element-wise against the largest amplitude: one U
application rounds each amplitude about L + 3 times, so complex128 results agree with the
float64 oracle to ~1e-15 of the largest amplitude and complex64 results to ~(L + 3) * 6e-8.
A k-term filter accumulates k such applications: the error grows at most ~k times
(complex128: < 1e-12 here; complex64: < 5e-7 * sqrt(k) * L, taken with margin).
"""

import math

import numpy as np
import pytest

from oracle import geosum, model
from paper_2102_05054_gb300 import inputs

from gpu_util import from_dev, require_gpu, to_dev

pytestmark = pytest.mark.gpu


def _rel(a, b):
    """Element-wise error: max_i |a_i - b_i| / max_i |b_i|. Every amplitude is held to the
    bound, not only their 2-norm (one wrong amplitude among 2^20 would hide in a norm)."""
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _make(L, J, g, W, seed):
    from paper_2102_05054_gb300 import floquet
    h = inputs.disorder(L, W, seed)
    return floquet.Floquet(L, J, g, h), model.KickedIsing(L, J, g, h)


@pytest.mark.parametrize("L", [3, 4, 5, 7, 10, 11, 12, 13, 14, 16])
@pytest.mark.parametrize("g", [0.3, 0.9045])   # tan form (|tan g| < 1) and cot form
def test_apply_u_c128_matches_oracle(L, g):
    torch = require_gpu()
    fq, op = _make(L, 1.0, g, 1.0, 100 + L)
    X = inputs.random_states(1 << L, 3, 7)
    t_in = to_dev(X, torch.complex128)
    t_out = torch.empty_like(t_in)
    fq.apply_u(t_in, t_out)
    torch.cuda.synchronize()
    got = from_dev(t_out, 1 << L)
    want = op.apply_u_block(X)
    assert np.abs(got - want).max() < 1e-13 * np.abs(want).max() * L


@pytest.mark.parametrize("L", [3, 4, 6, 9, 12, 13, 15, 17])
@pytest.mark.parametrize("g", [0.3, 0.9045, -2.2])
def test_apply_u_c64_matches_oracle(L, g):
    torch = require_gpu()
    fq, op = _make(L, 0.8, g, 2.0, 200 + L)
    X = inputs.random_states(1 << L, 2, 8)
    t_in = to_dev(X, torch.complex64)
    t_out = torch.empty_like(t_in)
    fq.apply_u(t_in, t_out)
    torch.cuda.synchronize()
    got = from_dev(t_out, 1 << L)
    want = op.apply_u_block(X)
    assert _rel(got, want) < 2e-7 * (L + 3)


@pytest.mark.parametrize("dtype_name", ["complex128", "complex64"])
def test_apply_u_in_place_and_special_cases(dtype_name):
    torch = require_gpu()
    dt = getattr(torch, dtype_name)
    tol = 1e-13 if dtype_name == "complex128" else 5e-6
    for (L, J, g) in [(12, 1.0, 0.0), (13, 0.0, 0.7), (14, 1.0, math.pi / 2), (18, 1.0, 0.9045)]:
        fq, op = _make(L, J, g, 1.0, 300 + L)
        x = inputs.complex_gaussian(1 << L, 9)
        t = to_dev(x, dt)
        fq.apply_u(t, t)  # in place
        torch.cuda.synchronize()
        assert _rel(from_dev(t), op.apply_u(x)) < tol


@pytest.mark.parametrize("L", [20])
def test_apply_u_L20_both_dtypes(L):
    # the bench configuration: L = 20, two passes per U (tile bits 12 + 8 for complex64,
    # 11 + 9 for complex128)
    torch = require_gpu()
    fq, op = _make(L, 1.0, 0.9045, 1.0, 1)
    x = inputs.complex_gaussian(1 << L, 5)
    want = op.apply_u(x)
    for dt, tol in [(torch.complex128, 1e-14), (torch.complex64, 5e-6)]:
        t_in = to_dev(x, dt)
        t_out = torch.empty_like(t_in)
        fq.apply_u(t_in, t_out)
        torch.cuda.synchronize()
        assert _rel(from_dev(t_out), want) < tol
    # unitarity at full size: ||U^5 psi|| = ||psi||
    t = to_dev(x, torch.complex128)
    for _ in range(5):
        fq.apply_u(t, t)
    torch.cuda.synchronize()
    assert abs(torch.linalg.norm(t).item() - 1.0) < 1e-13


@pytest.mark.parametrize("L,k,phi", [(6, 1, 0.0), (6, 2, 0.3), (10, 64, 0.0), (12, 37, 1.0),
                                     (14, 50, math.pi / 3), (16, 20, 2.0)])
@pytest.mark.parametrize("form", [0, 1])
def test_filter_c128_matches_oracle(L, k, phi, form):
    torch = require_gpu()
    fq, op = _make(L, 1.0, 0.9045, 1.0, 400 + L)
    X = inputs.random_states(1 << L, 2, 10)
    t_in = to_dev(X, torch.complex128)
    t_out = torch.empty_like(t_in)
    fq.filter_apply(phi, k, t_in, t_out, form=form)
    torch.cuda.synchronize()
    got = from_dev(t_out, 1 << L)
    want = np.stack([geosum.filter_acc(op, X[:, i], phi, k) for i in range(2)], axis=1)
    assert _rel(got, want) < 1e-13 * k


@pytest.mark.parametrize("L,k,phi", [(10, 64, 0.0), (13, 100, 0.5), (16, 40, math.pi / 3)])
@pytest.mark.parametrize("form", [0, 1])
def test_filter_c64_matches_oracle(L, k, phi, form):
    torch = require_gpu()
    fq, op = _make(L, 1.0, 0.9045, 1.0, 500 + L)
    x = inputs.complex_gaussian(1 << L, 11)
    t_in = to_dev(x, torch.complex64)
    t_out = torch.empty_like(t_in)
    fq.filter_apply(phi, k, t_in, t_out, form=form)
    torch.cuda.synchronize()
    want = geosum.filter_acc(op, x, phi, k)
    assert _rel(from_dev(t_out), want) < 5e-7 * math.sqrt(k) * L


def test_filter_repeat_uses_cached_graph_and_is_deterministic():
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    fq, _ = _make(12, 1.0, 0.9045, 1.0, 7)
    x = to_dev(inputs.complex_gaussian(1 << 12, 3), torch.complex64)
    a = torch.empty_like(x)
    b = torch.empty_like(x)
    fq.filter_apply(0.2, 33, x, a)
    floquet.reset_launch_count()
    fq.filter_apply(0.2, 33, x, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    # init + 32 steps of one pass + final conversion
    assert floquet.launch_count() == 1 + 32 + 1


def _g_from_phase(x, k):
    """g_k(e^{ix}) = e^{i(k-1)x/2} sin(kx/2)/sin(x/2), evaluated from the exact phase x
    (no cancellation near x = 0, unlike (1 - w^k)/(1 - w) from a rounded w)."""
    x = math.remainder(x, 2 * math.pi)
    if abs(x) < 1e-300:
        return complex(k)
    return np.exp(0.5j * (k - 1) * x) * math.sin(0.5 * k * x) / math.sin(0.5 * x)


@pytest.mark.parametrize("dtype_name", ["complex128", "complex64"])
def test_filter_full_length_L20_on_exact_eigenvectors(dtype_name):
    # L = 20, k = 16384 (the large workload's filter) on exact eigenvectors from closed-form
    # special cases: g = 0 (basis states, eigenphase -theta_s) and J = 0 (product states).
    # Bound: each U application is exact up to a relative rounding eps = (L + 3) u, and on an
    # eigenvector that rounding is coherent (the same perturbed eigenvalue every step), so the
    # filter output can drift by up to ~ k^2 eps / 2 in absolute terms. complex128: checked
    # against that bound. complex64: that bound is a few percent of |g| at this k, so the
    # check is on what the sweeps must keep: the output is parallel to the eigenvector.
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    dt = getattr(torch, dtype_name)
    L, k, phi = 20, 16384, 0.0
    d = 1 << L
    u = 1.1e-16 if dtype_name == "complex128" else 6e-8
    eps = (L + 3) * u

    def check(fq, v, x):
        t_in = to_dev(v, dt)
        t_out = torch.empty_like(t_in)
        fq.filter_apply(phi, k, t_in, t_out)
        torch.cuda.synchronize()
        out = from_dev(t_out)
        g = _g_from_phase(x, k)
        along = np.vdot(v, out)
        perp = np.linalg.norm(out - along * v)
        if dtype_name == "complex128":
            assert np.linalg.norm(out - g * v) < k * k * eps
            assert perp < 1e-10 * abs(g)
        else:
            # random rounding adds ~ k * eps absolute off the eigenvector direction
            assert perp < k * eps
            assert abs(along - g) < 0.5 * k * eps * k

    # g = 0: basis state |s>, U|s> = exp(-i theta_s)|s>
    h = inputs.disorder(L, 1.0, 1)
    theta = model.diagonal_phases(L, 1.0, h)
    fq = floquet.Floquet(L, 1.0, 0.0, h)
    s = int(np.argmin(np.abs(np.remainder(-theta - phi + np.pi, 2 * np.pi) - np.pi)))
    e = np.zeros(d, dtype=np.complex128)
    e[s] = 1.0
    check(fq, e, -theta[s] - phi)
    # J = 0: product of single-site eigenvectors; the eigenphase is the sum of site phases
    g = 0.9045
    fq = floquet.Floquet(L, 0.0, g, h)
    X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    v = np.ones(1, dtype=np.complex128)
    x = 0.0
    for i in range(L):
        u1 = np.diag([np.exp(-1j * h[i]), np.exp(1j * h[i])]) @ (np.cos(g) * np.eye(2)
                                                                 - 1j * np.sin(g) * X)
        w, vecs = np.linalg.eig(u1)
        j = int(np.argmin(np.abs(np.angle(w))))
        v = np.kron(vecs[:, j] / np.linalg.norm(vecs[:, j]), v)  # qubit i on the higher bits
        x += float(np.angle(w[j]))
    check(fq, v, x - phi)


@pytest.mark.parametrize("L", [3, 5, 10, 11, 12, 16, 20])
def test_apply_u_double_float_sweeps_match_oracle(L):
    # double-float sweeps: ~48-bit significands, so ~(L + 3) * 2^-47 relative per application
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    fq, op = _make(L, 1.0, 0.9045, 1.0, 600 + L)
    X = inputs.random_states(1 << L, 2, 12)
    t_in = to_dev(X, torch.complex128)
    t_out = torch.empty_like(t_in)
    fq.apply_u(t_in, t_out, sweep=floquet.C128_DF)
    torch.cuda.synchronize()
    assert _rel(from_dev(t_out, 1 << L), op.apply_u_block(X)) < 1e-14 * (L + 3)


@pytest.mark.parametrize("L,k,phi,form", [(10, 64, 0.0, 0), (12, 200, 1.0, 0), (13, 50, 0.4, 1),
                                          (16, 40, math.pi / 3, 0)])
def test_filter_double_float_matches_oracle(L, k, phi, form):
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    fq, op = _make(L, 1.0, 0.9045, 1.0, 700 + L)
    x = inputs.complex_gaussian(1 << L, 13)
    t_in = to_dev(x, torch.complex128)
    t_out = torch.empty_like(t_in)
    fq.filter_apply(phi, k, t_in, t_out, form=form, sweep=floquet.C128_DF)
    torch.cuda.synchronize()
    want = geosum.filter_acc(op, x, phi, k)
    assert _rel(from_dev(t_out), want) < 1e-14 * k * (L + 3)


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("L", [13, 15, 18, 20])
def test_every_launch_shape_matches_oracle(variant, L, monkeypatch):
    # the autotuner may pick any launch shape (2, 3 or 4 passes per U); force each one
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    monkeypatch.setenv("FLOQUET_PASS_VARIANT", str(variant))
    fq, op = _make(L, 1.0, 0.9045, 1.0, 800 + L)
    X = inputs.random_states(1 << L, 3, 14)
    want = op.apply_u_block(X)
    for dt, sweep, tol in [(torch.complex128, None, 1e-13 * (L + 3)),
                           (torch.complex64, None, 2e-7 * (L + 3)),
                           (torch.complex128, floquet.C128_DF, 1e-14 * (L + 3))]:
        t_in = to_dev(X, dt)
        t_out = torch.empty_like(t_in)
        fq.apply_u(t_in, t_out, sweep=sweep)
        torch.cuda.synchronize()
        assert _rel(from_dev(t_out, 1 << L), want) < tol, (dt, sweep)
    # and the filter (last pass with the accumulate epilogue) in the same shape
    x = inputs.complex_gaussian(1 << L, 15)
    t_in = to_dev(x, torch.complex128)
    t_out = torch.empty_like(t_in)
    fq.filter_apply(0.3, 5, t_in, t_out, sweep=floquet.C128_DF)
    torch.cuda.synchronize()
    assert _rel(from_dev(t_out), geosum.filter_acc(op, x, 0.3, 5)) < 1e-13


@pytest.mark.parametrize("variant,L", [(4, 18), (4, 19), (4, 20), (4, 21),
                                       (5, 16), (5, 17), (5, 18), (5, 19),
                                       (6, 20), (6, 21), (7, 18), (7, 20),
                                       (8, 18), (8, 19), (8, 20), (8, 21)])
@pytest.mark.parametrize("g", [0.4, 0.9045])   # tan and cot forms of the butterfly
def test_pipelined_double_float_passes_match_oracle(variant, L, g, monkeypatch):
    # double-float shapes 4-8 run the persistent cp.async-pipelined pass kernel (shape 8: its
    # two-CTA cluster form, the tile's top bit exchanged through distributed shared memory) for the
    # first pass and for later passes with 2-4 column bits (L = 21 and 19 add a third pass
    # that falls back to the one-tile-per-CTA kernel); several vectors, in place, and every
    # epilogue (plain phase, accumulate, Horner)
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    monkeypatch.setenv("FLOQUET_PASS_VARIANT", str(variant))
    fq, op = _make(L, 1.0, g, 1.0, 900 + L)
    X = inputs.random_states(1 << L, 3, 16)
    want = op.apply_u_block(X)
    t = to_dev(X, torch.complex128)
    t_out = torch.empty_like(t)
    fq.apply_u(t, t_out, sweep=floquet.C128_DF)
    fq.apply_u(t, t, sweep=floquet.C128_DF)  # in place
    torch.cuda.synchronize()
    assert _rel(from_dev(t_out, 1 << L), want) < 1e-14 * (L + 3)
    assert _rel(from_dev(t, 1 << L), want) < 1e-14 * (L + 3)
    Y = inputs.random_states(1 << L, 2, 17)
    for form in (floquet.FORM_ACC, floquet.FORM_HORNER):
        t_in = to_dev(Y, torch.complex128)
        t_out = torch.empty_like(t_in)
        fq.filter_apply(1.1, 5, t_in, t_out, form=form, sweep=floquet.C128_DF)
        torch.cuda.synchronize()
        got = from_dev(t_out, 1 << L)
        for j in range(2):
            assert _rel(got[:, j], geosum.filter_acc(op, Y[:, j], 1.1, 5)) < 1e-13, form


@pytest.mark.slow
@pytest.mark.parametrize("L", [22, 24])
def test_maximum_sizes_match_oracle(L):
    # the largest states the library accepts (L <= 24: 256 MiB per complex128 state), three
    # or more passes per U with the autotuned shapes; every sweep precision and the Horner
    # filter in double-float
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    fq, op = _make(L, 1.0, 0.9045, 1.0, 1000 + L)
    x = inputs.complex_gaussian(1 << L, 18)
    want = op.apply_u(x)
    for dt, sweep, tol in [(torch.complex128, None, 1e-13 * (L + 3)),
                           (torch.complex64, None, 2e-7 * (L + 3)),
                           (torch.complex128, floquet.C128_DF, 1e-14 * (L + 3))]:
        t_in = to_dev(x, dt)
        t_out = torch.empty_like(t_in)
        fq.apply_u(t_in, t_out, sweep=sweep)
        torch.cuda.synchronize()
        assert _rel(from_dev(t_out), want) < tol, (dt, sweep)
        del t_in, t_out
    t_in = to_dev(x, torch.complex128)
    t_out = torch.empty_like(t_in)
    fq.filter_apply(0.7, 3, t_in, t_out, form=floquet.FORM_HORNER, sweep=floquet.C128_DF)
    torch.cuda.synchronize()
    assert _rel(from_dev(t_out), geosum.filter_acc(op, x, 0.7, 3)) < 1e-13
