"""Pins of the CPU oracle against quantities fixed independently of it.

Each test checks the oracle against something it does not compute itself: dense matrix
exponentials of Kronecker-product generators, brute-force loops on tiny inputs, closed-form
spectra of special cases, the paper's statements about g_k (tests/golden), unitarity and
exact algebraic identities. The ``planted`` tests put a plausible mistake into the oracle
(on the CPU) and check that one of these pins catches it.
"""

import math
import os

import numpy as np
import pytest

from oracle import geosum, krylov, model
from paper_2102_05054_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _sorted_on_circle(w):
    w = np.asarray(w)
    return w[np.lexsort((np.abs(w), np.angle(w)))]


def _same_multiset_on_circle(a, b, tol):
    """Every value of a has a partner in b within tol (bipartite by greedy nearest)."""
    a = list(np.asarray(a))
    b = list(np.asarray(b))
    assert len(a) == len(b)
    bb = np.array(b)
    used = np.zeros(len(bb), dtype=bool)
    for x in a:
        dist = np.abs(bb - x)
        dist[used] = np.inf
        j = int(np.argmin(dist))
        assert dist[j] <= tol, (x, dist[j])
        used[j] = True


# ---------------------------------------------------------------- model: U = D K


@pytest.mark.parametrize("L", [3, 4, 5])
def test_phases_brute_force(L):
    rng = np.random.default_rng(7 + L)
    J = 0.7
    h = rng.uniform(-1, 1, L)
    theta = model.diagonal_phases(L, J, h)
    for s in range(1 << L):
        zs = [1 if ((s >> i) & 1) == 0 else -1 for i in range(L)]
        want = 0.0
        for i in range(L):
            want += J * zs[i] * zs[(i + 1) % L] + h[i] * zs[i]
        assert abs(theta[s] - want) < 1e-13


@pytest.mark.parametrize("L,J,g", [(3, 1.0, 0.9045), (4, 0.3, 0.2), (5, 1.0, 1.3),
                                   (6, -0.8, 0.9045), (7, 1.0, 2.5)])
def test_apply_u_matches_dense_expm(L, J, g):
    h = inputs.disorder(L, 1.5, 100 + L)
    op = model.KickedIsing(L, J, g, h)
    U_ref = model.dense_u_expm(L, J, g, h)
    assert np.abs(op.dense() - U_ref).max() < 1e-13


def test_unitarity_dense():
    L = 8
    op = model.KickedIsing(L, 1.0, 0.9045, inputs.disorder(L, 1.0, 3))
    U = op.dense()
    assert np.abs(U.conj().T @ U - np.eye(1 << L)).max() < 1e-13


def test_norm_preserved_L14():
    L = 14
    op = model.KickedIsing(L, 1.0, 0.9045, inputs.disorder(L, 1.0, 4))
    psi = inputs.complex_gaussian(1 << L, 9)
    for _ in range(5):
        psi = op.apply_u(psi)
    assert abs(np.linalg.norm(psi) - 1.0) < 1e-13


def test_special_case_g0_any_L():
    # g = 0: U = D, eigenpairs (exp(-i theta_s), |s>) in closed form, checked at L = 16.
    L = 16
    h = inputs.disorder(L, 2.0, 5)
    op = model.KickedIsing(L, 1.0, 0.0, h)
    lam = model.spectrum_g0(L, 1.0, h)
    rng = np.random.default_rng(0)
    for s in rng.integers(0, 1 << L, 20):
        e = np.zeros(1 << L, dtype=np.complex128)
        e[s] = 1.0
        u = op.apply_u(e)
        assert abs(u[s] - lam[s]) < 1e-14
        u[s] = 0
        assert np.abs(u).max() < 1e-14


def test_special_case_g0_dense_spectrum():
    L = 7
    h = inputs.disorder(L, 1.0, 6)
    op = model.KickedIsing(L, 1.0, 0.0, h)
    _same_multiset_on_circle(np.linalg.eigvals(op.dense()), model.spectrum_g0(L, 1.0, h), 1e-12)


def test_special_case_j0_spectrum():
    L = 7
    h = inputs.disorder(L, 1.0, 8)
    op = model.KickedIsing(L, 0.0, 0.9045, h)
    _same_multiset_on_circle(np.linalg.eigvals(op.dense()), model.spectrum_j0(L, 0.9045, h),
                             1e-11)


@pytest.mark.parametrize("L", [6, 7])
def test_special_case_g_half_pi_spectrum(L):
    h = inputs.disorder(L, 1.0, 9)
    op = model.KickedIsing(L, 1.0, math.pi / 2, h)
    _same_multiset_on_circle(np.linalg.eigvals(op.dense()),
                             model.spectrum_g_half_pi(L, 1.0, h), 1e-11)


# ---------------------------------------------------------------- filter g_k(U)


def _paper_facts():
    facts = {}
    with open(os.path.join(GOLDEN, "paper_gk_facts.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, value, _cite = [x.strip() for x in line.split("|")]
            facts[name] = value
    return facts


@pytest.mark.parametrize("k", [2, 7, 30, 64, 1024])
def test_gk_paper_facts(k):
    facts = _paper_facts()
    n_terms = k
    phi = 0.37
    peak = eval(facts["peak_modulus"], {"n_terms": n_terms})
    zero = eval(facts["first_zero_offset"], {"n_terms": n_terms, "pi": math.pi})
    assert abs(geosum.gk_closed(np.exp(1j * phi), phi, k)[0] - peak) < 1e-12
    # closed form of the paper against direct summation of the series
    x = np.linspace(-math.pi, math.pi, 41) + 1e-3
    w = np.exp(1j * x)
    direct = sum(w ** j for j in range(k))
    paper = eval(facts["closed_form"], {"n_terms": n_terms, "w": w})
    assert np.abs(paper - direct).max() < 1e-9 * k
    assert np.abs(geosum.gk_closed(np.exp(1j * (x + phi)), phi, k) - direct).max() < 1e-9 * k
    # zeros at +-2 pi / k, and |g| falls monotonically across the main lobe
    for sgn in (+1, -1):
        assert abs(geosum.gk_closed(np.exp(1j * (phi + sgn * zero)), phi, k)[0]) < 1e-9 * k
    t = np.linspace(0, zero, 200)
    mod = geosum.gk_on_circle(phi + t, phi, k)
    assert np.all(np.diff(mod) <= 1e-9 * k)
    # the sine-ratio form agrees with the closed form
    assert np.allclose(mod, np.abs(geosum.gk_closed(np.exp(1j * (phi + t)), phi, k)),
                       atol=1e-9 * k)


def test_lobe_count_statistics():
    # 2d/k eigenvalues on the outer lobe on average (Sec. 3); across targets the mean count
    # over 16 targets must be close to 2d/k.
    L, k = 10, 32
    op = model.KickedIsing(L, 1.0, 0.9045, inputs.disorder(L, 1.0, 11))
    ev = np.linalg.eigvals(op.dense())
    counts = [np.sum(krylov.angular_distance(ev, phi) < 2 * math.pi / k)
              for phi in np.linspace(0, 2 * math.pi, 16, endpoint=False)]
    expect = eval(_paper_facts()["lobe_count"], {"d": 1 << L, "n_terms": k})
    assert abs(np.mean(counts) - expect) < 0.15 * expect


def test_filter_closed_form_on_exact_eigenvectors():
    L, k, phi = 8, 37, 0.4
    op = model.KickedIsing(L, 1.0, 0.9045, inputs.disorder(L, 1.0, 12))
    w, v = np.linalg.eig(op.dense())
    for i in range(0, 1 << L, 17):
        out = geosum.filter_acc(op, v[:, i], phi, k)
        want = geosum.gk_closed(w[i:i + 1], phi, k)[0] * v[:, i]
        assert np.abs(out - want).max() < 1e-11 * k


def test_filter_peaks_at_target_eigenvalue():
    # Sec. 3: the phase factor rotates the target to 1, where |g_k| peaks at the number of
    # terms. Choose phi = arg(omega) for an exact eigenvalue: g_k(U) v = k v.
    L, k = 7, 23
    op = model.KickedIsing(L, 1.0, 0.9045, inputs.disorder(L, 1.0, 23))
    w, v = np.linalg.eig(op.dense())
    for i in (0, 5, 40):
        phi = float(np.angle(w[i]))
        out = geosum.filter_acc(op, v[:, i], phi, k)
        assert np.abs(out - k * v[:, i]).max() < 1e-11 * k
        out = geosum.filter_horner(op, v[:, i], phi, k)
        assert np.abs(out - k * v[:, i]).max() < 1e-11 * k


def test_filter_forms_agree_with_dense_definition():
    L, k, phi = 6, 11, 1.1
    op = model.KickedIsing(L, 1.0, 0.9045, inputs.disorder(L, 1.0, 13))
    psi = inputs.complex_gaussian(1 << L, 14)
    G = geosum.filter_dense(op.dense(), phi, k)
    a = geosum.filter_acc(op, psi, phi, k)
    b = geosum.filter_horner(op, psi, phi, k)
    assert np.abs(a - G @ psi).max() < 1e-12
    assert np.abs(b - G @ psi).max() < 1e-12


def test_filter_telescoping_identity():
    # (1 - z U) g_k(U) psi = psi - z^k U^k psi
    L, k, phi = 12, 50, math.pi / 3
    op = model.KickedIsing(L, 1.0, 0.9045, inputs.disorder(L, 2.0, 15))
    psi = inputs.complex_gaussian(1 << L, 16)
    acc = geosum.filter_acc(op, psi, phi, k)
    lhs = acc - geosum.zpow(phi, 1) * op.apply_u(acc)
    uk = psi.copy()
    for _ in range(k):
        uk = op.apply_u(uk)
    rhs = psi - geosum.zpow(phi, k) * uk
    assert np.abs(lhs - rhs).max() < 1e-12


def test_filter_commutes_with_u():
    L, k, phi = 10, 20, 0.9
    op = model.KickedIsing(L, 1.0, 0.9045, inputs.disorder(L, 1.0, 17))
    psi = inputs.complex_gaussian(1 << L, 18)
    a = op.apply_u(geosum.filter_acc(op, psi, phi, k))
    b = geosum.filter_acc(op, op.apply_u(psi), phi, k)
    assert np.abs(a - b).max() < 1e-12


# ---------------------------------------------------------------- Arnoldi and eigenpairs


def test_arnoldi_relation():
    L, k, phi, m = 8, 16, 0.0, 24
    op = model.KickedIsing(L, 1.0, 0.9045, inputs.disorder(L, 1.0, 19))
    v0 = inputs.complex_gaussian(1 << L, 20)
    A = lambda x: geosum.filter_acc(op, x, phi, k)  # noqa: E731
    V, H = krylov.arnoldi(A, v0, m)
    assert np.abs(V.conj().T @ V - np.eye(m + 1)).max() < 1e-13
    AV = np.stack([A(V[:, j]) for j in range(m)], axis=1)
    assert np.abs(AV - V @ H).max() < 1e-12 * np.abs(H).max()
    assert np.abs(np.tril(H, -2)).max() == 0.0
    # H_m equals the projection V^H g_k(U) V (Eq. arnoldi)
    assert np.abs(V[:, :m].conj().T @ AV - H[:m]).max() < 1e-12 * np.abs(H).max()


def test_rayleigh_residual_identity_off_eigenvectors():
    # For unitary U and a unit vector x that is NOT an eigenvector, omega = <x|U|x> and
    # ||U x - omega x||^2 = ||U x||^2 - 2 Re(conj(omega) <x|U x>) + |omega|^2 = 1 - |omega|^2
    # (exact algebra, independent of the code). A residual that dropped the omega term,
    # returned its square, or forgot the normalisation of x fails it; so does omega taken as
    # <Ux|x> (its conjugate) unless the residual is also computed with that conjugate.
    L = 8
    op = model.KickedIsing(L, 1.0, 0.9045, inputs.disorder(L, 1.0, 21))
    X = inputs.random_states(1 << L, 6, 40) * np.array([1.0, 3.0, 0.25, 1.0, 7.0, 0.5])
    omega, resid, Xn = krylov.rayleigh_residual(op, X)
    assert np.allclose(np.linalg.norm(Xn, axis=0), 1.0, atol=1e-14)
    for i in range(X.shape[1]):
        x = X[:, i] / np.linalg.norm(X[:, i])
        w = np.vdot(x, op.apply_u(x))
        assert abs(omega[i] - w) < 1e-14
        assert abs(omega[i]) < 0.5                        # random vectors: far from the circle
        assert abs(resid[i] ** 2 - (1.0 - abs(omega[i]) ** 2)) < 1e-13
    # and on a mixture of two exact eigenvectors with weights (a, b): omega = a^2 l1 + b^2 l2,
    # residual^2 = a^2 b^2 |l1 - l2|^2
    w_all, V = np.linalg.eig(op.dense())
    a, b = 0.8, 0.6
    x = a * V[:, 3] / np.linalg.norm(V[:, 3]) + b * V[:, 7] / np.linalg.norm(V[:, 7])
    om2, r2, _ = krylov.rayleigh_residual(op, x[:, None])
    assert abs(om2[0] - (a * a * w_all[3] + b * b * w_all[7])) < 1e-12
    assert abs(r2[0] ** 2 - (a * b * abs(w_all[3] - w_all[7])) ** 2) < 1e-12


def test_select_closest_brute_force():
    rng = np.random.default_rng(21)
    ang = rng.uniform(-math.pi, math.pi, 50)
    omega = np.exp(1j * ang)
    phi = 2.5
    idx = krylov.select_closest(omega, phi, 7)
    dist = [abs((a - phi + math.pi) % (2 * math.pi) - math.pi) for a in ang]
    want = sorted(range(50), key=lambda i: dist[i])[:7]
    assert list(idx) == want


def test_dense_eigs_special_case_g0():
    L, phi, nev = 8, 1.0, 12
    h = inputs.disorder(L, 1.0, 22)
    op = model.KickedIsing(L, 1.0, 0.0, h)
    om, X, r = krylov.dense_eigs(op, phi, nev)
    lam = model.spectrum_g0(L, 1.0, h)
    want = lam[krylov.select_closest(lam, phi, nev)]
    assert np.abs(om - want).max() < 1e-13
    assert r.max() < 1e-13


@pytest.mark.slow
def test_arpack_route_matches_dense_L10():
    cfg = inputs.WORKLOADS["kicked_ising_L10"]
    L = cfg["L"]
    op = model.KickedIsing(L, inputs.J_DEFAULT, inputs.G_DEFAULT,
                           inputs.disorder(L, cfg["W"], cfg["seed"]))
    om_d, X_d, r_d = krylov.dense_eigs(op, cfg["phi"], cfg["nev"])
    om_a, X_a, r_a = krylov.arpack_eigs(op, cfg["phi"], cfg["k"], cfg["nev"], cfg["m"],
                                        inputs.start_vector(L))
    assert np.abs(om_d - om_a).max() < 1e-10
    ov = np.abs(np.sum(X_d.conj() * X_a, axis=0))
    assert ov.min() > 1 - 1e-9
    assert r_a.max() < 1e-10
    # the paper's float64 residuals sit near 1e-15 (Tab. bench); the oracle's too
    facts = _paper_facts()
    assert r_a.max() < 100 * float(facts["fp64_resid_geosum_max"])


# ---------------------------------------------------------------- planted mistakes


def _planted(monkeypatch, target, name, bad):
    monkeypatch.setattr(target, name, bad)


def test_planted_dropped_periodic_bond_is_caught(monkeypatch):
    orig = model.diagonal_phases

    def open_chain(L, J, h):
        z = 1 - 2 * model.bit_table(L)
        return J * (z[:, :-1] * z[:, 1:]).sum(1) + z.astype(float) @ np.asarray(h)

    monkeypatch.setattr(model, "diagonal_phases", open_chain)
    with pytest.raises(AssertionError):
        test_apply_u_matches_dense_expm(5, 1.0, 0.9045)
    monkeypatch.setattr(model, "diagonal_phases", orig)


def test_planted_kick_sign_is_caught(monkeypatch):
    orig = model.apply_kick
    monkeypatch.setattr(model, "apply_kick", lambda psi, L, g: orig(psi, L, -g))
    with pytest.raises(AssertionError):
        test_apply_u_matches_dense_expm(4, 0.3, 0.2)


def test_planted_kd_order_is_caught(monkeypatch):
    # U = K D instead of D K: same spectrum, different operator
    def apply_kd(self, psi):
        return model.apply_kick(self.phase * psi, self.L, self.g)

    monkeypatch.setattr(model.KickedIsing, "apply_u", apply_kd)
    with pytest.raises(AssertionError):
        test_apply_u_matches_dense_expm(3, 1.0, 0.9045)


def test_planted_filter_off_by_one_is_caught(monkeypatch):
    orig = geosum.filter_acc
    monkeypatch.setattr(geosum, "filter_acc",
                        lambda op, psi, phi, k: orig(op, psi, phi, k + 1))
    with pytest.raises(AssertionError):
        test_filter_closed_form_on_exact_eigenvectors()


def test_planted_filter_phase_sign_is_caught(monkeypatch):
    orig = geosum.zpow
    monkeypatch.setattr(geosum, "zpow", lambda phi, j: orig(-phi, j))
    with pytest.raises(AssertionError):
        test_filter_peaks_at_target_eigenvalue()


def test_planted_single_gram_schmidt_pass_is_caught(monkeypatch):
    def cgs1(V, w):
        h1 = V.T @ w                       # missing conjugate
        w = w - V @ h1
        beta = np.linalg.norm(w)
        return h1, beta, w / beta

    monkeypatch.setattr(krylov, "cgs2", cgs1)
    with pytest.raises(AssertionError):
        test_arnoldi_relation()


def test_paper_params_pins():
    # Sec. 5 fixes n_cv = floor(2^(L/2+1)) and k = 0.8 * 2^(L+1) / n_cv; for even L the
    # Krylov dimension is a power of two, and in every case the Krylov dimension is about
    # 80 % of the outer-lobe count 2d/k and more than twice the number of wanted pairs
    assert krylov.paper_params(12, 50) == (51, 128)    # 0.8 * 8192 / 128 = 51.2
    assert krylov.paper_params(14, 50) == (102, 256)   # 0.8 * 32768 / 256 = 102.4
    assert krylov.paper_params(16, 50) == (205, 512)   # 0.8 * 131072 / 512 = 204.8
    assert krylov.paper_params(13, 10) == (72, 181)    # floor(2^7.5) = 181
    for L in range(6, 25):
        for nev in (1, 10, 50, 100):
            if 2 * nev + 1 > min(512, (1 << L) - 1):
                with pytest.raises(ValueError):
                    krylov.paper_params(L, nev)
                continue
            k, m = krylov.paper_params(L, nev)
            assert m > 2 * nev and m <= 512
            lobe = 2 * (1 << L) / k
            assert abs(m / lobe - 0.8) < 0.8 * (0.5 / k) + 1e-12
            if L % 2 == 0 and 2 ** (L // 2 + 1) <= 512 and 2 ** (L // 2 + 1) > 2 * nev:
                assert m == 2 ** (L // 2 + 1)


# ---------------------------------------------------------------- entanglement entropy (Eq. ee)

def _bell_chain(L):
    # Bell pairs (|00> + |11>)/sqrt 2 on qubits (0,1), (2,3), ...
    bell = np.array([1, 0, 0, 1], dtype=np.complex128) / np.sqrt(2)  # index b0 + 2 b1
    psi = np.array([1.0 + 0j])
    for _ in range(L // 2):
        psi = np.kron(bell, psi)  # new pair on the next two (higher) bits
    return psi


def test_entropy_pins():
    from oracle import entropy
    L = 8
    # product state: zero for every cut
    prod = np.array([1.0 + 0j])
    rng = np.random.default_rng(3)
    for _ in range(L):
        q = rng.standard_normal(2) + 1j * rng.standard_normal(2)
        prod = np.kron(q / np.linalg.norm(q), prod)
    for LA in range(L + 1):
        assert abs(entropy.entanglement_entropy(prod, L, LA)) < 1e-12
    # Bell pairs on (0,1), (2,3), ...: ln 2 for a cut through one pair, 0 between pairs
    bc = _bell_chain(L)
    for LA in range(L + 1):
        want = np.log(2) if LA % 2 == 1 else 0.0
        assert abs(entropy.entanglement_entropy(bc, L, LA) - want) < 1e-12
    # one Bell pair on qubits (0, 1), the other qubits in |0>: subsystem A is the LOW bits,
    # so only the cut after qubit 0 is entangled
    one = np.zeros(1 << L, dtype=np.complex128)
    one[0] = one[3] = 1 / np.sqrt(2)
    for LA in range(L + 1):
        want = np.log(2) if LA == 1 else 0.0
        assert abs(entropy.entanglement_entropy(one, L, LA) - want) < 1e-12
    # GHZ: ln 2 for every proper cut
    ghz = np.zeros(1 << L, dtype=np.complex128)
    ghz[0] = ghz[-1] = 1 / np.sqrt(2)
    for LA in range(1, L):
        assert abs(entropy.entanglement_entropy(ghz, L, LA) - np.log(2)) < 1e-12
    # maximally entangled across the middle cut: LA ln 2
    LA = L // 2
    mx = np.zeros(1 << L, dtype=np.complex128)
    for a in range(1 << LA):
        mx[a + (a << LA)] = 1
    mx /= np.linalg.norm(mx)
    assert abs(entropy.entanglement_entropy(mx, L, LA) - LA * np.log(2)) < 1e-12
    # S_A = S_B for any pure state: the spectrum of rho_B = tr_A |psi><psi|, formed by an
    # explicit partial trace, gives the same entropy as the singular values
    x = inputs.complex_gaussian(1 << L, 4)
    for LA in range(1, L):
        M = np.array([[x[a + (b << LA)] for b in range(1 << (L - LA))] for a in range(1 << LA)])
        rho_B = np.einsum("ab,ac->bc", M, M.conj())
        lam = np.clip(np.linalg.eigvalsh(rho_B), 1e-300, None)
        assert abs(entropy.entanglement_entropy(x, L, LA) + np.sum(lam * np.log(lam))) < 1e-12


def test_page_value_pins():
    from oracle import entropy
    # two qubits: 1/4 + 1/3 - 1/4 = 1/3 nats, the known mean for random two-qubit states
    assert abs(entropy.page_entropy(1, 1) - 1.0 / 3.0) < 1e-15
    # large systems: ln m - m / (2 n) up to O(1/n)
    for LA, LB in [(4, 12), (6, 10), (8, 8)]:
        m, n = 2 ** LA, 2 ** LB
        assert abs(entropy.page_entropy(LA, LB) - (np.log(m) - m / (2 * n))) < 2.0 / n
    assert entropy.page_entropy(7, 3) == entropy.page_entropy(3, 7)
    # random states average to the Page value
    L, LA = 10, 4
    s = [entropy.entanglement_entropy(inputs.complex_gaussian(1 << L, 100 + i), L, LA)
         for i in range(40)]
    assert abs(np.mean(s) - entropy.page_entropy(LA, L - LA)) < 4 * np.std(s) / np.sqrt(40) + 1e-3


def test_entropy_of_product_eigenstates_J0():
    # J = 0: U is a product of single-qubit unitaries, its (non-degenerate) eigenvectors are
    # product states, so every cut has zero entanglement
    from oracle import entropy
    L = 6
    op = model.KickedIsing(L, 0.0, 0.7, inputs.disorder(L, 1.0, 9))
    w, V = np.linalg.eig(op.dense())
    for j in range(0, 1 << L, 7):
        v = V[:, j] / np.linalg.norm(V[:, j])
        for LA in range(1, L):
            assert entropy.entanglement_entropy(v, L, LA) < 1e-9


# ---------------------------------------------------------------- brickwork circuit (Sec. 2)

def _brick(L, g2=None, g1=None, seed=5):
    from oracle import brickwork
    r2, r1 = inputs.brickwork_gates(L, seed)
    return brickwork.Brickwork(L, r2 if g2 is None else g2, r1 if g1 is None else g1)


def test_brickwork_unitary_and_dense():
    op = _brick(6)
    U = op.dense()
    assert np.abs(U.conj().T @ U - np.eye(64)).max() < 1e-13
    # Haar gates give a dense U in the computational basis (Sec. 2)
    assert np.mean(np.abs(U) > 1e-12) == 1.0
    x = inputs.complex_gaussian(64, 3)
    assert np.allclose(U @ x, op.apply_u(x), atol=1e-14)


def test_brickwork_gate_index_convention():
    # bond gates I (x) X act on the LOW qubit of each bond (index b_i + 2 b_{i+1}); the
    # boundary gates are identities: U_b flips qubits 1, 3, .., L-3 and U_a flips 0, 2, ..,
    # L-2, so U |s> = |s xor (2^(L-1) - 1)>
    L = 6
    X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    g2 = np.stack([np.kron(np.eye(2), X)] * (L - 1))
    g1 = np.stack([np.eye(2, dtype=np.complex128)] * 2)
    op = _brick(L, g2, g1)
    for s in range(1 << L):
        e = np.zeros(1 << L, dtype=np.complex128)
        e[s] = 1
        y = op.apply_u(e)
        assert abs(y[s ^ ((1 << (L - 1)) - 1)] - 1) < 1e-15 and np.abs(y).sum() - 1 < 1e-14


def test_brickwork_layer_order():
    # U = U_a U_b: U_b acts first. With X on qubit 0 in U_b and a CNOT (control qubit 0,
    # target qubit 1) on bond (0,1) in U_a, |00..0> goes to |..011> (index 3); the other
    # order would give index 1
    L = 4
    I4 = np.eye(4, dtype=np.complex128)
    cnot = I4[:, [0, 3, 2, 1]]  # column b0 + 2 b1 -> row b0 + 2 (b1 xor b0)
    g2 = np.stack([cnot, I4, I4])
    g1 = np.stack([np.array([[0, 1], [1, 0]], dtype=np.complex128), np.eye(2)])
    op = _brick(L, g2, g1)
    e = np.zeros(16, dtype=np.complex128)
    e[0] = 1
    y = op.apply_u(e)
    assert abs(y[3] - 1) < 1e-15


def test_brickwork_product_gates_spectrum():
    # bond gates that are products of single-qubit unitaries make U a product over qubits:
    # its eigenvalues are the products of the per-qubit 2 x 2 eigenvalues (closed form)
    L = 6
    rng = np.random.default_rng(11)
    A = [inputs.haar_unitary(2, rng) for _ in range(L - 1)]  # low factor of bond i
    B = [inputs.haar_unitary(2, rng) for _ in range(L - 1)]  # high factor of bond i
    g2 = np.stack([np.kron(B[i], A[i]) for i in range(L - 1)])
    g1 = np.stack([inputs.haar_unitary(2, rng) for _ in range(2)])
    op = _brick(L, g2, g1)
    per_qubit = []
    for q in range(L):
        # factor from U_b (first), then from U_a
        if q == 0:
            fb = g1[0]
        elif q == L - 1:
            fb = g1[1]
        else:
            fb = A[q] if q % 2 == 1 else B[q - 1]
        fa = A[q] if q % 2 == 0 else B[q - 1]
        per_qubit.append(np.linalg.eigvals(fa @ fb))
    lam = np.array([1.0 + 0j])
    for ev in per_qubit:
        lam = np.outer(ev, lam).ravel()
    got = np.linalg.eigvals(op.dense())
    for x in lam:
        assert np.min(np.abs(got - x)) < 1e-12


def test_defect_coefficients_identity():
    # g_k(U) x - g_k(omega) x = q(U) (U - omega) x for any x and any complex omega (not only
    # eigenvalues), checked with dense U; a wrong power or a dropped z fails it
    L, k, phi = 6, 12, 0.7
    op = model.KickedIsing(L, 1.0, 0.9045, inputs.disorder(L, 1.0, 12))
    U = op.dense()
    x = inputs.complex_gaussian(1 << L, 5)
    for omega in (np.exp(0.3j), 0.9 * np.exp(-2.0j), 1.1 + 0.2j):
        a = geosum.defect_coefficients(omega, phi, k)
        assert a.shape == (k - 1,)
        lhs = geosum.filter_dense(U, phi, k) @ x - geosum.gk_closed(omega, phi, k) * x
        r = U @ x - omega * x
        rhs = np.zeros_like(x)
        p = r.copy()
        for coef in a:  # sum_l a_l U^l r
            rhs += coef * p
            p = U @ p
        assert np.linalg.norm(lhs - rhs) < 1e-12 * np.linalg.norm(lhs)


def test_block_arnoldi_reduces_to_arnoldi_and_keeps_its_relation():
    L = 8
    op = model.KickedIsing(L, 1.0, 0.9045, inputs.disorder(L, 1.0, 31))
    d = 1 << L
    # b = 1: the same basis and Hessenberg matrix as the single-vector Arnoldi
    v0 = inputs.complex_gaussian(d, 5)
    V1, H1 = krylov.arnoldi(op.apply_u, v0, 12)
    Vb, Hb = krylov.block_arnoldi(op.apply_u_block, v0[:, None], 12)
    assert np.abs(V1 - Vb).max() < 1e-12 and np.abs(H1 - Hb).max() < 1e-12
    # b = 3 on g_k(U): orthonormal basis, A V_n = V H, band structure below the b-th diagonal
    b, nb = 3, 7
    V0 = inputs.random_states(d, b, 6)
    apply_g = lambda X: np.stack([geosum.filter_acc(op, X[:, i], 0.4, 9)
                                  for i in range(X.shape[1])], axis=1)
    V, H = krylov.block_arnoldi(apply_g, V0, nb)
    assert np.abs(V.conj().T @ V - np.eye(V.shape[1])).max() < 1e-12
    assert np.abs(apply_g(V[:, :nb * b]) - V @ H).max() < 1e-11 * np.abs(H).max()
    rows, cols = np.nonzero(np.abs(H) > 0)
    assert np.all(rows <= cols + b)
    # the start block lies in the space (its columns are combinations of the first b)
    P = V[:, :b] @ (V[:, :b].conj().T @ V0)
    assert np.abs(P - V0).max() < 1e-12


def test_block_arnoldi_spans_the_block_krylov_space():
    # span V[:, :(j+1) b] = span{V0, U V0, ..., U^j V0} (the definition of the space), checked
    # against the explicit power basis; and with d = (nblocks + 1) b the basis is all of C^d,
    # so V^H U V has U's eigenvalues, its first nblocks b columns being H
    L = 6
    op = model.KickedIsing(L, 0.8, 0.6, inputs.disorder(L, 1.0, 32))
    d, b, nb = 1 << L, 3, 4
    V0 = inputs.random_states(d, b, 7)
    V, H = krylov.block_arnoldi(op.apply_u_block, V0, nb)
    K = V0.copy()
    P = V0.copy()
    for j in range(nb + 1):
        Q = V[:, :(j + 1) * b]
        assert np.abs(K - Q @ (Q.conj().T @ K)).max() < 1e-10 * np.abs(K).max(), j
        P = op.apply_u_block(P)
        K = np.concatenate([K, P], axis=1)
    L2 = 4
    op2 = model.KickedIsing(L2, 0.8, 0.6, inputs.disorder(L2, 1.0, 33))
    V2, H2 = krylov.block_arnoldi(op2.apply_u_block, inputs.random_states(16, 4, 8), 3)
    G = V2.conj().T @ op2.apply_u_block(V2)
    assert np.abs(G[:, :12] - H2).max() < 1e-12
    lam = np.linalg.eigvals(G)
    want = np.linalg.eigvals(op2.dense())
    assert np.abs(np.sort_complex(lam)[:, None] - want[None, :]).min(axis=1).max() < 1e-11
