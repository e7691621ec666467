"""ctypes binding of libfloquet.so (include/floquet.h).

Argument marshalling only: every step of the computation runs in the library's CUDA
kernels. PyTorch supplies device memory (torch.Tensor on cuda) and streams. The names
follow the C ABI. There is no CPU fallback: if the library is missing or cannot be loaded,
``lib()`` raises.
"""

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfloquet.so")

OK, EINVAL, ENOMEM, ECUDA, ENOCONV, ETIMEOUT = 0, -1, -2, -3, -4, -5
C128, C64, C128_DF = 0, 1, 2
FP64, FILTER_FP32, FILTER_DF = 0, 1, 2
FORM_ACC, FORM_HORNER = 0, 1

_lib = None

_c_int, _c_double, _c_void_p, _c_int64 = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, \
    ctypes.c_int64
_dptr = ctypes.POINTER(ctypes.c_double)
_iptr = ctypes.POINTER(ctypes.c_int)

# name -> (restype, argtypes); mirrors include/floquet.h
SIGNATURES = {
    "floquet_create": (_c_int, [_c_int, _c_double, _c_double, _dptr, ctypes.POINTER(_c_void_p)]),
    "floquet_destroy": (_c_int, [_c_void_p]),
    "brickwork_create": (_c_int, [_c_int, _dptr, _dptr, ctypes.POINTER(_c_void_p)]),
    "floquet_dim": (_c_int, [_c_void_p, ctypes.POINTER(_c_int64)]),
    "floquet_apply_u": (_c_int, [_c_void_p, _c_void_p, _c_void_p, _c_int, _c_int, _c_void_p]),
    "filter_apply": (_c_int, [_c_void_p, _c_double, _c_int64, _c_void_p, _c_void_p, _c_int,
                              _c_int, _c_int, _c_void_p]),
    "gram_schmidt": (_c_int, [_c_int64, _c_void_p, _c_int, _c_void_p, _dptr, _c_void_p]),
    "floquet_pass_plan": (_c_int, [_c_int, _c_int, _c_int, ctypes.POINTER(_c_int), _c_int,
                                   ctypes.POINTER(_c_int)]),
    "floquet_polish_correction": (_c_int, [_c_void_p, _c_double, _c_int64, _dptr, _c_void_p,
                                           _c_void_p, _c_int, _c_int, _c_void_p]),
    "gram_schmidt_noalloc": (_c_int, [_c_int64, _c_void_p, _c_int, _c_void_p, _c_void_p,
                                      _c_void_p]),
    "small_eig": (_c_int, [_c_int, _c_void_p, _dptr, _c_void_p, _c_void_p]),
    "ritz_residuals": (_c_int, [_c_void_p, _c_void_p, _c_int, _dptr, _dptr, _c_void_p]),
    "arnoldi_eigs": (_c_int, [_c_void_p, _c_double, _c_int64, _c_int, _c_int, _c_int, _c_double,
                              _c_double, _c_int, _c_void_p, _dptr, _c_void_p, _dptr, _iptr,
                              _c_void_p]),
    "arnoldi_eigs_batched": (_c_int, [_c_int, _c_double, _c_double, _dptr, _c_int, _dptr, _c_int,
                                      _c_int64, _c_int, _c_int, _c_int, _c_double, _c_double,
                                      _c_int, _c_void_p, _dptr, _dptr, _iptr, _c_void_p]),
    "floquet_profile_enable": (_c_int, [_c_int]),
    "floquet_profile_read": (_c_int, [_dptr, ctypes.POINTER(_c_int64), _dptr]),
    "floquet_launch_count": (_c_int64, []),
    "entanglement_entropy": (_c_int, [_c_int, _c_void_p, _c_int, ctypes.POINTER(_c_int), _c_int,
                                      _dptr, _c_void_p]),
    "floquet_suggest_params": (_c_int, [_c_int, _c_int, _c_int, ctypes.POINTER(_c_int64),
                                        ctypes.POINTER(_c_int)]),
    "floquet_reset_launch_count": (None, []),
    "floquet_last_error": (ctypes.c_char_p, []),
}


class FloquetError(RuntimeError):
    def __init__(self, code, where):
        msg = lib().floquet_last_error().decode()
        super().__init__(f"{where} failed with status {code}: {msg}")
        self.code = code


def lib():
    """Load libfloquet.so (raises if it is absent: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} not found; build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            if not hasattr(L, name):
                continue  # reported by exported_symbols(); calling it raises AttributeError
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    """Names of SIGNATURES that the loaded library exports."""
    L = lib()
    return [n for n in SIGNATURES if hasattr(L, n)]


def _check(code, where):
    if code != OK:
        raise FloquetError(code, where)
    return code


def _stream(stream):
    import torch
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(x):
    """Device or host pointer of a torch tensor or numpy array (must be contiguous)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"] or x.flags["F_CONTIGUOUS"]
        return ctypes.c_void_p(x.ctypes.data)
    assert x.is_contiguous(), "tensor must be contiguous"
    return ctypes.c_void_p(x.data_ptr())


def _dtype_code(t):
    import torch
    if t.dtype == torch.complex128:
        return C128
    if t.dtype == torch.complex64:
        return C64
    raise TypeError(f"unsupported dtype {t.dtype}")


def _dp(a):
    return a.ctypes.data_as(_dptr)


class Floquet:
    """Owns a floquet_t: U = D K for one chain (L, J, g, h)."""

    def __init__(self, L, J, g, h):
        h = np.ascontiguousarray(h, dtype=np.float64)
        if h.shape != (L,):
            raise ValueError("h must have length L")
        handle = ctypes.c_void_p()
        _check(lib().floquet_create(L, J, g, _dp(h), ctypes.byref(handle)), "floquet_create")
        self.handle = handle
        self.L, self.J, self.g, self.h = L, J, g, h.copy()
        d = ctypes.c_int64()
        _check(lib().floquet_dim(self.handle, ctypes.byref(d)), "floquet_dim")
        self.d = d.value

    @classmethod
    def brickwork(cls, L, g2, g1):
        """The paper's brickwork random circuit (brickwork_create): g2 ((L-1) x 4 x 4) bond
        gates with indices b_i + 2 b_{i+1}, g1 (2 x 2 x 2) boundary gates on qubits 0 and
        L-1; complex128 sweeps and the FP64 eigensolver only."""
        g2 = np.ascontiguousarray(g2, dtype=np.complex128)
        g1 = np.ascontiguousarray(g1, dtype=np.complex128)
        if g2.shape != (L - 1, 4, 4) or g1.shape != (2, 2, 2):
            raise ValueError("g2 must be (L-1) x 4 x 4 and g1 2 x 2 x 2")
        self = cls.__new__(cls)
        handle = ctypes.c_void_p()
        _check(lib().brickwork_create(int(L), g2.view(np.float64).ctypes.data_as(_dptr),
                                      g1.view(np.float64).ctypes.data_as(_dptr),
                                      ctypes.byref(handle)), "brickwork_create")
        self.handle = handle
        self.L, self.J, self.g, self.h = L, None, None, None
        d = ctypes.c_int64()
        _check(lib().floquet_dim(self.handle, ctypes.byref(d)), "floquet_dim")
        self.d = d.value
        return self

    def close(self):
        if self.handle:
            lib().floquet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _nvec(self, t):
        n = t.numel()
        if n % self.d:
            raise ValueError("tensor size must be a multiple of d")
        return n // self.d

    def apply_u(self, psi_in, psi_out, stream=None, sweep=None):
        """sweep=C128_DF runs complex128 states through double-float sweeps."""
        dt = _dtype_code(psi_in) if sweep is None else sweep
        _check(lib().floquet_apply_u(self.handle, _ptr(psi_in), _ptr(psi_out),
                                     self._nvec(psi_in), dt, _stream(stream)),
               "floquet_apply_u")
        return psi_out

    def filter_apply(self, phi, k, psi_in, psi_out, form=FORM_ACC, stream=None, sweep=None):
        dt = _dtype_code(psi_in) if sweep is None else sweep
        _check(lib().filter_apply(self.handle, float(phi), int(k), _ptr(psi_in), _ptr(psi_out),
                                  self._nvec(psi_in), dt, int(form), _stream(stream)),
               "filter_apply")
        return psi_out

    def polish_correction(self, phi, K, omega, R, out, sweep=C64, stream=None):
        """out_j = q_j(U) R_j, q_j the defect polynomial of the K-term filter at phi and
        omega_j; R, out: device complex128 tensors of nvec states; omega: nvec complex
        numbers; sweep: C64 or C128_DF."""
        om = np.ascontiguousarray(np.asarray(omega, dtype=np.complex128).ravel())
        n = self._nvec(R)
        if om.size != n:
            raise ValueError("one omega per state")
        _check(lib().floquet_polish_correction(self.handle, float(phi), int(K),
                                               om.view(np.float64).ctypes.data_as(_dptr),
                                               _ptr(R), _ptr(out), n, int(sweep),
                                               _stream(stream)), "floquet_polish_correction")
        return out

    def ritz_residuals(self, X, stream=None):
        n = self._nvec(X)
        om = np.zeros(2 * n)
        res = np.zeros(n)
        _check(lib().ritz_residuals(self.handle, _ptr(X), n, _dp(om), _dp(res), _stream(stream)),
               "ritz_residuals")
        return om[0::2] + 1j * om[1::2], res

    def arnoldi_eigs(self, phi, k, nev, m, v0, precision=FP64, tol=0.0, tol_resid=0.0,
                     max_restarts=50, evecs=None, stream=None, check=True):
        """Returns (omega, resid, n_conv, status); eigenvectors go to `evecs` if given."""
        ev = np.zeros(2 * nev)
        res = np.zeros(nev)
        nconv = ctypes.c_int(0)
        rc = lib().arnoldi_eigs(self.handle, float(phi), int(k), int(nev), int(m), int(precision),
                                float(tol), float(tol_resid), int(max_restarts), _ptr(v0),
                                _dp(ev), _ptr(evecs), _dp(res), ctypes.byref(nconv),
                                _stream(stream))
        if check and rc not in (OK, ENOCONV):
            raise FloquetError(rc, "arnoldi_eigs")
        return ev[0::2] + 1j * ev[1::2], res, nconv.value, rc


def pass_plan(L, NB, min_cols):
    """The U application's pass plan: a list of (NB, c, start, kick_from, midbits, topshift)."""
    out = (_c_int * (6 * 64))()
    n = _c_int()
    _check(lib().floquet_pass_plan(int(L), int(NB), int(min_cols), out, 64, ctypes.byref(n)),
           "floquet_pass_plan")
    return [tuple(out[6 * i: 6 * i + 6]) for i in range(n.value)]


def gram_schmidt(V, n, w, stream=None):
    """CGS2 of w (d complex128, device) against the first n columns of V (d x >=n)."""
    d = w.numel()
    h = np.zeros(2 * (n + 1))
    _check(lib().gram_schmidt(d, _ptr(V), n, _ptr(w), _dp(h), _stream(stream)), "gram_schmidt")
    return h[0::2] + 1j * h[1::2]


def gram_schmidt_noalloc(V, n, w, h, stream=None):
    """gram_schmidt with no device allocation: h is a caller-owned device tensor of n+1
    complex128 (coefficients, then beta); asynchronous on the stream."""
    _check(lib().gram_schmidt_noalloc(w.numel(), _ptr(V), n, _ptr(w), _ptr(h), _stream(stream)),
           "gram_schmidt_noalloc")
    return h


def small_eig(A, Y=None, stream=None):
    """Eigen-decomposition of a small complex128 matrix (column-major, host or device)."""
    n = A.shape[0]
    lam = np.zeros(2 * n)
    _check(lib().small_eig(n, _ptr(A), _dp(lam), _ptr(Y), _stream(stream)), "small_eig")
    return lam[0::2] + 1j * lam[1::2]


def arnoldi_eigs_batched(L, J, g, hs, phis, k, nev, m, v0, tol=0.0, tol_resid=0.0,
                         max_restarts=50, stream=None, check=True, precision=None):
    hs = np.ascontiguousarray(hs, dtype=np.float64)
    phis = np.ascontiguousarray(phis, dtype=np.float64)
    R, P = hs.shape[0], phis.shape[0]
    ev = np.zeros(2 * nev * R * P)
    res = np.zeros(nev * R * P)
    nconv = np.zeros(R * P, dtype=np.int32)
    prec = FP64 if precision is None else int(precision)
    rc = lib().arnoldi_eigs_batched(int(L), float(J), float(g), _dp(hs), R, _dp(phis), P, int(k),
                                    int(nev), int(m), prec, float(tol), float(tol_resid),
                                    int(max_restarts), _ptr(v0), _dp(ev), _dp(res),
                                    nconv.ctypes.data_as(_iptr), _stream(stream))
    if check and rc not in (OK, ENOCONV):
        raise FloquetError(rc, "arnoldi_eigs_batched")
    om = (ev[0::2] + 1j * ev[1::2]).reshape(R, P, nev)
    return om, res.reshape(R, P, nev), nconv.reshape(R, P), rc


def profile_enable(on=True):
    _check(lib().floquet_profile_enable(1 if on else 0), "floquet_profile_enable")


def profile_read():
    """{'c128'|'c64'|'df': (sweep_ms, u_applications, algorithmic_bytes)} since enable."""
    ms = np.zeros(3)
    apps = (ctypes.c_int64 * 3)()
    by = np.zeros(3)
    _check(lib().floquet_profile_read(_dp(ms), apps, _dp(by)), "floquet_profile_read")
    return {"c128": (ms[0], apps[0], by[0]), "c64": (ms[1], apps[1], by[1]),
            "df": (ms[2], apps[2], by[2])}


def launch_count():
    return lib().floquet_launch_count()


def reset_launch_count():
    lib().floquet_reset_launch_count()


def suggest_params(L, nev, max_m=512):
    """(k, m) by the paper's rule (Secs. 4-5): m = max(floor(2^(L/2+1)), 2 nev + 1) capped at
    min(max_m, d - 1), k = round(0.8 * 2^(L+1) / m). Host only."""
    k = _c_int64(0)
    m = _c_int(0)
    _check(lib().floquet_suggest_params(int(L), int(nev), int(max_m), ctypes.byref(k),
                                        ctypes.byref(m)), "floquet_suggest_params")
    return int(k.value), int(m.value)


def entanglement_entropy(L, X, cuts, stream=None):
    """S[j, c] (numpy, nvec x ncut): entanglement entropy of state j of X (device complex128,
    shape (nvec, 2^L) or (2^L,)) for subsystem A = the low cuts[c] qubits."""
    cuts = np.ascontiguousarray(np.asarray(cuts, dtype=np.int32).ravel())
    nvec = int(X.numel() // (1 << L))
    S = np.zeros(nvec * len(cuts))
    _check(lib().entanglement_entropy(int(L), _ptr(X), nvec,
                                      cuts.ctypes.data_as(ctypes.POINTER(_c_int)), len(cuts),
                                      _dp(S), _stream(stream)), "entanglement_entropy")
    return S.reshape(nvec, len(cuts))
