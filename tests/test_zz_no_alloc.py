"""gram_schmidt_noalloc against gram_schmidt, through the C ABI.

gram_schmidt_noalloc serves callers that cannot allocate device memory while they run; it
keeps its scratch in one fixed device array that persists between calls. The check: two
calls in a row (the second on an array still holding the first call's values) give the same
coefficients, norm and unit vector as the allocating entry point, to the CGS2 tolerance of
the other Gram-Schmidt tests (1e-13 relative), the oracle's CGS2 gives the same results on
sizes that are not multiples of the kernels' blocks and with no columns at all (n = 0: w is
only normalised), and oversized inputs are refused.
"""

import numpy as np
import pytest

from oracle import krylov

from gpu_util import from_dev, require_gpu, to_dev

pytestmark = pytest.mark.gpu


def _case(d, n, seed):
    rng = np.random.default_rng(seed)
    V, _ = np.linalg.qr(rng.standard_normal((d, max(n, 1))) + 1j * rng.standard_normal((d, max(n, 1))))
    w = rng.standard_normal(d) + 1j * rng.standard_normal(d)
    return V, w


def test_noalloc_matches_allocating_entry_point_twice():
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    for (d, n, seed) in [(65536, 64, 1), (4096, 17, 2)]:
        V, w = _case(d, n, seed)
        tV = to_dev(V)
        w_ref = to_dev(w)
        h_ref = floquet.gram_schmidt(tV, n, w_ref)
        w_new = to_dev(w)
        h_new = torch.zeros(n + 1, dtype=torch.complex128, device="cuda")
        floquet.gram_schmidt_noalloc(tV, n, w_new, h_new)
        torch.cuda.synchronize()
        h_new = h_new.cpu().numpy()
        scale = np.linalg.norm(w)
        assert np.abs(h_new[:n] - h_ref[:n]).max(initial=0) < 1e-13 * scale
        assert abs(h_new[n].real - h_ref[n].real) < 1e-13 * scale
        assert np.abs(from_dev(w_new) - from_dev(w_ref)).max() < 1e-13


@pytest.mark.parametrize("d,n", [(3000, 5), (1000, 0), (4097, 37), (65536, 0)])
def test_noalloc_matches_oracle_cgs2(d, n):
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    V, w = _case(d, n, 10 + n)
    V = V[:, :n]
    tV = to_dev(V) if n > 0 else to_dev(np.zeros((d, 1), dtype=np.complex128))
    tw = to_dev(w)
    th = torch.full((n + 1,), float("nan"), dtype=torch.complex128, device="cuda")
    floquet.gram_schmidt_noalloc(tV, n, tw, th)
    torch.cuda.synchronize()
    got_h = th.cpu().numpy()
    if n > 0:
        h, beta, q = krylov.cgs2(V, w)
    else:
        beta = np.linalg.norm(w)
        h, q = np.zeros(0, dtype=np.complex128), w / beta
    scale = np.linalg.norm(w)
    assert np.abs(got_h[:n] - h).max(initial=0) < 1e-13 * scale
    assert abs(got_h[n] - beta) < 1e-13 * scale
    assert np.abs(from_dev(tw) - q).max() < 1e-13


def test_noalloc_rejects_sizes_beyond_its_array():
    torch = require_gpu()
    from paper_2102_05054_gb300 import floquet
    w = torch.zeros(8, dtype=torch.complex128, device="cuda")
    h = torch.zeros(300, dtype=torch.complex128, device="cuda")
    lib = floquet.lib()
    rc = lib.gram_schmidt_noalloc((1 << 20) + 1, floquet._ptr(w), 0, floquet._ptr(w),
                                  floquet._ptr(h), None)
    assert rc == floquet.EINVAL and b"capacity" in lib.floquet_last_error()
    rc = lib.gram_schmidt_noalloc(8, floquet._ptr(w), 257, floquet._ptr(w), floquet._ptr(h), None)
    assert rc == floquet.EINVAL and b"capacity" in lib.floquet_last_error()
