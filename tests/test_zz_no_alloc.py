"""gram_schmidt_noalloc against gram_schmidt, through the C ABI.

gram_schmidt_noalloc serves callers that cannot allocate device memory while they run; it
keeps its scratch in one fixed device array that persists between calls. The check: two
calls in a row (the second on an array still holding the first call's values) give the same
coefficients, norm and unit vector as the allocating entry point, to the CGS2 tolerance of
the other Gram-Schmidt tests (1e-13 relative), and oversized inputs are refused.
"""

import numpy as np
import pytest

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
