"""Host-side checks of the C ABI (no GPU needed): the library builds and loads, exports every
function include/floquet.h declares, and rejects invalid arguments before touching the GPU."""

import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "floquet.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2102_05054_gb300 import build, floquet
    build.build()
    return floquet.lib()


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b([a-z_][a-z0-9_]*)\s*\(", text)
    skip = {"if", "for", "while", "sizeof", "return", "defined"}
    return sorted({n for n in names if n not in skip})


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ["floquet_create", "floquet_destroy", "floquet_apply_u", "filter_apply",
              "gram_schmidt", "small_eig", "ritz_residuals", "arnoldi_eigs",
              "arnoldi_eigs_batched", "floquet_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2102_05054_gb300 import floquet
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(floquet.SIGNATURES) >= set(_declared_functions())


def test_create_rejects_bad_arguments(lib):
    from paper_2102_05054_gb300 import floquet
    h = np.zeros(30)
    handle = ctypes.c_void_p()
    for L in (2, 25, -1):
        rc = lib.floquet_create(L, 1.0, 0.9, h.ctypes.data_as(floquet._dptr), ctypes.byref(handle))
        assert rc == floquet.EINVAL
        assert b"outside" in lib.floquet_last_error()
    assert lib.floquet_create(4, 1.0, 0.9, None, ctypes.byref(handle)) == floquet.EINVAL
    bad = np.array([0.0, np.nan, 0.0, 0.0])
    assert lib.floquet_create(4, 1.0, 0.9, bad.ctypes.data_as(floquet._dptr),
                              ctypes.byref(handle)) == floquet.EINVAL
    assert lib.floquet_create(4, np.inf, 0.9, h.ctypes.data_as(floquet._dptr),
                              ctypes.byref(handle)) == floquet.EINVAL


def test_calls_reject_null_handles(lib):
    from paper_2102_05054_gb300 import floquet
    assert lib.floquet_destroy(None) == floquet.OK
    assert lib.floquet_apply_u(None, None, None, 1, 0, None) == floquet.EINVAL
    assert lib.filter_apply(None, 0.0, 4, None, None, 1, 0, 0, None) == floquet.EINVAL
    ev = np.zeros(4)
    nc = ctypes.c_int()
    assert lib.arnoldi_eigs(None, 0.0, 8, 2, 4, 0, 0.0, 0.0, 1, None,
                            ev.ctypes.data_as(floquet._dptr), None,
                            ev.ctypes.data_as(floquet._dptr), ctypes.byref(nc),
                            None) == floquet.EINVAL
    assert lib.small_eig(0, None, None, None, None) == floquet.EINVAL
    assert lib.small_eig(513, None, None, None, None) == floquet.EINVAL
    assert lib.gram_schmidt(0, None, 0, None, None, None) == floquet.EINVAL
    assert lib.floquet_polish_correction(None, 0.0, 8, None, None, None, 1, 1,
                                         None) == floquet.EINVAL


def test_launch_counter_resets(lib):
    lib.floquet_reset_launch_count()
    assert lib.floquet_launch_count() == 0


def test_suggest_params_matches_oracle(lib):
    # the paper's (k, n_cv) rule: the C ABI (integer arithmetic) against the oracle (the
    # formula in floating point); no GPU needed
    from oracle import krylov
    from paper_2102_05054_gb300 import floquet
    for L in range(3, 25):
        for nev in (1, 2, 5, 10, 50, 100, 200):
            for max_m in (512, 300, 64):
                try:
                    want = krylov.paper_params(L, nev, max_m)
                except ValueError:
                    k = ctypes.c_int64()
                    m = ctypes.c_int()
                    assert lib.floquet_suggest_params(L, nev, max_m, ctypes.byref(k),
                                                      ctypes.byref(m)) == floquet.EINVAL
                    continue
                assert floquet.suggest_params(L, nev, max_m) == want, (L, nev, max_m)
    assert lib.floquet_suggest_params(2, 1, 512, None, None) == floquet.EINVAL


def test_create_without_a_usable_device_fails_cleanly(lib):
    # failure detection on the host: with no usable CUDA device (this CPU container) the
    # device allocation inside floquet_create fails; the call must return FLOQUET_ECUDA, leave
    # the handle NULL, name the failing call in the thread's error message, and leave the
    # library usable (a host-only query still works)
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present: the allocation does not fail")
    from paper_2102_05054_gb300 import floquet
    h = np.zeros(8)
    handle = ctypes.c_void_p()
    rc = lib.floquet_create(8, 1.0, 0.9, h.ctypes.data_as(floquet._dptr), ctypes.byref(handle))
    assert rc == floquet.ECUDA
    assert handle.value is None
    assert b"cudaMalloc" in lib.floquet_last_error()
    assert floquet.pass_plan(20, 11, 2)[0][:4] == (11, 11, 11, 0)


def test_header_compiles_as_c99_and_cxx(tmp_path):
    # the boundary is a C ABI: the public header must be valid C as well as C++
    import shutil
    src = tmp_path / "use_header.c"
    src.write_text('#include "floquet.h"\nint main(void) { return 0; }\n')
    inc = os.path.join(ROOT, "include")
    for cc, flags in [("gcc", ["-std=c99"]), ("g++", ["-std=c++17", "-x", "c++"])]:
        if shutil.which(cc) is None:
            pytest.skip(f"{cc} not found")
        r = subprocess.run([cc, *flags, "-Wall", "-Werror", "-I", inc, "-c", str(src), "-o",
                            str(tmp_path / "out.o")], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
