"""The C-ABI library builds for sm_103a, loads, and exports every entry
point declared in include/spsvm.h; host-only entry points agree with the
oracle.  No GPU needed (no compute call touches the device)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(spsvm_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    import paper_1404_1066_gb300 as sp
    lib = sp.load()
    declared = _declared()
    assert len(declared) >= 25
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    from paper_1404_1066_gb300 import _lib
    assert declared == set(_lib.SIGNATURES), declared ^ set(_lib.SIGNATURES)


def test_built_for_sm103a():
    from paper_1404_1066_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_strerror_and_version():
    import paper_1404_1066_gb300 as sp
    lib = sp.load()
    assert b"sm_103a" in lib.spsvm_version()
    for code in range(0, -8, -1):
        assert lib.spsvm_strerror(code)
    assert lib.spsvm_strerror(-99) == b"unknown status"


@pytest.mark.parametrize("n,J,kappa,seed,rnd", [
    (1000, [3, 17, 999, 0, 500], 256, 42, 3),
    (10, list(range(7)), 256, 1, 0),
    (5000, [], 64, 2 ** 63 + 5, 7),
    (70000, list(range(0, 70000, 97)), 256, 123456789, 2 ** 31 + 1),
])
def test_candidate_draw_matches_oracle(n, J, kappa, seed, rnd):
    import paper_1404_1066_gb300 as sp
    from oracle import spsvm as O
    np.testing.assert_array_equal(sp.spsvm_draw_candidates(n, J, kappa, seed, rnd),
                                  O.draw_candidates(n, J, kappa, seed, rnd))


def test_workspace_size_and_argument_checks():
    import ctypes as C
    import paper_1404_1066_gb300 as sp
    lib = sp.load()
    o, _ = sp.make_options(precision="bf16split")
    b = lib.spsvm_fit_workspace_bytes(500_000, 128, 4096, C.byref(o))
    # two kernel-matrix copies of 4096 x 500,096 x 4 bytes dominate
    assert 2 * 4096 * 500_096 * 4 <= b < 2 * 4096 * 500_096 * 4 + 2 * 10 ** 9
    assert lib.spsvm_fit_workspace_bytes(0, 128, 4096, C.byref(o)) == 0
    # bad arguments are rejected before any device work
    h = C.c_void_p()
    assert lib.spsvm_fit(None, 10, 2, 2, None, 1.0, 1.0, 1, 0.0, None, None, 0, C.byref(h)) == -1
    assert lib.spsvm_cholesky(None, 4, 4, None, None, 0, None) == -1
    assert b"NULL" in lib.spsvm_last_error() or b"bad" in lib.spsvm_last_error()
