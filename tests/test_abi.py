"""The C-ABI library builds, loads and exports every symbol include/stkkt.h declares (no GPU needed)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "stkkt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:long\s+|unsigned\s+)*\w+\**\s+\**(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1508_06103_gb300 import _lib, build

    build.build()
    return _lib.load()


def test_header_declares_the_documented_entry_points():
    names = _declared()
    for n in ("kkt_create", "kkt_apply", "kkt_rhs", "ras_setup", "ras_apply", "coarse_setup", "gmres_solve",
              "recover_source", "kkt_destroy", "ras_destroy", "coarse_destroy", "two_level_apply", "kkt_residual"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_signatures_cover_the_header(lib):
    from paper_1508_06103_gb300 import _lib

    assert set(_declared()) == set(_lib.SIGNATURES)


def test_version_and_error_strings(lib):
    assert b"sm_103a" in lib.kkt_version()
    assert isinstance(lib.kkt_last_error(), bytes)


def test_destroy_null_is_a_noop(lib):
    lib.kkt_destroy(None)
    lib.ras_destroy(None)
    lib.coarse_destroy(None)


def test_argument_errors_are_reported_without_a_gpu(lib):
    from paper_1508_06103_gb300 import _lib

    h = ctypes.c_void_p()
    # null grid -> KKT_ERR_ARG, no device work attempted
    assert lib.kkt_create(None, 4, 0.25, None, None, None, 0, 1e-3, 1e-1, 0.5, ctypes.byref(h)) == -1
    g = _lib.KktGrid(2, 2, 2, 1.0, 1.0, 1.0, 1)
    a = (ctypes.c_double * 8)(*([0.1] * 8))
    v = (ctypes.c_double * 24)()
    # theta outside [1/2, 1]
    assert lib.kkt_create(ctypes.byref(g), 4, 0.25, a, v, None, 0, 1e-3, 1e-1, 0.2, ctypes.byref(h)) == -1
    # sensor out of range
    s = (ctypes.c_int * 1)(999)
    assert lib.kkt_create(ctypes.byref(g), 4, 0.25, a, v, s, 1, 1e-3, 1e-1, 0.5, ctypes.byref(h)) == -1
    assert b"sensor" in lib.kkt_last_error()
    assert lib.kkt_apply(None, None, None, 64, None) == -1
    assert lib.kkt_set_regularization(None, 1) == -1
    assert b"kkt_set_regularization" in lib.kkt_last_error()
    assert lib.reduced_solve(None, None, None, None, 30, 1e-8, 10, 1e-12, None, None, None, None) == -1
    assert b"reduced_solve" in lib.kkt_last_error()
    assert lib.kkt_mma_peak(None, None, None) == -1
    assert lib.ras_local_pattern(2, None) == -1
    assert lib.ras_local_pattern(1, (ctypes.c_int * 3)()) == -1   # exact LU has no slot pattern
    assert lib.kkt_set_element(None, 1) == -1
    assert b"kkt_set_element" in lib.kkt_last_error()
    assert lib.gmres_solve(None, None, None, None, None, 30, 1e-8, 10, 0, None, None, None) == -1


def test_local_patterns_of_an_interior_point():
    """Host logic of the pattern-driven local solvers (no device work): ILU(0) keeps F_h's
    structural pattern (C: 2 levels x 27 x 2 components, G: 2 x 27 + 2 sensor couplings,
    f: 3 x 27 x 2), the point-block ILU(0) the 81-point neighbourhood in all three components,
    and ILU(1) the level-1 pattern, a strict superset of ILU(0)'s."""
    from paper_1508_06103_gb300 import api

    assert api.local_pattern("ilu0") == [108, 56, 162]
    assert api.local_pattern("bilu0") == [243, 243, 243]
    # ILU(1): the oracle's levels of fill (iluk_pattern) at the centre of a 5^4-point box with
    # a sensor at every node and no Dirichlet face (every level-1 path stays inside)
    import numpy as np
    from oracle import kkt, schwarz

    p = kkt.Problem((4, 4, 4), (1.0, 1.0, 1.0), 1.0, 4, 0.5, 0, np.full(64, 0.1), np.ones((64, 3)),
                    np.arange(125), 1e-3, 1e-2)
    box = schwarz.boxes(p, (1, 1, 1, 1), 0)[0]
    idx, _ = schwarz.box_unknowns(p, box)
    A = kkt.assemble(p)[idx][:, idx].tocsr()
    pat1 = schwarz.iluk_pattern(A, schwarz.local_pattern(p, idx), 1)
    centre = 2 + 5 * (2 + 5 * (2 + 5 * 2))
    assert api.local_pattern("ilu1") == [len(pat1[3 * centre + c]) for c in range(3)] == [780, 199, 667]


def test_header_is_plain_c():
    """include/stkkt.h is the C ABI: it compiles as C99 and as C++17 without warnings (the
    exports themselves are checked against the header by the binding-coverage test)."""
    import os
    import shutil
    import subprocess

    import pytest

    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    hdr = os.path.join(root, "include", "stkkt.h")
    subprocess.run([cc, "-x", "c", "-std=c99", "-Wall", "-Werror", "-fsyntax-only", hdr], check=True)
    cxx = shutil.which("g++")
    if cxx is not None:
        subprocess.run([cxx, "-x", "c++", "-std=c++17", "-Wall", "-Werror", "-fsyntax-only", hdr], check=True)
