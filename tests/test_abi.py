"""C ABI checks that need no GPU: the library builds, loads and exports every declared entry
point; host-side helpers (constitutive law, Bond rotation, validation) agree with the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2602_07354_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_2602_07354_gb300 import build

    build.build()
    return B.lib()


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:int|void|const char\*)\s+(elas_\w+)\s*\(", txt, re.M))
    return sorted(names)


def test_every_declared_symbol_is_exported(built):
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(built, n), n  # ctypes resolves the exported symbol


def test_library_has_sm103a_code():
    # the in-tree library is built for sm_103a only
    from paper_2602_07354_gb300 import build

    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_host_constitutive_helpers_match_oracle(built, oracle):
    rng = np.random.default_rng(0)
    for E, nu in [(200.0, 0.3), (194.0, 0.2934), (400.0, 0.25)]:
        assert np.allclose(B.elas_isotropic_stiffness(E, nu), oracle.iso_stiffness(E, nu), rtol=1e-14, atol=1e-12)
    C = B.elas_cubic_stiffness(204.6, 137.7, 126.2)
    assert np.array_equal(C, oracle.cubic_stiffness(204.6, 137.7, 126.2))
    for _ in range(10):
        rho = rng.normal(size=3) * rng.choice([0.1, 1.0, 10.0])
        Cg = B.elas_rotated_stiffness(C, rho)  # Bond-matrix route
        Co = oracle.rotate_stiffness(C, oracle.rodrigues_to_R(rho))  # 4-index route
        assert np.allclose(Cg, Co, rtol=0, atol=1e-12 * np.abs(C).max())
    Cg = B.elas_rotated_stiffness(C, [1e9, 0, 0])  # the generator's |q_w| < 1e-8 guard
    Co = oracle.rotate_stiffness(C, oracle.rodrigues_to_R([1e9, 0, 0]))
    assert np.allclose(Cg, Co, atol=1e-9 * np.abs(C).max())


def test_invalid_arguments_fail_cleanly_without_gpu(built):
    with pytest.raises(B.ElasError):
        B.elas_workspace_bytes(1, 4, 4, 1, B.PREC_FP64)
    with pytest.raises(B.ElasError):
        B.elas_workspace_bytes(4, 4, 4, 1, 7)
    with pytest.raises(B.ElasError):
        B.elas_isotropic_stiffness(200.0, 0.5)
    with pytest.raises(B.ElasError):
        B.elas_rotated_stiffness(np.eye(6), [np.nan, 0, 0])
    L = built
    h = ctypes.c_void_p(0)
    phase = np.zeros(8, np.int32)
    C = np.eye(6).ravel()
    # dims < 2 and out-of-range ids are rejected before any device work
    assert L.elas_create(ctypes.byref(h), 1, 2, 4, phase.ctypes.data, 1, C.ctypes.data, None, 0, None, 0, None) == -1
    bad = phase.copy()
    bad[3] = 5
    n = B.elas_workspace_bytes(2, 2, 2, 1, 0)
    assert L.elas_create(ctypes.byref(h), 2, 2, 2, bad.ctypes.data, 1, C.ctypes.data, None, 0,
                         ctypes.c_void_p(256 * 1024), n, None) == -1
    assert b"outside" in L.elas_last_error(None)
    assert L.elas_create(ctypes.byref(h), 2, 2, 2, phase.ctypes.data, 1, C.ctypes.data, None, 0, None, n, None) == -2
    asym = np.eye(6)
    asym[0, 1] = 1.0
    assert L.elas_create(ctypes.byref(h), 2, 2, 2, phase.ctypes.data, 1, asym.ravel().ctypes.data, None, 0,
                         ctypes.c_void_p(256 * 1024), n, None) == -1
    nanC = np.eye(6)
    nanC[2, 2] = np.nan
    assert L.elas_create(ctypes.byref(h), 2, 2, 2, phase.ctypes.data, 1, nanC.ravel().ctypes.data, None, 0,
                         ctypes.c_void_p(256 * 1024), n, None) == -1
    assert b"non-finite" in L.elas_last_error(None)


def test_workspace_size_scales_with_grid(built):
    a = B.elas_workspace_bytes(100, 100, 100, 500, B.PREC_FP64)
    b = B.elas_workspace_bytes(100, 100, 100, 500, B.PREC_MIXED)
    assert a > 100 ** 3 * (4 + 48 + 5 * 24) * 0.99  # ids + Minv + w,g,h,Ah,z in FP64
    assert b < a
