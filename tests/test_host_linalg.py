"""CPU tests of the library's host FP64 linear algebra (Cholesky, Hermitian Jacobi) used by rb_build."""
import ctypes as C
import os

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2110_13115_gb300 import _native as N, build

    if not os.path.exists(N.LIB_PATH):
        build.build()
    return N.load()


@pytest.mark.parametrize("n", [1, 2, 5, 40, 130])
def test_hermitian_jacobi_against_definition(lib, n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    a = x @ x.conj().T + np.diag(np.linspace(0, 3, n))
    a2 = np.ascontiguousarray(a.copy())
    w = np.zeros(n)
    v = np.zeros((n, n), np.complex128)
    assert lib.rbx_herm_eig(n, a2.ctypes.data, w.ctypes.data, v.ctypes.data) == 0
    assert np.all(np.diff(w) <= 0)
    # A V = V diag(w), V unitary (the definition), and the spectrum matches LAPACK's
    np.testing.assert_allclose(a @ v, v * w[None, :], atol=1e-10 * np.abs(w).max())
    np.testing.assert_allclose(v.conj().T @ v, np.eye(n), atol=1e-12)
    np.testing.assert_allclose(w, np.linalg.eigvalsh(a)[::-1], rtol=1e-11, atol=1e-11 * w.max())


def test_degenerate_spectrum(lib):
    n = 6
    q, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((n, n)) + 1j * np.random.default_rng(2).standard_normal((n, n)))
    d = np.array([3.0, 3.0, 1.0, 1.0, 1.0, 0.0])
    a = q @ np.diag(d) @ q.conj().T
    w = np.zeros(n)
    v = np.zeros((n, n), np.complex128)
    a2 = np.array(a, order="C", copy=True)
    lib.rbx_herm_eig(n, a2.ctypes.data, w.ctypes.data, v.ctypes.data)
    np.testing.assert_allclose(w, d, atol=1e-12)
    np.testing.assert_allclose(a @ v, v * w[None, :], atol=1e-12)


def test_cholesky(lib):
    rng = np.random.default_rng(3)
    n = 30
    x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    a = np.ascontiguousarray(x @ x.conj().T + np.eye(n))
    lo = np.zeros((n, n), np.complex128)
    assert lib.rbx_cholesky(n, a.ctypes.data, lo.ctypes.data) == 0
    np.testing.assert_allclose(lo @ lo.conj().T, a, atol=1e-10)
    assert np.allclose(np.triu(lo, 1), 0)
    bad = np.ascontiguousarray(-a)
    assert lib.rbx_cholesky(n, bad.ctypes.data, lo.ctypes.data) == 1
