"""The C-ABI library builds, loads without a GPU and exports every declared entry point."""
import os
import re
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2607_20728_gb300 as p
    return p


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(bse_\w+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(pkg):
    lib = pkg.load_library()
    names = _declared()
    assert "bse_setup" in names and "bse_apply_liouville" in names and "bse_forces" in names
    for n in names:
        assert hasattr(lib, n), n


def test_host_eigensolver_without_gpu(pkg):
    rng = np.random.default_rng(0)
    for n in (1, 3, 16, 90):
        M = rng.standard_normal((n, n))
        M = M + M.T
        w, V = pkg.host_sym_eig(M)
        assert np.abs(w - np.linalg.eigvalsh(M)).max() < 1e-12 * max(1.0, np.abs(w).max())
        assert np.abs(V.T @ V - np.eye(n)).max() < 1e-13
    # repeated eigenvalues
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    M = Q @ np.diag([1.0] * 4 + [2.0] * 4 + [-3.0] * 4) @ Q.T
    w, V = pkg.host_sym_eig(M)
    assert np.abs(w - np.sort([1.0] * 4 + [2.0] * 4 + [-3.0] * 4)).max() < 1e-13
    assert np.abs(M @ V - V * w).max() < 1e-13


def test_errors_are_status_codes(pkg):
    with pytest.raises(pkg.BSEError) as e:
        pkg.host_sym_eig(np.array([[np.nan]]))
    assert e.value.status == 1


def test_host_eigensolver_lowest_vectors(pkg):
    """k lowest eigenvectors by inverse iteration on the tridiagonal form, including clusters of
    equal and nearly equal eigenvalues (Gram-Schmidt inside a cluster)."""
    rng = np.random.default_rng(11)
    n = 120
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([np.repeat([-2.0, -1.0, -1.0 + 1e-9], [5, 4, 3]), np.linspace(0.0, 5.0, n - 12)])
    cases = [(Q * lam) @ Q.T]
    R = rng.standard_normal((n, n))
    cases.append(R + R.T)
    for A in cases:
        for k in (1, 7, 40):
            w, V = pkg.host_sym_eig_lowest(A, k)
            assert np.abs(w - np.linalg.eigvalsh(A)).max() < 1e-12 * np.abs(A).max() * n
            assert np.abs(A @ V - V * w[:k]).max() < 1e-12 * np.abs(A).max() * n
            assert np.abs(V.T @ V - np.eye(k)).max() < 1e-12


def test_host_eigensolver_rayleigh_ritz_sizes(pkg):
    """Matrices of the sizes the Davidson Rayleigh-Ritz steps reach (the pool's reduction, the
    root-free QR sweep): a dense spectrum with close pairs, a graded one, and a matrix that splits
    into two blocks (zero off-diagonal entries in the reduction)."""
    rng = np.random.default_rng(5)
    for n in (64, 131, 200, 241):
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        lam = np.sort(np.concatenate([np.linspace(-1.0, 0.0, n // 2), np.linspace(0.1, 3.0, n - n // 2)]))
        lam[3] = lam[2] + 1e-11
        graded = np.sort(np.logspace(-6, 2, n) * np.where(np.arange(n) % 2 == 0, 1.0, -1.0))
        B = np.zeros((n, n))
        h = n // 3
        R1 = rng.standard_normal((h, h))
        R2 = rng.standard_normal((n - h, n - h))
        B[:h, :h] = R1 + R1.T
        B[h:, h:] = R2 + R2.T
        for A in ((Q * lam) @ Q.T, (Q * graded) @ Q.T, B):
            ref = np.linalg.eigvalsh(A)
            scale = np.abs(ref).max()
            for k in (1, 44, min(80, n)):
                w, V = pkg.host_sym_eig_lowest(A, k)
                assert np.abs(w - ref).max() < 1e-13 * scale * 8
                assert np.abs(A @ V - V * w[:k]).max() < 1e-12 * scale * 8
                assert np.abs(V.T @ V - np.eye(k)).max() < 1e-11
                # the k lowest alone (bisection on the Sturm count, the Davidson's form)
                wk, Vk = pkg.host_sym_eig_k(A, k)
                assert np.abs(wk - ref[:k]).max() < 1e-13 * scale * 8
                assert np.abs(A @ Vk - Vk * wk).max() < 1e-12 * scale * 8
                assert np.abs(Vk.T @ Vk - np.eye(k)).max() < 1e-11

