"""Pins for oracle.screening (Eq. 3) against its definition and a closed form."""
import numpy as np

import bse_inputs as bi
from oracle.basis import PWBasis
from oracle.screening import Screening


def _basis():
    s = bi.micro()
    return s, PWBasis(s.lattice, s.ecut, s.grid)


def test_single_plane_wave_pdep_closed_form():
    """One PDEP supported on a +-G0 pair: W cos(G0.r) = 4 pi/|G0|^2 (1 + c) cos(G0.r)."""
    s, b = _basis()
    k = 5
    coef = np.zeros((1, b.npw))
    coef[0, 2 * k - 1] = 1.0                       # cosine function of half-sphere vector k
    lam = np.array([-0.7])
    W = Screening(b, coef, lam)
    G0 = b.G[b.i_plus[k - 1]]
    j = np.stack(np.meshgrid(*[np.arange(n) / n for n in b.grid], indexing="ij"), -1)
    r = j @ b.lattice
    c = lam[0] / (1 - lam[0])
    out = W.apply(np.cos(r @ G0))
    assert np.abs(out - 4 * np.pi / (G0 @ G0) * (1 + c) * np.cos(r @ G0)).max() < 1e-12
    # the orthogonal sine partner is only bare-screened
    out = W.apply(np.sin(r @ G0))
    assert np.abs(out - 4 * np.pi / (G0 @ G0) * np.sin(r @ G0)).max() < 1e-12


def test_apply_equals_dense_definition():
    s, b = _basis()
    W = Screening(b, s.pdep_coef, s.pdep_lambda)
    rng = np.random.default_rng(7)
    rho = b.to_grid(b.real_to_full(rng.standard_normal(b.npw))) * b.to_grid(
        b.real_to_full(rng.standard_normal(b.npw)))
    rh = b.density_coeffs(rho)
    ref = W.dense_matrix() @ rh
    got = b.density_coeffs(W.apply(rho))
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_symmetric_and_screened():
    s, b = _basis()
    W = Screening(b, s.pdep_coef, s.pdep_lambda)
    Wd = W.dense_matrix()
    assert np.abs(Wd - Wd.conj().T).max() < 1e-13
    # lambda < 0 makes W = v_c + negative semi-definite part
    V0 = Screening(b, s.pdep_coef, s.pdep_lambda, n_pdep=0).dense_matrix()
    assert np.linalg.eigvalsh(Wd - V0).max() < 1e-12


def test_no_pdep_is_bare_coulomb():
    s, b = _basis()
    rng = np.random.default_rng(8)
    rho = b.to_grid(b.real_to_full(rng.standard_normal(b.npw))).real ** 2
    W = Screening(b, s.pdep_coef, s.pdep_lambda, n_pdep=0)
    assert np.abs(W.apply(rho) - b.coulomb(rho)).max() < 1e-13
