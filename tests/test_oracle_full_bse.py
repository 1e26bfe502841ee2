"""Pins for the oracle's BSE beyond the TDA (coupling block B = 2 K2e - K2d, Sec. SI).

The DMPT apply of B (liouville.apply_B, grid products through W) and the transition-basis matrix
(dense_bse.coupling_matrix, pair-density integrals) are independent constructions; the excitation
energies (dense_bse.full_lowest, the square-root route) are checked against the eigenvalues of
the non-Hermitian block matrix itself, and a dense eigenvector is checked against the DMPT
operators in the form the paper writes the equation.
"""
import numpy as np
import pytest

import bse_inputs as bi
from oracle import dense_bse, liouville, model


@pytest.fixture(scope="module")
def micro():
    spec = bi.micro()
    gs = model.GroundState(spec, all_states=True)
    return spec, gs


@pytest.mark.parametrize("spin", [0, 1])
def test_apply_b_columns_equal_the_transition_matrix(micro, spin):
    spec, gs = micro
    op = liouville.Liouville(spec, gs=gs, spin=spin)
    Bm, _ = dense_bse.coupling_matrix(spec, gs=gs, spin=spin)
    assert np.abs(Bm - Bm.T).max() < 1e-14
    eps_c, phi_c = gs.empty_states()
    ne, no = len(eps_c), spec.n_occ
    for v in range(no):
        for c in (0, 1, 5, ne - 1):
            a = np.zeros((no, gs.basis.npw), complex)
            a[v] = phi_c[c]
            col = (op.apply_B(a) @ phi_c.conj().T).real.ravel()
            assert np.abs(col - Bm[:, v * ne + c]).max() < 1e-12 * max(1.0, np.abs(Bm).max())


def test_full_energies_are_the_block_matrix_eigenvalues(micro):
    spec, gs = micro
    A, _ = dense_bse.bse_matrix(spec, gs=gs)
    Bm, _ = dense_bse.coupling_matrix(spec, gs=gs)
    ev = np.linalg.eigvals(np.block([[A, Bm], [-Bm, -A]]))
    assert np.abs(ev.imag).max() < 1e-10
    pos = np.sort(ev.real[ev.real > 0])
    neg = np.sort(-ev.real[ev.real < 0])
    assert np.abs(pos - neg).max() < 1e-12                    # +-omega pairs
    w = dense_bse.full_lowest(spec, k=4)
    assert np.abs(w - pos[:4]).max() < 1e-12


def test_kernels_off_reduce_to_the_transition_energies(micro):
    spec, gs = micro
    w = dense_bse.full_lowest(spec, k=1, k1e=False, k1d=False, scissor=0.07)
    assert abs(w[0] - (gs.eps_all[spec.n_occ] - gs.eps_all[spec.n_occ - 1] + 0.07)) < 1e-12


@pytest.mark.parametrize("spin", [0, 1])
def test_dense_eigenvector_solves_the_dmpt_equations(micro, spin):
    """(A, B; B*, A*)(X; Y) = omega (X; -Y) with the DMPT operators (L = D + 2K1e - K1d, B), for the
    dense solution mapped to orbital vectors a_v = sum_c X_vc phi_c, b_v = sum_c Y_vc phi_c."""
    spec, gs = micro
    A, _ = dense_bse.bse_matrix(spec, gs=gs, spin=spin)
    Bm, _ = dense_bse.coupling_matrix(spec, gs=gs, spin=spin)
    ev, V = np.linalg.eig(np.block([[A, Bm], [-Bm, -A]]))
    i = np.argmin(np.where(ev.real > 0, ev.real, np.inf))
    w = ev[i].real
    n = A.shape[0]
    X, Y = V[:n, i].real, V[n:, i].real
    eps_c, phi_c = gs.empty_states()
    no = spec.n_occ
    a = X.reshape(no, -1) @ phi_c
    bv = Y.reshape(no, -1) @ phi_c
    op = liouville.Liouville(spec, gs=gs, spin=spin)
    r1 = op.apply(a) + op.apply_B(bv) - w * a
    r2 = op.apply_B(a) + op.apply(bv) + w * bv
    scale = np.abs(a).max()
    assert np.abs(r1).max() < 1e-10 * scale and np.abs(r2).max() < 1e-10 * scale


def test_full_bse_on_tiny_differs_from_tda():
    """On the 2-well cell the coupling lowers the lowest singlet by about half (small-gap model):
    a dropped B would show."""
    spec = bi.tiny()
    w_full = dense_bse.full_lowest(spec, k=1)[0]
    w_tda = dense_bse.lowest(spec, k=1)[0]
    assert 0 < w_full < w_tda - 1e-3
