"""Pins for the oracle's Liouville operator (Eqs. 1-2) and Davidson solver."""
import numpy as np
import pytest

import bse_inputs as bi
from oracle import dense_bse, forces, liouville, model


@pytest.fixture(scope="module")
def tiny_all():
    spec = bi.tiny()
    return spec, model.GroundState(spec, all_states=True)


@pytest.fixture(scope="module")
def micro_all():
    spec = bi.micro()
    return spec, model.GroundState(spec, all_states=True)


def _rand_pc(op, seed, k=1):
    b = op.basis
    X = bi.random_trial_block(seed, k, op.spec.n_occ, b.npw)
    return np.stack([op.Pc(b.real_to_full(x)) for x in X])


def test_hermitian_on_pc_space(tiny_all):
    spec, gs = tiny_all
    op = liouville.Liouville(spec, gs=gs)
    A, B = _rand_pc(op, 1, 2)
    lhs = np.vdot(B, op.apply(A))
    rhs = np.vdot(op.apply(B), A)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)
    assert np.abs(gs.phi.conj() @ op.apply(A).T).max() < 1e-13   # output lies in P_c


def test_davidson_equals_dense_transition_basis(tiny_all):
    """Check (a): DMPT + Davidson reproduces the explicit electron-hole matrix."""
    spec, gs = tiny_all
    M, _ = dense_bse.bse_matrix(spec, gs=gs)
    ref = np.linalg.eigvalsh(M)[:2]
    w, A, op = forces.excitation(spec.__class__(**{**spec.__dict__, "n_roots": 2}), gs=gs)
    assert np.abs(w - ref).max() < 1e-10
    assert abs(np.vdot(A[0], A[0]) - 1) < 1e-12                  # A^dagger A = 1 (Sec. SI)


def test_matrix_elements_equal_apply(micro_all):
    spec, gs = micro_all
    M, _ = dense_bse.bse_matrix(spec, gs=gs)
    op = liouville.Liouville(spec, gs=gs)
    eps_c, phi_c = gs.empty_states()
    ne = len(eps_c)
    for (vp, cp) in [(0, 0), (1, 3), (0, 17)]:
        A = np.zeros((spec.n_occ, gs.basis.npw), complex)
        A[vp] = phi_c[cp]
        LA = op.apply(A)
        col = np.concatenate([phi_c.conj() @ LA[v] for v in range(spec.n_occ)])
        assert np.abs(col.real - M[:, vp * ne + cp]).max() < 1e-12


@pytest.mark.parametrize("spin", [0, 1])
def test_davidson_vs_dense_micro(micro_all, spin):
    spec, gs = micro_all
    s2 = spec.__class__(**{**spec.__dict__, "spin": spin})
    ref = dense_bse.lowest(s2, gs=gs)[0]
    w, _, _ = forces.excitation(s2, gs=gs)
    assert abs(w[0] - ref) < 1e-10


def test_kernels_off_gives_homo_lumo_gap(tiny_all):
    """Closed form: with K1e = K1d = 0, Omega = eps_LUMO - eps_HOMO + Delta."""
    spec, gs = tiny_all
    for delta in (0.0, 0.37):
        w, _, _ = forces.excitation(spec, gs=gs, k1e=False, k1d=False, scissor=delta)
        assert abs(w[0] - (gs.eps_all[spec.n_occ] - gs.eps_all[spec.n_occ - 1] + delta)) < 1e-11


def test_scissor_shifts_every_root(tiny_all):
    spec, gs = tiny_all
    w0, _, _ = forces.excitation(spec, gs=gs)
    w1, _, _ = forces.excitation(spec, gs=gs, scissor=0.25)
    assert abs((w1[0] - w0[0]) - 0.25) < 1e-11


def test_exchange_raises_singlet_above_triplet(micro_all):
    """2 K1e is positive semi-definite, so the singlet lies above the triplet."""
    spec, gs = micro_all
    ws = dense_bse.lowest(spec, gs=gs, spin=0)[0]
    wt = dense_bse.lowest(spec, gs=gs, spin=1)[0]
    assert ws > wt


def test_bare_coulomb_davidson_vs_dense(micro_all):
    """W = v_c (no PDEPs, CIS-like row of Table S1): Davidson equals the dense matrix."""
    spec, gs = micro_all
    ref = dense_bse.lowest(spec, gs=gs, n_pdep=0)[0]
    w, _, _ = forces.excitation(spec, gs=gs, n_pdep=0)
    assert abs(w[0] - ref) < 1e-10


@pytest.mark.slow
def test_davidson_finds_the_lowest_root_small16():
    """On the 8-well model a random-start Davidson settles on an excited root; the oracle's start
    block of lowest transitions must give the lowest eigenvalue of the dense transition-basis
    matrix (the definition of Omega)."""
    from oracle import dense_bse
    spec = bi.small16()
    w, _, _ = forces.excitation(spec, tol=1e-11)
    assert abs(w[0] - dense_bse.lowest(spec)[0]) < 1e-9
