"""Pins for the oracle's U vector, Z-vector and forces (Eqs. 4-7, Sec. SI).

The strongest pin is check (d): central finite differences of omega(R) with W held
fixed in G-space (the validation protocol of Sec. SII), with a freshly solved
ground state at every displaced geometry.
"""
import copy

import numpy as np
import pytest

import bse_inputs as bi
from oracle import forces, liouville, model


@pytest.fixture(scope="module")
def micro_result():
    return forces.bse_forces(bi.micro(), tol=1e-11)


@pytest.fixture(scope="module")
def tiny_result():
    return forces.bse_forces(bi.tiny(), tol=1e-11)


def _perturbed_op(op, dphi):
    """A copy of op whose occupied orbitals are phi + dphi (eps re-evaluated)."""
    gs = copy.copy(op.gs)
    gs.phi = op.gs.phi + dphi
    gs.phi_r = gs.basis.to_grid(gs.phi)
    gs.eps = np.real(np.einsum("vg,gh,vh->v", gs.phi.conj(), gs.H, gs.phi))
    new = copy.copy(op)
    new.gs = gs
    new._tau = {} if op._tau is not None else None
    return new


def test_u_vector_is_the_orbital_gradient(micro_result):
    """dE/dt of E = (P_c A)^dagger L (P_c A) along phi + t dphi (dphi in P_c) is 2 Re sum <u|dphi>."""
    r = micro_result
    op = r.op
    b = op.basis
    rng = np.random.default_rng(11)
    A = op.Pc(b.real_to_full(rng.standard_normal((op.spec.n_occ, b.npw))))
    U = forces.u_vector(op, A)
    dphi = op.Pc(b.real_to_full(rng.standard_normal((op.spec.n_occ, b.npw))))
    h = 1e-4
    E = []
    for t in (h, -h, h / 2, -h / 2):
        o2 = _perturbed_op(op, t * dphi)
        E.append(o2.energy(o2.Pc(A)))
    d1 = (E[0] - E[1]) / (2 * h)
    d2 = (E[2] - E[3]) / h
    fd = (4 * d2 - d1) / 3
    ana = 2 * np.real(np.vdot(U, dphi))
    assert abs(fd - ana) < 1e-8 * max(1.0, abs(ana))


def test_zvector_cg_equals_sum_over_states(tiny_result):
    r = tiny_result
    gs_all = model.GroundState(r.op.spec, all_states=True)
    Z = forces.zvector_sos(r.op, r.U, gs_all)
    assert np.abs(Z - r.Z).max() < 1e-10
    assert np.abs(r.op.gs.phi.conj() @ r.Z.T).max() < 1e-12      # <Z_w|phi_v> = 0 (Sec. SI)


def test_forces_match_finite_differences_micro(micro_result):
    r = micro_result
    for atom in range(2):
        for alpha in range(3):
            fd = forces.omega_fd_richardson(r.op.spec, atom, alpha)
            assert abs(r.domega_dR[atom, alpha] - fd) < 1e-7


@pytest.mark.slow
def test_forces_match_finite_differences_tiny(tiny_result):
    r = tiny_result
    for atom, alpha in [(0, 0), (1, 2)]:
        fd = forces.omega_fd_richardson(r.op.spec, atom, alpha)
        assert abs(r.domega_dR[atom, alpha] - fd) < 1e-7


def test_forces_by_sum_over_states(tiny_result):
    """Independent of the Z-vector: plug the DFPT orbital response
    dphi_v = -sum_c phi_c <phi_c|dV|phi_v>/(eps_c - eps_v) into the orbital gradient."""
    r = tiny_result
    op = r.op
    spec = op.spec
    gs_all = model.GroundState(spec, all_states=True)
    eps_c, phi_c = gs_all.empty_states()
    b = op.basis
    dm = b.mill[:, None, :] - b.mill[None, :, :]
    dG = dm @ b.B
    rho_x, _ = forces.densities(op, r.A, np.zeros_like(r.Z))
    hf = forces.force_contraction(op, rho_x.real)
    for atom in range(spec.n_atoms):
        s2 = spec.sigma[atom] ** 2
        g2 = np.sum(dG * dG, -1)
        Va = (-spec.Z[atom] * (2 * np.pi * s2) ** 1.5 / b.omega * np.exp(-0.5 * s2 * g2)
              * np.exp(-1j * (dG @ spec.pos[atom])))
        for alpha in range(3):
            dH = -1j * dG[..., alpha] * Va                      # dH_GG'/dR = -i(G-G')_alpha V_a(G-G')
            mel = phi_c.conj() @ dH @ op.gs.phi.T               # <phi_c|dV|phi_v>
            dphi = -((mel / (eps_c[:, None] - op.gs.eps[None, :])).T @ phi_c)
            tot = hf[atom, alpha] + 2 * np.real(np.vdot(r.U, dphi))
            assert abs(tot - r.domega_dR[atom, alpha]) < 1e-10


def test_zero_net_force_with_bare_coulomb():
    """Check (c): with W = v_c everything is translation invariant, so sum_a F_a = 0."""
    r = forces.bse_forces(bi.tiny(), n_pdep=0, tol=1e-11)
    assert np.abs(r.F.sum(axis=0)).max() < 1e-9
    assert np.abs(r.F).max() > 1e-4


def test_hellmann_feynman_without_kernels():
    """K1e = K1d = 0: A is the HOMO->LUMO transition, U = Z = 0 and
    d omega/dR = int dV/dR (|phi_L|^2 - |phi_H|^2)."""
    spec = bi.tiny()
    r = forces.bse_forces(spec, k1e=False, k1d=False, tol=1e-11)
    assert np.abs(r.U).max() < 1e-10 and np.abs(r.Z).max() < 1e-10
    gs_all = model.GroundState(spec, all_states=True)
    b = r.op.basis
    phl = b.to_grid(b.real_to_full(gs_all.X_all[[spec.n_occ - 1, spec.n_occ]]))
    rho = np.abs(phl[1]) ** 2 - np.abs(phl[0]) ** 2
    ref = forces.force_contraction(r.op, rho)
    assert np.abs(ref - r.domega_dR).max() < 1e-10


def test_triplet_forces_match_finite_differences():
    spec = bi.micro(spin=1)
    r = forces.bse_forces(spec, tol=1e-11)
    fd = forces.omega_fd_richardson(spec, 0, 1)
    assert abs(r.domega_dR[0, 1] - fd) < 1e-7


def test_forces_match_finite_differences_hexagonal_cell():
    """Non-orthogonal (honeycomb) lattice and a non-cubic grid: reciprocal vectors, the sphere and
    dV/dR all go through the general cell matrix."""
    spec = bi.hexcell()
    r = forces.bse_forces(spec, tol=1e-11)
    for atom, alpha in [(0, 0), (1, 1), (0, 2)]:
        fd = forces.omega_fd_richardson(spec, atom, alpha)
        assert abs(r.domega_dR[atom, alpha] - fd) < 1e-7


def test_forces_match_finite_differences_small16():
    """8 wells, 16 occupied orbitals: the case where an unconverged excitation vector shows up in
    the forces first."""
    spec = bi.small16()
    r = forces.bse_forces(spec, tol=1e-12)
    for atom, alpha in [(0, 0), (5, 1)]:
        fd = forces.omega_fd_richardson(spec, atom, alpha, tol=1e-12)
        assert abs(r.domega_dR[atom, alpha] - fd) < 1e-8
