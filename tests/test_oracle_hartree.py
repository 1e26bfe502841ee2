"""Pins for the oracle's Hartree-SCF model (f_Hxc = v_c, Kohn-Sham response kernels of Sec. SI).

The model adds to the non-SCF one: the Coulomb potential of Gaussian ionic charges in V_ext, the
self-consistent Hartree potential of rho = 2 sum_v |phi_v|^2 in H^KS, the f_Hxc term of the D
contribution to U, and the kernel terms 2 K1e,KS + 2 K2e,KS of the Z-vector operator (Eq. 7).
Each is pinned by something other than its own formula: a closed form for the ionic potential,
the fixed-point property for the SCF, a finite-difference orbital gradient for U, a direct solve
with G-space Coulomb integrals for the Z-vector, and finite differences of omega(R) (Sec. SII
protocol) for the whole chain, which also fail when a factor is planted wrong.
"""
import copy

import numpy as np
import pytest
import scipy.special

import bse_inputs as bi
from oracle import forces, liouville, model
from oracle.basis import PWBasis


@pytest.fixture(scope="module")
def micro_h():
    return bi.hartree_model(bi.micro())


@pytest.fixture(scope="module")
def micro_h_result(micro_h):
    return forces.bse_forces(micro_h, tol=1e-11)


def test_ionic_potential_matches_isolated_gaussian_charge():
    """Electron potential of one Gaussian ion (charge q, width s) in a large cubic cell with the
    G = 0 term dropped: near the ion it is -q erf(r/(sqrt2 s))/r, the uniform compensating
    background's -(2 pi q / 3 Omega) r^2 and a constant (image terms start at r^4/L^5)."""
    L, q, s = 24.0, 2.0, 0.8
    b = PWBasis(np.eye(3) * L, 20.0, (72, 72, 72))
    V = model.vloc_atoms(b, b.dG, np.zeros((1, 3)), [0.0], [s], [q]).sum(axis=0)
    F = np.zeros(b.grid, dtype=np.complex128)
    F[b.didx] = V
    Vr = (np.fft.ifftn(F) * b.nr).real
    j = np.arange(2, 10)
    r = j * L / 72
    ref = -q * scipy.special.erf(r / (np.sqrt(2) * s)) / r - 2 * np.pi * q / (3 * b.omega) * r ** 2
    got = Vr[j, 0, 0]
    # the periodic images add a cubic-harmonic r^4 term, bounded here by 4 q r^4 / L^5
    bound = 1e-7 + 4 * q * (r ** 4 + r[0] ** 4) / L ** 5
    assert np.all(np.abs((got - got[0]) - (ref - ref[0])) < bound)
    got_diag = np.array([Vr[i, i, 0] for i in range(1, 7)])
    rd = np.sqrt(2) * np.arange(1, 7) * L / 72
    refd = -q * scipy.special.erf(rd / (np.sqrt(2) * s)) / rd - 2 * np.pi * q / (3 * b.omega) * rd ** 2
    bound = 1e-7 + 4 * q * (rd ** 4 + r[0] ** 4) / L ** 5
    assert np.all(np.abs((got_diag - got[0]) - (refd - ref[0])) < bound)


def test_scf_fixed_point(micro_h_result, micro_h):
    gs = micro_h_result.op.gs
    b = gs.basis
    assert gs.scf_residual <= 1e-12
    # the cell is neutral: 2 N_occ electrons against sum q = 2 N_occ
    assert abs(b.integrate(gs.rho) - 2 * micro_h.n_occ) < 1e-10
    assert abs(np.sum(micro_h.q_ion) - 2 * micro_h.n_occ) < 1e-14
    # the occupied orbitals of H^KS reproduce the density that built its Hartree potential
    assert np.abs(gs.density(gs.X) - gs.rho).max() < 1e-9
    # and are its eigenvectors
    HX = gs.phi @ gs.H.T
    assert np.abs(HX - gs.eps[:, None] * gs.phi).max() < 1e-10
    # v_H solves Poisson's equation for rho - <rho> (spectral Laplacian on the grid)
    N = np.array(b.grid)
    m = [np.fft.fftfreq(n, 1.0 / n) for n in N]
    M = np.stack(np.meshgrid(*m, indexing="ij"), axis=-1)
    G = M @ b.B
    lap = -np.sum(G * G, axis=-1) * np.fft.fftn(gs.vH)
    rho_t = np.fft.fftn(gs.rho)
    rho_t[0, 0, 0] = 0.0
    assert np.abs(np.fft.ifftn(-lap - 4 * np.pi * rho_t)).max() < 1e-9 * np.abs(gs.rho).max() * 4 * np.pi


def _hartree_energy(op, phi, A):
    """E = A^dagger (D + 2 K1e - K1d) A at orbitals phi (not necessarily eigenstates), with H^KS
    rebuilt from rho(phi) and the D term's full matrix eps_v'v'' = <phi_v'|H|phi_v''>."""
    gs = op.gs
    b = gs.basis
    g2 = copy.copy(gs)
    g2.phi = phi
    g2.phi_r = b.to_grid(phi)
    rho = 2.0 * np.sum(np.abs(g2.phi_r) ** 2, axis=0)
    H_ext = model.hamiltonian(b, gs.pos, gs.spec.Z, gs.spec.sigma, gs.q)
    g2.H = H_ext + model.potential_matrix(b, b.coulomb(rho).real)
    E_mat = phi.conj() @ g2.H @ phi.T
    g2.eps = np.real(np.diag(E_mat))
    o2 = copy.copy(op)
    o2.gs = g2
    o2._tau = {} if op._tau is not None else None
    Ap = o2.Pc(A)
    E = np.real(np.vdot(Ap, o2.apply(Ap)))
    O = Ap.conj() @ Ap.T                                   # O[v', v] = <a_v'|a_v>
    off = E_mat - np.diag(np.diag(E_mat))
    return E - np.real(np.sum(O * off.T))


def test_u_vector_is_the_orbital_gradient_with_hartree(micro_h_result):
    """dE/dt along phi + t dphi (dphi in P_c) is 2 Re sum <u|dphi>, H^KS following rho(phi)."""
    op = micro_h_result.op
    b = op.basis
    rng = np.random.default_rng(12)
    A = op.Pc(b.real_to_full(rng.standard_normal((op.spec.n_occ, b.npw))))
    U = forces.u_vector(op, A)
    dphi = op.Pc(b.real_to_full(rng.standard_normal((op.spec.n_occ, b.npw))))
    h = 1e-4
    E = [_hartree_energy(op, op.gs.phi + t * dphi, A) for t in (h, -h, h / 2, -h / 2)]
    d1 = (E[0] - E[1]) / (2 * h)
    d2 = (E[2] - E[3]) / h
    fd = (4 * d2 - d1) / 3
    ana = 2 * np.real(np.vdot(U, dphi))
    assert abs(fd - ana) < 1e-8 * max(1.0, abs(ana))


def test_coupled_zvector_equals_direct_solve(micro_h):
    """Z from the coupled CG against a dense solve in the (v, c) transition basis, whose matrix is
    (eps_c - eps_v) delta + 4 Omega sum_G 4 pi/G^2 rho_vc(G)^* rho_v'c'(G) (Coulomb integrals of
    the pair densities in G space)."""
    gs = model.GroundState(micro_h, all_states=True)
    op = liouville.Liouville(micro_h, gs=gs)
    b = gs.basis
    rng = np.random.default_rng(5)
    U = op.Pc(b.real_to_full(rng.standard_normal((micro_h.n_occ, b.npw))))
    Z = forces.zvector_cg(op, U, tol=1e-13)
    eps_c, phi_c = gs.empty_states()
    no, nc = micro_h.n_occ, len(eps_c)
    pc_r = b.to_grid(phi_c)
    pair = np.einsum("vxyz,cxyz->vcxyz", np.conj(gs.phi_r), pc_r).reshape(no * nc, *b.grid)
    rh = b.density_coeffs(pair)                              # (no*nc, n_dens)
    vc = np.zeros(len(b.dg2))
    vc[b.dg2 > 0] = 4 * np.pi / b.dg2[b.dg2 > 0]
    K = b.omega * np.real((rh.conj() * vc) @ rh.T)
    Mx = np.diag((eps_c[None, :] - gs.eps[:, None]).ravel()) + 4.0 * K
    rhs = -(U @ phi_c.conj().T).ravel()                      # -<phi_c|u_v>
    x = np.linalg.solve(Mx, rhs.real)
    Zd = x.reshape(no, nc) @ phi_c
    assert np.abs(Z - Zd).max() < 1e-9 * max(1.0, np.abs(Zd).max())


@pytest.mark.parametrize("name,comps", [("micro", [(0, 0), (1, 2)]), ("tiny", [(0, 0)]),
                                        ("hexcell", [(1, 2)])])
def test_forces_match_finite_differences(name, comps):
    spec = bi.hartree_model(getattr(bi, name)())
    r = forces.bse_forces(spec, tol=1e-11)
    for atom, alpha in comps:
        fd = forces.omega_fd_richardson(spec, atom, alpha, h=1e-3, tol=1e-11)
        assert abs(r.domega_dR[atom, alpha] - fd) < 1e-9 * max(1.0, abs(fd)), (name, atom, alpha)


def test_planted_factor_errors_fail_finite_differences(micro_h, monkeypatch):
    """The finite-difference pin is sensitive to both Hartree factors: the D-term coefficient of
    U taken as 1 instead of 2, or the Z-vector kernel as 2 K1e,KS instead of 2 K1e,KS + 2 K2e,KS."""
    fd = forces.omega_fd_richardson(micro_h, 0, 0, h=1e-3, tol=1e-11)
    orig_u = forces.u_vector

    def u_half(op, A):
        rho_x, _ = forces.densities(op, A, np.zeros_like(A))
        b = op.basis
        return orig_u(op, A) - op.Pc(b.from_grid(b.coulomb(rho_x)[None] * op.gs.phi_r))

    monkeypatch.setattr(forces, "u_vector", u_half)
    bad = forces.bse_forces(micro_h, tol=1e-11).domega_dR[0, 0]
    assert abs(bad - fd) > 1e-4
    monkeypatch.setattr(forces, "u_vector", orig_u)
    orig_z = liouville.Liouville.apply_zop

    def z_half(self, Z):
        b, gs = self.basis, self.gs
        vz = b.coulomb(np.sum(np.conj(gs.phi_r) * b.to_grid(Z), axis=0))
        return orig_z(self, Z) - self.Pc(2.0 * b.from_grid(vz[None] * gs.phi_r))

    monkeypatch.setattr(liouville.Liouville, "apply_zop", z_half)
    bad = forces.bse_forces(micro_h, tol=1e-11).domega_dR[0, 0]
    assert abs(bad - fd) > 1e-4
