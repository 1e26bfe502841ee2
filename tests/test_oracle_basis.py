"""Pins for oracle.basis and oracle.model against brute force and closed forms."""
import numpy as np
import pytest

import bse_inputs as bi
from oracle import model
from oracle.basis import PWBasis


@pytest.fixture(scope="module")
def micro_gs():
    return model.GroundState(bi.micro(), all_states=True)


def _random_real_coeffs(b, rng, n):
    return b.real_to_full(rng.standard_normal((n, b.npw)))


def test_real_basis_unitary():
    s = bi.micro()
    b = PWBasis(s.lattice, s.ecut, s.grid)
    U = b.real_basis_matrix()
    assert np.abs(U.conj().T @ U - np.eye(b.npw)).max() < 1e-14
    x = np.random.default_rng(1).standard_normal((3, b.npw))
    assert np.abs(b.full_to_real(b.real_to_full(x)) - x).max() < 1e-14
    f = b.to_grid(b.real_to_full(x))
    assert np.abs(f.imag).max() < 1e-13          # real-basis functions are real in r


def test_grid_normalisation_parseval():
    s = bi.micro()
    b = PWBasis(s.lattice, s.ecut, s.grid)
    c = _random_real_coeffs(b, np.random.default_rng(2), 2)
    f = b.to_grid(c)
    assert np.allclose(b.integrate(np.conj(f[0]) * f[1]), np.vdot(c[0], c[1]), atol=1e-12)
    assert np.abs(b.from_grid(f) - c).max() < 1e-13


def test_pair_density_equals_direct_convolution():
    """(f g)^(G) = (1/Omega) sum_G' c_f(G') c_g(G - G'), summed explicitly."""
    s = bi.micro()
    b = PWBasis(s.lattice, s.ecut, s.grid)
    c = _random_real_coeffs(b, np.random.default_rng(3), 2)
    grid = b.density_coeffs(b.to_grid(c[0]) * b.to_grid(c[1]))
    look = {tuple(m): i for i, m in enumerate(b.mill)}
    rng = np.random.default_rng(4)
    for gi in rng.choice(len(b.dmill), 25, replace=False):
        G = b.dmill[gi]
        acc = 0.0
        for i, m in enumerate(b.mill):
            j = look.get(tuple(G - m))
            if j is not None:
                acc += c[0][i] * c[1][j]
        assert abs(grid[gi] - acc / b.omega) < 1e-14


def test_coulomb_closed_form():
    """v_c * cos(G0.r) = 4 pi/|G0|^2 cos(G0.r); a constant has no G != 0 part."""
    s = bi.micro()
    b = PWBasis(s.lattice, s.ecut, s.grid)
    j = np.stack(np.meshgrid(*[np.arange(n) / n for n in b.grid], indexing="ij"), -1)
    r = j @ b.lattice
    G0 = np.array([1, 2, -1]) @ b.B
    rho = np.cos(r @ G0) + 3.0
    v = b.coulomb(rho)
    assert np.abs(v - 4 * np.pi / (G0 @ G0) * np.cos(r @ G0)).max() < 1e-12


def test_vloc_formula_vs_real_space_images():
    """V(G) of the periodic Gaussian sum equals the FFT of V(r) built by image sums."""
    s = bi.micro()
    b = PWBasis(s.lattice, s.ecut, (40, 40, 40))
    j = np.stack(np.meshgrid(*[np.arange(n) / n for n in b.grid], indexing="ij"), -1)
    r = j @ b.lattice
    V = np.zeros(b.grid)
    for a in range(len(s.pos)):
        for t in np.array(np.meshgrid([-1, 0, 1], [-1, 0, 1], [-1, 0, 1])).reshape(3, -1).T:
            d = r - (s.pos[a] + t @ b.lattice)
            V += -s.Z[a] * np.exp(-np.sum(d * d, -1) / (2 * s.sigma[a] ** 2))
    Vg = np.fft.fftn(V)[b.idx] / b.nr
    ref = model.vloc_atoms(b, b.G, s.pos, s.Z, s.sigma).sum(axis=0)
    assert np.abs(Vg - ref).max() < 1e-9


def test_dense_hamiltonian_vs_grid_route(micro_gs):
    """H a by the dense matrix equals 1/2 G^2 a + FFT[V(r) a(r)] on an alias-free grid."""
    gs = micro_gs
    b = gs.basis
    c = _random_real_coeffs(b, np.random.default_rng(5), 3)
    dense = c @ gs.H.T
    grid = 0.5 * b.g2 * c + b.from_grid(gs.vloc_grid()[None] * b.to_grid(c))
    assert np.abs(dense - grid).max() < 1e-12


def test_ground_state_residual_orthonormal(micro_gs):
    gs = micro_gs
    phi = gs.phi
    res = phi @ gs.H.T - gs.eps[:, None] * phi
    assert np.abs(res).max() < 1e-11
    assert np.abs(phi.conj() @ phi.T - np.eye(len(phi))).max() < 1e-13
    assert np.abs(gs.phi_r.imag).max() < 1e-12


def test_free_electron_spectrum():
    """Z = 0: the eigenvalues are 1/2 |G|^2 of the sphere (textbook)."""
    s = bi.micro()
    s = s.__class__(**{**s.__dict__, "Z": np.zeros_like(s.Z)})
    gs = model.GroundState(s, all_states=True)
    assert np.abs(np.sort(gs.eps_all) - np.sort(0.5 * gs.basis.g2)).max() < 1e-12


@pytest.mark.parametrize("make", [bi.micro, bi.tiny])
def test_configs_have_a_gap(make):
    gs = model.GroundState(make())
    assert gs.gap > 1e-3
