"""Synthetic ground state (oracle): H = -1/2 nabla^2 + sum_a V_a, non-self-consistent.

The paper's ground states are Quantum ESPRESSO DFT runs (Sec. SIV); the
synthetic stand-in replaces the pseudopotential by Gaussian wells
V_a(r) = -Z_a exp(-|r - R_a|^2 / (2 sigma_a^2)) summed over periodic images, whose
derivative plays the role of dV_ext/dR in Eq. 4.
"""
import numpy as np
import scipy.linalg

from .basis import PWBasis


def vloc_atoms(basis, G, pos, Z, sigma):
    """Per-atom Fourier coefficients V_a(G) = -Z (2 pi s^2)^{3/2}/Omega e^{-s^2 G^2/2} e^{-iG.R_a}.

    Returns (n_atoms, len(G)) complex."""
    g2 = np.sum(G * G, axis=1)
    pref = -np.asarray(Z)[:, None] * (2 * np.pi * np.asarray(sigma)[:, None] ** 2) ** 1.5 / basis.omega
    return pref * np.exp(-0.5 * np.asarray(sigma)[:, None] ** 2 * g2[None, :]) * np.exp(
        -1j * (np.asarray(pos) @ G.T))


def hamiltonian(basis, pos, Z, sigma):
    """Dense H_GG' = 1/2 |G|^2 delta_GG' + V(G - G') on the wave-function sphere."""
    box = 2 * np.abs(basis.mill).max(axis=0)
    axes = [np.arange(-box[i], box[i] + 1) for i in range(3)]
    M = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, 3)
    Vbox = vloc_atoms(basis, M @ basis.B, pos, Z, sigma).sum(axis=0).reshape(
        tuple(2 * box + 1))
    H = np.empty((basis.npw, basis.npw), dtype=np.complex128)
    mill = basis.mill.astype(np.int64)
    step = max(1, 2_000_000 // basis.npw)
    for i0 in range(0, basis.npw, step):
        d = mill[i0:i0 + step, None, :] - mill[None, :, :] + box
        H[i0:i0 + step] = Vbox[d[..., 0], d[..., 1], d[..., 2]]
    H[np.diag_indices(basis.npw)] += 0.5 * basis.g2
    return H


class GroundState:
    """Occupied orbitals phi_v (real in r), energies eps_v and, optionally, all empty states."""

    def __init__(self, spec, all_states=False, pos=None):
        self.spec = spec
        self.basis = PWBasis(spec.lattice, spec.ecut, spec.grid)
        b = self.basis
        self.pos = np.asarray(spec.pos if pos is None else pos, dtype=np.float64)
        self.H = hamiltonian(b, self.pos, spec.Z, spec.sigma)
        U = b.real_basis_matrix()
        Hr = U.conj().T @ self.H @ U
        if np.abs(Hr.imag).max() > 1e-10 * max(1.0, np.abs(Hr).max()):
            raise AssertionError("Hamiltonian is not real in the real basis")
        Hr = 0.5 * (Hr.real + Hr.real.T)
        n_occ = spec.n_occ
        if all_states:
            eps, X = np.linalg.eigh(Hr)
        else:
            eps, X = scipy.linalg.eigh(Hr, subset_by_index=[0, n_occ])
        X = X.T                                    # rows = states, real basis
        from bse_inputs import gauge_vector
        g = gauge_vector(spec.lattice, spec.ecut)
        sgn = np.sign(X @ g)
        sgn[sgn == 0] = 1.0
        X = X * sgn[:, None]
        self.eps_all = eps
        self.X_all = X
        self.eps = eps[:n_occ].copy()
        self.X = X[:n_occ].copy()                  # real-basis occupied orbitals
        self.phi = b.real_to_full(self.X)          # (n_occ, npw) complex
        self.phi_r = b.to_grid(self.phi)           # (n_occ, N1, N2, N3)
        self.gap = eps[n_occ] - eps[n_occ - 1]

    def empty_states(self):
        if self.X_all.shape[0] <= self.spec.n_occ + 1 and self.X_all.shape[0] < self.basis.npw:
            raise ValueError("ground state computed without all empty states")
        return self.eps_all[self.spec.n_occ:], self.basis.real_to_full(self.X_all[self.spec.n_occ:])

    def vloc_grid(self):
        """V(r_j) on the grid from its density-sphere Fourier series (used only in tests)."""
        b = self.basis
        V = vloc_atoms(b, b.dG, self.pos, self.spec.Z, self.spec.sigma).sum(axis=0)
        F = np.zeros(b.grid, dtype=np.complex128)
        F[b.didx] = V
        return np.fft.ifftn(F) * b.nr
