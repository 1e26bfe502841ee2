"""Synthetic ground state (oracle): H = -1/2 nabla^2 + sum_a V_a (+ v_H[rho] in the Hartree model).

The paper's ground states are Quantum ESPRESSO DFT runs (Sec. SIV); the
synthetic stand-in replaces the pseudopotential by Gaussian wells
V_a(r) = -Z_a exp(-|r - R_a|^2 / (2 sigma_a^2)) summed over periodic images, whose
derivative plays the role of dV_ext/dR in Eq. 4.

Two ground-state models:
  * non-self-consistent (default): H = -1/2 nabla^2 + V_ext, f_Hxc = 0;
  * Hartree-SCF (spec.hartree): H^KS = -1/2 nabla^2 + V_ext + v_c * rho with the closed-shell
    density rho = 2 sum_v |phi_v|^2, solved to self-consistency; each site also carries a
    Gaussian ionic charge q_a (width sigma_a) whose Coulomb potential -v_c * rho_ion is part of
    V_ext, so that the cell is neutral.  This is the f_Hxc = v_c, alpha_EXX = 0 case of the
    Kohn-Sham response kernels of Sec. SI.
"""
import numpy as np
import scipy.linalg

from .basis import PWBasis


def vloc_atoms(basis, G, pos, Z, sigma, q=None):
    """Per-atom Fourier coefficients of the external potential,
       V_a(G) = -[Z_a (2 pi s_a^2)^{3/2} + 4 pi q_a / |G|^2] e^{-s_a^2 G^2/2} e^{-iG.R_a} / Omega,
    the well plus, when q is given, the Coulomb potential of the Gaussian ionic charge
    q_a (2 pi s_a^2)^{-3/2} e^{-|r-R_a|^2/(2 s_a^2)} (G = 0 term dropped: neutralising background).

    Returns (n_atoms, len(G)) complex."""
    g2 = np.sum(G * G, axis=1)
    s2 = np.asarray(sigma)[:, None] ** 2
    amp = np.asarray(Z)[:, None] * (2 * np.pi * s2) ** 1.5 * np.ones_like(g2)[None, :]
    if q is not None:
        inv = np.zeros_like(g2)
        nz = g2 > 0
        inv[nz] = 4 * np.pi / g2[nz]
        amp = amp + np.asarray(q)[:, None] * inv[None, :]
    return -amp / basis.omega * np.exp(-0.5 * s2 * g2[None, :]) * np.exp(-1j * (np.asarray(pos) @ G.T))


def _sphere_matrix(basis, Vbox, box):
    """Dense <G|V|G'> = V(G - G') on the wave-function sphere from Fourier coefficients on a box."""
    H = np.empty((basis.npw, basis.npw), dtype=np.complex128)
    mill = basis.mill.astype(np.int64)
    step = max(1, 2_000_000 // basis.npw)
    for i0 in range(0, basis.npw, step):
        d = mill[i0:i0 + step, None, :] - mill[None, :, :] + box
        H[i0:i0 + step] = Vbox[d[..., 0], d[..., 1], d[..., 2]]
    return H


def hamiltonian(basis, pos, Z, sigma, q=None):
    """Dense H_GG' = 1/2 |G|^2 delta_GG' + V_ext(G - G') on the wave-function sphere."""
    box = 2 * np.abs(basis.mill).max(axis=0)
    axes = [np.arange(-box[i], box[i] + 1) for i in range(3)]
    M = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, 3)
    Vbox = vloc_atoms(basis, M @ basis.B, pos, Z, sigma, q).sum(axis=0).reshape(
        tuple(2 * box + 1))
    H = _sphere_matrix(basis, Vbox, box)
    H[np.diag_indices(basis.npw)] += 0.5 * basis.g2
    return H


def potential_matrix(basis, v_r):
    """<G|v|G'> for a real potential v(r) given on the grid (band-limited to the density sphere)."""
    F = np.fft.fftn(v_r) / basis.nr
    N = np.array(basis.grid)
    box = 2 * np.abs(basis.mill).max(axis=0)
    axes = [np.arange(-box[i], box[i] + 1) for i in range(3)]
    M = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1)
    w = np.mod(M, N)
    Vbox = F[w[..., 0], w[..., 1], w[..., 2]]
    return _sphere_matrix(basis, Vbox, box)


class GroundState:
    """Occupied orbitals phi_v (real in r), energies eps_v and, optionally, all empty states."""

    def __init__(self, spec, all_states=False, pos=None, scf_tol=1e-12, scf_max_iter=200):
        self.spec = spec
        self.basis = PWBasis(spec.lattice, spec.ecut, spec.grid)
        b = self.basis
        self.pos = np.asarray(spec.pos if pos is None else pos, dtype=np.float64)
        self.hartree = bool(getattr(spec, "hartree", False))
        self.q = getattr(spec, "q_ion", None)
        self.H = hamiltonian(b, self.pos, spec.Z, spec.sigma, self.q)
        self._U = b.real_basis_matrix()
        n_occ = spec.n_occ
        if self.hartree:
            self._scf(scf_tol, scf_max_iter)
        eps, X = self._solve(n_occ, all_states)
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

    def _real_h(self, H):
        Hr = self._U.conj().T @ H @ self._U
        if np.abs(Hr.imag).max() > 1e-10 * max(1.0, np.abs(Hr).max()):
            raise AssertionError("Hamiltonian is not real in the real basis")
        return 0.5 * (Hr.real + Hr.real.T)

    def _solve(self, n_occ, all_states, H=None):
        Hr = self._real_h(self.H if H is None else H)
        if all_states:
            eps, X = np.linalg.eigh(Hr)
        else:
            eps, X = scipy.linalg.eigh(Hr, subset_by_index=[0, n_occ])
        return eps, X.T                            # rows = states, real basis

    def density(self, X):
        """Closed-shell density rho(r) = 2 sum_v |phi_v(r)|^2 of real-basis occupied rows X."""
        phi_r = self.basis.to_grid(self.basis.real_to_full(X))
        return 2.0 * np.sum(np.abs(phi_r) ** 2, axis=0)

    def _scf(self, tol, max_iter, depth=8, beta=0.5):
        """Self-consistent Hartree ground state: rho = 2 sum_v |phi_v|^2 with phi_v the lowest
        eigenstates of H_ext + v_c * rho.  The fixed point is reached by Anderson mixing of the
        density (any convergent mixing reaches the same fixed point); converged when
        (int |rho_out - rho_in|^2)^{1/2} <= tol."""
        b = self.basis
        H_ext = self.H
        rho = np.zeros(b.grid)
        hist_x, hist_r = [], []
        for it in range(max_iter):
            vH = b.coulomb(rho).real
            H = H_ext + potential_matrix(b, vH)
            _, X = self._solve(self.spec.n_occ, False, H)
            res = self.density(X[:self.spec.n_occ]) - rho
            nres = float(np.sqrt(b.integrate(res * res)))
            if nres <= tol:
                break
            hist_x.append(rho.ravel().copy())
            hist_r.append(res.ravel().copy())
            hist_x, hist_r = hist_x[-depth:], hist_r[-depth:]
            new = rho.ravel() + beta * res.ravel()
            if len(hist_r) > 1:
                dR = np.diff(np.array(hist_r), axis=0)
                dX = np.diff(np.array(hist_x), axis=0)
                gam = np.linalg.lstsq(dR.T, res.ravel(), rcond=None)[0]
                new = new - (dX + beta * dR).T @ gam
            rho = new.reshape(b.grid)
        else:
            raise RuntimeError(f"oracle SCF did not converge: residual {nres:.3e}")
        self.scf_iterations = it
        self.scf_residual = nres
        self.rho = rho
        self.vH = vH
        self.H = H

    def empty_states(self):
        if self.X_all.shape[0] <= self.spec.n_occ + 1 and self.X_all.shape[0] < self.basis.npw:
            raise ValueError("ground state computed without all empty states")
        return self.eps_all[self.spec.n_occ:], self.basis.real_to_full(self.X_all[self.spec.n_occ:])

    def vloc_grid(self):
        """V(r_j) on the grid from its density-sphere Fourier series (used only in tests)."""
        b = self.basis
        V = vloc_atoms(b, b.dG, self.pos, self.spec.Z, self.spec.sigma, self.q).sum(axis=0)
        F = np.zeros(b.grid, dtype=np.complex128)
        F[b.didx] = V
        return np.fft.ifftn(F) * b.nr
