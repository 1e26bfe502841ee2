"""Bare and screened Coulomb interactions (oracle).

W(r, r') = v_c(r, r') + (1/Omega) sum_a phitilde_a(r) lambda_a/(1 - lambda_a) phitilde_a*(r'),
phitilde_a = v_c^{1/2} phi_a  (Eq. 3, PDEP form).

Readings of the paper's silent points:
 * PDEP vectors phi_a(r) = sum_G phi_a(G) e^{iG.r} with sum_G |phi_a(G)|^2 = 1 on
   the wave-function sphere (G = 0 excluded), so the 1/Omega of Eq. 3 cancels the
   Omega of the r'-integral;
 * v_c(G) = 4 pi / |G|^2 for 0 < |G|^2 <= 4 Ecut, zero at G = 0 and outside;
 * v_c^{1/2}(G) = sqrt(4 pi) / |G| on the wave-function sphere, zero at G = 0.
"""
import numpy as np


class Screening:
    def __init__(self, basis, pdep_coef, pdep_lambda, n_pdep=None):
        self.basis = basis
        coef = np.asarray(pdep_coef, dtype=np.float64)
        lam = np.asarray(pdep_lambda, dtype=np.float64)
        if n_pdep is not None:
            coef, lam = coef[:n_pdep], lam[:n_pdep]
        self.npdep = coef.shape[0]
        self.c = lam / (1.0 - lam)                             # lambda_a / (1 - lambda_a)
        self.phi = basis.real_to_full(coef) if self.npdep else np.zeros((0, basis.npw), complex)
        g = np.sqrt(basis.g2)
        self.s = np.where(basis.g2 > 0, np.sqrt(4 * np.pi) / np.where(g > 0, g, 1.0), 0.0)
        self.vc = np.where(basis.dg2 > 0, 4 * np.pi / np.where(basis.dg2 > 0, basis.dg2, 1.0), 0.0)

    def apply_G(self, rhohat_grid):
        """(W rho)^ on the full FFT grid given rhohat on the full FFT grid (Fourier series coeffs)."""
        b = self.basis
        out = np.zeros_like(rhohat_grid)
        out[(Ellipsis,) + b.didx] = self.vc * rhohat_grid[(Ellipsis,) + b.didx]
        if self.npdep:
            x = self.s * rhohat_grid[(Ellipsis,) + b.idx]          # v_c^{1/2} rho on the sphere
            p = x @ self.phi.conj().T                              # <phi_a | v_c^{1/2} rho>
            out[(Ellipsis,) + b.idx] += self.s * ((p * self.c) @ self.phi)
        return out

    def apply(self, rho):
        """W * rho for grid functions rho (..., N1, N2, N3)."""
        b = self.basis
        F = np.fft.fftn(rho, axes=(-3, -2, -1)) / b.nr
        return np.fft.ifftn(self.apply_G(F), axes=(-3, -2, -1)) * b.nr

    def dense_matrix(self):
        """W as an explicit matrix on the density sphere (its definition, for tests)."""
        b = self.basis
        n = len(b.dg2)
        W = np.diag(self.vc).astype(np.complex128)
        if self.npdep:
            lookup = {tuple(m): i for i, m in enumerate(b.dmill)}
            pos = np.array([lookup[tuple(m)] for m in b.mill])
            ph = np.zeros((self.npdep, n), dtype=np.complex128)
            ph[:, pos] = self.phi * self.s[None, :]
            W += ph.T @ np.diag(self.c) @ ph.conj()
        return W
