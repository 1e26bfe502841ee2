"""Plane-wave basis at the Gamma point (oracle).

Conventions (Hartree atomic units, Ecut in Ry so the sphere is |G|^2 <= Ecut):
an orbital is f(r) = Omega^{-1/2} sum_G c(G) exp(iG.r) with sum_G |c(G)|^2 = 1;
a density or potential is rho(r) = sum_G rhohat(G) exp(iG.r).  The FFT grid has
points r_j = sum_i (j_i/N_i) a_i.  The paper works at Gamma only (Sec. SIV).
"""
import numpy as np


class PWBasis:
    """Full wave-function sphere |G|^2 <= ecut and density sphere |G|^2 <= 4 ecut."""

    def __init__(self, lattice, ecut, grid):
        self.lattice = np.asarray(lattice, dtype=np.float64)
        self.ecut = float(ecut)
        self.grid = tuple(int(n) for n in grid)
        self.nr = int(np.prod(self.grid))
        self.omega = abs(np.linalg.det(self.lattice))
        self.B = 2.0 * np.pi * np.linalg.inv(self.lattice).T       # rows b_i
        self.mill, self.G, self.g2 = self._sphere(self.ecut)
        self.dmill, self.dG, self.dg2 = self._sphere(4.0 * self.ecut)
        self.npw = len(self.mill)
        self.idx = self._grid_index(self.mill)
        self.didx = self._grid_index(self.dmill)
        self._check_alias_free()
        self._real_basis_maps()

    def _sphere(self, gmax2):
        nmax = [int(np.floor(np.sqrt(gmax2) * np.linalg.norm(self.lattice[i]) / (2 * np.pi))) + 1
                for i in range(3)]
        m = np.array([(a, b, c) for a in range(-nmax[0], nmax[0] + 1)
                      for b in range(-nmax[1], nmax[1] + 1)
                      for c in range(-nmax[2], nmax[2] + 1)])
        G = m @ self.B
        g2 = np.sum(G * G, axis=1)
        keep = g2 <= gmax2
        return m[keep], G[keep], g2[keep]

    def _grid_index(self, m):
        N = np.array(self.grid)
        w = np.mod(m, N)
        return (w[:, 0], w[:, 1], w[:, 2])

    def _check_alias_free(self):
        # products of a density-sphere function with a wave-function-sphere
        # function must not alias back into the wave-function sphere
        kw = np.abs(self.mill).max(axis=0)
        kd = np.abs(self.dmill).max(axis=0)
        if np.any(np.array(self.grid) < kd + 2 * kw + 1):
            raise ValueError("FFT grid too small for alias-free products")

    # --- real basis of the input format (see bse_inputs) -----------------
    def _real_basis_maps(self):
        m = self.mill
        pos = (m[:, 2] > 0) | ((m[:, 2] == 0) & (m[:, 1] > 0)) | (
            (m[:, 2] == 0) & (m[:, 1] == 0) & (m[:, 0] > 0))
        half = np.nonzero(pos)[0]
        order = np.lexsort((m[half, 0], m[half, 1], m[half, 2]))   # by (n3, n2, n1)
        half = half[order]
        lookup = {tuple(x): i for i, x in enumerate(m)}
        neg = np.array([lookup[tuple(-m[i])] for i in half])
        zero = lookup[(0, 0, 0)]
        self.i_zero, self.i_plus, self.i_minus = zero, half, neg
        self.nhalf = len(half)
        assert 2 * self.nhalf + 1 == self.npw

    def real_to_full(self, x):
        """Real-basis rows (..., npw) -> complex full-sphere coefficients (..., npw)."""
        x = np.asarray(x, dtype=np.float64)
        c = np.zeros(x.shape, dtype=np.complex128)
        c[..., self.i_zero] = x[..., 0]
        cp = (x[..., 1::2] + 1j * x[..., 2::2]) / np.sqrt(2.0)
        c[..., self.i_plus] = cp
        c[..., self.i_minus] = np.conj(cp)
        return c

    def full_to_real(self, c):
        """Inverse of real_to_full for coefficients of real-in-r functions."""
        c = np.asarray(c)
        x = np.zeros(c.shape, dtype=np.float64)
        x[..., 0] = c[..., self.i_zero].real
        cp = c[..., self.i_plus]
        x[..., 1::2] = np.sqrt(2.0) * cp.real
        x[..., 2::2] = np.sqrt(2.0) * cp.imag
        return x

    def real_basis_matrix(self):
        """Unitary U with c_full = U x_real (columns = real basis functions)."""
        return self.real_to_full(np.eye(self.npw)).T

    # --- grid transforms ----------------------------------------------------
    def to_grid(self, c):
        """Orbital coefficients (..., npw) -> f(r_j) on the grid (..., N1, N2, N3)."""
        c = np.asarray(c, dtype=np.complex128)
        F = np.zeros(c.shape[:-1] + self.grid, dtype=np.complex128)
        F[(Ellipsis,) + self.idx] = c
        return np.fft.ifftn(F, axes=(-3, -2, -1)) * (self.nr / np.sqrt(self.omega))

    def from_grid(self, f):
        """Grid function (..., N1, N2, N3) -> orbital coefficients on the wave-function sphere."""
        F = np.fft.fftn(f, axes=(-3, -2, -1)) * (np.sqrt(self.omega) / self.nr)
        return F[(Ellipsis,) + self.idx]

    def density_coeffs(self, rho):
        """rhohat(G) on the density sphere for rho(r) = sum_G rhohat(G) e^{iG.r}."""
        F = np.fft.fftn(rho, axes=(-3, -2, -1)) / self.nr
        return F[(Ellipsis,) + self.didx]

    def integrate(self, f):
        """int_cell f(r) dr, exact for functions band-limited to the grid."""
        return np.sum(f, axis=(-3, -2, -1)) * (self.omega / self.nr)

    def coulomb(self, rho):
        """v_c * rho: 4 pi/|G|^2 on the density sphere, G = 0 dropped."""
        F = np.fft.fftn(rho, axes=(-3, -2, -1)) / self.nr
        out = np.zeros_like(F)
        v = np.zeros(len(self.dg2))
        nz = self.dg2 > 0
        v[nz] = 4.0 * np.pi / self.dg2[nz]
        out[(Ellipsis,) + self.didx] = F[(Ellipsis,) + self.didx] * v
        return np.fft.ifftn(out, axes=(-3, -2, -1)) * self.nr
