"""DMPT form of the TDA Bethe-Salpeter operator (oracle), Eqs. 1-2, and the coupling block B of
the BSE beyond the TDA (Sec. SI).

  (D A)_v    = P_c (H^QP - eps_v^QP) a_v,   H^QP = H^KS + P_c Delta_sci   (Eq. 2a; Table S1)
  (K1e A)_v  = P_c [v_c * Delta rho] phi_v,  Delta rho = sum_v phi_v^* a_v  (Eq. 2b)
  (K1d A)_v  = P_c sum_v' [W * (phi_v'^* phi_v)] a_v'                     (Eq. 2c)
  P_c        = 1 - sum_v |phi_v><phi_v|

The singlet operator is D + 2 K1e - K1d (Eq. 1); the triplet channel drops the
exchange term (D - K1d).  ``k1e``/``k1d`` switch terms off for the special cases
of Table S1 (K1d = 0: semi-local-TDDFT-like; W = v_c: CIS-like).

The D term uses the dense Hamiltonian matrix; the kernel terms use real-space
products on the FFT grid.  Trial vectors are full-sphere complex coefficient
arrays of shape (n_occ, npw).
"""
import numpy as np

from .model import GroundState
from .screening import Screening


class Liouville:
    def __init__(self, spec, gs=None, n_pdep=None, k1e=True, k1d=True, spin=None, scissor=None,
                 tau_cache_bytes=2 << 30):
        self.spec = spec
        self.gs = gs if gs is not None else GroundState(spec)
        self.basis = self.gs.basis
        self.W = Screening(self.basis, spec.pdep_coef, spec.pdep_lambda, n_pdep=n_pdep)
        self.k1e = bool(k1e)
        self.k1d = bool(k1d)
        self.spin = spec.spin if spin is None else int(spin)
        self.scissor = spec.scissor if scissor is None else float(scissor)
        no = spec.n_occ
        self._tau = None
        if no * no * self.basis.nr * 16 <= tau_cache_bytes:
            self._tau = {}

    # ---- occupied-space projector ---------------------------------------------
    def Pc(self, X):
        """P_c = 1 - sum_v |phi_v><phi_v| applied to each row."""
        phi = self.gs.phi
        S = X @ phi.conj().T
        return X - S @ phi

    # ---- tau_{v'v} = W * (phi_v'^* phi_v) (Eq. 2c) --------------------------------
    def tau(self, vp, v):
        if self._tau is not None and (vp, v) in self._tau:
            return self._tau[(vp, v)]
        pr = self.gs.phi_r
        t = self.W.apply(np.conj(pr[vp]) * pr[v])
        if self._tau is not None:
            self._tau[(vp, v)] = t
        return t

    # ---- the operator ------------------------------------------------------------
    def unprojected(self, A):
        """M A with L A = P_c M A; returns (M A, a_r, Delta rho, v_H)."""
        gs, b = self.gs, self.basis
        A = np.asarray(A, dtype=np.complex128)
        no = self.spec.n_occ
        a_r = b.to_grid(A)
        # D, Eq. 2a with the scissor shift acting on P_c A = A
        MA = A @ gs.H.T - gs.eps[:, None] * A + self.scissor * A
        drho = np.sum(np.conj(gs.phi_r) * a_r, axis=0)
        vH = b.coulomb(drho)
        if self.k1e and self.spin == 0:
            MA = MA + 2.0 * b.from_grid(vH[None] * gs.phi_r)              # 2 K1e, Eq. 2b
        if self.k1d:
            acc = np.zeros_like(a_r)
            for v in range(no):
                for vp in range(no):
                    acc[v] += self.tau(vp, v) * a_r[vp]
            MA = MA - b.from_grid(acc)                                    # -K1d, Eq. 2c
        return MA, a_r, drho, vH

    def apply(self, A):
        """L A = (D + 2 K1e - K1d) A (singlet) or (D - K1d) A (triplet), Eq. 1."""
        return self.Pc(self.unprojected(A)[0])

    def apply_B(self, A):
        """B A, the coupling block of the BSE beyond the TDA (Sec. SI):
        (K2e A)_v = P_c [v_c * sum_v' a_v'^* phi_v'] phi_v,
        (K2d A)_v = P_c sum_v' [W * (a_v'^* phi_v)] phi_v',
        B = 2 K2e - K2d (singlet) or -K2d (triplet), terms switched like K1e/K1d."""
        gs, b = self.gs, self.basis
        A = np.asarray(A, dtype=np.complex128)
        no = self.spec.n_occ
        a_r = b.to_grid(A)
        out = np.zeros_like(a_r)
        if self.k1e and self.spin == 0:
            rho2 = np.sum(np.conj(a_r) * gs.phi_r, axis=0)
            out += 2.0 * b.coulomb(rho2)[None] * gs.phi_r
        if self.k1d:
            for v in range(no):
                for vp in range(no):
                    out[v] -= self.W.apply(np.conj(a_r[vp]) * gs.phi_r[v]) * gs.phi_r[vp]
        return self.Pc(b.from_grid(out))

    def apply_zop(self, Z):
        """The Z-vector operator of Eq. 7 with alpha_EXX = 0 (K1d,KS = K2d,KS = 0):
        P_c (H^KS - eps_v) Z_v, plus, in the Hartree-SCF model (f_Hxc = v_c), the kernel terms
        2 K1e,KS + 2 K2e,KS, which for real orbitals and real Z are both
        P_c [v_c * sum_v' phi_v' Z_v'] phi_v, i.e. 4 P_c [v_c * sum_v' phi_v' Z_v'] phi_v."""
        gs, b = self.gs, self.basis
        Z = np.asarray(Z, dtype=np.complex128)
        out = Z @ gs.H.T - gs.eps[:, None] * Z
        if gs.hartree:
            z_r = b.to_grid(Z)
            vz = b.coulomb(np.sum(np.conj(gs.phi_r) * z_r, axis=0))
            out = out + 4.0 * b.from_grid(vz[None] * gs.phi_r)
        return self.Pc(out)

    def energy(self, A):
        """A^dagger L A for a (not necessarily normalised) P_c-space A."""
        return np.real(np.vdot(A, self.apply(A)))

    def diag_precond(self):
        """Diagonal of D in the plane-wave basis, used by the Davidson preconditioner."""
        gs = self.gs
        v0 = np.real(np.trace(gs.H) - 0.5 * np.sum(self.basis.g2)) / self.basis.npw
        return 0.5 * self.basis.g2[None, :] + v0 - gs.eps[:, None] + self.scissor
