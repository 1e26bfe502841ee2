"""TDA-BSE matrix, and the coupling block of the full BSE, in the explicit transition basis
(oracle check (a)).

With every empty eigenstate phi_c of H in the plane-wave sphere, the response
orbitals are a_v = sum_c X_vc phi_c and Eq. 1 becomes the familiar matrix
  M_{vc,v'c'} = (eps_c - eps_v + Delta) delta_vv' delta_cc'
              + 2 (phi_c phi_v | v_c | phi_v' phi_c')        [K1e, Eq. 2b]
              -   (phi_c phi_c' | W | phi_v' phi_v)          [K1d, Eq. 2c]
for real orbitals.  Its lowest eigenvalue is Omega.  This is the conventional
electron-hole-basis form that the paper's DMPT formulation avoids (main text,
after Eq. 3); it is used here only as an independent definition.
"""
import numpy as np

from .model import GroundState
from .screening import Screening


def bse_matrix(spec, gs=None, n_pdep=None, k1e=True, k1d=True, spin=None, scissor=None):
    if gs is None:
        gs = GroundState(spec, all_states=True)
    b = gs.basis
    spin = spec.spin if spin is None else spin
    scissor = spec.scissor if scissor is None else scissor
    W = Screening(b, spec.pdep_coef, spec.pdep_lambda, n_pdep=n_pdep)
    eps_c, phi_c = gs.empty_states()
    no, ne = spec.n_occ, len(eps_c)
    occ_r = gs.phi_r.real
    emp_r = b.to_grid(phi_c)
    assert np.abs(emp_r.imag).max() < 1e-10
    emp_r = emp_r.real
    dv = b.omega / b.nr
    n = no * ne
    M = np.zeros((n, n))
    M[np.diag_indices(n)] = (eps_c[None, :] - gs.eps[:, None] + scissor).ravel()
    E = emp_r.reshape(ne, -1)
    if k1e and spin == 0:
        P = (occ_r[:, None] * emp_r[None]).reshape(n, *b.grid)           # phi_v phi_c
        VP = b.coulomb(P).real.reshape(n, -1)
        M += 2.0 * dv * (P.reshape(n, -1) @ VP.T)
    if k1d:
        for v in range(no):
            for vp in range(no):
                tau = W.apply(occ_r[vp] * occ_r[v]).real.ravel()
                M[v * ne:(v + 1) * ne, vp * ne:(vp + 1) * ne] -= dv * (E * tau[None, :]) @ E.T
    return M, gs


def lowest(spec, k=1, **kw):
    M, gs = bse_matrix(spec, **kw)
    w = np.linalg.eigvalsh(0.5 * (M + M.T))
    return w[:k]


def coupling_matrix(spec, gs=None, n_pdep=None, k1e=True, k1d=True, spin=None):
    """The coupling block B of the BSE beyond the TDA (Sec. SI) in the transition basis, real orbitals:
      B_{vc,v'c'} = 2 (phi_c phi_v | v_c | phi_v' phi_c')      [K2e]
                  -   (phi_c phi_v' | W | phi_c' phi_v)        [K2d]."""
    if gs is None:
        gs = GroundState(spec, all_states=True)
    b = gs.basis
    spin = spec.spin if spin is None else spin
    W = Screening(b, spec.pdep_coef, spec.pdep_lambda, n_pdep=n_pdep)
    eps_c, phi_c = gs.empty_states()
    no, ne = spec.n_occ, len(eps_c)
    occ_r = gs.phi_r.real
    emp_r = b.to_grid(phi_c).real
    dv = b.omega / b.nr
    n = no * ne
    Bm = np.zeros((n, n))
    P = (occ_r[:, None] * emp_r[None]).reshape(n, *b.grid)               # P[(v, c)] = phi_v phi_c
    if k1e and spin == 0:
        Bm += 2.0 * dv * (P.reshape(n, -1) @ b.coulomb(P).real.reshape(n, -1).T)
    if k1d:
        # G[(v', c), (v, c')] = (phi_v' phi_c | W | phi_v phi_c');  B[v, c, v', c'] -= G[v', c, v, c']
        WP = W.apply(P).real.reshape(n, -1)
        G = dv * (P.reshape(n, -1) @ WP.T)
        Bm -= G.reshape(no, ne, no, ne).transpose(2, 1, 0, 3).reshape(n, n)
    return Bm, gs


def full_lowest(spec, k=1, **kw):
    """Lowest k excitation energies of the BSE beyond the TDA (Sec. SI): the positive eigenvalues
    of [[A, B], [-B, -A]], computed for real A, B with A - B positive definite as the square roots
    of the eigenvalues of (A - B)^{1/2} (A + B) (A - B)^{1/2}."""
    A, gs = bse_matrix(spec, **kw)
    kw.pop("scissor", None)
    kw.pop("gs", None)
    Bm, _ = coupling_matrix(spec, gs=gs, **kw)
    A = 0.5 * (A + A.T)
    Bm = 0.5 * (Bm + Bm.T)
    em, Um = np.linalg.eigh(A - Bm)
    if em.min() <= 0:
        raise ValueError("A - B is not positive definite: the BSE has no real spectrum here")
    S = (Um * np.sqrt(em)) @ Um.T
    w2 = np.linalg.eigvalsh(S @ (A + Bm) @ S)
    if w2.min() <= 0:
        raise ValueError("A + B is not positive definite: the BSE has no real spectrum here")
    return np.sqrt(w2[:k])
