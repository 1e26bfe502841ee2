"""Wannier-localised occupied orbitals and the pair-pruned Liouville operator (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The paper evaluates the integrals of the
screened Coulomb potential with the KS orbitals using Wannier localisation (the accelerations
paragraph of the main text, citing Gygi, Fattebert and Schwegler's simultaneous-diagonalisation
algorithm).  At the Gamma point the maximally localised rotation w_i = sum_v U_vi phi_v maximises
sum_k g_k sum_i |<w_i| e^{-i b_k.r} |w_i>|^2 over the reciprocal vectors b_k, with weights
g_k = |a_k|^2 / (2 pi)^2 (the Gamma-point spread functional); for real orbitals the matrices are
C_k = <phi|cos(b_k.r)|phi> and S_k = <phi|sin(b_k.r)|phi>, real symmetric, and the maximisation is
their joint diagonalisation by Jacobi rotations.  The rotation angle of a pair (p, q) maximises
sum_k g_k [(A'_pp - A'_qq)^2] over the six matrices, whose (cos 2t, sin 2t) is the leading
eigenvector of the 2 x 2 matrix sum_k g_k h_k h_k^T, h_k = (A_pp - A_qq, 2 A_pq) (Cardoso and
Souloumiac's closed form).

The Liouville operator of Eqs. 1-2 is covariant under the rotation: in the Wannier basis,
  (L~ A~)_i = P_c [ H a~_i - sum_j eps~_ji a~_j + Delta a~_i + 2 v_H[sum_j w_j a~_j] w_i
                    - sum_j tau~_ji a~_j ],   eps~ = U^T diag(eps) U,  tau~_ji = W * (w_j w_i),
so L~ = U^T L U.  Pruning keeps tau~_ji only for the pairs whose Wannier centres are within a
cutoff distance (minimum image); it is an approximation, exact in the limit of a large cutoff.
"""
import numpy as np

from .forces import densities, force_contraction, u_vector, zvector_cg
from .liouville import Liouville
from .model import GroundState


def position_matrices(gs):
    """[(g_k, C_k, S_k, M_k)] for k = 1..3: M_k = <phi_v| e^{-i b_k.r} |phi_w>, C = Re M, S = -Im M."""
    b = gs.basis
    N = np.array(b.grid)
    j = np.stack(np.meshgrid(*[np.arange(n) for n in N], indexing="ij"), axis=-1)
    frac = j / N                                            # r = frac @ lattice
    out = []
    pr = gs.phi_r.real.reshape(gs.phi_r.shape[0], -1)
    dv = b.omega / b.nr
    for k in range(3):
        ph = 2 * np.pi * frac[..., k].ravel()               # b_k . r = 2 pi s_k
        M = dv * (pr * np.exp(-1j * ph)[None, :]) @ pr.T
        g = np.dot(b.lattice[k], b.lattice[k]) / (2 * np.pi) ** 2
        out.append((g, M.real.copy(), -M.imag.copy(), M))
    return out


def spread_objective(mats, U):
    """sum_k g_k sum_i |<w_i| e^{-i b_k.r} |w_i>|^2 for the rotation U."""
    t = 0.0
    for g, C, S, _ in mats:
        c = np.einsum("vi,vw,wi->i", U, C, U)
        s = np.einsum("vi,vw,wi->i", U, S, U)
        t += g * np.sum(c * c + s * s)
    return t


def localize(gs, tol=1e-13, max_sweeps=200):
    """Maximally localising rotation U (n_occ x n_occ, w_i = sum_v U_vi phi_v) by Jacobi sweeps of
    the joint diagonalisation; returns (U, centres [n_occ, 3] bohr, sweeps)."""
    mats = position_matrices(gs)
    n = gs.phi_r.shape[0]
    A = []
    for g, C, S, _ in mats:
        A += [(g, C.copy()), (g, S.copy())]
    U = np.eye(n)
    for sweep in range(max_sweeps):
        biggest = 0.0
        for p in range(n - 1):
            for q in range(p + 1, n):
                G = np.zeros((2, 2))
                for g, M in A:
                    h = np.array([M[p, p] - M[q, q], 2.0 * M[p, q]])
                    G += g * np.outer(h, h)
                ev, vec = np.linalg.eigh(G)
                x, y = vec[:, 1]
                if x < 0:
                    x, y = -x, -y
                t = 0.5 * np.arctan2(y, x)
                if abs(t) < 1e-15:
                    continue
                biggest = max(biggest, abs(t))
                c, s = np.cos(t), np.sin(t)
                R = np.array([[c, -s], [s, c]])                # w_p = c phi_p + s phi_q, w_q = -s phi_p + c phi_q
                for _, M in A:
                    M[:, [p, q]] = M[:, [p, q]] @ R
                    M[[p, q], :] = R.T @ M[[p, q], :]
                U[:, [p, q]] = U[:, [p, q]] @ R
        if biggest < tol:
            break
    centres = wannier_centres(gs, U, mats)
    return U, centres, sweep + 1


def wannier_centres(gs, U, mats=None):
    """r_i = sum_k s_ik a_k with s_ik = -arg(<w_i| e^{-i b_k.r} |w_i>) / (2 pi), in [0, 1)."""
    mats = mats or position_matrices(gs)
    s = np.zeros((U.shape[1], 3))
    for k, (_, _, _, M) in enumerate(mats):
        d = np.einsum("vi,vw,wi->i", U, M, U)
        s[:, k] = np.mod(-np.angle(d) / (2 * np.pi), 1.0)
    return s @ gs.basis.lattice


def canonical_order(gs, U, centres):
    """Order the Wannier functions by their fractional centres (rounded) and fix each sign with the
    gauge vector g (<w_i|g> > 0), so both sides of a comparison hold the same basis."""
    from bse_inputs import gauge_vector
    frac = np.mod(centres @ np.linalg.inv(gs.basis.lattice), 1.0)
    key = np.round(frac, 4)
    order = np.lexsort((key[:, 2], key[:, 1], key[:, 0]))
    U = U[:, order]
    centres = centres[order]
    g = gauge_vector(gs.spec.lattice, gs.spec.ecut)
    sgn = np.sign((U.T @ gs.X) @ g)
    sgn[sgn == 0] = 1.0
    return U * sgn[None, :], centres


def pair_mask(lattice, centres, cutoff):
    """kept[i, j] when the minimum-image distance of the centres is <= cutoff (i = j always)."""
    lat = np.asarray(lattice)
    inv = np.linalg.inv(lat)
    d = centres[:, None, :] - centres[None, :, :]
    f = d @ inv
    f -= np.round(f)
    best = np.full(d.shape[:2], np.inf)
    for s in np.array(np.meshgrid([-1, 0, 1], [-1, 0, 1], [-1, 0, 1], indexing="ij")).reshape(3, -1).T:
        best = np.minimum(best, np.linalg.norm((f + s) @ lat, axis=-1))
    keep = best <= cutoff
    np.fill_diagonal(keep, True)
    return keep


class WannierLiouville:
    """L~ of Eqs. 1-2 in the Wannier basis with the K1d pairs pruned by centre distance."""

    def __init__(self, op, U, centres, cutoff):
        self.op = op
        self.gs, self.basis, self.spec = op.gs, op.basis, op.spec
        self.U = U
        self.w = U.T @ op.gs.phi                               # Wannier coefficients (full sphere)
        self.w_r = self.basis.to_grid(self.w)
        self.eps_t = U.T @ np.diag(op.gs.eps) @ U
        self.keep = pair_mask(self.spec.lattice, centres, cutoff)
        self.n_pairs = int((np.count_nonzero(self.keep) + self.keep.shape[0]) // 2)

    def Pc(self, X):
        return self.op.Pc(X)

    def diag_precond(self):
        return self.op.diag_precond()

    def apply(self, At):
        op, b, gs = self.op, self.basis, self.gs
        At = np.asarray(At, dtype=np.complex128)
        a_r = b.to_grid(At)
        MA = At @ gs.H.T - self.eps_t @ At + op.scissor * At
        if op.k1e and op.spin == 0:
            vH = b.coulomb(np.sum(np.conj(self.w_r) * a_r, axis=0))
            MA = MA + 2.0 * b.from_grid(vH[None] * self.w_r)
        if op.k1d:
            no = self.spec.n_occ
            acc = np.zeros_like(a_r)
            for i in range(no):
                for j in range(no):
                    if self.keep[i, j]:
                        acc[i] += op.W.apply(np.conj(self.w_r[j]) * self.w_r[i]) * a_r[j]
            MA = MA - b.from_grid(acc)
        return self.Pc(MA)


def pruned_forces(spec, cutoff, tol=1e-10, seed=0, n_guess=8):
    """Omega from the pruned operator (Davidson in the Wannier basis, started from the rotated
    lowest transitions, with the rotated exact kernel-free preconditioner) and the forces of the
    exact U / Z / contraction evaluated on its eigenvector rotated back to the canonical orbitals.
    Returns (omega, F, A, n_pairs, U, centres)."""
    from bse_inputs import random_trial_block
    from .davidson import davidson
    gs = GroundState(spec, all_states=True)
    op = Liouville(spec, gs=gs)
    U, centres, _ = localize(gs)
    U, centres = canonical_order(gs, U, centres)
    wop = WannierLiouville(op, U, centres, cutoff)
    b = gs.basis
    k = spec.n_roots
    blocks = [b.real_to_full(random_trial_block(seed, k + 2, spec.n_occ, b.npw))]
    de = gs.eps_all[spec.n_occ:][None, :] - gs.eps[:, None]
    phi_c = b.real_to_full(gs.X_all[spec.n_occ:])
    for flat in np.argsort(de, axis=None)[:n_guess]:
        v, c = np.unravel_index(flat, de.shape)
        A = np.zeros((spec.n_occ, b.npw), dtype=complex)
        A[v] = phi_c[c]
        blocks.append(A[None])
    X0 = np.einsum("vi,kvg->kig", U, np.concatenate(blocks, axis=0))        # A~ = U^T A
    eps_c = gs.eps_all[spec.n_occ:]

    def precond(Rt, th):
        R = U @ Rt                                                         # back to canonical
        ov = R @ phi_c.conj().T
        d = eps_c[None, :] - gs.eps[:, None] + spec.scissor - th
        d = np.where(np.abs(d) < 1e-3, np.where(d < 0, -1e-3, 1e-3), d)
        return U.T @ ((ov / d) @ phi_c)

    w, At, rn, it = davidson(wop, X0, n_roots=min(k + 2, X0.shape[0]), tol=tol, precond=precond)
    if not np.all(rn[:k] < tol):
        raise RuntimeError(f"oracle pruned Davidson did not converge: {rn[:k]}")
    A = U @ At[0]
    Uv = u_vector(op, A)
    Z = zvector_cg(op, Uv)
    rho_x, rho_z = densities(op, A, Z)
    F = -force_contraction(op, (rho_x + rho_z).real)
    return w[:k], F, A, wop.n_pairs, U, centres
