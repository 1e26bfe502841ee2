"""Analytical TDA-BSE forces (oracle): U vector, Z-vector, densities and Eq. 4.

Lagrangian route of Sec. SI (alpha_EXX = 0, fixed scissor, dW/d<phi| = 0).  For the
non-self-consistent model (f_Hxc = 0):

  u_w = P_c [ 2 v_c*(Delta rho^*) a_w - sum_v W*(a_v^* a_w) phi_v ] - sum_v S_wv a_v,
  S_wv = <phi_w | (M A)_v>,   L A = P_c M A,

which is the sum of the K1e and K1d contributions printed in Sec. SI (their
second terms are the S-terms); the D contribution vanishes because its
f_Hxc and alpha_EXX terms do.  The Z-vector equation (Eq. 7) then reduces to
  P_c (H - eps_w) Z_w = -u_w,  <Z_w|phi_v> = 0.
In the Hartree-SCF model (f_Hxc = v_c, rho = 2 sum_v |phi_v|^2) the D contribution keeps its
f_Hxc term, u_w += 2 P_c [v_c * Delta rho^(x)] phi_w (the factor is the closed-shell 2 of rho:
the derivative of int v_H[rho] Delta rho^(x) with respect to phi_w is 2 * 2 v_c*(Delta rho^(x)) phi_w
and u is half the real-variable gradient, as for the K1e term above), and the Z-vector operator
gains 2 K1e,KS + 2 K2e,KS (Liouville.apply_zop); the coupled system is solved by one CG.
Then
  d omega / dR = int dV/dR [Delta rho^(x) + Delta rho^(z)]          (Eq. 4)
  Delta rho^(x) = sum_v |a_v|^2 - sum_vv' phi_v^* phi_v' <a_v'|a_v>  (Eq. 5)
  Delta rho^(z) = sum_v (Z_v^* phi_v + phi_v^* Z_v)                  (Eq. 6)
The force reported is F = -d omega/dR (the excited-state increment).
"""
import numpy as np

from .davidson import davidson
from .liouville import Liouville
from .model import GroundState, vloc_atoms


def u_vector(op, A):
    gs, b = op.gs, op.basis
    MA, a_r, drho, vH = op.unprojected(A)
    S = gs.phi.conj() @ MA.T                                   # S[w, v] = <phi_w | (MA)_v>
    no = op.spec.n_occ
    t = np.zeros_like(a_r)
    if op.k1e and op.spin == 0:
        t += 2.0 * b.coulomb(np.conj(drho))[None] * a_r            # 2 v_c*(Delta rho^*) a_w
    if op.k1d:
        for w in range(no):
            for v in range(no):
                t[w] -= op.W.apply(np.conj(a_r[v]) * a_r[w]) * gs.phi_r[v]   # -W*(a_v^* a_w) phi_v
    if gs.hartree:
        rho_x, _ = densities(op, A, np.zeros_like(A))
        t += 2.0 * b.coulomb(rho_x)[None] * gs.phi_r                    # D term, f_Hxc = v_c
    return op.Pc(b.from_grid(t)) - S @ A


def zvector_cg(op, U, tol=1e-12, max_iter=2000):
    """Solve the Z-vector equation (Eq. 7) by preconditioned conjugate gradients on P_c: one CG
    per orbital when the operator is block diagonal (non-SCF model), one CG over all orbitals
    when the Hartree kernel couples them."""
    if op.gs.hartree:
        return _zvector_cg_coupled(op, U, tol, max_iter)
    gs = op.gs
    Z = np.zeros_like(U)
    R = -op.Pc(U)
    diag = 0.5 * op.basis.g2[None, :] + 1.0
    P = op.Pc(R / diag)
    Zr = P.copy()
    rz = np.real(np.sum(R.conj() * Zr, axis=1))
    b0 = np.linalg.norm(R, axis=1)
    for it in range(max_iter):
        AP = op.apply_zop(P)
        pap = np.real(np.sum(P.conj() * AP, axis=1))
        # rows whose residual is already zero (e.g. solved exactly) take no further step
        alpha = np.divide(rz, pap, out=np.zeros_like(rz), where=(pap > 0) & (rz > 0))
        Z = Z + alpha[:, None] * P
        R = R - alpha[:, None] * AP
        if np.all(np.linalg.norm(R, axis=1) <= tol * np.maximum(b0, 1e-300)):
            break
        Zr = op.Pc(R / diag)
        rz_new = np.real(np.sum(R.conj() * Zr, axis=1))
        beta = np.divide(rz_new, rz, out=np.zeros_like(rz), where=rz > 0)
        P = Zr + beta[:, None] * P
        rz = rz_new
    return op.Pc(Z)


def _zvector_cg_coupled(op, U, tol, max_iter):
    """CG for the symmetric positive-definite coupled operator of Eq. 7 over the whole block."""
    R = -op.Pc(U)
    Z = np.zeros_like(U)
    diag = 0.5 * op.basis.g2[None, :] + 1.0
    Zr = op.Pc(R / diag)
    P = Zr.copy()
    rz = np.real(np.vdot(R, Zr))
    b0 = np.linalg.norm(R)
    if b0 == 0.0:
        return Z
    for it in range(max_iter):
        AP = op.apply_zop(P)
        alpha = rz / np.real(np.vdot(P, AP))
        Z = Z + alpha * P
        R = R - alpha * AP
        if np.linalg.norm(R) <= tol * b0:
            break
        Zr = op.Pc(R / diag)
        rz_new = np.real(np.vdot(R, Zr))
        P = Zr + (rz_new / rz) * P
        rz = rz_new
    else:
        raise RuntimeError("oracle Z-vector CG did not converge")
    return op.Pc(Z)


def zvector_sos(op, U, gs_all):
    """Z by the sum over all empty states (only for small bases; non-SCF model, where the
    Z-vector operator is diagonal in the empty states)."""
    if op.gs.hartree:
        raise ValueError("the sum over states solves the non-SCF Z-vector equation only")
    eps_c, phi_c = gs_all.empty_states()
    ov = phi_c.conj() @ U.T                                     # <phi_c | u_w>
    return -((ov / (eps_c[:, None] - op.gs.eps[None, :])).T @ phi_c)


def densities(op, A, Z):
    gs, b = op.gs, op.basis
    a_r = b.to_grid(A)
    O = A.conj() @ A.T                                          # O[v', v] = <a_v'|a_v>
    rho_x = np.sum(np.abs(a_r) ** 2, axis=0) - np.einsum(
        "vxyz,wxyz,wv->xyz", np.conj(gs.phi_r), gs.phi_r, O)
    z_r = b.to_grid(Z)
    rho_z = np.sum(np.conj(z_r) * gs.phi_r + np.conj(gs.phi_r) * z_r, axis=0)
    return rho_x, rho_z


def force_contraction(op, rho):
    """d omega/dR_{a,alpha} = Omega sum_{G in density sphere} Re[i G_alpha V_a(G)^* rhohat(G)]."""
    b = op.basis
    rh = b.density_coeffs(rho)
    Va = vloc_atoms(b, b.dG, op.gs.pos, op.spec.Z, op.spec.sigma, op.gs.q)
    dw = np.einsum("ag,gx->ax", np.conj(Va) * rh[None, :], 1j * b.dG)
    return b.omega * dw.real


class ForceResult:
    pass


def excitation(spec, pos=None, gs=None, n_pdep=None, tol=1e-10, seed=0, n_guess=8, **kw):
    """Lowest spec.n_roots eigenpairs of Eq. 1.

    Davidson converges to whichever roots its subspace resolves first, and from a random start it
    can settle on an excited root whose residual vanishes before the lowest one enters the
    subspace.  So the start block holds the n_guess lowest single transitions phi_v -> phi_c
    (ordered by eps_c - eps_v, the diagonal of the D term of Eq. 2a) next to k + 2 seeded random
    vectors, and k + 2 roots are converged, of which the lowest k are returned."""
    if gs is None:
        gs = GroundState(spec, pos=pos, all_states=True)
    op = Liouville(spec, gs=gs, n_pdep=n_pdep, **kw)
    from bse_inputs import random_trial_block
    k = spec.n_roots
    b = gs.basis
    blocks = [b.real_to_full(random_trial_block(seed, k + 2, spec.n_occ, b.npw))]
    n_states = gs.X_all.shape[0]
    if n_states > spec.n_occ:
        de = gs.eps_all[spec.n_occ:][None, :] - gs.eps[:, None]          # (v, c)
        order = np.argsort(de, axis=None)[:n_guess]
        phi_c = b.real_to_full(gs.X_all[spec.n_occ:])
        for flat in order:
            v, c = np.unravel_index(flat, de.shape)
            A = np.zeros((spec.n_occ, b.npw), dtype=complex)
            A[v] = phi_c[c]
            blocks.append(A[None])
    X0 = np.concatenate(blocks, axis=0)
    n_track = min(k + 2, X0.shape[0])
    precond = None
    if n_states == b.npw:
        # with every empty state known, correct with the exact inverse of (D - theta) for the
        # kernel-free D of Eq. 2a: r_vc / (eps_c - eps_v + scissor - theta) in the empty states
        eps_c = gs.eps_all[spec.n_occ:]
        shift = kw.get("scissor", spec.scissor)

        def precond(R, th):
            ov = R @ phi_c.conj().T                                    # <phi_c | r_v>
            d = eps_c[None, :] - gs.eps[:, None] + shift - th
            d = np.where(np.abs(d) < 1e-3, np.where(d < 0, -1e-3, 1e-3), d)
            return (ov / d) @ phi_c
    w, A, rn, it = davidson(op, X0, n_roots=n_track, tol=tol, precond=precond)
    if not np.all(rn[:k] < tol):
        raise RuntimeError(f"oracle Davidson did not converge: residuals {rn[:k]}")
    return w[:k], A[:k], op


def bse_forces(spec, root=0, pos=None, n_pdep=None, tol=1e-10, **kw):
    """Full oracle pipeline: ground state, Davidson, U, Z (CG), densities, forces."""
    w, A, op = excitation(spec, pos=pos, n_pdep=n_pdep, tol=tol, **kw)
    a = A[root]
    U = u_vector(op, a)
    Z = zvector_cg(op, U)
    rho_x, rho_z = densities(op, a, Z)
    dw = force_contraction(op, (rho_x + rho_z).real)
    r = ForceResult()
    r.omega, r.A, r.U, r.Z, r.op = w, a, U, Z, op
    r.rho_x, r.rho_z = rho_x, rho_z
    r.domega_dR = dw
    r.F = -dw
    return r


def omega_fd(spec, atom, alpha, h=1e-3, root=0, n_pdep=None, tol=1e-11, **kw):
    """Central finite difference of omega(R) with W held fixed in G-space (Sec. SII)."""
    vals = []
    for s in (+1, -1):
        p = spec.pos.copy()
        p[atom, alpha] += s * h
        w, _, _ = excitation(spec, pos=p, n_pdep=n_pdep, tol=tol, **kw)
        vals.append(w[root])
    return (vals[0] - vals[1]) / (2 * h)


def omega_fd_richardson(spec, atom, alpha, h=1e-3, **kw):
    d1 = omega_fd(spec, atom, alpha, h=h, **kw)
    d2 = omega_fd(spec, atom, alpha, h=h / 2, **kw)
    return (4 * d2 - d1) / 3
