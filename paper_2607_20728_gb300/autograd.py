"""Differentiable excitation energy: Omega(R) with a hand-written adjoint.

``ExcitationEnergy.apply(R, system)`` returns the lowest (or ``root``-th) TDA-BSE excitation
energy at atomic positions R (bohr, shape (n_atoms, 3), float64).  Its backward pass does not
differentiate through the Davidson iterations: by the Lagrangian construction of Sec. 2 (Eq. 4-6)
the total derivative of Omega is the Hellmann-Feynman-like contraction of the relaxed
excited-state density (the excitation density of A plus the orbital-response density of the
Z-vector, which solves P_c (H - eps_v) Z_v = -u_v) with dV_loc/dR.  So backward is one Z-vector
solve plus the force contraction, both in the CUDA library: grad_R = -F * grad_Omega.

W is held fixed under the displacement (the screening enters through fixed PDEP vectors in
reciprocal space), which is the derivative the library's forces are.
"""
import numpy as np
import torch


class ExcitationEnergy(torch.autograd.Function):
    """forward(R, system, root=0, tol=1e-9, z_tol=1e-10) -> Omega (0-dim float64 tensor on R's device)."""

    @staticmethod
    def forward(ctx, R, system, root=0, tol=1e-9, z_tol=1e-10, max_iter=300):
        pos = R.detach().to("cpu", torch.float64).numpy().copy()
        if pos.shape != (system.n_atoms, 3):
            raise ValueError(f"positions must have shape ({system.n_atoms}, 3), got {tuple(pos.shape)}")
        system.set_positions(pos)
        w, _ = system.davidson(n_roots=root + 1, tol=tol, max_iter=max_iter)
        ctx.system, ctx.root, ctx.tol, ctx.z_tol, ctx.max_iter = system, root, tol, z_tol, max_iter
        ctx.pos = pos
        ctx.generation = system.generation
        ctx.device = R.device
        return torch.tensor(float(w[root]), dtype=torch.float64, device=R.device)

    @staticmethod
    def backward(ctx, grad_omega):
        s = ctx.system
        if s.generation != ctx.generation:
            # another forward ran on this system since ours: restore our geometry and roots
            s.set_positions(ctx.pos)
            s.davidson(n_roots=ctx.root + 1, tol=ctx.tol, max_iter=ctx.max_iter)
        s.zvector(root=ctx.root, tol=ctx.z_tol, max_iter=10 * ctx.max_iter)
        F = s.forces(root=ctx.root)                        # -dOmega/dR, Ha/bohr
        g = torch.as_tensor(-np.asarray(F), dtype=torch.float64, device=ctx.device)
        return g * grad_omega, None, None, None, None, None


def excitation_energy(R, system, root=0, tol=1e-9, z_tol=1e-10, max_iter=300):
    """Omega(R) for ``system`` (a ``BSESystem``), differentiable with respect to R."""
    return ExcitationEnergy.apply(R, system, root, tol, z_tol, max_iter)
