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


class BatchExcitationEnergies(torch.autograd.Function):
    """forward(R_1, ..., R_n, batch=...) -> Omega of every system of a ``BSEBatch``.

    The batch solve already runs the Z-vector and the force contraction for every system, so the
    forward pass keeps the forces and the backward pass is grad_R_i = -F_i * grad_Omega_i."""

    @staticmethod
    def forward(ctx, batch, tols, *Rs):
        pos = [R.detach().to("cpu", torch.float64).numpy().copy() for R in Rs]
        for p, na in zip(pos, batch.n_atoms):
            if p.shape != (na, 3):
                raise ValueError(f"positions must have shape ({na}, 3), got {tuple(p.shape)}")
        st = batch.set_positions(pos)
        w, F, st2 = batch.solve(*tols)
        if st != 0 or st2 != 0 or not np.all(np.isfinite(w)):
            raise RuntimeError("batch solve failed: " + "; ".join(
                f"system {i}: {batch.error(i)}" for i in range(len(w)) if batch.status(i) != 0))
        ctx.F = F
        ctx.devices = [R.device for R in Rs]
        return torch.tensor(w, dtype=torch.float64, device=Rs[0].device)

    @staticmethod
    def backward(ctx, grad_w):
        g = grad_w.detach().to("cpu", torch.float64).numpy()
        grads = tuple(torch.as_tensor(-gi * Fi, dtype=torch.float64, device=d)
                      for gi, Fi, d in zip(g, ctx.F, ctx.devices))
        return (None, None) + grads


def batch_excitation_energies(Rs, batch, davidson_tol=1e-9, zvector_tol=1e-10, max_iter=500):
    """Omega of every system of ``batch`` (a ``BSEBatch``) at positions Rs, differentiable in each R."""
    return BatchExcitationEnergies.apply(batch, (davidson_tol, zvector_tol, max_iter), *Rs)
