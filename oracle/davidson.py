"""Block Davidson eigensolver for the lowest roots of the TDA operator (oracle).

The paper's WEST code solves Eq. 1 iteratively; it does not describe the
solver, so this is the textbook block Davidson method (Rayleigh-Ritz on a growing
subspace, diagonal preconditioner, restart to the current Ritz vectors), kept
on the P_c space.  Vectors are flattened (n_occ * npw) complex arrays.
"""
import numpy as np


def _orth_against(V, T):
    for _ in range(2):
        if V.shape[0]:
            T = T - (T @ V.conj().T) @ V
    out = []
    for t in T:
        for q in out:
            t = t - np.vdot(q, t) * q
        nrm = np.linalg.norm(t)
        if nrm > 1e-8:
            t = t / nrm
            for q in out:
                t = t - np.vdot(q, t) * q
            t = t / np.linalg.norm(t)
            out.append(t)
    return np.array(out) if out else np.zeros((0, V.shape[1]), V.dtype)


def davidson(op, X0, n_roots=1, tol=1e-9, max_iter=300, max_sub=None):
    """Lowest ``n_roots`` eigenpairs of the TDA operator ``op`` (a Liouville).

    X0: initial trial block (k, n_occ, npw).  Returns (omega, A, residual_norms, iters)."""
    shape = X0.shape[1:]
    proj = lambda X: op.Pc(X.reshape(-1, *shape)).reshape(X.shape[0], -1)
    apply = lambda X: np.stack([op.apply(x.reshape(shape)).ravel() for x in X])
    diag = op.diag_precond().ravel()
    k = X0.shape[0]
    max_sub = max_sub or max(8 * k, 24)
    V = _orth_against(np.zeros((0, X0[0].size), complex), proj(X0.reshape(k, -1).astype(complex)))
    AV = apply(V)
    it = 0
    while True:
        it += 1
        Hs = V.conj() @ AV.T
        Hs = 0.5 * (Hs + Hs.conj().T)
        th, y = np.linalg.eigh(Hs)
        th, y = th[:n_roots], y[:, :n_roots]
        X = y.T @ V
        AX = y.T @ AV
        R = AX - th[:, None] * X
        rn = np.linalg.norm(R, axis=1)
        if np.all(rn < tol) or it >= max_iter:
            return th, X.reshape(n_roots, *shape), rn, it
        T = []
        for j in range(n_roots):
            if rn[j] >= tol:
                d = diag - th[j]
                d = np.where(np.abs(d) < 0.1, np.where(d < 0, -0.1, 0.1), d)
                T.append(R[j] / d)
        T = proj(np.array(T))
        if V.shape[0] + T.shape[0] > max_sub:
            V = _orth_against(np.zeros((0, V.shape[1]), complex), X)
            AV = apply(V)
        T = _orth_against(V, T)
        if T.shape[0] == 0:
            return th, X.reshape(n_roots, *shape), rn, it
        V = np.vstack([V, T])
        AV = np.vstack([AV, apply(T)])
