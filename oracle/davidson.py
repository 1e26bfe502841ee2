"""Block Davidson eigensolver for the lowest roots of the TDA operator (oracle).

The paper's WEST code solves Eq. 1 iteratively; it does not describe the
solver, so this is the textbook block Davidson method (Rayleigh-Ritz on a growing
subspace, diagonal preconditioner, restart to the current Ritz vectors), kept
on the P_c space.  Vectors are flattened (n_occ * npw) complex arrays.
"""
import numpy as np


def _orth_against(V, T):
    """Orthonormalise the rows of T against the orthonormal rows of V and each other (Gram-Schmidt
    twice); a row is dropped when less than 1e-10 of its norm survives the projections (a relative
    test, so that the small corrections of a nearly converged solve are kept)."""
    n0 = np.linalg.norm(T, axis=1) if T.shape[0] else np.zeros(0)
    for _ in range(2):
        if V.shape[0]:
            T = T - (T @ V.conj().T) @ V
    out = []
    for t, t0 in zip(T, n0):
        for q in out:
            t = t - np.vdot(q, t) * q
        nrm = np.linalg.norm(t)
        if t0 > 0 and nrm > 1e-10 * t0:
            t = t / nrm
            for q in out:
                t = t - np.vdot(q, t) * q
            t = t / np.linalg.norm(t)
            out.append(t)
    return np.array(out) if out else np.zeros((0, V.shape[1]), V.dtype)


def davidson(op, X0, n_roots=1, tol=1e-9, max_iter=300, max_sub=None, precond=None):
    """Lowest ``n_roots`` eigenpairs of the TDA operator ``op`` (a Liouville).

    X0: initial trial block (k, n_occ, npw).  precond(R, theta), optional, returns the correction
    for residual R (n_occ, npw) of a Ritz value theta; default: the diagonal of D (Eq. 2a) in
    the plane-wave basis.  Returns (omega, A, residual_norms, iters)."""
    shape = X0.shape[1:]
    proj = lambda X: op.Pc(X.reshape(-1, *shape)).reshape(X.shape[0], -1)
    apply = lambda X: np.stack([op.apply(x.reshape(shape)).ravel() for x in X])
    diag = op.diag_precond().ravel()
    k = X0.shape[0]
    max_sub = max_sub or max(8 * k, 24)
    keep = min(k, max_sub // 2)           # Ritz vectors kept at a restart
    V = _orth_against(np.zeros((0, X0[0].size), complex), proj(X0.reshape(k, -1).astype(complex)))
    AV = apply(V)
    it = 0
    while True:
        it += 1
        Hs = V.conj() @ AV.T
        Hs = 0.5 * (Hs + Hs.conj().T)
        th_all, y_all = np.linalg.eigh(Hs)
        th, y = th_all[:n_roots], y_all[:, :n_roots]
        X = y.T @ V
        AX = y.T @ AV
        R = AX - th[:, None] * X
        rn = np.linalg.norm(R, axis=1)
        if np.all(rn < tol) or it >= max_iter:
            return th, X.reshape(n_roots, *shape), rn, it
        T = []
        for j in range(n_roots):
            if rn[j] >= tol:
                if precond is not None:
                    T.append(precond(R[j].reshape(shape), th[j]).ravel())
                    continue
                d = diag - th[j]
                d = np.where(np.abs(d) < 0.1, np.where(d < 0, -0.1, 0.1), d)
                T.append(R[j] / d)
        T = proj(np.array(T))
        if V.shape[0] + T.shape[0] > max_sub:
            nk = min(max(keep, n_roots), V.shape[0])
            V = _orth_against(np.zeros((0, V.shape[1]), complex), y_all[:, :nk].T @ V)
            AV = apply(V)
        T = _orth_against(V, T)
        if T.shape[0] == 0:
            return th, X.reshape(n_roots, *shape), rn, it
        V = np.vstack([V, T])
        AV = np.vstack([AV, apply(T)])
