"""Mixed-precision path (FP32 grids, FFTs, tau and products; FP64 subspace, residuals,
Z-vector refinement and force reduction) against the FP64 oracle on the 2-well model.

Bounds: |dOmega| <= 1e-6 Ha and |dF| <= 1e-5 Ha/bohr, the stated targets of the mixed form.
Operator rows: FP32 grids carry ~1e-7 relative error per product, so rows are compared to
2e-5 of the largest entry.
"""
import numpy as np
import pytest

import bse_inputs as bi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2607_20728_gb300 as p
    return p


@pytest.fixture(scope="module")
def spec():
    return bi.tiny()


@pytest.fixture(scope="module")
def mixed(pkg, spec):
    s = pkg.BSESystem(spec, gs_tol=3e-13, precision=1)
    yield s
    s.close()


@pytest.fixture(scope="module")
def oracle(spec):
    from oracle import forces
    return forces.bse_forces(spec, tol=1e-12)


def test_mixed_apply_rows(mixed, oracle, spec):
    b = oracle.op.basis
    g = bi.gauge_vector(spec.lattice, spec.ecut)
    _, phi = mixed.ground_state()
    P = phi.cpu().numpy()
    sg = np.sign(P @ g)
    d = bi.covariant_weights(spec.lattice, spec.ecut, 0)
    A = P * d[None, :]
    A = A - (A @ P.T) @ P
    LA = mixed.apply(torch.tensor(A[None], device="cuda")).cpu().numpy()[0] * sg[:, None]
    Xo = oracle.op.gs.X
    Ao = Xo * d[None, :]
    Ao = Ao - (Ao @ Xo.T) @ Xo
    LAo = b.full_to_real(oracle.op.apply(b.real_to_full(Ao)))
    assert np.abs(LA - LAo).max() < 2e-5 * np.abs(LAo).max()


def test_mixed_omega_and_forces(mixed, oracle):
    w, _ = mixed.davidson(n_roots=1, tol=2e-6, max_iter=400)
    assert abs(w[0] - oracle.omega[0]) < 1e-6
    mixed.zvector(0, tol=1e-9)
    F = mixed.forces(0)
    assert np.abs(F - oracle.F).max() < 1e-5


@pytest.fixture(scope="module")
def small_spec():
    return bi.small16()


@pytest.fixture(scope="module")
def small_oracle(small_spec):
    from oracle import liouville, model
    gs = model.GroundState(small_spec)
    return liouville.Liouville(small_spec, gs=gs)


@pytest.mark.parametrize("precision", [0, 1])
def test_blocked_k1d_rows_small16(pkg, small_spec, small_oracle, precision):
    """16-orbital blocks: FP64 combine kernel and the TMA-fed FP32 kernel, 1..5 trial vectors
    (every per-launch vector count), against the oracle's rows."""
    spec = small_spec
    s = pkg.BSESystem(spec, gs_tol=1e-12, precision=precision)
    assert s.stats()["k1d_tma"] == (1 if precision == 1 else 0)
    b = small_oracle.basis
    g = bi.gauge_vector(spec.lattice, spec.ecut)
    _, phi = s.ground_state()
    P = phi.cpu().numpy()
    sg = np.sign(P @ g)
    Xo = small_oracle.gs.X
    kinds = [0, 1, 2, 0, 1]
    trials_g, trials_o = [], []
    for i, kd in enumerate(kinds):
        d = bi.covariant_weights(spec.lattice, spec.ecut, kd) * (1.0 + 0.1 * i)
        A = P * d[None, :]
        trials_g.append(A - (A @ P.T) @ P)
        Ao = Xo * d[None, :]
        trials_o.append(Ao - (Ao @ Xo.T) @ Xo)
    tol = 1e-10 if precision == 0 else 2e-5
    for nb in (1, 2, 3, 4, 5):
        LA = s.apply(torch.tensor(np.stack(trials_g[:nb]), device="cuda")).cpu().numpy()
        for i in range(nb):
            LAo = b.full_to_real(small_oracle.apply(b.real_to_full(trials_o[i])))
            got = LA[i] * sg[:, None]
            assert np.abs(got - LAo).max() < tol * np.abs(LAo).max(), (nb, i)
    s.close()
