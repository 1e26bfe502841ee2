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
