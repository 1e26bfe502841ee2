"""torch.autograd wrapper of Omega(R): backward = Z-vector adjoint + force contraction (Eq. 4-6).

Expected gradients come from the FP64 CPU oracle (its forces are pinned to Richardson finite
differences of its own Omega(R) in the CPU suite) and from finite differences of the wrapper's
own forward pass with W held fixed (h = 1e-3 bohr, central, and its Richardson extrapolation).
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
def oracle_result(spec):
    from oracle import forces
    return forces.bse_forces(spec, tol=1e-12)


@pytest.fixture(scope="module")
def fp64_sys(pkg, spec):
    s = pkg.BSESystem(spec, gs_tol=3e-13)
    yield s
    s.close()


def _omega(pkg, R, s, **kw):
    from paper_2607_20728_gb300.autograd import excitation_energy
    return excitation_energy(R, s, **kw)


def test_gradient_matches_oracle_forces(pkg, spec, fp64_sys, oracle_result):
    R = torch.tensor(spec.pos, dtype=torch.float64, requires_grad=True)
    om = _omega(pkg, R, fp64_sys, tol=1e-11, z_tol=1e-12)
    assert abs(om.item() - oracle_result.omega[0]) < 1e-9
    om.backward()
    assert np.abs(R.grad.numpy() + oracle_result.F).max() < 1e-7


def test_gradient_matches_finite_differences(pkg, spec, fp64_sys):
    R0 = torch.tensor(spec.pos, dtype=torch.float64, requires_grad=True)
    om = _omega(pkg, R0, fp64_sys, tol=1e-11, z_tol=1e-12)
    (g,) = torch.autograd.grad(om, R0)

    def omega_at(p):
        with torch.no_grad():
            return _omega(pkg, torch.tensor(p), fp64_sys, tol=1e-11).item()

    for atom, alpha in [(0, 0), (1, 2), (0, 1)]:
        fd = {}
        for h in (1e-3, 5e-4):
            vals = []
            for sgn in (+1, -1):
                p = spec.pos.copy()
                p[atom, alpha] += sgn * h
                vals.append(omega_at(p))
            fd[h] = (vals[0] - vals[1]) / (2 * h)
        rich = (4 * fd[5e-4] - fd[1e-3]) / 3
        assert abs(fd[1e-3] - g[atom, alpha].item()) < 1e-6       # O(h^2) at h = 1e-3 bohr
        assert abs(rich - g[atom, alpha].item()) < 1e-8


def test_backward_after_another_forward(pkg, spec, fp64_sys, oracle_result):
    """A later forward at another geometry must not change an earlier graph's gradient."""
    R1 = torch.tensor(spec.pos, dtype=torch.float64, requires_grad=True)
    om1 = _omega(pkg, R1, fp64_sys, tol=1e-11, z_tol=1e-12)
    p2 = spec.pos.copy()
    p2[0, 0] += 0.05
    R2 = torch.tensor(p2, dtype=torch.float64, requires_grad=True)
    om2 = _omega(pkg, R2, fp64_sys, tol=1e-11, z_tol=1e-12)
    assert abs(om2.item() - om1.item()) > 1e-6
    om1.backward()
    assert np.abs(R1.grad.numpy() + oracle_result.F).max() < 1e-7


def test_chain_rule_through_a_function_of_omega(pkg, spec, fp64_sys, oracle_result):
    """d(Omega^2 + 3 Omega)/dR = (2 Omega + 3) dOmega/dR: the incoming gradient is honoured."""
    R = torch.tensor(spec.pos, dtype=torch.float64, requires_grad=True)
    om = _omega(pkg, R, fp64_sys, tol=1e-11, z_tol=1e-12)
    (om * om + 3 * om).backward()
    w = oracle_result.omega[0]
    assert np.abs(R.grad.numpy() + (2 * w + 3) * oracle_result.F).max() < 1e-6


def test_gradcheck(pkg, spec, fp64_sys):
    R = torch.tensor(spec.pos, dtype=torch.float64, requires_grad=True)
    f = lambda r: _omega(pkg, r, fp64_sys, tol=1e-11, z_tol=1e-12)   # noqa: E731
    assert torch.autograd.gradcheck(f, (R,), eps=1e-4, atol=1e-7, rtol=1e-4)


def test_mixed_precision_gradient(pkg, spec, oracle_result):
    s = pkg.BSESystem(spec, precision=1)
    try:
        R = torch.tensor(spec.pos, dtype=torch.float64, requires_grad=True)
        om = _omega(pkg, R, s, tol=1e-7, z_tol=1e-10)
        assert abs(om.item() - oracle_result.omega[0]) < 1e-6
        om.backward()
        assert np.abs(R.grad.numpy() + oracle_result.F).max() < 1e-5
    finally:
        s.close()


def test_wrong_shape_rejected(pkg, fp64_sys):
    with pytest.raises(ValueError):
        _omega(pkg, torch.zeros(3, 3, dtype=torch.float64), fp64_sys)
