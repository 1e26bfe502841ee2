"""The FIRE minimiser of the relaxation driver (bse_fire_minimize, host only): closed-form minima.

FIRE (Bitzek et al., PRL 97, 170201 (2006)) is the stepper of bse_relax; these checks run it on
functions whose minimisers are known, through the C ABI, without a GPU.
"""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def pkg():
    import paper_2607_20728_gb300 as p
    try:
        p.load_library()
    except Exception as e:       # the library is built by __graft_entry__.build()
        pytest.skip(f"library not built: {e}")
    return p


def test_anisotropic_quadratic(pkg):
    """E = 1/2 sum k_i (x_i - c_i)^2 with stiffnesses over two decades: x -> c within fmax / k_min."""
    rng = np.random.default_rng(3)
    k = np.geomspace(0.1, 10.0, 12)
    c = rng.standard_normal(12)
    fun = lambda x: (0.5 * np.sum(k * (x - c) ** 2), -k * (x - c))  # noqa: E731
    x, E, n = pkg.bse_fire_minimize(fun, np.zeros(12), fmax=1e-8, max_steps=5000)
    assert np.abs(k * (x - c)).max() <= 1e-8
    assert np.abs(x - c).max() <= 1e-8 / k.min() * 1.0001
    assert E < 1e-14


def test_double_well_chain(pkg):
    """E = sum (x_i^2 - 1)^2 + 0.1 sum x_i x_{i+1}: a stationary point with a positive-definite
    Hessian (a minimum), reached from a generic start with the energy below the start's."""
    def fun(x):
        E = np.sum((x * x - 1) ** 2) + 0.1 * np.sum(x[:-1] * x[1:])
        g = 4 * x * (x * x - 1)
        g[:-1] += 0.1 * x[1:]
        g[1:] += 0.1 * x[:-1]
        return E, -g
    x0 = np.linspace(-0.3, 0.4, 9)
    x, E, n = pkg.bse_fire_minimize(fun, x0, fmax=1e-9, max_steps=5000)
    assert np.abs(fun(x)[1]).max() <= 1e-9
    H = np.diag(12 * x * x - 4) + 0.1 * (np.eye(9, k=1) + np.eye(9, k=-1))
    assert np.linalg.eigvalsh(H).min() > 0
    assert E < fun(x0)[0]


def test_failures_are_reported(pkg):
    def bad(x):
        raise RuntimeError("no energy here")
    with pytest.raises(pkg.BSEError) as e:
        pkg.bse_fire_minimize(bad, np.zeros(3), fmax=1e-6)
    assert e.value.status == 1
    with pytest.raises(pkg.BSEError) as e:
        pkg.bse_fire_minimize(lambda x: (np.sum(x * x), -2 * x), np.ones(3), fmax=1e-12, max_steps=3)
    assert e.value.status == 4
