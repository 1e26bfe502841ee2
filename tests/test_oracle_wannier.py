"""Pins for the oracle's Wannier localisation and pair-pruned Liouville operator.

The localisation is checked against what fixes it: the centre formula on a function whose centre
is known, the rotation's orthogonality, the objective's increase and local maximality, and the
centres of the Hartree model's one-orbital-per-site states sitting on the wells.  The operator is
checked by covariance: without pruning L~ = U^T L U exactly, and omega and the forces equal the
canonical path's; with pruning the error vanishes as the cutoff passes the largest pair distance.
"""
import numpy as np
import pytest

import bse_inputs as bi
from oracle import forces, liouville, model, wannier
from oracle.basis import PWBasis


@pytest.fixture(scope="module")
def small_h():
    spec = bi.hartree_model(bi.small16())
    gs = model.GroundState(spec, all_states=True)
    U, c, sweeps = wannier.localize(gs)
    U, c = wannier.canonical_order(gs, U, c)
    return spec, gs, U, c


def test_centre_formula_on_a_gaussian():
    """A normalised Gaussian centred at r0 (symmetric about r0): the Gamma-point centre is r0."""
    lat = np.array([[9.0, 0, 0], [2.0, 8.0, 0], [0.5, 1.0, 10.0]])
    b = PWBasis(lat, 12.0, (32, 32, 36))
    r0 = np.array([3.1, 2.2, 4.7])
    N = np.array(b.grid)
    j = np.stack(np.meshgrid(*[np.arange(n) for n in N], indexing="ij"), axis=-1) / N
    d = j - (r0 @ np.linalg.inv(lat))
    d -= np.round(d)
    rr = np.linalg.norm(d @ lat, axis=-1)
    f = np.exp(-rr ** 2 / (2 * 0.9 ** 2))
    f /= np.sqrt(np.sum(f * f) * b.omega / b.nr)

    class G:
        pass
    g = G()
    g.basis, g.phi_r = b, f[None].astype(complex)
    c = wannier.wannier_centres(g, np.eye(1))
    df = (c[0] - r0) @ np.linalg.inv(lat)
    df -= np.round(df)
    assert np.linalg.norm(df @ lat) < 1e-8


def test_localisation(small_h):
    spec, gs, U, c = small_h
    assert np.abs(U.T @ U - np.eye(spec.n_occ)).max() < 1e-12
    mats = wannier.position_matrices(gs)
    o_loc = wannier.spread_objective(mats, U)
    assert o_loc > wannier.spread_objective(mats, np.eye(spec.n_occ)) + 1.0
    # a local maximum: small rotations of any pair lower the objective
    rng = np.random.default_rng(2)
    for _ in range(10):
        p, q = rng.choice(spec.n_occ, 2, replace=False)
        for t in (1e-3, -1e-3):
            R = np.eye(spec.n_occ)
            R[p, p] = R[q, q] = np.cos(t)
            R[p, q], R[q, p] = -np.sin(t), np.sin(t)
            assert wannier.spread_objective(mats, U @ R) <= o_loc + 1e-12
    # one localised orbital per well
    inv = np.linalg.inv(spec.lattice)
    for ci in c:
        d = (ci - spec.pos) @ inv
        d -= np.round(d)
        assert np.min(np.linalg.norm(d @ spec.lattice, axis=1)) < 0.1


def test_unpruned_operator_is_the_rotated_operator(small_h):
    spec, gs, U, c = small_h
    op = liouville.Liouville(spec, gs=gs)
    wop = wannier.WannierLiouville(op, U, c, cutoff=1e9)
    rng = np.random.default_rng(4)
    b = gs.basis
    A = op.Pc(b.real_to_full(rng.standard_normal((spec.n_occ, b.npw))))
    lhs = wop.apply(U.T @ A)
    rhs = U.T @ op.apply(A)
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(rhs).max()


def test_pruning_error_vanishes_with_the_cutoff(small_h):
    spec, gs, U, c = small_h
    ref = forces.bse_forces(spec, tol=1e-11)
    errs = []
    for cut in (3.0, 4.0, 6.0, 1e9):
        w, F, A, npairs, _, _ = wannier.pruned_forces(spec, cut, tol=1e-11)
        errs.append((npairs, abs(w[0] - ref.omega[0]), np.abs(F - ref.F).max()))
    assert errs[-1][0] == spec.n_occ * (spec.n_occ + 1) // 2
    assert errs[-1][1] < 1e-10 and errs[-1][2] < 1e-8
    assert errs[0][0] < errs[1][0] < errs[2][0] < errs[3][0]
    assert errs[0][1] > errs[2][1] and errs[0][2] > errs[2][2]
