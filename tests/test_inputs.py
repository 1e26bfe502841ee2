"""The seeded input generator: determinism and the documented input format."""
import numpy as np

import bse_inputs as bi
from oracle.basis import PWBasis


def test_deterministic():
    a, b = bi.tiny(), bi.tiny()
    assert np.array_equal(a.pos, b.pos)
    assert np.array_equal(a.pdep_coef, b.pdep_coef)


def test_pdep_orthonormal_and_no_g0():
    for spec in (bi.micro(), bi.tiny()):
        P = spec.pdep_coef
        assert np.abs(P @ P.T - np.eye(spec.n_pdep)).max() < 1e-13
        assert np.all(P[:, 0] == 0.0)
        assert np.all(spec.pdep_lambda < 0)


def test_npdep_is_twice_nocc_in_production_shapes():
    # Sec. SIV: the number of PDEPs is twice the number of occupied orbitals
    t = bi.tiny()
    assert t.n_pdep >= 2 * t.n_occ


def test_half_sphere_matches_full_sphere():
    for spec in (bi.micro(), bi.tiny()):
        b = PWBasis(spec.lattice, spec.ecut, spec.grid)
        n = bi.half_sphere_miller(spec.lattice, spec.ecut)
        assert 2 * len(n) + 1 == b.npw == spec.n_pw
        # the oracle's own ordering of the half sphere agrees with the generator's
        assert np.array_equal(b.mill[b.i_plus], n)
        assert np.array_equal(b.mill[b.i_minus], -n)


def test_configured_grids_are_alias_free():
    for spec in (bi.micro(), bi.tiny()):
        PWBasis(spec.lattice, spec.ecut, spec.grid)      # raises when too small
