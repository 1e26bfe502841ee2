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


def test_hartree_model_variant():
    """hartree_model: one doubly occupied orbital and an ionic charge 2 per site (a neutral cell),
    everything else of the workload unchanged."""
    for base in (bi.tiny(), bi.hexcell(), bi.small16()):
        h = bi.hartree_model(base)
        assert h.hartree and not base.hartree and base.q_ion is None
        assert h.n_occ == base.n_atoms
        assert np.array_equal(h.q_ion, np.full(base.n_atoms, 2.0))
        assert abs(h.q_ion.sum() - 2 * h.n_occ) == 0.0
        for f in ("lattice", "pos", "Z", "sigma", "pdep_coef", "pdep_lambda"):
            assert np.array_equal(getattr(h, f), getattr(base, f))
        assert h.grid == base.grid and h.ecut == base.ecut and h.seed == base.seed
        # positions can be replaced without losing the model
        h2 = h.with_positions(h.pos + 0.01)
        assert h2.hartree and np.array_equal(h2.q_ion, h.q_ion)
