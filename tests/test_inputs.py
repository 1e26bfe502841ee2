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


def test_midsize_parity_cells():
    """The mid-size parity cells have the shapes their docstrings promise: several 16-orbital
    blocks and pair batches of 256, ragged grid tiles, N_pdep = 2 N_occ, alias-free grids."""
    m48, m40 = bi.mid48(), bi.mid40()
    assert m48.n_occ == 48 and m48.n_occ % 16 == 0 and m48.n_occ // 16 == 3
    assert m48.n_occ * (m48.n_occ + 1) // 2 == 1176 > 4 * 256
    nr48 = int(np.prod(m48.grid))
    assert nr48 % 32 == 0 and nr48 % 128 != 0
    assert m40.n_occ % 16 != 0 and int(np.prod(m40.grid)) % 32 != 0
    for spec in (m48, m40):
        assert spec.n_pdep == 2 * spec.n_occ
        P = spec.pdep_coef
        assert np.abs(P @ P.T - np.eye(spec.n_pdep)).max() < 1e-12
        PWBasis(spec.lattice, spec.ecut, spec.grid)
    assert np.array_equal(bi.CONFIGS["mid48"]().pos, m48.pos)
    assert np.array_equal(bi.CONFIGS["mid40"]().pos, m40.pos)


def test_midsize_cells_are_gapped():
    """All occupied states bound (s- and p-like states of the 8 Ha wells): a HOMO-LUMO gap far
    above the 1e-2 Ha that keeps the excitation and its derivative well conditioned."""
    from oracle import model
    for spec in (bi.mid48(), bi.mid40()):
        gs = model.GroundState(spec)
        assert gs.gap > 0.4 and gs.eps[-1] < -0.4
