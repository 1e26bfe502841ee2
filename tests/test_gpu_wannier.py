"""GPU parity for Wannier pair pruning of K1d (BSE_FLAG_WANNIER_PRUNE), through the C ABI.

Expected values come from the FP64 CPU oracle (oracle/wannier.py: its own localisation, pair
selection and pruned Davidson, then the exact U / Z / forces on the pruned eigenvector).  Both
sides localise independently; the kept-pair count is compared, then omega and the forces.
Without pruning (a cutoff beyond every pair) the result is the canonical one.  Tolerances: FP64
|dOmega| <= 1e-9 Ha, |dF| <= 1e-7 Ha/bohr; mixed 1e-6 / 1e-5.
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


_REF = {}


def ref(name, cutoff):
    key = (name, cutoff)
    if key not in _REF:
        from oracle import wannier
        spec = bi.hartree_model(getattr(bi, name)())
        w, F, A, npairs, U, cen = wannier.pruned_forces(spec, cutoff, tol=1e-11)
        _REF[key] = (spec, w[0], F, npairs)
    return _REF[key]


@pytest.mark.parametrize("name,cutoff,precision,flags", [("small16", 1e9, 0, 0), ("small16", 6.0, 0, 0),
                                                          ("small16", 4.0, 0, 0), ("small16", 4.0, 1, 0),
                                                          ("small16", 4.0, 0, 4), ("hexcell", 2.0, 0, 0)])
def test_pruned_omega_and_forces(pkg, name, cutoff, precision, flags):
    spec, w_ref, F_ref, npairs = ref(name, cutoff)
    s = pkg.BSESystem(spec, gs_tol=1e-12, scf_tol=1e-11, precision=precision, flags=flags, pair_cutoff=cutoff)
    try:
        st = s.stats()
        assert st["wannier_pairs"] == npairs and st["wannier_sweeps"] >= 1
        w, _ = s.davidson(n_roots=1, tol=1e-11 if precision == 0 else 1e-7, max_iter=400)
        s.zvector(0, tol=1e-12 if precision == 0 else 1e-10)
        F = s.forces(0)
        lw, lf = (1e-9, 1e-7) if precision == 0 else (1e-6, 1e-5)
        assert abs(w[0] - w_ref) < lw
        assert np.abs(F - F_ref).max() < lf
    finally:
        s.close()


def test_unpruned_equals_the_canonical_path(pkg):
    from oracle import forces
    spec = bi.hartree_model(bi.small16())
    r = forces.bse_forces(spec, tol=1e-11)
    s = pkg.BSESystem(spec, gs_tol=1e-12, scf_tol=1e-11, pair_cutoff=1e9)
    try:
        w, _ = s.davidson(n_roots=1, tol=1e-11)
        s.zvector(0, tol=1e-12)
        F = s.forces(0)
        assert abs(w[0] - r.omega[0]) < 1e-9
        assert np.abs(F - r.F).max() < 1e-7
        assert s.stats()["wannier_pairs"] == spec.n_occ * (spec.n_occ + 1) // 2
    finally:
        s.close()
