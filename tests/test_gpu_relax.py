"""Excited-state relaxation driver (bse_relax, bse_relax_batch) on E = E_gs + omega.

The ground-state surface is a harmonic well E_gs = 1/2 k |R - R0|^2 supplied by the caller (the
synthetic model has none of its own).  The check is independent of the driver: at the geometry it
returns, the FP64 CPU oracle's excited-state forces plus the harmonic force must vanish to within
the convergence threshold (the GPU forces agree with the oracle's to 1e-7 Ha/bohr elsewhere in
the suite), and the energy must be below the starting one.
"""
import numpy as np
import pytest

import bse_inputs as bi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K = 0.2  # Ha/bohr^2


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2607_20728_gb300 as p
    return p


def _harmonic(R0):
    def fn(pos):
        d = pos - R0
        return 0.5 * K * float(np.sum(d * d)), -K * d
    return fn


def _oracle_total_force(spec, pos):
    from oracle import forces
    r = forces.bse_forces(spec.with_positions(pos), tol=1e-12)
    return r.F - K * (pos - spec.pos), r.omega[0]


@pytest.mark.parametrize("name,hartree,inexact,precision", [("tiny", False, True, 0), ("tiny", False, False, 0),
                                                             ("tiny", True, True, 0), ("tiny", False, True, 1)])
def test_relaxed_geometry_is_stationary(pkg, name, hartree, inexact, precision):
    spec = getattr(bi, name)()
    if hartree:
        spec = bi.hartree_model(spec)
    s = pkg.BSESystem(spec, gs_tol=1e-12, precision=precision)
    try:
        w0, _ = s.davidson(n_roots=1, tol=1e-10 if precision == 0 else 1e-7)
        fmax = 2e-5 if precision == 0 else 1e-4
        pos, E, w, evals = s.relax(_harmonic(spec.pos), fmax=fmax, max_steps=400, inexact=inexact,
                                   davidson_tol=1e-10 if precision == 0 else 1e-7, zvector_tol=1e-11)
        assert E < w0[0]
        Ft, wo = _oracle_total_force(spec, pos)
        assert abs(w - wo) < (1e-9 if precision == 0 else 1e-6)
        assert np.abs(Ft).max() < fmax + (1e-7 if precision == 0 else 1e-5)
        assert np.abs(pos - spec.pos).max() > 1e-4       # the excitation moved the atoms
    finally:
        s.close()


def test_batch_relaxation(pkg):
    specs = [bi.tiny(), bi.micro(), bi.hartree_model(bi.micro())]
    b = pkg.BSEBatch(specs, n_workers=3, precision=0, gs_tol=1e-12)
    try:
        calls = []

        def gs(system, pos):
            calls.append(system)
            return _harmonic(specs[system].pos)(pos)

        out, E, w, evals, st = b.relax(gs, fmax=2e-5, max_steps=400, davidson_tol=1e-10, zvector_tol=1e-11)
        assert st == 0, [b.error(i) for i in range(len(specs))]
        assert sorted(set(calls)) == [0, 1, 2]
        for i, sp in enumerate(specs):
            Ft, wo = _oracle_total_force(sp, out[i])
            assert abs(w[i] - wo) < 1e-9
            assert np.abs(Ft).max() < 2e-5 + 1e-7
            assert evals[i] > 1
    finally:
        b.close()
