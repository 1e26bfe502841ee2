"""The Z-vector conjugate gradients as one captured CUDA graph (a WHILE conditional node whose body
is one iteration, with the step lengths, residuals and stop decision on the device) against the
same solve looping on the host (BSE_FLAG_NO_GRAPHS), and against the oracle's forces.

The first Z-vector solve of a context loops on the host (it sizes every buffer the loop touches);
later solves replay the captured loop.  Cases: the non-SCF operator (one CG per orbital) and the
Hartree-SCF operator (one coupled CG), FP64 and the mixed path's FP32 inner solves.  The two loops
do the same arithmetic; the coupled step lengths sum over orbitals in a different order, so the
results agree to rounding: 1e-10 Ha/bohr (FP64) and 1e-8 (mixed, FP32 inner solves).
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


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("model", ["small16", "hartree-tiny"])
def test_captured_zvector_loop_matches_host_loop(pkg, model, precision):
    spec = bi.small16() if model == "small16" else bi.hartree_model(bi.tiny())
    out = {}
    for flags in (0, pkg.FLAG_NO_GRAPHS):
        s = pkg.BSESystem(spec, gs_tol=3e-13 if precision == 0 else 1e-10, precision=precision, flags=flags)
        try:
            s.davidson(1, tol=1e-10 if precision == 0 else 1e-7, max_iter=400)
            s.zvector(0, tol=1e-11)
            if precision == 0:
                # the first solve loops on the host (the mixed path's later inner solves of the
                # same call already replay the loop its first inner solve sized)
                assert s.stats()["zvector_graphed"] == 0
            s.zvector(0, tol=1e-11)
            st = s.stats()
            assert st["zvector_graphed"] == (1 if flags == 0 else 0)
            out[flags] = (s.forces(0), st["zvector_iterations"], st["zvector_residual"])
        finally:
            s.close()
    F_graph, it_graph, res_graph = out[0]
    F_host, it_host, res_host = out[pkg.FLAG_NO_GRAPHS]
    assert res_graph <= 1e-11 and res_host <= 1e-11
    assert abs(it_graph - it_host) <= 1
    tol = 1e-10 if precision == 0 else 1e-8
    assert np.abs(F_graph - F_host).max() < tol


def test_captured_zvector_loop_matches_oracle(pkg):
    from oracle import forces
    spec = bi.tiny()
    ref = forces.bse_forces(spec, tol=1e-12)
    s = pkg.BSESystem(spec, gs_tol=3e-13)
    try:
        s.davidson(1, tol=1e-11, max_iter=400)
        s.zvector(0, tol=1e-12)
        s.set_positions(spec.pos)                  # a new geometry: buffers keep their addresses
        w, _ = s.davidson(1, tol=1e-11, max_iter=400)
        s.zvector(0, tol=1e-12)
        assert s.stats()["zvector_graphed"] == 1
        F = s.forces(0)
    finally:
        s.close()
    assert abs(w[0] - ref.omega[0]) < 1e-9
    assert np.abs(F - ref.F).max() < 1e-7
