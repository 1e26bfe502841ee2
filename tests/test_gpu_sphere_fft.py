"""Sphere-pruned transforms (column z pass + plane xy pass, scatter/gather and the D term fused)
against the FP64 oracle, and against the library's own full-grid FFT path.

Cases: the cubic 2-well model (24^3) and the honeycomb cell (non-orthogonal lattice, 24x24x36
grid), FP64 and mixed precision, Liouville operator (op 0) and the Z-vector operator
P_c (H - eps_v) (op 1, which runs the fused H product).  Tolerances as in the other parity
tests: FP64 rows to 1e-11 of the largest entry, FP32-grid rows to 2e-5.
"""
import numpy as np
import pytest

import bse_inputs as bi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FULL_GRID = 4   # BSE_FLAG_FULL_GRID_FFT


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2607_20728_gb300 as p
    return p


@pytest.fixture(scope="module", params=["tiny", "hexcell"])
def case(request):
    from oracle import liouville, model
    spec = bi.CONFIGS[request.param]()
    gs = model.GroundState(spec, all_states=True)
    return spec, liouville.Liouville(spec, gs=gs)


def _trials(X, spec):
    out = []
    for k in (0, 1):
        d = bi.covariant_weights(spec.lattice, spec.ecut, k)
        A = X * d[None, :]
        out.append(A - (A @ X.T) @ X)
    return np.stack(out)


def _rows(pkg, spec, op_oracle, flags, precision, op):
    s = pkg.BSESystem(spec, flags=flags, gs_tol=3e-13, precision=precision)
    try:
        g = bi.gauge_vector(spec.lattice, spec.ecut)
        _, phi = s.ground_state()
        P = phi.cpu().numpy()
        sg = np.sign(P @ g)
        got = s.apply(torch.tensor(_trials(P, spec), device="cuda"), op=op).cpu().numpy() * sg[None, :, None]
    finally:
        s.close()
    b = op_oracle.basis
    Ao = _trials(op_oracle.gs.X, spec)
    ref = []
    for a in Ao:
        full = b.real_to_full(a)
        ref.append(b.full_to_real(op_oracle.apply(full) if op == 0 else op_oracle.apply_zop(full)))
    return got, np.stack(ref)


@pytest.mark.parametrize("op", [0, 1])
@pytest.mark.parametrize("flags", [0, FULL_GRID])
def test_fp64_rows(pkg, case, flags, op):
    spec, o = case
    got, ref = _rows(pkg, spec, o, flags, 0, op)
    assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("op", [0, 1])
def test_mixed_rows(pkg, case, op):
    spec, o = case
    got, ref = _rows(pkg, spec, o, 0, 1, op)
    assert np.abs(got - ref).max() < 2e-5 * np.abs(ref).max()


def test_omega_and_forces_both_paths(pkg, case):
    from oracle import forces
    spec, _ = case
    r = forces.bse_forces(spec, tol=1e-12)
    for flags in (0, FULL_GRID):
        s = pkg.BSESystem(spec, flags=flags, gs_tol=3e-13)
        try:
            w, _ = s.davidson(1, tol=1e-11, max_iter=400)
            s.zvector(0, tol=1e-12)
            F = s.forces(0)
        finally:
            s.close()
        assert abs(w[0] - r.omega[0]) < 1e-9
        assert np.abs(F - r.F).max() < 1e-7


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("flags", [0, FULL_GRID])
def test_transform_utilities_match_numpy(pkg, case, flags, precision):
    """bse_sphere_to_grid / bse_grid_to_sphere (the apply's first and last transforms) against
    numpy's FFT of the same real-basis rows: f(r) = Omega^-1/2 sum_G c(G) e^{iG.r}, and back.
    An odd row count leaves the last packed grid half used."""
    spec, o = case
    b = o.basis
    rng = np.random.default_rng(5)
    X = rng.standard_normal((5, b.npw))
    ref = b.to_grid(b.real_to_full(X)).real                    # (5, N1, N2, N3)
    s = pkg.BSESystem(spec, flags=flags, gs_tol=1e-10, precision=precision)
    try:
        P = s.sphere_to_grid(torch.tensor(X, device="cuda"))
        got = P.cpu().numpy()
        Y = s.grid_to_sphere(P, 5).cpu().numpy()
    finally:
        s.close()
    re_ = np.stack([got[q].real if k == 0 else got[q].imag for q in range(3) for k in (0, 1)])[:5]
    tol = 1e-13 if precision == 0 else 2e-6
    assert np.abs(got[2].imag).max() < tol * np.abs(ref).max()
    assert np.abs(re_.transpose(0, 3, 2, 1) - ref).max() < tol * np.abs(ref).max()
    assert np.abs(Y - X).max() < tol * np.abs(X).max()
