"""Batches of independent systems (bse_setup_batch / bse_solve_batch): concurrent worker
streams, graph-captured Liouville applies, per-system failure isolation, and the batched
autograd form, against the FP64 oracle of each system and central finite differences."""
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
def specs():
    return [bi.tiny(), bi.small16(), bi.hexcell(), bi.micro()]


@pytest.fixture(scope="module")
def oracle(specs):
    from oracle import forces
    return [forces.bse_forces(s, tol=1e-12) for s in specs]


@pytest.mark.parametrize("precision,tol_w,tol_f", [(0, 1e-9, 1e-7), (1, 1e-6, 1e-5)])
def test_batch_matches_oracle(pkg, specs, oracle, precision, tol_w, tol_f):
    b = pkg.BSEBatch(specs, n_workers=3, precision=precision, gs_tol=3e-13)
    try:
        assert b.setup_status == 0
        w, F, st = b.solve(davidson_tol=1e-11 if precision == 0 else 1e-7, zvector_tol=1e-12)
        assert st == 0
        for i, r in enumerate(oracle):
            assert abs(w[i] - r.omega[0]) < tol_w, i
            assert np.abs(F[i] - r.F).max() < tol_f, i
            assert b.system_stats(i)["n_applies"] > 0
    finally:
        b.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-7)])
def test_graph_replay_matches_plain_launches(pkg, specs, precision, tol):
    """Graph-replayed applies give the same solution as plain launches of the same batch."""
    out = []
    for flags in (0, pkg.FLAG_NO_GRAPHS):
        b = pkg.BSEBatch(specs[:3], n_workers=2, precision=precision, gs_tol=3e-13, flags=flags)
        try:
            w, F, st = b.solve(davidson_tol=1e-11 if precision == 0 else 1e-7, zvector_tol=1e-12)
            assert st == 0
            out.append((w, F))
        finally:
            b.close()
    (w0, F0), (w1, F1) = out
    assert np.abs(w0 - w1).max() < tol
    for a, c in zip(F0, F1):
        assert np.abs(a - c).max() < 100 * tol


def test_failed_system_is_isolated(pkg, specs):
    bad = bi.tiny()
    bad.grid = (12, 12, 12)      # below the alias-free minimum: BSE_ERR_INVALID at setup
    b = pkg.BSEBatch([specs[0], bad, specs[3]], n_workers=2, precision=0, gs_tol=3e-13)
    try:
        assert b.setup_status == 1 and b.status(1) == 1 and b.status(0) == 0 and b.status(2) == 0
        w, F, st = b.solve(davidson_tol=1e-10, zvector_tol=1e-11)
        assert np.isnan(w[1]) and np.all(np.isnan(F[1]))
        assert np.isfinite(w[0]) and np.isfinite(w[2])
    finally:
        b.close()


def test_batched_autograd_matches_finite_differences(pkg, specs):
    from paper_2607_20728_gb300.autograd import batch_excitation_energies
    sub = [specs[3], specs[0]]
    b = pkg.BSEBatch(sub, n_workers=2, precision=0, gs_tol=3e-13)
    try:
        Rs = [torch.tensor(s.pos, dtype=torch.float64, requires_grad=True) for s in sub]
        w = batch_excitation_energies(Rs, b, davidson_tol=1e-11, zvector_tol=1e-12)
        (w.sum() + 2.0 * w[1]).backward()
        h = 1e-3
        for k, (atom, alpha) in enumerate([(0, 0), (1, 2)]):
            for i in range(2):
                vals = []
                for sgn in (+1, -1):
                    P = [s.pos.copy() for s in sub]
                    P[i][atom, alpha] += sgn * h
                    with torch.no_grad():
                        wp = batch_excitation_energies([torch.tensor(p) for p in P], b, davidson_tol=1e-11,
                                                       zvector_tol=1e-12)
                    vals.append(float(wp[i]) * (3.0 if i == 1 else 1.0))
                fd = (vals[0] - vals[1]) / (2 * h)
                assert abs(fd - Rs[i].grad[atom, alpha].item()) < 2e-6
    finally:
        b.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-6)])
def test_autotuned_context_matches_oracle(pkg, specs, oracle, precision, tol):
    """BSE_FLAG_AUTOTUNE times the candidate launch shapes on the first apply; whatever it picks,
    the solution is the oracle's."""
    s = pkg.BSESystem(specs[1], gs_tol=3e-13, precision=precision, flags=pkg.FLAG_AUTOTUNE)
    try:
        w, _ = s.davidson(1, tol=1e-11 if precision == 0 else 1e-7, max_iter=400)
        st = s.stats()
        assert st["tuned"] == 1
        assert st["tuned_full_grid_fft"] in (0, 1)
        assert st["tuned_xy_threads"] in (0, 256)
        assert st["tuned_gemm_split_pct"] in (50, 100, 200)
        if precision == 1:
            assert 1 <= st["tuned_k1d_nb"] <= 4
        assert abs(w[0] - oracle[1].omega[0]) < tol
    finally:
        s.close()


def test_batch_systems_are_tuned(pkg, specs):
    b = pkg.BSEBatch(specs[:2], n_workers=2, precision=1, gs_tol=1e-10)
    try:
        b.solve(davidson_tol=1e-5)
        assert all(b.system_stats(i)["tuned"] == 1 for i in range(2))
    finally:
        b.close()


@pytest.mark.parametrize("precision,tol_w,tol_f", [(0, 1e-10, 1e-8), (1, 1e-7, 2e-6)])
def test_warm_start_reaches_the_cold_solution(pkg, specs, precision, tol_w, tol_f):
    """BSE_FLAG_WARM_START seeds the next geometry's solves with the previous states and roots;
    the converged results are the cold ones, in fewer ground-state iterations."""
    spec = specs[1]
    p2 = spec.pos.copy()
    p2[2, 1] += 0.01
    warm = pkg.BSESystem(spec, gs_tol=3e-13, precision=precision, flags=pkg.FLAG_WARM_START)
    cold = pkg.BSESystem(spec.with_positions(p2), gs_tol=3e-13, precision=precision)
    try:
        dtol = 1e-11 if precision == 0 else 1e-7
        warm.davidson(1, tol=dtol, max_iter=400)
        warm.set_positions(p2)
        gs_warm = warm.stats()["gs_iterations"]
        ww, _ = warm.davidson(1, tol=dtol, max_iter=400)
        warm.zvector(0, tol=1e-12)
        Fw = warm.forces(0)
        wc, _ = cold.davidson(1, tol=dtol, max_iter=400)
        cold.zvector(0, tol=1e-12)
        Fc = cold.forces(0)
        assert abs(ww[0] - wc[0]) < tol_w
        assert np.abs(Fw - Fc).max() < tol_f
        assert gs_warm < cold.stats()["gs_iterations"]
    finally:
        warm.close()
        cold.close()


@pytest.fixture(scope="module")
def batch48_smallest():
    """The four cheapest systems of the 48-system workload (grid points x N_occ^2): 36^3 and 64^3
    grids, N_occ 18-36, N_pdep 64-72, with their oracle force pipelines."""
    from oracle import forces
    specs = bi.batch48()
    order = sorted(range(len(specs)), key=lambda i: np.prod(specs[i].grid) * specs[i].n_occ ** 2)[:4]
    sub = [specs[i] for i in order]
    return sub, [forces.bse_forces(s, tol=1e-10) for s in sub]


@pytest.mark.parametrize("precision,tol_w,tol_f", [(0, 1e-9, 1e-7), (1, 1e-6, 1e-5)])
def test_config5_systems_match_oracle(pkg, batch48_smallest, precision, tol_w, tol_f):
    """Systems of the 48-system workload itself (uneven grids and N_occ, N_occ not a multiple of
    16, 36^3 and 64^3 grids) solved as one batch against the oracle, FP64 and mixed."""
    sub, ref = batch48_smallest
    b = pkg.BSEBatch(sub, n_workers=4, precision=precision, gs_tol=3e-13 if precision == 0 else 1e-10)
    try:
        assert b.setup_status == 0
        w, F, st = b.solve(davidson_tol=1e-10 if precision == 0 else 1e-6, zvector_tol=1e-11)
        assert st == 0
        for i, r in enumerate(ref):
            assert abs(w[i] - r.omega[0]) < tol_w, (sub[i].name, w[i], r.omega[0])
            assert np.abs(F[i] - r.F).max() < tol_f, sub[i].name
    finally:
        b.close()
