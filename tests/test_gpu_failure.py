"""Failure detection on the GPU without a fault: the device-side bounded waits give up and report.

The K1d pipeline's mbarrier waits are bounded by one second of %globaltimer (and an iteration
cap); when one runs out, the kernel sets a device error flag and returns, and the host turns the
flag into BSE_ERR_TIMEOUT.  bse_selftest_bounded_wait makes such a wait run out on a barrier that
nothing completes; the test checks the status, the time it took, and that the context still
computes correctly afterwards.  bse_selftest_k1d_stall runs the whole multi-warp K1d pipeline
with a producer that issues no copies: every consumer warp's wait runs out, and the warps must
leave together (a warp left at a named barrier that another warp quit would never return).
"""
import time

import numpy as np
import pytest

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


def test_bounded_wait_gives_up_and_the_context_survives(pkg):
    lib = pkg.load_library()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = lib.bse_selftest_bounded_wait(None)
    dt = time.perf_counter() - t0
    assert st == 6, pkg.STATUS.get(st, st)            # BSE_ERR_TIMEOUT
    assert 0.5 < dt < 60.0
    # the context is intact: an FFT round trip on the device is exact
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 12, 10, 8)) + 1j * rng.standard_normal((2, 12, 10, 8))
    t = torch.tensor(x, dtype=torch.complex128, device="cuda")
    pkg.bse_fft3d(t, -1)
    pkg.bse_fft3d(t, +1)
    assert np.abs(t.cpu().numpy() / (8 * 10 * 12) - x).max() < 1e-13


def test_k1d_pipeline_stall_times_out_for_all_warps(pkg):
    import bse_inputs as bi
    spec = bi.small16()
    s = pkg.BSESystem(spec, gs_tol=1e-11, precision=1)
    try:
        assert s.stats()["k1d_tma"] == 1
        _, phi = s.ground_state()
        A = phi[None].clone() * 0.5
        A = A - (A[0] @ phi.T) @ phi
        before = s.apply(A).cpu().numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = pkg.load_library().bse_selftest_k1d_stall(s.ctx)
        dt = time.perf_counter() - t0
        assert st == 6, pkg.STATUS.get(st, st)        # BSE_ERR_TIMEOUT
        assert 0.5 < dt < 60.0
        # the context still computes the same operator, bit for bit up to rounding order
        after = s.apply(A).cpu().numpy()
        assert np.abs(after - before).max() <= 1e-12 * np.abs(before).max()
    finally:
        s.close()
