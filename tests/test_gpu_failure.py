"""Failure detection on the GPU without a fault: the device-side bounded waits give up and report.

The K1d pipeline's mbarrier waits are bounded by one second of %globaltimer (and an iteration
cap); when one runs out, the kernel sets a device error flag and returns, and the host turns the
flag into BSE_ERR_TIMEOUT.  bse_selftest_bounded_wait makes such a wait run out on a barrier that
nothing completes; the test checks the status, the time it took, and that the context still
computes correctly afterwards.
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
