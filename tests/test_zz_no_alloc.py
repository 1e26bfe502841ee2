"""The allocation-free FFT entry point (bse_fft3d_noalloc) against bse_fft3d.

Some callers cannot allocate device memory themselves (their memory belongs to another
allocator, or they cannot afford the device-wide synchronisation of cudaMalloc/cudaFree);
bse_fft3d_noalloc serves them with its twiddle tables in a fixed device array.  Two calls in
a row with different sizes check that the shared table is rewritten correctly between
calls.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_fft_matches_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2607_20728_gb300 as pkg
    lib = pkg.load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(11)
    for (n1, n2, n3), direction in (((24, 24, 24), -1), ((16, 30, 27), +1)):
        x = rng.standard_normal((2, n3, n2, n1)) + 1j * rng.standard_normal((2, n3, n2, n1))
        a = torch.tensor(x, dtype=torch.complex128, device="cuda")
        b = a.clone()
        st = lib.bse_fft3d(n1, n2, n3, 2, ctypes.c_void_p(a.data_ptr()), direction, stream)
        assert st == 0, lib.bse_last_error(None).decode()
        st = lib.bse_fft3d_noalloc(n1, n2, n3, 2, ctypes.c_void_p(b.data_ptr()), direction, stream)
        assert st == 0, lib.bse_last_error(None).decode()
        ref, got = a.cpu().numpy(), b.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max()
    # sizes beyond the table are rejected before anything runs
    st = lib.bse_fft3d_noalloc(1024, 2, 2, 1, ctypes.c_void_p(b.data_ptr()), -1, stream)
    assert st == 1
