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
    cases = (((24, 24, 24), -1), ((16, 30, 27), +1))
    tensors = []
    for (n1, n2, n3), direction in cases:
        x = rng.standard_normal((2, n3, n2, n1)) + 1j * rng.standard_normal((2, n3, n2, n1))
        a = torch.tensor(x, dtype=torch.complex128, device="cuda")
        tensors.append((a, a.clone(), a.clone()))
    # warm-up calls: the first call on a device may load the library's device code (lazy module
    # loading takes device memory once) and looks up the table's address
    for ((n1, n2, n3), direction), (_, _, w) in zip(cases, tensors):
        assert lib.bse_fft3d_noalloc(n1, n2, n3, 2, ctypes.c_void_p(w.data_ptr()), direction, stream) == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    got = []
    for ((n1, n2, n3), direction), (_, b, _) in zip(cases, tensors):
        st = lib.bse_fft3d_noalloc(n1, n2, n3, 2, ctypes.c_void_p(b.data_ptr()), direction, stream)
        assert st == 0, lib.bse_last_error(None).decode()
    torch.cuda.synchronize()
    # the property the entry point exists for: two calls in a row take no device memory
    assert torch.cuda.mem_get_info()[0] == free0
    for ((n1, n2, n3), direction), (a, b, _) in zip(cases, tensors):
        st = lib.bse_fft3d(n1, n2, n3, 2, ctypes.c_void_p(a.data_ptr()), direction, stream)
        assert st == 0, lib.bse_last_error(None).decode()
        ref, out = a.cpu().numpy(), b.cpu().numpy()
        assert np.abs(out - ref).max() <= 1e-14 * np.abs(ref).max()
    # sizes beyond the table are rejected before anything runs
    b = tensors[0][1]
    st = lib.bse_fft3d_noalloc(1024, 2, 2, 1, ctypes.c_void_p(b.data_ptr()), -1, stream)
    assert st == 1
