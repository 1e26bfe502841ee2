"""Thin Python binding of the GB300 plane-wave TDA-BSE force library (C ABI in include/bse_gb300.h).

Argument marshalling only: every step of the computation runs in the CUDA library.
The functions carry the C names (``bse_setup``, ``bse_apply_liouville``,
``bse_davidson``, ``bse_zvector``, ``bse_forces``); ``BSESystem`` wraps a context.
PyTorch provides device memory and the stream.  There is no CPU fallback: if the
library has not been built, importing the binding raises.
"""
import ctypes
import os

import numpy as np

from ._build import LIB, build  # noqa: F401

BSE_OK = 0
STATUS = {0: "BSE_OK", 1: "BSE_ERR_INVALID", 2: "BSE_ERR_OOM", 3: "BSE_ERR_CUDA",
          4: "BSE_ERR_NOT_CONVERGED", 5: "BSE_ERR_DEGENERATE", 6: "BSE_ERR_TIMEOUT",
          7: "BSE_ERR_STATE"}
FLAG_NO_K1E = 1
FLAG_NO_K1D = 2
FLAG_FULL_GRID_FFT = 4
FLAG_NO_GRAPHS = 8
FLAG_AUTOTUNE = 16
FLAG_WARM_START = 32
FLAG_HARTREE_SCF = 64
FLAG_WANNIER_PRUNE = 128
KERNEL_K1D = 0
KERNEL_FFT = 1
KERNEL_SPHERE_FFT = 2

_dp = ctypes.POINTER(ctypes.c_double)
# bse_grad_fn and bse_gs_energy_fn (include/bse_gb300.h)
_GRAD_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, ctypes.c_void_p)
_GS_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, ctypes.c_void_p)


class BSEError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class SystemDesc(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_double * 9), ("grid", ctypes.c_int * 3), ("ecut", ctypes.c_double),
                ("n_atoms", ctypes.c_int), ("pos", _dp), ("Z", _dp), ("sigma", _dp),
                ("n_occ", ctypes.c_int), ("n_pdep", ctypes.c_int), ("pdep_coef", _dp),
                ("pdep_lambda", _dp), ("pdep_on_device", ctypes.c_int), ("scissor", ctypes.c_double),
                ("spin", ctypes.c_int), ("precision", ctypes.c_int), ("flags", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("gs_tol", ctypes.c_double), ("q_ion", _dp),
                ("scf_tol", ctypes.c_double), ("pair_cutoff", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("gs_iterations", ctypes.c_int), ("davidson_iterations", ctypes.c_int),
                ("zvector_iterations", ctypes.c_int), ("n_applies", ctypes.c_int),
                ("gs_residual", ctypes.c_double), ("davidson_residual", ctypes.c_double),
                ("zvector_residual", ctypes.c_double), ("homo_lumo_gap", ctypes.c_double),
                ("ms_setup", ctypes.c_double), ("ms_ground_state", ctypes.c_double),
                ("ms_tau", ctypes.c_double), ("ms_davidson", ctypes.c_double),
                ("ms_uvec", ctypes.c_double), ("ms_zvector", ctypes.c_double),
                ("ms_forces", ctypes.c_double), ("bytes_tau", ctypes.c_double), ("k1d_tma", ctypes.c_int),
                ("ms_host_eig", ctypes.c_double), ("gs_chunks", ctypes.c_int), ("tuned", ctypes.c_int),
                ("tuned_full_grid_fft", ctypes.c_int), ("tuned_k1d_nb", ctypes.c_int),
                ("scf_iterations", ctypes.c_int), ("scf_residual", ctypes.c_double),
                ("wannier_pairs", ctypes.c_int), ("wannier_sweeps", ctypes.c_int),
                ("tuned_xy_threads", ctypes.c_int), ("tuned_gemm_split_pct", ctypes.c_int),
                ("zvector_graphed", ctypes.c_int)]


class RelaxOpts(ctypes.Structure):
    _fields_ = [("fmax", ctypes.c_double), ("max_steps", ctypes.c_int), ("dt", ctypes.c_double),
                ("dt_max", ctypes.c_double), ("max_move", ctypes.c_double), ("root", ctypes.c_int),
                ("davidson_tol", ctypes.c_double), ("zvector_tol", ctypes.c_double), ("inexact", ctypes.c_int)]


def _relax_opts(fmax, max_steps, root, inexact, davidson_tol, zvector_tol, dt, dt_max, max_move):
    return RelaxOpts(float(fmax), int(max_steps), float(dt), float(dt_max), float(max_move), int(root),
                     float(davidson_tol), float(zvector_tol), 1 if inexact else 0)


def _gs_callback(fn):
    """Wrap fn(system, pos[n_atoms, 3]) -> (E, F[n_atoms, 3]) as a bse_gs_energy_fn."""
    def cb(system, n_atoms, pos, energy, F, user):
        try:
            P = np.ctypeslib.as_array(pos, shape=(n_atoms * 3,)).reshape(n_atoms, 3).copy()
            E, Fg = fn(system, P)
            energy[0] = float(E)
            np.ctypeslib.as_array(F, shape=(n_atoms * 3,))[:] = np.asarray(Fg, dtype=np.float64).ravel()
            return 0
        except Exception:
            return 1
    return _GS_FN(cb)


_lib = None


def load_library():
    """Load the in-tree shared library; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise RuntimeError(f"CUDA library not built ({LIB}); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB)
    vp = ctypes.c_void_p
    sigs = {
        "bse_setup": (ctypes.c_int, [ctypes.POINTER(SystemDesc), ctypes.POINTER(vp)]),
        "bse_set_positions": (ctypes.c_int, [vp, _dp]),
        "bse_get_dims": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int)]),
        "bse_get_ground_state": (ctypes.c_int, [vp, _dp, vp]),
        "bse_get_empty_states": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _dp, vp]),
        "bse_apply_liouville": (ctypes.c_int, [vp, ctypes.c_int, vp, vp, ctypes.c_int]),
        "bse_davidson": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, vp]),
        "bse_zvector": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, vp, vp]),
        "bse_davidson_full": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, vp, vp]),
        "bse_fire_minimize": (ctypes.c_int, [ctypes.c_int, _dp, _GRAD_FN, vp, ctypes.c_double, ctypes.c_int,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.POINTER(ctypes.c_int), _dp]),
        "bse_relax": (ctypes.c_int, [vp, ctypes.POINTER(RelaxOpts), _GS_FN, vp, _dp, _dp, _dp,
                                     ctypes.POINTER(ctypes.c_int)]),
        "bse_relax_batch": (ctypes.c_int, [vp, ctypes.POINTER(RelaxOpts), _GS_FN, vp, _dp, _dp, _dp,
                                           ctypes.POINTER(ctypes.c_int)]),
        "bse_forces": (ctypes.c_int, [vp, ctypes.c_int, _dp]),
        "bse_get_density": (ctypes.c_int, [vp, ctypes.c_int, _dp]),
        "bse_get_stats": (ctypes.c_int, [vp, ctypes.POINTER(Stats)]),
        "bse_fft3d": (ctypes.c_int, [ctypes.c_int] * 4 + [vp, ctypes.c_int, vp]),
        "bse_fft3d_noalloc": (ctypes.c_int, [ctypes.c_int] * 4 + [vp, ctypes.c_int, vp]),
        "bse_host_sym_eig": (ctypes.c_int, [ctypes.c_int, _dp, _dp, _dp]),
        "bse_selftest_bounded_wait": (ctypes.c_int, [vp]),
        "bse_selftest_k1d_stall": (ctypes.c_int, [vp]),
        "bse_sphere_to_grid": (ctypes.c_int, [vp, ctypes.c_int, vp, vp]),
        "bse_batch_timing": (ctypes.c_int, [vp, _dp, _dp]),
        "bse_grid_to_sphere": (ctypes.c_int, [vp, ctypes.c_int, vp, vp]),
        "bse_host_sym_eig_lowest": (ctypes.c_int, [ctypes.c_int, _dp, ctypes.c_int, _dp, _dp]),
        "bse_host_sym_eig_k": (ctypes.c_int, [ctypes.c_int, _dp, ctypes.c_int, _dp, _dp]),
        "bse_gemm": (ctypes.c_int, [ctypes.c_char, ctypes.c_char] + [ctypes.c_int] * 3 +
                     [ctypes.c_double, vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_double, vp, ctypes.c_int, vp]),
        "bse_profile": (ctypes.c_int, [vp, ctypes.c_int]),
        "bse_gemm_bf16x3": (ctypes.c_int, [ctypes.c_int] * 3 + [ctypes.c_float, vp, ctypes.c_int, vp, ctypes.c_int,
                                                                 ctypes.c_float, vp, ctypes.c_int, vp]),
        "bse_get_kernel_timing": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong), _dp, _dp, _dp]),
        "bse_launch_count": (ctypes.c_longlong, []),
        "bse_last_error": (ctypes.c_char_p, [vp]),
        "bse_destroy": (None, [vp]),
        "bse_setup_batch": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(SystemDesc), ctypes.c_int,
                                           ctypes.POINTER(vp)]),
        "bse_solve_batch": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp, _dp]),
        "bse_batch_set_positions": (ctypes.c_int, [vp, _dp]),
        "bse_batch_size": (ctypes.c_int, [vp]),
        "bse_batch_status": (ctypes.c_int, [vp, ctypes.c_int]),
        "bse_batch_system": (vp, [vp, ctypes.c_int]),
        "bse_destroy_batch": (None, [vp]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status, ctx=None):
    if status != BSE_OK:
        msg = load_library().bse_last_error(ctx).decode()
        raise BSEError(status, msg)


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _dev_ptr(t):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _grid_ptr(t, precision, nq, grid):
    """Pointer to packed complex grids of the context's precision, shape checked."""
    import torch
    dt = torch.complex128 if precision == 0 else torch.complex64
    n1, n2, n3 = grid
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.is_contiguous()
            and t.numel() >= nq * n1 * n2 * n3):
        raise TypeError(f"expected a contiguous {dt} CUDA tensor of at least {nq} grids")
    return ctypes.c_void_p(t.data_ptr())


# ---- functions with the C names ------------------------------------------------------
def bse_setup(lattice, grid, ecut, pos, Z, sigma, n_occ, pdep_coef, pdep_lambda, scissor=0.0, spin=0,
              flags=0, precision=0, stream=None, gs_tol=0.0, q_ion=None, scf_tol=0.0, pair_cutoff=0.0):
    """Returns an opaque context handle (ctypes.c_void_p); see include/bse_gb300.h."""
    lib = load_library()
    keep = []
    d = _make_desc(keep, lattice, grid, ecut, pos, Z, sigma, n_occ, pdep_coef, pdep_lambda, scissor, spin,
                   flags, precision, stream, gs_tol, q_ion, scf_tol, pair_cutoff)
    h = ctypes.c_void_p()
    st = lib.bse_setup(ctypes.byref(d), ctypes.byref(h))
    if st != BSE_OK:
        msg = lib.bse_last_error(h if h.value else None).decode()
        if h.value:
            lib.bse_destroy(h)
        raise BSEError(st, msg)
    return h


def _make_desc(keep, lattice, grid, ecut, pos, Z, sigma, n_occ, pdep_coef, pdep_lambda, scissor=0.0, spin=0,
               flags=0, precision=0, stream=None, gs_tol=0.0, q_ion=None, scf_tol=0.0, pair_cutoff=0.0):
    """Fill a SystemDesc; arrays it points to are appended to `keep` (the caller holds them)."""

    def arr(x):
        a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
        keep.append(a)
        return a

    d = SystemDesc()
    lat = arr(lattice).ravel()
    for i in range(9):
        d.lattice[i] = lat[i]
    for i in range(3):
        d.grid[i] = int(grid[i])
    d.ecut = float(ecut)
    p = arr(pos)
    d.n_atoms = p.shape[0]
    d.pos, d.Z, d.sigma = _ptr(p), _ptr(arr(Z)), _ptr(arr(sigma))
    d.n_occ = int(n_occ)
    d.pdep_on_device = 0
    coef = pdep_coef
    try:
        import torch
        if isinstance(coef, torch.Tensor) and coef.is_cuda:
            d.pdep_on_device = 1
            d.n_pdep = int(coef.shape[0])
            d.pdep_coef = ctypes.cast(ctypes.c_void_p(coef.data_ptr()), _dp)
            keep.append(coef)
    except ImportError:
        pass
    if not d.pdep_on_device:
        c = arr(coef) if coef is not None and np.size(coef) else np.zeros((0, 1))
        d.n_pdep = int(c.shape[0])
        d.pdep_coef = _ptr(c) if d.n_pdep else None
    lam = arr(pdep_lambda if pdep_lambda is not None else np.zeros(0))
    d.pdep_lambda = _ptr(lam) if lam.size else None
    d.scissor, d.spin, d.precision, d.flags = float(scissor), int(spin), int(precision), int(flags)
    d.stream = stream
    d.gs_tol = float(gs_tol)
    d.q_ion = _ptr(arr(q_ion)) if q_ion is not None else None
    d.scf_tol = float(scf_tol)
    d.pair_cutoff = float(pair_cutoff)
    return d


def _spec_model(spec, flags):
    """Flags and ionic charges of a spec's ground-state model (Hartree-SCF or not)."""
    if getattr(spec, "hartree", False):
        flags |= FLAG_HARTREE_SCF
    return flags, getattr(spec, "q_ion", None)


def bse_apply_liouville(ctx, A, LA, op=0):
    n_vec = A.shape[0]
    _check(load_library().bse_apply_liouville(ctx, n_vec, _dev_ptr(A), _dev_ptr(LA), int(op)), ctx)


def bse_davidson(ctx, n_roots, tol, max_iter, A_out=None):
    w = np.zeros(n_roots)
    _check(load_library().bse_davidson(ctx, n_roots, float(tol), int(max_iter), _ptr(w),
                                       _dev_ptr(A_out) if A_out is not None else None), ctx)
    return w


def bse_zvector(ctx, root, tol, max_iter, Z_out=None, U_out=None):
    _check(load_library().bse_zvector(ctx, int(root), float(tol), int(max_iter),
                                      _dev_ptr(Z_out) if Z_out is not None else None,
                                      _dev_ptr(U_out) if U_out is not None else None), ctx)


def bse_forces(ctx, root, n_atoms):
    F = np.zeros((n_atoms, 3))
    _check(load_library().bse_forces(ctx, int(root), _ptr(F)), ctx)
    return F


def bse_fft3d(data, direction):
    """In-place batched 3D FFT of a complex128 CUDA tensor shaped (batch, n3, n2, n1)."""
    import torch
    if not (data.is_cuda and data.dtype == torch.complex128 and data.is_contiguous() and data.dim() == 4):
        raise TypeError("expected a contiguous complex128 CUDA tensor (batch, n3, n2, n1)")
    b, n3, n2, n1 = data.shape
    stream = ctypes.c_void_p(torch.cuda.current_stream(data.device).cuda_stream)
    _check(load_library().bse_fft3d(n1, n2, n3, b, ctypes.c_void_p(data.data_ptr()), int(direction), stream))


def bse_gemm(ta, tb, alpha, A, B, beta, C):
    """C = alpha op(A) op(B) + beta C for contiguous float64 CUDA matrices (row-major)."""
    import torch
    M, N = C.shape
    K = A.shape[0] if ta == "T" else A.shape[1]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _check(load_library().bse_gemm(ta.encode(), tb.encode(), M, N, K, float(alpha), _dev_ptr(A), A.shape[1],
                                   _dev_ptr(B), B.shape[1], float(beta), _dev_ptr(C), C.shape[1], stream))


def bse_gemm_bf16x3(alpha, A, B, beta, C):
    """C = alpha A B^T + beta C on the tensor cores (split-BF16); contiguous float32 CUDA matrices."""
    import torch
    for t in (A, B, C):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise TypeError("expected contiguous float32 CUDA tensors")
    M, N = C.shape
    K = A.shape[1]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _check(load_library().bse_gemm_bf16x3(M, N, K, float(alpha), ctypes.c_void_p(A.data_ptr()), A.shape[1],
                                          ctypes.c_void_p(B.data_ptr()), B.shape[1], float(beta),
                                          ctypes.c_void_p(C.data_ptr()), C.shape[1], stream))


def bse_launch_count():
    return int(load_library().bse_launch_count())


def host_sym_eig_lowest(A, k):
    """All eigenvalues of the symmetric A and the k lowest eigenvectors (columns 0..k-1)."""
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float64))
    n = A.shape[0]
    w = np.zeros(n)
    V = np.zeros((n, n))
    _check(load_library().bse_host_sym_eig_lowest(n, _ptr(A), int(k), _ptr(w), _ptr(V)))
    return w, V[:, :k]


def host_sym_eig_k(A, k):
    """The k lowest eigenvalues of the symmetric A and their eigenvectors (columns 0..k-1)."""
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float64))
    n = A.shape[0]
    w = np.zeros(n)
    V = np.zeros((n, n))
    _check(load_library().bse_host_sym_eig_k(n, _ptr(A), int(k), _ptr(w), _ptr(V)))
    return w[:k], V[:, :k]


def host_sym_eig(A):
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float64))
    n = A.shape[0]
    w = np.zeros(n)
    V = np.zeros((n, n))
    _check(load_library().bse_host_sym_eig(n, _ptr(A), _ptr(w), _ptr(V)))
    return w, V


def bse_fire_minimize(fun, x0, fmax, max_steps=1000, dt=0.1, dt_max=0.5, max_move=0.1):
    """FIRE minimisation of fun(x) -> (E, F = -dE/dx) on the host (no GPU): returns (x, E, evaluations)."""
    x = np.ascontiguousarray(np.asarray(x0, dtype=np.float64).copy())
    n = x.size

    def cb(nn, xp, ep, fp, user):
        try:
            E, F = fun(np.ctypeslib.as_array(xp, shape=(nn,)).copy())
            ep[0] = float(E)
            np.ctypeslib.as_array(fp, shape=(nn,))[:] = np.asarray(F, dtype=np.float64).ravel()
            return 0
        except Exception:
            return 1

    c_cb = _GRAD_FN(cb)
    steps = ctypes.c_int()
    E = ctypes.c_double()
    _check(load_library().bse_fire_minimize(n, _ptr(x), c_cb, None, float(fmax), int(max_steps), float(dt),
                                            float(dt_max), float(max_move), ctypes.byref(steps), ctypes.byref(E)))
    return x, E.value, steps.value


# ---- convenience wrapper -----------------------------------------------------------------
class BSESystem:
    """One system on the current CUDA device; accepts any object with the fields of
    ``bse_inputs.SystemSpec``."""

    def __init__(self, spec, flags=0, scissor=None, spin=None, n_pdep=None, stream=None, gs_tol=0.0, precision=0,
                 scf_tol=0.0, pair_cutoff=None):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device())
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        coef, lam = spec.pdep_coef, spec.pdep_lambda
        if n_pdep is not None:
            coef, lam = coef[:n_pdep], lam[:n_pdep]
        flags, q_ion = _spec_model(spec, flags)
        if pair_cutoff is not None:
            flags |= FLAG_WANNIER_PRUNE
        self.ctx = bse_setup(spec.lattice, spec.grid, spec.ecut, spec.pos, spec.Z, spec.sigma, spec.n_occ,
                             coef, lam, scissor=spec.scissor if scissor is None else scissor,
                             spin=spec.spin if spin is None else spin, flags=flags,
                             stream=ctypes.c_void_p(stream), gs_tol=gs_tol, precision=precision,
                             q_ion=q_ion, scf_tol=scf_tol,
                             pair_cutoff=0.0 if pair_cutoff is None else float(pair_cutoff))
        dims = (ctypes.c_int * 8)()
        _check(load_library().bse_get_dims(self.ctx, dims), self.ctx)
        (self.n_pw, self.n_occ, self.n_pdep, self.n_atoms, n1, n2, n3, self.n_dens) = list(dims)
        self.grid = (n1, n2, n3)
        self.precision = int(precision)
        self.generation = 0            # bumped by every call that replaces the geometry or the roots
        self._pos = np.asarray(spec.pos, dtype=np.float64).copy()

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            load_library().bse_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def zeros(self, *shape):
        return self.torch.zeros(*shape, dtype=self.torch.float64, device=self.device)

    def ground_state(self):
        eps = np.zeros(self.n_occ)
        phi = self.zeros(self.n_occ, self.n_pw)
        _check(load_library().bse_get_ground_state(self.ctx, _ptr(eps), _dev_ptr(phi)), self.ctx)
        return eps, phi

    def empty_states(self):
        """The unoccupied states solved with the ground state: (eps[n_empty], phi[n_empty, n_pw])."""
        n = ctypes.c_int(0)
        lib = load_library()
        _check(lib.bse_get_empty_states(self.ctx, 0, ctypes.byref(n), None, None), self.ctx)
        eps = np.zeros(max(1, n.value))
        phi = self.zeros(max(1, n.value), self.n_pw)
        _check(lib.bse_get_empty_states(self.ctx, n.value, ctypes.byref(n), _ptr(eps), _dev_ptr(phi)), self.ctx)
        return eps[:n.value], phi[:n.value]

    def set_positions(self, pos):
        p = np.ascontiguousarray(np.asarray(pos, dtype=np.float64))
        _check(load_library().bse_set_positions(self.ctx, _ptr(p)), self.ctx)
        self.generation += 1
        self._pos = p.copy()

    def apply(self, A, op=0):
        A = A.contiguous()
        LA = self.torch.empty_like(A)
        bse_apply_liouville(self.ctx, A, LA, op)
        return LA

    def relax(self, gs_energy, fmax=1e-4, max_steps=300, root=0, inexact=True, davidson_tol=0.0, zvector_tol=0.0,
              dt=0.0, dt_max=0.0, max_move=0.0, pos=None):
        """Excited-state relaxation (bse_relax) on E = E_gs + omega from pos (default: the current
        positions); gs_energy(pos[n_atoms, 3]) -> (E_gs, F_gs).  Returns (pos, E, omega, evaluations)."""
        P = np.ascontiguousarray(np.asarray(self._pos if pos is None else pos, dtype=np.float64).copy())
        opts = _relax_opts(fmax, max_steps, root, inexact, davidson_tol, zvector_tol, dt, dt_max, max_move)
        cb = _gs_callback(lambda system, p: gs_energy(p))
        E, w, steps = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        st = load_library().bse_relax(self.ctx, ctypes.byref(opts), cb, None, _ptr(P), ctypes.byref(E),
                                      ctypes.byref(w), ctypes.byref(steps))
        self.generation += 1
        self._pos = P.copy()
        _check(st, self.ctx)
        return P, E.value, w.value, steps.value

    def davidson_full(self, n_roots=1, tol=1e-9, max_iter=300):
        """Lowest roots of the BSE beyond the TDA (bse_davidson_full): (omega, X, Y)."""
        X = self.zeros(n_roots, self.n_occ, self.n_pw)
        Y = self.zeros(n_roots, self.n_occ, self.n_pw)
        w = np.zeros(n_roots)
        _check(load_library().bse_davidson_full(self.ctx, int(n_roots), float(tol), int(max_iter), _ptr(w),
                                                _dev_ptr(X), _dev_ptr(Y)), self.ctx)
        self.generation += 1
        return w, X, Y

    def davidson(self, n_roots=1, tol=1e-9, max_iter=200):
        A = self.zeros(n_roots, self.n_occ, self.n_pw)
        w = bse_davidson(self.ctx, n_roots, tol, max_iter, A)
        self.generation += 1
        return w, A

    def zvector(self, root=0, tol=1e-10, max_iter=1000):
        Z = self.zeros(self.n_occ, self.n_pw)
        U = self.zeros(self.n_occ, self.n_pw)
        bse_zvector(self.ctx, root, tol, max_iter, Z, U)
        return Z, U

    def forces(self, root=0):
        return bse_forces(self.ctx, root, self.n_atoms)

    def density(self, which):
        n1, n2, n3 = self.grid
        rho = np.zeros((n3, n2, n1))
        _check(load_library().bse_get_density(self.ctx, int(which), _ptr(rho)), self.ctx)
        return rho

    def sphere_to_grid(self, X, out=None):
        """Real-basis rows X (float64 CUDA tensor [n][n_pw]) -> packed grids [(n+1)/2][N3][N2][N1]
        (complex128 for FP64 contexts, complex64 for mixed ones), bse_sphere_to_grid."""
        X = X.contiguous()
        n = X.shape[0]
        n1, n2, n3 = self.grid
        dt = self.torch.complex128 if self.precision == 0 else self.torch.complex64
        if out is None:
            out = self.torch.empty(((n + 1) // 2, n3, n2, n1), dtype=dt, device=self.device)
        _check(load_library().bse_sphere_to_grid(self.ctx, int(n), _dev_ptr(X),
                                                 _grid_ptr(out, self.precision, (n + 1) // 2, self.grid)), self.ctx)
        return out

    def grid_to_sphere(self, P, n, out=None):
        """Packed grids P (overwritten) -> real-basis rows [n][n_pw] (float64), bse_grid_to_sphere."""
        if out is None:
            out = self.zeros(n, self.n_pw)
        _check(load_library().bse_grid_to_sphere(self.ctx, int(n), _grid_ptr(P, self.precision, (n + 1) // 2, self.grid),
                                                 _dev_ptr(out)), self.ctx)
        return out

    def profile(self, enable=True):
        _check(load_library().bse_profile(self.ctx, 1 if enable else 0), self.ctx)

    def kernel_timing(self, kernel):
        n = ctypes.c_longlong()
        ms, by, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(load_library().bse_get_kernel_timing(self.ctx, int(kernel), ctypes.byref(n), ctypes.byref(ms),
                                                    ctypes.byref(by), ctypes.byref(fl)), self.ctx)
        return {"launches": n.value, "ms": ms.value, "alg_bytes": by.value, "alg_flops": fl.value}

    def stats(self):
        s = Stats()
        _check(load_library().bse_get_stats(self.ctx, ctypes.byref(s)), self.ctx)
        return {k: getattr(s, k) for k, _ in Stats._fields_}


class BSEBatch:
    """Many independent systems on the current CUDA device (bse_setup_batch): each spec is any
    object with the fields of ``bse_inputs.SystemSpec``.  ``solve()`` returns the lowest
    excitation energy of every system and the forces, one (n_atoms, 3) array per system."""

    def __init__(self, specs, n_workers=8, precision=1, gs_tol=0.0, flags=0):
        lib = load_library()
        self.specs = list(specs)
        self.n_atoms = [int(np.asarray(sp.pos).shape[0]) for sp in self.specs]
        keep = []
        descs = (SystemDesc * len(self.specs))()
        for i, sp in enumerate(self.specs):
            fl, q_ion = _spec_model(sp, flags)
            descs[i] = _make_desc(keep, sp.lattice, sp.grid, sp.ecut, sp.pos, sp.Z, sp.sigma, sp.n_occ,
                                  sp.pdep_coef, sp.pdep_lambda, sp.scissor, sp.spin, fl, precision, None,
                                  gs_tol, q_ion)
        h = ctypes.c_void_p()
        st = lib.bse_setup_batch(len(self.specs), descs, int(n_workers), ctypes.byref(h))
        self.h = h
        self.setup_status = st
        if not h.value:
            raise BSEError(st, lib.bse_last_error(None).decode())

    def status(self, i):
        return load_library().bse_batch_status(self.h, int(i))

    def timing(self):
        """Device time (ms) of the last setup and the last solve (bse_batch_timing)."""
        su, so = ctypes.c_double(), ctypes.c_double()
        _check(load_library().bse_batch_timing(self.h, ctypes.byref(su), ctypes.byref(so)))
        return su.value, so.value

    def error(self, i):
        lib = load_library()
        ctx = lib.bse_batch_system(self.h, int(i))
        return lib.bse_last_error(ctypes.c_void_p(ctx) if ctx else None).decode()

    def system_stats(self, i):
        lib = load_library()
        ctx = lib.bse_batch_system(self.h, int(i))
        if not ctx:
            return None
        s = Stats()
        _check(lib.bse_get_stats(ctypes.c_void_p(ctx), ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def set_positions(self, pos_list):
        allp = np.ascontiguousarray(np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in pos_list]))
        return load_library().bse_batch_set_positions(self.h, _ptr(allp))

    def relax(self, gs_energy, pos_list=None, fmax=1e-4, max_steps=300, root=0, inexact=True, davidson_tol=0.0,
              zvector_tol=0.0, dt=0.0, dt_max=0.0, max_move=0.0):
        """bse_relax_batch: every system relaxed concurrently on E = E_gs + omega; gs_energy(system,
        pos[n_atoms, 3]) -> (E_gs, F_gs) (called from the workers' threads).  Returns (list of
        positions, E, omega, evaluations, status)."""
        if pos_list is None:
            pos_list = [sp.pos for sp in self.specs]
        allp = np.ascontiguousarray(np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in pos_list]))
        n = len(self.specs)
        E, w = np.zeros(n), np.zeros(n)
        steps = (ctypes.c_int * n)()
        opts = _relax_opts(fmax, max_steps, root, inexact, davidson_tol, zvector_tol, dt, dt_max, max_move)
        cb = _gs_callback(gs_energy)
        st = load_library().bse_relax_batch(self.h, ctypes.byref(opts), cb, None, _ptr(allp), _ptr(E), _ptr(w),
                                            steps)
        out, o = [], 0
        for na in self.n_atoms:
            out.append(allp[o:o + 3 * na].reshape(na, 3).copy())
            o += 3 * na
        return out, E, w, list(steps), st

    def solve(self, davidson_tol=1e-5, zvector_tol=1e-10, max_iter=500):
        w = np.zeros(len(self.specs))
        F = np.zeros(3 * sum(self.n_atoms))
        st = load_library().bse_solve_batch(self.h, float(davidson_tol), float(zvector_tol), int(max_iter),
                                            _ptr(w), _ptr(F))
        out, o = [], 0
        for na in self.n_atoms:
            out.append(F[o:o + 3 * na].reshape(na, 3))
            o += 3 * na
        return w, out, st

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load_library().bse_destroy_batch(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
