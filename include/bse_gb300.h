/*
 * bse_gb300.h -- C ABI of the GB300 (sm_103a) plane-wave TDA-BSE force library.
 *
 * The library computes the lowest TDA Bethe-Salpeter excitation energies of a
 * Gamma-point plane-wave model system in the density-matrix (DMPT) form of
 * arXiv 2607.20728, Eqs. 1-3, and their nuclear forces by the Lagrangian /
 * Z-vector route of Eqs. 4-7 and Supplemental Sec. SI.  Everything after
 * bse_setup runs on one GPU; the host sees small matrices and scalars only.
 *
 * Conventions shared by every call
 *  - Hartree atomic units; ecut in Ry, i.e. the wave-function sphere is
 *    |G|^2 <= ecut in bohr^-2 and the density sphere |G|^2 <= 4 ecut.
 *  - Real basis of length n_pw for Gamma-point functions (real in r):
 *    index 0 is G = 0; half-sphere vector k = 1..(n_pw-1)/2 gives index 2k-1
 *    (cosine part) and 2k (sine part), c(G_k) = (x[2k-1] + i x[2k])/sqrt(2),
 *    c(-G_k) = conj(c(G_k)).  The half sphere holds Miller triples n != 0 with
 *    n3 > 0, or n3 == 0 and n2 > 0, or n3 == n2 == 0 and n1 > 0, in ascending
 *    (n3, n2, n1) order.  Orbitals are f(r) = Omega^-1/2 sum_G c(G) e^{iG.r}.
 *  - Real-space grids are row-major with the first lattice index fastest:
 *    r(j1, j2, j3) = sum_i (j_i/N_i) a_i, linear index j1 + N1 (j2 + N2 j3).
 *  - Trial blocks A are [n_vec][n_occ][n_pw] FP64 row-major device arrays;
 *    a_{b,v} belongs to occupied orbital v (Eq. 1).
 *  - Every call is ordered on the context's stream and returns a bse_status;
 *    no C++ exception crosses this boundary.  On error, bse_last_error()
 *    returns a one-line message and the context stays usable unless the status
 *    is BSE_ERR_CUDA (a CUDA failure: destroy the context).
 *  - Device pointers passed in are owned by the caller and must stay valid for
 *    the duration of the call; the context owns all memory it allocates.
 */
#ifndef BSE_GB300_H
#define BSE_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bse_ctx bse_ctx;

typedef enum {
  BSE_OK = 0,
  BSE_ERR_INVALID = 1,        /* bad argument, non-finite input, grid too small */
  BSE_ERR_OOM = 2,            /* device allocation failed */
  BSE_ERR_CUDA = 3,           /* CUDA runtime error */
  BSE_ERR_NOT_CONVERGED = 4,  /* iteration limit reached; outputs hold the last iterate */
  BSE_ERR_DEGENERATE = 5,     /* HOMO-LUMO gap or root spacing below 1e-6 Ha */
  BSE_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up */
  BSE_ERR_STATE = 7           /* call out of order (e.g. forces before davidson) */
} bse_status;

/* Kernel switches for the special cases of Table S1 (tests); 0 = full BSE. */
#define BSE_FLAG_NO_K1E 1     /* drop the bare exchange term 2 K1e (Eq. 2b) */
#define BSE_FLAG_NO_K1D 2     /* drop the screened direct term K1d (Eq. 2c) */
/* Run the wave-function-sphere transforms as full-grid 3D FFTs instead of the default
 * sphere-pruned column/plane passes (same results up to rounding; for comparisons). */
#define BSE_FLAG_FULL_GRID_FFT 4
/* Run without captured CUDA graphs: in a batch (bse_setup_batch) this system's Liouville applies
 * become plain launches, and in any context the Z-vector conjugate gradients loop on the host
 * instead of running as one captured device-side loop (same results; for comparisons). */
#define BSE_FLAG_NO_GRAPHS 8
/* Choose the launch shapes by timing the candidates on the first Liouville apply: the transform
 * path (sphere-pruned or full-grid), the trial vectors per K1d pass, the threads per plane-pass CTA
 * of the sphere-pruned transforms and the split-K of the occupied-projection GEMMs (a coordinate
 * search in that order); choices are cached per problem shape for the process.  On by default for
 * the systems of a batch. */
#define BSE_FLAG_AUTOTUNE 16
/* Warm start for sequences of nearby geometries (a relaxation or dynamics step): after
 * bse_set_positions the ground-state Davidson starts from the previous geometry's states and
 * bse_davidson from the previous excitation vectors.  Results are converged to the same
 * tolerances; only the number of iterations changes. */
#define BSE_FLAG_WARM_START 32
/* Hartree-SCF ground-state model (f_Hxc = v_c, alpha_EXX = 0: the Kohn-Sham response kernels of
 * Sec. SI with the Hartree kernel only).  The occupied orbitals are the lowest n_occ eigenstates
 * of H^KS = -1/2 nabla^2 + V_ext + v_c * rho, rho = 2 sum_v |phi_v|^2, iterated to
 * self-consistency (Anderson mixing of rho until (int |rho_out - rho_in|^2)^{1/2} <= scf_tol).
 * The BSE operator (Eqs. 1-2) uses that H^KS; the U vector gains the f_Hxc term of its D
 * contribution, 2 P_c [v_c * Delta rho^(x)] phi_w; the Z-vector operator (Eq. 7) gains
 * 2 K1e,KS + 2 K2e,KS = 4 P_c [v_c * sum_v phi_v Z_v] phi_w and is solved as one coupled system.
 * A cell with q_ion = 2 on every site and n_occ = n_atoms is neutral. */
#define BSE_FLAG_HARTREE_SCF 64
/* Wannier pair pruning of K1d (an approximation): after the ground state the occupied orbitals are
 * localised at Gamma (maximally localised rotation w_i = sum_v U_vi phi_v by joint Jacobi
 * diagonalisation of the cos/sin position matrices), tau~_ij = W * (w_i w_j) is cached only for
 * the pairs whose Wannier centres are within pair_cutoff (minimum image), and the Liouville
 * operator (op 0, and so bse_davidson) is U L~ U^T with L~ the Wannier-gauge operator of
 * Eqs. 1-2 (full eps matrix in D) restricted to those pairs.  U vector, Z-vector and forces stay
 * exact (their one K1d product is evaluated on the fly) on the pruned eigenvector.  Exact for a
 * cutoff beyond every pair distance. */
#define BSE_FLAG_WANNIER_PRUNE 128

/* System description.  All pointers are host pointers unless stated; the
 * library copies what it needs during bse_setup. */
typedef struct {
  double lattice[9];          /* rows a1, a2, a3 (bohr) */
  int grid[3];                /* FFT grid; each N_i >= kd_i + 2 kw_i + 1 where kw/kd are the
                                 largest |n_i| in the wave-function/density spheres, else
                                 BSE_ERR_INVALID (products must not alias, Eq. 2) */
  double ecut;                /* Ry */
  int n_atoms;
  const double *pos;          /* [n_atoms][3] bohr */
  const double *Z;            /* [n_atoms] Gaussian well depth: V_a(r) = -Z exp(-r^2/(2 sigma^2)) */
  const double *sigma;        /* [n_atoms] bohr */
  int n_occ;                  /* occupied orbitals (lowest eigenstates of H) */
  int n_pdep;                 /* PDEP vectors (Eq. 3); 0 gives W = v_c */
  const double *pdep_coef;    /* [n_pdep][n_pw] real-basis rows, orthonormal, zero G = 0
                                 component; host, or device if pdep_on_device */
  const double *pdep_lambda;  /* [n_pdep] host, each < 0 */
  int pdep_on_device;
  double scissor;             /* Ha: H^QP = H^KS + P_c scissor (Table S1, "BSE-Scissor") */
  int spin;                   /* 0 singlet D + 2K1e - K1d; 1 triplet D - K1d */
  int precision;              /* 0 = FP64 throughout */
  int flags;                  /* BSE_FLAG_* */
  void *stream;               /* cudaStream_t to order all work on; NULL = context-owned stream */
  double gs_tol;              /* ground-state residual-norm target ||H phi - eps phi||; 0 = 1e-11 */
  const double *q_ion;        /* [n_atoms] Gaussian ionic charges (width sigma), or NULL for none:
                                 V_ext gains -v_c * sum_a q_a (2 pi sigma_a^2)^{-3/2}
                                 exp(-|r - R_a|^2/(2 sigma_a^2)), G = 0 term dropped */
  double scf_tol;             /* BSE_FLAG_HARTREE_SCF density-residual target; 0 = 1e-10 (FP64),
                                 1e-9 (mixed) */
  double pair_cutoff;         /* BSE_FLAG_WANNIER_PRUNE: largest Wannier-centre distance of a kept
                                 K1d pair (bohr, > 0) */
} bse_system_desc;

/* Per-context statistics (bse_get_stats). */
typedef struct {
  int gs_iterations;          /* ground-state Davidson iterations (all chunks) */
  int davidson_iterations;
  int zvector_iterations;
  int n_applies;              /* trial vectors passed through the Liouville operator */
  double gs_residual;         /* max ground-state residual norm */
  double davidson_residual;   /* max residual norm of the converged roots */
  double zvector_residual;    /* max relative Z-vector residual */
  double homo_lumo_gap;       /* Ha */
  double ms_setup, ms_ground_state, ms_tau, ms_davidson, ms_uvec, ms_zvector, ms_forces;
  double bytes_tau;           /* bytes of the cached tau_{v'v}(r) */
  int k1d_tma;                /* 1 when the TMA-fed FP32 kernel serves the K1d term (mixed precision) */
  double ms_host_eig;         /* host time in the Rayleigh-Ritz / orthonormalisation eigensolves */
  int gs_chunks;              /* Davidson chunks of the ground state */
  int tuned;                  /* 1 once the autotuner has chosen this context's launch shapes */
  int tuned_full_grid_fft;    /* its choice: 1 full-grid transforms, 0 sphere-pruned */
  int tuned_k1d_nb;           /* its choice: trial vectors per K1d pass (0: not applicable) */
  int scf_iterations;         /* Hartree-SCF iterations of the last geometry (0: non-SCF model) */
  double scf_residual;        /* final (int |rho_out - rho_in|^2)^{1/2} */
  int wannier_pairs;          /* K1d pairs kept under BSE_FLAG_WANNIER_PRUNE (of n_occ (n_occ + 1)/2) */
  int wannier_sweeps;         /* Jacobi sweeps of the localisation */
  int tuned_xy_threads;       /* its choice: threads per plane-pass CTA of the sphere-pruned transforms
                                 (0: the default, 512) */
  int tuned_gemm_split_pct;   /* its choice: split-K of the occupied-projection GEMMs, percent of the
                                 library's heuristic (100: the heuristic) */
  int zvector_graphed;        /* 1 when the last Z-vector conjugate-gradient solve ran as one captured
                                 CUDA graph (a device-side loop), 0 when it looped on the host: the
                                 first solve of a context, BSE_FLAG_NO_GRAPHS, or profiling on */
} bse_stats;

/* Build a context: enumerate the spheres, upload the PDEP basis, and run the
 * geometry stage of bse_set_positions for desc->pos.  The non-self-consistent
 * ground state (lowest n_occ eigenpairs of H = -1/2 nabla^2 + sum_a V_a), or with
 * BSE_FLAG_HARTREE_SCF the self-consistent one, is found by a block Davidson on the GPU; tau_{v'v}(r) = [W * phi_v' phi_v](r)
 * (Eq. 2c with Eq. 3) is cached for v' <= v.  Returns BSE_ERR_DEGENERATE if the
 * HOMO-LUMO gap is below 1e-6 Ha, BSE_ERR_NOT_CONVERGED if the Hartree SCF has not
 * reached scf_tol in 200 iterations. */
bse_status bse_setup(const bse_system_desc *desc, bse_ctx **out);

/* New atomic positions ([n_atoms][3] host, bohr): rebuild V, the ground state
 * and the tau cache.  W stays fixed in G-space (dW/d<phi| = 0, Sec. SI). */
bse_status bse_set_positions(bse_ctx *ctx, const double *pos);

/* dims[0..7] = n_pw, n_occ, n_pdep, n_atoms, N1, N2, N3, number of density-sphere G. */
bse_status bse_get_dims(const bse_ctx *ctx, int *dims);

/* Occupied energies eps_host[n_occ] and, if phi_dev != NULL, the real-basis
 * orbitals phi_dev[n_occ][n_pw] (device).  Each orbital's sign is arbitrary. */
bse_status bse_get_ground_state(bse_ctx *ctx, double *eps_host, double *phi_dev);

/* The unoccupied states solved with the ground state (the lowest few to the ground-state
 * tolerance, then up to 64 more to 1e-3 in the residual norm; they span the low-energy part of
 * the P_c space in which the BSE preconditioner of Eqs. 1-2 is exact).  *n_empty: their number.
 * eps_host[max_states] (may be NULL): their energies, ascending; phi_dev[max_states][n_pw]
 * (device, may be NULL): real-basis coefficients, orthonormal and orthogonal to the occupied
 * orbitals.  Only min(max_states, *n_empty) states are written.  BSE_ERR_STATE before a ground
 * state exists. */
bse_status bse_get_empty_states(bse_ctx *ctx, int max_states, int *n_empty, double *eps_host, double *phi_dev);

/* LA = L A for n_vec trial vectors (device, [n_vec][n_occ][n_pw]):
 *   op 0: L = D + 2 K1e - K1d (singlet) or D - K1d (triplet), Eqs. 1-2, output projected by P_c;
 *   op 1: L = P_c (H - eps_v), the Z-vector operator of Eq. 7 for the non-SCF model;
 *   op 2: the Z-vector operator of Eq. 7 of the context's ground-state model: op 1, or with
 *         BSE_FLAG_HARTREE_SCF P_c (H - eps_v) Z_v + 4 P_c [v_c * sum_v' phi_v' Z_v'] phi_v;
 *   op 3: B, the coupling block of the BSE beyond the TDA (Sec. SI), real orbitals:
 *         (2 K2e - K2d) A (singlet) or -K2d A (triplet), K2e A = P_c [v_c * sum_v' a_v' phi_v'] phi_v,
 *         K2d A = P_c sum_v' [W * (a_v' phi_v)] phi_v' (W applied to N_occ^2 pair densities per vector).
 * A is used as given (callers keep it in the P_c space).  A and LA must not overlap. */
bse_status bse_apply_liouville(bse_ctx *ctx, int n_vec, const double *A_dev, double *LA_dev, int op);

/* Lowest n_roots eigenpairs of op 0 by block Davidson with FP64 Rayleigh-Ritz.
 * Convergence: residual norm ||L A - omega A|| <= tol for every root.  omega_host
 * [n_roots] receives the energies (Ha); A_dev (optional, [n_roots][n_occ][n_pw])
 * the normalised eigenvectors (A^dagger A = 1).  The context keeps the roots
 * for bse_zvector / bse_forces. */
bse_status bse_davidson(bse_ctx *ctx, int n_roots, double tol, int max_iter,
                        double *omega_host, double *A_dev);

/* Lowest n_roots excitation energies of the BSE beyond the TDA (Sec. SI), for real orbitals
 * (A B; B A)(X; Y) = omega (X; -Y) with A = L (op 0) and B (op 3 of bse_apply_liouville), solved
 * as (A - B)(A + B)(X + Y) = omega^2 (X + Y) by a Davidson on X + Y and X - Y.  omega_host
 * [n_roots] ascending; X_dev, Y_dev (device [n_roots][n_occ][n_pw], either may be NULL) with
 * X.X - Y.Y = 1.  Energies only: bse_zvector/bse_forces keep referring to the last TDA solve
 * (the paper's forces are TDA).  BSE_ERR_DEGENERATE when A - B or A + B is not positive definite
 * (no real spectrum, e.g. a negative TDA root), BSE_ERR_NOT_CONVERGED at max_iter. */
bse_status bse_davidson_full(bse_ctx *ctx, int n_roots, double tol, int max_iter, double *omega_host,
                             double *X_dev, double *Y_dev);

/* U vector of root `root` (Sec. SI) and the Z-vector solve P_c (H - eps_v) Z_v = -u_v
 * (Eq. 7 with f_Hxc = 0, alpha_EXX = 0) by batched preconditioned CG, to relative
 * residual tol per orbital; with BSE_FLAG_HARTREE_SCF the coupled operator of op 2 by one
 * CG over the block, to the block's relative residual.  Z_dev (optional) receives Z
 * [n_occ][n_pw]; U_dev (optional) receives U [n_occ][n_pw]. */
bse_status bse_zvector(bse_ctx *ctx, int root, double tol, int max_iter, double *Z_dev,
                       double *U_dev);

/* Forces F = -d omega/dR (Ha/bohr), F_host[n_atoms][3], from Eq. 4 with the
 * densities of Eqs. 5-6.  Runs bse_zvector (tol 1e-10) first if it has not been
 * run for this root. */
bse_status bse_forces(bse_ctx *ctx, int root, double *F_host);

/* Density grids, host [N3][N2][N1] (first index fastest): which 0 = Delta rho^(x) (Eq. 5) and
 * 1 = Delta rho^(z) (Eq. 6) of the last bse_forces call (else BSE_ERR_STATE); 2 = the ground-state
 * density rho = 2 sum_v |phi_v|^2 of the current geometry. */
bse_status bse_get_density(bse_ctx *ctx, int which, double *rho_host);

bse_status bse_get_stats(const bse_ctx *ctx, bse_stats *out);

/* Utility: the sphere -> grid transform of the Liouville apply (its first step, the trial vectors
 * a_v on the real-space grid for the products of Eq. 2) on its own.  n real-basis rows X_dev
 * [n][n_pw] (device, FP64) -> packed grids P_dev [(n+1)/2][N3][N2][N1] of complex numbers
 * (device; complex128 for an FP64 context, complex64 for a mixed-precision one): grid q holds
 * f_2q(r) + i f_2q+1(r), f(r) = Omega^-1/2 sum_G c(G) e^{iG.r} (for odd n the last imaginary
 * part is 0).  Sphere-pruned column and plane passes, or full-grid FFTs under
 * BSE_FLAG_FULL_GRID_FFT, exactly as inside the apply.  Ordered on the context's stream and
 * synchronised before returning. */
bse_status bse_sphere_to_grid(bse_ctx *ctx, int n, const double *X_dev, void *P_dev);

/* Utility: the grid -> sphere transform of the Liouville apply (its last step before P_c) on its
 * own: packed grids P_dev as written by bse_sphere_to_grid (overwritten: the transform runs in
 * place) -> real-basis rows Y_dev [n][n_pw] of c(G) = Omega^1/2 / N_r sum_r f(r) e^{-iG.r}. */
bse_status bse_grid_to_sphere(bse_ctx *ctx, int n, void *P_dev, double *Y_dev);

/* Batched in-place 3D complex FFT (no normalisation) of `batch` contiguous
 * grids data_dev[batch][n3][n2][n1] of interleaved FP64 complex numbers;
 * direction -1 computes sum_j x_j e^{-2 pi i k.j/N}, +1 the inverse sign.
 * Sizes 2 <= n_i <= 512 with prime factors 2, 3, 5 only.  The transform the
 * Liouville operator uses for every real-space product of Eq. 2. */
bse_status bse_fft3d(int n1, int n2, int n3, int batch, double *data_dev, int direction,
                     void *stream);

/* Allocation-free form of bse_fft3d, for callers that must not allocate device memory:
 * code whose device memory belongs to another allocator (a framework's caching pool that
 * accounts for every byte), or loops that cannot afford the implicit device-wide
 * synchronisation of cudaMalloc/cudaFree.  The paper has no counterpart; this is a library
 * convenience.  Same arguments, layout and result as bse_fft3d, sizes up to 512 per axis
 * (else BSE_ERR_INVALID, nothing launched).  The twiddle tables live in one file-scope device
 * array of 24 KB that every GPU loading the library keeps until the process exits; each call
 * rewrites the entries it reads, so no clearing is needed.  All calls on a device share that
 * array: calls whose transforms overlap on the GPU (different streams, or different host
 * threads) race and must be ordered by the caller.  The first call on each device looks up
 * the array's device address with that device current; it may also be the call that loads the
 * library's device code (CUDA's lazy module loading), which takes device memory once, so make
 * that first call at set-up, before any stream capture.  Later calls allocate nothing.
 * Synchronises `stream` before returning. */
bse_status bse_fft3d_noalloc(int n1, int n2, int n3, int batch, double *data_dev, int direction,
                             void *stream);

/* Utility: the library's FP64 GEMM, C = alpha op(A) op(B) + beta C on device arrays,
 * row-major: ta 'N' op(A) = A [M][lda], 'T' op(A) = A^T with A [K][lda]; tb 'N' op(B) = B [K][ldb],
 * 'T' op(B) = B^T with B [N][ldb]; C [M][ldc].  It carries the occupied-space projector
 * (S = Phi^T Y, Y -= Phi S) and the Davidson / PDEP products.  Ordered on `stream`,
 * synchronised before returning. */
bse_status bse_gemm(char ta, char tb, int M, int N, int K, double alpha, const double *A, int lda,
                    const double *B, int ldb, double beta, double *C, int ldc, void *stream);

/* Utility: C = alpha A B^T + beta C on the 5th-generation tensor cores with split-BF16
 * operands (x = hi + lo, three BF16 products, FP32 accumulation): A [M][lda], B [N][ldb],
 * C [M][ldc], FP32 device arrays, K >= 1.  The mixed-precision path uses it for the PDEP
 * projection and back-projection of Eq. 3.  Relative error per product about 3 * 2^-18.
 * BSE_ERR_TIMEOUT if a bounded device-side wait gave up.  Synchronises `stream`. */
bse_status bse_gemm_bf16x3(int M, int N, int K, float alpha, const float *A, int lda, const float *B, int ldb,
                           float beta, float *C, int ldc, void *stream);

/* Kernel classes timed by bse_profile (CUDA events on the context's stream). */
#define BSE_KERNEL_K1D 0      /* fused grid combine: V a + 2 v_H phi - sum_v' tau_{v'v} a_v' (Eq. 2a-2c) */
#define BSE_KERNEL_FFT 1      /* one batched 3D FFT (three axis passes) */
#define BSE_KERNEL_SPHERE_FFT 2  /* one sphere-pruned transform (z pass + plane pass, or the fused H product) */
#define BSE_KERNEL_COUNT 3

/* enable != 0 starts per-kernel timing (and clears the counters), 0 stops it.  While it
 * is on, every launch of the classes above is bracketed by CUDA events on the context's
 * stream; the elapsed times are summed at the end of each call.  Off by default. */
bse_status bse_profile(bse_ctx *ctx, int enable);

/* Launches, summed device time (ms) and algorithmic work of one kernel class since
 * bse_profile(ctx, 1): alg_bytes is the minimum HBM traffic the kernel must move
 * (inputs read once, outputs written once), alg_flops its useful floating-point
 * operations, both counted from the launch's sizes. */
bse_status bse_get_kernel_timing(const bse_ctx *ctx, int kernel, long long *launches, double *total_ms,
                                 double *alg_bytes, double *alg_flops);

/* Number of kernels this library has launched in this process (all contexts). */
long long bse_launch_count(void);

/* Host-only utility: eigenvalues w[n] (ascending) and eigenvectors (columns of V[n][n],
 * row-major) of the symmetric matrix A[n][n] by Householder tridiagonalisation and the
 * implicit QR iteration with Wilkinson shifts.  The Davidson solvers use it for their
 * FP64 Rayleigh-Ritz matrices.  Needs no GPU. */
bse_status bse_host_sym_eig(int n, const double *A, double *w, double *V);

/* Failure-detection self-test of the device-side bounded waits (the mbarrier waits of the K1d
 * pipeline): one thread waits on an mbarrier that nothing completes; the wait gives up after one
 * second of %globaltimer, the kernel sets the device error flag and returns.  Returns
 * BSE_ERR_TIMEOUT when that happened (the expected outcome; the context stays usable),
 * BSE_ERR_CUDA otherwise.  stream: a cudaStream_t or NULL. */
bse_status bse_selftest_bounded_wait(void *stream);

/* Failure-detection self-test of the whole K1d pipeline (Eq. 2c, the TMA-fed FP32 contraction of
 * a mixed-precision context with n_occ a multiple of 16): one launch over every 32-point tile with
 * all consumer warps, in which the producer warp issues no copies.  Every consumer's bounded wait
 * gives up after one second; the consumer warps leave the kernel together (no warp waits at a
 * barrier another has quit), the device error flag is set, nothing is written.  Returns
 * BSE_ERR_TIMEOUT when that happened (expected; the context stays usable), BSE_ERR_STATE for a
 * context without that pipeline, BSE_ERR_CUDA otherwise. */
bse_status bse_selftest_k1d_stall(bse_ctx *ctx);

/* Host-only utility: all eigenvalues w[n] (ascending) of the symmetric A[n][n] and the
 * eigenvectors of the k lowest (columns 0..k-1 of V[n][n]; the other columns are left as
 * they are): Householder tridiagonalisation, eigenvalues by implicit QR without vectors,
 * vectors by inverse iteration with Gram-Schmidt inside clusters of close eigenvalues.  The
 * Davidson solvers use it for their Rayleigh-Ritz steps. */
bse_status bse_host_sym_eig_lowest(int n, const double *A, int k, double *w, double *V);

/* Host-only utility, the Davidson's Rayleigh-Ritz form: the k lowest eigenvalues w[0..k)
 * (ascending; w[k..n) are left unspecified) and their eigenvectors (columns 0..k-1 of V[n][n]).
 * From 64 rows on the eigenvalues come from bisection on the Sturm count of the tridiagonal
 * form, split over the host thread pool, instead of a QR sweep over all n. */
bse_status bse_host_sym_eig_k(int n, const double *A, int k, double *w, double *V);

/* Last error message of ctx, or of the last context-free call (bse_setup failure,
 * bse_fft3d, bse_host_sym_eig) on this thread when ctx is NULL. */
const char *bse_last_error(const bse_ctx *ctx);   /* never NULL */
void bse_destroy(bse_ctx *ctx);                   /* NULL is a no-op */

/* ---- Batches of independent systems -------------------------------------------
 * Many independent systems of uneven size (each one bse_setup's problem: own cell, atoms,
 * PDEP basis, precision) solved concurrently on one GPU.  The paper's method treats each
 * system on its own (Sec. 2); batching is a throughput form with no counterpart there.
 * n_workers host threads each own one CUDA stream; every system is bound to one worker
 * (largest estimated cost first, to the least loaded worker), so the kernels of different
 * systems interleave on the GPU.  Within a system, each block of trial vectors of the
 * Liouville apply (op 0) is replayed from a CUDA graph captured at its first use.
 * Systems whose setup fails keep their status (bse_batch_status) and are skipped by the
 * solve; the calls return the first failing status, all systems having been attempted. */
/* ---- Excited-state relaxation --------------------------------------------------------
 * The forces of Eq. 4 drive excited-state geometry relaxations (Sec. SIV relaxes until the
 * largest force component is below a threshold).  The excited-state energy is
 * E(R) = E_gs(R) + omega(R): the synthetic model has no ground-state energy of its own, so the
 * caller supplies E_gs and F_gs = -dE_gs/dR; omega and its forces come from bse_davidson,
 * bse_zvector and bse_forces of the chosen root. */

/* Generic energy/force callback: n coordinates x, returns 0 on success and fills energy and
 * F = -dE/dx (host arrays). */
typedef int (*bse_grad_fn)(int n, const double *x, double *energy, double *F, void *user);

/* FIRE minimisation (Bitzek, Koskinen, Gaehler, Moseler, Gumbsch, Phys. Rev. Lett. 97, 170201
 * (2006); unit masses) of E(x) until max_i |F_i| <= fmax.  dt: initial time step, dt_max its cap,
 * max_move: largest displacement of one coordinate per step.  Host only, no GPU work of its own.
 * x (host [n]) is updated in place; BSE_ERR_NOT_CONVERGED after max_steps, BSE_ERR_INVALID if
 * the callback fails or returns non-finite values. */
bse_status bse_fire_minimize(int n, double *x, bse_grad_fn fn, void *user, double fmax, int max_steps, double dt,
                             double dt_max, double max_move, int *steps_out, double *energy_out);

/* Ground-state energy callback of a relaxation: system index (0 for bse_relax), atoms, positions
 * (host [n_atoms][3]); fills energy and F_gs = -dE_gs/dR (host [n_atoms][3]); returns 0 on success. */
typedef int (*bse_gs_energy_fn)(int system, int n_atoms, const double *pos, double *energy, double *F,
                                void *user);

typedef struct {
  double fmax;                /* converged when max |F_alpha| <= fmax (Ha/bohr) */
  int max_steps;
  double dt, dt_max, max_move;  /* FIRE parameters (bohr, unit masses); 0 = 0.1, 0.5, 0.1 */
  int root;                   /* excitation root followed */
  double davidson_tol, zvector_tol;  /* tolerances of the converged step; 0 = 1e-8, 1e-10 */
  int inexact;                /* 1: inexact solves, each tolerance loosened in proportion to the
                                 current largest force (capped at 1e-4 / 1e-3) and brought back to
                                 the tight values to confirm convergence */
} bse_relax_opts;

/* Relax the excited state of ctx from pos_inout (host [n_atoms][3], updated in place) with FIRE on
 * E = E_gs + omega, warm-starting every geometry from the previous one (BSE_FLAG_WARM_START for
 * the duration).  energy_out: final E; omega_out: final omega; steps_out: force evaluations. */
bse_status bse_relax(bse_ctx *ctx, const bse_relax_opts *opts, bse_gs_energy_fn gs, void *user, double *pos_inout,
                     double *energy_out, double *omega_out, int *steps_out);

typedef struct bse_batch bse_batch;

/* descs[n]: as for bse_setup (the stream field is ignored); n_workers >= 1. */
bse_status bse_setup_batch(int n, const bse_system_desc *descs, int n_workers, bse_batch **out);

/* Every system: lowest excitation (bse_davidson with one root), Z-vector and forces.
 * omega_host[n] (Ha); F_host[sum_i 3 n_atoms_i] (Ha/bohr, systems in order); either may
 * be NULL.  Entries of failed systems are NaN. */
bse_status bse_solve_batch(bse_batch *b, double davidson_tol, double zvector_tol, int max_iter,
                           double *omega_host, double *F_host);

/* New positions for every system, pos_all[sum_i 3 n_atoms_i] (bohr); re-runs each system's
 * ground state and tau concurrently (bse_set_positions). */
bse_status bse_batch_set_positions(bse_batch *b, const double *pos_all);
/* bse_relax for every system of the batch concurrently (one worker thread each, the callback
 * called with the system index, possibly from several threads at once); pos_all_inout is the
 * concatenation of the systems' [n_atoms][3] arrays; energy_out, omega_out, steps_out [n].
 * Returns the first failing status; the other systems complete. */
bse_status bse_relax_batch(bse_batch *b, const bse_relax_opts *opts, bse_gs_energy_fn gs, void *user,
                           double *pos_all_inout, double *energy_out, double *omega_out, int *steps_out);

/* Device time of the last bse_setup_batch (setup_ms) and bse_solve_batch (solve_ms): from the first
 * worker stream's start to the last one's end, by CUDA events recorded on the workers' streams
 * around their systems (ms; either pointer may be NULL). */
bse_status bse_batch_timing(const bse_batch *b, double *setup_ms, double *solve_ms);

int bse_batch_size(const bse_batch *b);
bse_status bse_batch_status(const bse_batch *b, int i);     /* status of system i's last call */
bse_ctx *bse_batch_system(bse_batch *b, int i);              /* NULL if its setup failed */
void bse_destroy_batch(bse_batch *b);                        /* NULL is a no-op */

#ifdef __cplusplus
}
#endif
#endif /* BSE_GB300_H */
