// Internal declarations shared by the translation units of the BSE library.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/bse_gb300.h"

namespace bse {

// ----------------------------------------------------------------------------
// errors: internal code throws; the C ABI converts to bse_status
struct Error : std::runtime_error {
  bse_status status;
  Error(bse_status s, const std::string &m) : std::runtime_error(m), status(s) {}
};

#define BSE_CUDA(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      throw ::bse::Error(e_ == cudaErrorMemoryAllocation ? BSE_ERR_OOM : BSE_ERR_CUDA,   \
                         std::string(#call) + ": " + cudaGetErrorString(e_));            \
  } while (0)

// every kernel launch of the library is followed by BSE_CHECK_LAUNCH(), which also counts it
void count_launch();
#define BSE_CHECK_LAUNCH()            \
  do {                                \
    ::bse::count_launch();            \
    BSE_CUDA(cudaGetLastError());     \
  } while (0)

#define BSE_REQUIRE(cond, msg)                                       \
  do {                                                               \
    if (!(cond)) throw ::bse::Error(BSE_ERR_INVALID, (msg));         \
  } while (0)

// Device memory of the library's buffers, cached per host thread: cudaFree synchronises the
// whole device, which would serialise the streams of a batch at every temporary buffer.  A
// block released by a thread is only handed out again by the same thread; every library call
// synchronises its stream before returning, and within a call all work of the thread is on one
// stream, so a reused block is never still in use by an earlier kernel.  Blocks above 1 GB, and
// blocks beyond 8 GB of cache per thread, go straight back to cudaFree.
void *dev_alloc(size_t bytes, size_t *granted);
void dev_release(void *p, size_t bytes);

// owning device buffer
template <class T>
struct DevBuf {
  T *p = nullptr;
  size_t n = 0;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) dev_release(p, bytes);
    p = nullptr;
    n = 0;
    bytes = 0;
  }
  void alloc(size_t count) {
    if (count <= n && p) return;
    release();
    if (count == 0) return;
    p = static_cast<T *>(dev_alloc(count * sizeof(T), &bytes));
    n = bytes / sizeof(T);
  }
  T *get() const { return p; }
};

// complex type of a real type
template <class R> struct CxType;
template <> struct CxType<double> { using T = double2; };
template <> struct CxType<float> { using T = float2; };
template <class R> using CT = typename CxType<R>::T;

// ----------------------------------------------------------------------------
// FFT (fft.cu)
struct FFTAxis {
  int n = 0;
  int nstage = 0;
  int radix[12] = {0};
  double2 *tw = nullptr;   // device table exp(-2 pi i k/n), k < n, FP64
  float2 *tw32 = nullptr;  // the same rounded to FP32
};

struct FFTPlan {
  int n[3] = {0, 0, 0};
  long nr = 0;
  FFTAxis ax[3];
  std::vector<void *> owned;
  void init(int n1, int n2, int n3);
  void destroy();
  // in-place batched transform of `batch` grids; dir -1 forward, +1 inverse
  void exec(double2 *data, int batch, int dir, cudaStream_t s) const;
  void exec(float2 *data, int batch, int dir, cudaStream_t s) const;
};

bool fft_size_ok(int n);
// same transform as FFTPlan::exec with the twiddles in a file-scope device array (no allocation)
void fft3d_noalloc(int n1, int n2, int n3, int batch, double2 *data, int dir, cudaStream_t s);

// ----------------------------------------------------------------------------
// GEMM (linalg.cu): row-major FP64, C = alpha op(A) op(B) + beta C
//   'N' op(A) = A [M][K]; 'T' op(A) = A^T with A stored [K][M]
//   'N' op(B) = B [K][N]; 'T' op(B) = B^T with B stored [N][K]
// fixed: split-K partials go to this buffer, which is never resized (the split is clamped to
// it); the default is a per-thread buffer that grows on demand.  split_pct scales the number of
// K slices the heuristic picks (a tunable of the autotuner; 100 = the heuristic)
void dgemm(char ta, char tb, int M, int N, int K, double alpha, const double *A, int lda,
           const double *B, int ldb, double beta, double *C, int ldc, cudaStream_t s,
           DevBuf<double> *fixed = nullptr, int split_pct = 100);
// FP32 SIMT GEMM with FP32 accumulation (same conventions)
void sgemm(char ta, char tb, int M, int N, int K, float alpha, const float *A, int lda,
           const float *B, int ldb, float beta, float *C, int ldc, cudaStream_t s,
           DevBuf<float> *fixed = nullptr, int split_pct = 100);
// FP64 operands and output with FP32 products and sums (same conventions as dgemm): the operands
// are rounded to FP32 as they are staged, alpha, beta and the sum over K slices are applied in FP64
void mgemm(char ta, char tb, int M, int N, int K, double alpha, const double *A, int lda, const double *B, int ldb,
           double beta, double *C, int ldc, cudaStream_t s, int split_pct = 100);
// out[i] = sum_j X[i][j] * Y[i][j] for i < rows (part: scratch of the partial sums; the default is
// a per-thread buffer)
void rowdot(int rows, long len, const double *X, const double *Y, double *out, cudaStream_t s,
            DevBuf<double> *part = nullptr);
// X[i][:] = a[i] X[i][:] + b[i] Y[i][:]   (a,b device arrays of length rows, NULL = 1)
void row_axpby(int rows, long len, const double *a, double *X, const double *b, const double *Y,
               cudaStream_t s);

// host symmetric eigensolver (Householder tridiagonalisation + implicit QL):
// A [n][n] row-major symmetric, returns ascending eigenvalues w and eigenvectors
// as the columns of V [n][n]
void sym_eig(int n, const double *A, double *w, double *V);
// all eigenvalues, eigenvectors only of the k lowest (columns 0..k-1 of V)
// all_values: w[0..n) (implicit QR); otherwise only w[0..k) are computed (bisection on the host
// pool from 64 rows on), the form of the Davidson's Rayleigh-Ritz steps
void sym_eig_lowest(int n, const double *A, int k, double *w, double *V, bool all_values = true);

// ----------------------------------------------------------------------------
// the context
struct Stats {
  bse_stats s{};
};

// per-kernel-class CUDA-event timing (bse_profile)
struct KernelProf {
  bool on = false;
  struct Pending {
    cudaEvent_t a, b;
    int kind;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  long long launches[BSE_KERNEL_COUNT] = {};
  double ms[BSE_KERNEL_COUNT] = {};
  double bytes[BSE_KERNEL_COUNT] = {};
  double flops[BSE_KERNEL_COUNT] = {};
  cudaEvent_t get();
  // returns the event pair to record around one launch (nullptr pair when off)
  void begin(cudaStream_t s, int kind, double bytes, double flops, cudaEvent_t *stop_out);
  void flush();  // synchronise on pending stops and accumulate
  ~KernelProf();
};

// TMA-fed FP32 K1d contraction (k1d_tma.cu)
// tau in the tile-major layout of the bulk-copy K1d kernel: for every tile of 32 grid points,
// the orbital blocks (I <= J; column J outer, I inner) one after the other, each [jj][ii][32]
// (I < J) or the packed triangle [jj (jj + 1)/2 + ii][32] (I = J)
struct K1dTma {
  const float *tau = nullptr;
  long npairs = 0;
  int *err = nullptr;                  // device flag set when a bounded wait gives up
  bool ready = false;
};
// position (in pairs) of the pair (v', v), v' <= v, inside one 32-point tile of that layout
__host__ __device__ inline long k1d_tile_slot(int vp, int v, int nocc) {
  (void)nocc;
  const int I = vp / 16, J = v / 16, ii = vp % 16, jj = v % 16;
  const long col = 128L * J * (J - 1) + 136L * J;  // pairs of the columns before J
  if (I == J) return col + 256L * J + jj * (jj + 1) / 2 + ii;
  return col + 256L * I + jj * 16 + ii;
}

// an FP32 operand split into bf16 hi + lo, rows padded with zeros to kp (a multiple of 64) columns
struct SplitBF16 {
  DevBuf<unsigned short> hi, lo;
  int rows = 0, k = 0, kp = 0;
};
void split_bf16(int rows, int k, const float *X, int ldx, SplitBF16 &out, cudaStream_t s);
// C [M][N] = alpha A B^T + beta C on the tensor cores (split-BF16, 3 products, FP32 accumulation)
void umma_gemm_nt(int M, int N, float alpha, const SplitBF16 &A, const SplitBF16 &B, float beta, float *C, int ldc,
                  DevBuf<float> &partial, int *err, cudaStream_t s);
void transpose_f32(int rows, int cols, const float *X, float *Y, cudaStream_t s);

// grid-resident arrays of one precision
template <class R>
struct Grids {
  DevBuf<R> vloc;        // [nr] V(r)
  DevBuf<R> vcg;         // [nr] 4 pi/|G|^2 on the density sphere (0 elsewhere / G = 0)
  DevBuf<R> phir;        // [nocc][nr]
  DevBuf<R> tau;         // [npairs][nr], pair (v', v) with v' <= v at v (v + 1)/2 + v'
  DevBuf<CT<R>> work;    // packed complex grids
  DevBuf<CT<R>> work2;
  DevBuf<R> pdep;        // [npdep][npw]: PDEP rows times v_c^{1/2}(G)
  DevBuf<R> cpdep;       // [npdep] lambda/(1 - lambda)
  DevBuf<R> sbuf;        // [batch][npw] density coordinates
  DevBuf<R> qbuf;        // [batch][npdep]
  DevBuf<CT<R>> colbuf;  // occupied columns between the passes of the sphere-pruned transforms
  DevBuf<CT<R>> vh;      // packed v_H grids of one apply block
  DevBuf<CT<R>> colbuf_apply;  // column buffer of the Liouville apply (fixed size, see apply_scratch)
  DevBuf<CT<R>> colbuf_dens;   // density-sphere columns of the pair pipelines
  DevBuf<R> bar, bt;           // coupling-block apply: a_v(r) and the accumulated T_v(r) [nocc][nr]
  DevBuf<R> wphir;             // Wannier orbitals w_i(r) [nocc][nr] (pair pruning)
  DevBuf<R> wtau;              // tau~_p = W * (w_j w_i) for the kept pairs [npairs_kept][nr]
};

// Wannier pair pruning of K1d (BSE_FLAG_WANNIER_PRUNE)
struct WannierPrune {
  bool on = false;
  double cutoff = 0.0;
  int npairs = 0, sweeps = 0;
  std::vector<double> U_h;     // [nocc][nocc], w_i = sum_v U_vi phi_v
  DevBuf<double> U;            // device copy
  DevBuf<double> epst;         // eps~ = U^T diag(eps) U [nocc][nocc]
  DevBuf<int2> pairs;          // kept pairs (i, j), i <= j
  DevBuf<int> off;             // CSR offsets per orbital [nocc + 1]
  DevBuf<int2> nbr;            // (j, pair index) per kept neighbour of each orbital
  DevBuf<double> rot;          // rotated trial vectors (apply scratch)
};

// sphere-pruned transforms (sphere_fft.cu): column tables of the wave-function sphere
struct SphereFFT {
  bool ready = false, ok64 = false, ok32 = false, disabled = false;
  int ncols = 0, ncols_pad = 0, ngroups = 0, nxs = 0, cg = 32;
  DevBuf<int> colpos;   // [ncols_pad] plane position j1 + N1 j2 of each column, -1 for padding
  DevBuf<int> xs;       // [nxs] x indices whose y lines the sphere reaches
  DevBuf<int4> ent;     // coefficients by z-pass group: (kk, +G slot/z, -G slot/z, 0)
  DevBuf<int> ent_off;  // [ngroups + 1]
};

// Conjugate gradients of the Z-vector solve run as one CUDA graph: a WHILE conditional node whose
// body is one iteration (operator, step lengths and residuals on the device) and whose last kernel
// decides on the device whether to go on.  The vectors live here so that their addresses, which a
// captured graph records, stay fixed for the life of the context.
struct CgState {
  double tol, best, relmax;
  int maxit, stall, it, best_it, done;
};
struct CgWork {
  DevBuf<double> Rr, Zr, P, AP, dz;               // [nocc][npw]
  DevBuf<double> dots, rz, rr, r0, al, aln, be;  // [nocc]
  DevBuf<double> Cb, Ck, zth, vsh, part, s64;    // preconditioner and reduction scratch
  DevBuf<CgState> st;
  std::map<int, cudaGraphExec_t> graphs;          // key: 2 (FP32 grids) + (coupled)
  std::map<int, long long> body_kernels;          // kernels per iteration (launch accounting)
  std::map<int, std::vector<const void *>> fp;    // addresses each graph recorded
  std::map<int, bool> failed;                     // no capture possible: plain loop from then on
  std::map<int, int> plain_runs;                  // the first run sizes every lazily grown buffer
  ~CgWork() {
    for (auto &kv : graphs)
      if (kv.second) cudaGraphExecDestroy(kv.second);
  }
};

struct Ctx {
  bse_system_desc desc{};
  KernelProf prof;
  int prec = 0;           // 0 FP64, 1 mixed
  Grids<double> g64;
  Grids<float> g32;
  template <class R> Grids<R> &grids();
  std::string last_error;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bse_stats stats{};

  // geometry of the cell
  double lat[9], B[9], omega = 0;
  int N[3] = {0, 0, 0};
  long nr = 0;
  int npw = 0, nhalf = 0, nocc = 0, npdep = 0, natoms = 0, ndens = 0;
  int spin = 0, flags = 0;
  double scissor = 0;
  double gs_tol = 1e-11;        // ground-state residual norm target
  std::vector<double> pos, Z, sigma;
  std::vector<double> q;      // Gaussian ionic charges (empty: none)
  bool hartree = false;       // Hartree-SCF ground-state model (BSE_FLAG_HARTREE_SCF)
  double scf_tol = 1e-10;     // its density-residual target
  std::vector<double> kin_h;  // 1/2 |G|^2 per real-basis index

  FFTPlan fft;
  SphereFFT sfft;   // wave-function sphere columns
  SphereFFT dfft;   // density-sphere columns (pair pipelines of the tau build and the U vector)

  // static tables
  DevBuf<int> gp, gm;         // grid index of +G_k, -G_k (k = 1..nhalf), entry 0 = G = 0
  DevBuf<double> kin;         // [npw]

  // geometry-dependent state
  double v0 = 0;              // V(G = 0)
  DevBuf<double> vext;        // [nr] V_ext(r) (the Hartree model adds v_H[rho] to it in g64.vloc)
  DevBuf<double> rho_gs;      // [nr] ground-state density 2 sum_v phi_v(r)^2
  DevBuf<double> warm_rho;    // previous geometry's SCF density (warm start)
  bool have_warm_rho = false;
  DevBuf<double> phi;         // [nocc][npw]
  DevBuf<float> phi32;        // FP32 copy (mixed precision: P_c inside the FP32-grid operator)
  DevBuf<float> pc32;         // scratch of the FP32 P_c: [nf][npw] rows, then [nf][nocc] overlaps
  DevBuf<double> eps;         // [nocc]
  DevBuf<double> negeps;      // [nocc] -eps_v (D-term shift of the gather)
  std::vector<double> eps_h;
  DevBuf<double> empty;       // [n_empty][npw] lowest empty states (guesses, preconditioner)
  DevBuf<double> eps_empty_d;
  std::vector<double> eps_empty;
  long npairs = 0;
  bool have_gs = false;

  // roots
  int nroots = 0;
  DevBuf<double> roots;       // [nroots][nocc][npw]
  int warm_roots = 0;         // roots of the previous geometry kept in `roots` (warm start)
  DevBuf<double> warm_states;  // previous geometry's ground-state block (warm start)
  int warm_nstates = 0;
  std::vector<double> omega_h;
  int z_root = -1;
  DevBuf<double> zvec, uvec;  // [nocc][npw]
  DevBuf<double> rho_x, rho_z;  // [nr]
  bool have_rho = false;

  K1dTma k1d;                  // FP32 K1d with TMA staging (mixed precision)
  SplitBF16 pdep_split;        // PDEP rows x v_c^{1/2} (projection operand, mixed precision)
  SplitBF16 pdepT_split;       // their transpose (back-projection operand)
  SplitBF16 gemm_a;            // per-call split of the left operand
  DevBuf<float> gemm_part;     // split-K partials of the tensor-core GEMM
  DevBuf<int> dev_err;        // device-side error flag of bounded waits
  // launch shapes chosen by the autotuner (k1d_nb_cap 0: the largest that fits; xy_threads 0: the
  // default plane-pass width; gemm_split_pct: the occupied-projection GEMMs' split-K, in percent
  // of the heuristic's)
  bool autotune = false;
  int k1d_nb_cap = 0;
  int xy_threads = 0;
  int gemm_split_pct = 100;
  // CUDA graphs of the Liouville apply (op 0), one per block size, replayed on staging buffers
  bool use_graphs = false;
  std::map<int, cudaGraphExec_t> graphs;
  std::map<int, long long> graph_kernels;  // kernels per replay (launch accounting)
  DevBuf<double> gA, gLA;
  // split-K partials of the apply's occupied-space projections, sized once at setup: every
  // buffer a captured apply touches keeps its address for the life of the context
  DevBuf<double> apply_s64;
  DevBuf<float> apply_s32;
  std::vector<const void *> graph_fp;  // addresses the captured graphs were recorded with
  // scratch
  DevBuf<double> smat;        // small matrices
  DevBuf<int2> pairs;
  DevBuf<int2> pairs_full;    // all ordered pairs (v', v) (the coupling block's pair densities)
  WannierPrune wan;
  CgWork cg;                  // the Z-vector conjugate gradients (captured loop)

  ~Ctx();
};

bool k1d_tma_supported(int nocc, long nr);
// a bounded mbarrier wait on a barrier nothing completes: sets *err (device) when it gives up
void wait_selftest(cudaStream_t s, int *err);
int k1d_tma_max_nb(int nocc);
void k1d_tma_init(K1dTma &t, const float *tau, long npairs, long nr, int *err);
// packed grids of np pair products (pairs list + p0 .. + np - 1) -> tau in the tile-major layout
void k1d_unpack_tiled(const Ctx &c, int np, const int2 *pairs, const float2 *P, float *tau);
void k1d_tma(const Ctx &c, const K1dTma &t, int nb, const float *phir, const float *vloc, const float2 *Pa,
             const float2 *Pvh, float2 *Py, bool use_vloc, bool use_k1e);
void k1d_tma_stall_test(const Ctx &c, const K1dTma &t, const float *phir, const float *vloc, const float2 *Pa,
                        const float2 *Pvh, float2 *Py);

// sphere-pruned transforms (sphere_fft.cu).  miller_half holds (n1, n2, n3) of G_kk for
// kk = 0..nhalf (kk = 0 is G = 0) in the order of the real basis; dens_cols the (n1, n2) of every
// density-sphere G.
void sphere_fft_init(Ctx &c, const std::vector<int> &miller_half, const std::vector<int> &dens_cols);
// pair pipelines on the density sphere: P (packed pair grids) -> Coulomb-weighted columns and X
// (wave-function-sphere coefficients for the PDEP part); then X' added back and -> P
template <class R> bool dens_fft_ok(const Ctx &c);
template <class R>
void dens_forward(Ctx &c, int np, CT<R> *P, R *X, double scale, const R *vcg, R cscale);
template <class R> void dens_inverse(Ctx &c, int np, const R *X, double scale, CT<R> *P);
template <class R> bool sphere_fft_ok(const Ctx &c);
// X [nf][npw] (real basis) -> packed grids P [(nf+1)/2][nr], every point written
template <class R> void sphere_to_grid(Ctx &c, int nf, const double *X, CT<R> *P, double scale,
                                       CT<R> *colbuf = nullptr);
// packed grids -> Y [nf][npw] (the gather_pairs contract, D term included when Xd is given);
// P is left unchanged
// colbuf: column buffer to use (large enough for (nf + 1)/2 grids); default the context's
template <class R>
void grid_to_sphere(Ctx &c, int nf, CT<R> *P, double *Y, double scale, const double *Xd, const double *shift,
                    int period, double shift_const, CT<R> *colbuf = nullptr);
// HX = H X (+ shift_v X) without a grid in global memory
template <class R> void sphere_h(Ctx &c, int nf, const double *X, double *HX, const double *shift);

template <> inline Grids<double> &Ctx::grids<double>() { return g64; }
template <> inline Grids<float> &Ctx::grids<float>() { return g32; }

// ----------------------------------------------------------------------------
// kernels (kernels.cu)
namespace k {
// X [nf][npw] -> packed grids P [(nf+1)/2][nr]: pair q holds f = 2q (re), 2q+1 (im); P must be
// zeroed unless accumulate (then the coefficients are added)
template <class R, class I>
void scatter_pairs(const Ctx &c, int nf, const I *X, CT<R> *P, double scale, bool accumulate = false);
// packed grids -> Y [nf][npw] = scale * coeffs + (kin + shift[f % period] + shift_const) * Xd (Xd may be NULL)
template <class R, class O>
void gather_pairs(const Ctx &c, int nf, const CT<R> *P, O *Y, double scale, const double *Xd = nullptr,
                  const double *shift = nullptr, int period = 1, double shift_const = 0.0);
// P[q][r] *= scale w[r] for nq packed grids
template <class R> void mul_grid(long nr, int nq, CT<R> *P, const R *w, R scale, cudaStream_t s);
// unpack packed grids into real grids [nf][nr]
template <class R, class O> void unpack_real(long nr, int nf, const CT<R> *P, O *Rr, cudaStream_t s);
// pack real grids [nf][nr] into packed grids
template <class R> void pack_real(long nr, int nf, const R *Rr, CT<R> *P, cudaStream_t s);
// packed grids of A[x](r) * Bm[y](r) for the pairs (x, y) of list
template <class R>
void pair_products(long nr, int np, const int2 *list, const R *A, const R *Bm, CT<R> *P, cudaStream_t s);
// Q[i][a] *= s[a]
template <class T> void scale_cols(int rows, int cols, T *Q, const T *s, cudaStream_t st);
// Delta rho_b(r) = sum_v phi_v(r) a_{b,v}(r) -> packed grids over b
template <class R> void drho(const Ctx &c, int nb, const R *phir, const CT<R> *Pa, CT<R> *Pd);
// Y_{b,v} = V a + 2 vH_b phi_v - sum_v' tau_{v'v} a_{b,v'} (terms switched by the flags)
template <class R>
void combine_tau(const Ctx &c, int nb, const R *phir, const R *vloc, const R *tau, const CT<R> *Pa,
                 const CT<R> *Pvh, CT<R> *Py, bool use_vloc, bool use_k1e, bool use_k1d);
// T_w -= sigma_{vw} phi_v (and, when sym, T_v -= sigma_{vw} phi_w for v != w) for the pairs (v, w) of list
template <class R>
void sigma_contract(const Ctx &c, int np, const int2 *list, const CT<R> *Psig, const R *phir, R *T,
                    bool sym = true);
// Delta rho^(x) = sum_v a_v^2 - phi_v Psi_v, Delta rho^(z) = 2 sum_v Z_v phi_v (FP64 grids)
void rel_density(const Ctx &c, const double *phir, const double *ar, const double *psi, const double *zr,
                 double *rx, double *rz);
// V_ext(G) on the density sphere (Gaussian wells, and ionic Gaussian charges q_d unless NULL)
// -> packed grid (G space) ready for the inverse FFT
void vloc_G(const Ctx &c, const double *pos_d, const double *Z_d, const double *sig_d, const double *q_d,
            double2 *P);
// d omega/dR contraction over the density sphere; rho in G space (packed grid, re part = rho)
void force_reduce(const Ctx &c, const double2 *rhoG, const double *pos_d, const double *Z_d,
                  const double *sig_d, const double *q_d, double *partial, int nchunk, double *out);
// out[r] = scale sum_v phi_v(r)^2
void density_sum(long nr, int nocc, const double *phir, double scale, double *out, cudaStream_t s);
// out = sum_v a_v^2 - phi_v Psi_v  (Delta rho^(x), Eq. 5)
template <class R>
void xdensity(long nr, int nocc, const R *phir, const R *ar, const R *psi, R *out, cudaStream_t s);
// Y = V a + 2 vH w - sum over the kept pairs of the CSR lists (off, nbr = (j, tau index)) tau a
template <class R>
void combine_pruned(const Ctx &c, int nb, const R *phir, const R *vloc, const R *tau, const int *off, const int2 *nbr,
                    const CT<R> *Pa, const CT<R> *Pvh, CT<R> *Py, bool use_k1e, bool use_k1d);
// phi_v(r) cos / sin (2 pi j_k / N_k) along lattice vector k, [nocc][nr] each
void phase_rows(const Ctx &c, int k, const double *phir, double *oc, double *os);
// packed grids P += pairs of the real grids T
template <class R> void add_packed(long nr, int nf, const R *T, CT<R> *P, cudaStream_t s);
// out = sum_v X_v Y_v over nocc grids
template <class R> void pair_sum(long nr, int nocc, const R *X, const R *Y, R *out, cudaStream_t s);
// T_w += scale v phi_w for the nocc grids of T
template <class R> void add_product(long nr, int nocc, const R *v, const R *phir, R scale, R *T, cudaStream_t s);
// R = AX - theta X
void residual(int k, long n, const double *AX, const double *X, const double *theta, double *R,
              cudaStream_t s);
// T = R / d, d = kin[j % npw] + vshift[j / npw] - theta_scale theta[row], |d| >= floor (sign kept)
void precond_diag(int k, long n, const double *R, const double *kin, int npw, const double *vshift,
                  double theta_scale, const double *theta, double floor, double *T, cudaStream_t s);
void fill_real_grid(long nr, double2 *P, const double *R, cudaStream_t s);
// out[f][c] = C[f][c] / (eps_e[c] - eps_o[f % nocc] + shift - th[f / nocc]) - Ck[f][c]
void subspace_den(int rows, int ne, int nocc, const double *C, const double *Ck, const double *eps_e,
                  const double *eps_o, double shift, const double *th, double floor, double *out, cudaStream_t s);
// elementwise conversions
void convert(long n, const double *src, float *dst, cudaStream_t s);
// C[i][j] = alpha T[i][j] + beta C[i][j] (T FP32 [M][N], C FP64 with leading dimension ldc)
void axpby_f32(int M, int N, double alpha, const float *T, double beta, double *C, int ldc, cudaStream_t s);
// X -= T (FP64 -= FP32)
void sub_f32(long n, double *X, const float *T, cudaStream_t s);
}  // namespace k

}  // namespace bse
