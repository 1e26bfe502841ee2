// Context, solvers and C ABI of the plane-wave TDA-BSE force library.
//
// Flow of a force evaluation (arXiv 2607.20728):
//   bse_setup / bse_set_positions : V(G), non-SCF ground state (block Davidson on H),
//                                   tau_{v'v} = W * (phi_v' phi_v)   (Eq. 2c with Eq. 3)
//   bse_davidson                  : lowest roots of D + 2K1e - K1d   (Eqs. 1-2)
//   bse_zvector                   : U vector (Sec. SI), Z-vector solve (Eq. 7)
//   bse_forces                    : Delta rho^(x) + Delta rho^(z) (Eqs. 5-6) contracted with dV/dR (Eq. 4)
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <numeric>
#include <string>
#include <thread>
#include <tuple>
#include <mutex>
#include <type_traits>
#include <thread>
#include <tuple>
#include <mutex>
#include <type_traits>
#include <vector>

#include "internal.cuh"

namespace bse {

namespace {
std::atomic<long long> g_launches{0};
}
thread_local long long tl_launches = 0;  // this thread's launches (graph capture accounting)
void count_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ++tl_launches;
}
long long launch_count_now() { return tl_launches; }
// a replayed graph runs the kernels captured into it; a capture records launches that do not run
void add_launches(long long n) {
  g_launches.fetch_add(n, std::memory_order_relaxed);
  tl_launches += n;
}

cudaEvent_t KernelProf::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  BSE_CUDA(cudaEventCreate(&e));
  return e;
}

void KernelProf::begin(cudaStream_t s, int kind, double b, double f, cudaEvent_t *stop_out) {
  *stop_out = nullptr;
  if (!on) return;
  Pending p;
  p.a = get();
  p.b = get();
  p.kind = kind;
  BSE_CUDA(cudaEventRecord(p.a, s));
  pending.push_back(p);
  launches[kind] += 1;
  bytes[kind] += b;
  flops[kind] += f;
  *stop_out = p.b;
}

void KernelProf::flush() {
  for (auto &p : pending) {
    BSE_CUDA(cudaEventSynchronize(p.b));
    float t = 0.f;
    BSE_CUDA(cudaEventElapsedTime(&t, p.a, p.b));
    ms[p.kind] += t;
    pool.push_back(p.a);
    pool.push_back(p.b);
  }
  pending.clear();
}

KernelProf::~KernelProf() {
  for (auto &p : pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : pool) cudaEventDestroy(e);
}

namespace {
constexpr size_t kPoolGrain = 512;
constexpr size_t kPoolMaxBlock = 1ull << 30;
constexpr size_t kPoolCap = 8ull << 30;

// 0 before the pool's first use on this thread, 1 while it lives, 2 once destroyed.  Buffers of
// other thread-local objects can be released after the pool during thread exit (destruction
// order follows construction order): they then go straight to cudaFree.
thread_local int tl_pool_state = 0;

struct DevPool {
  std::multimap<size_t, void *> free;  // size -> block
  size_t cached = 0;
  DevPool() { tl_pool_state = 1; }
  ~DevPool() {
    tl_pool_state = 2;
    for (auto &kv : free) cudaFree(kv.second);
  }
};
thread_local DevPool tl_pool;
}  // namespace

thread_local long long tl_alloc_calls = 0;  // buffers handed out by this thread (graph capture check)

void *dev_alloc(size_t bytes, size_t *granted) {
  ++tl_alloc_calls;
  const size_t want = (bytes + kPoolGrain - 1) / kPoolGrain * kPoolGrain;
  if (tl_pool_state == 2) {
    void *p = nullptr;
    if (cudaMalloc(&p, want) != cudaSuccess) {
      cudaGetLastError();
      throw Error(BSE_ERR_OOM, "cudaMalloc of " + std::to_string(want) + " bytes failed");
    }
    *granted = want;
    return p;
  }
  auto it = tl_pool.free.lower_bound(want);
  if (it != tl_pool.free.end() && it->first <= 2 * want) {
    void *p = it->second;
    *granted = it->first;
    tl_pool.cached -= it->first;
    tl_pool.free.erase(it);
    return p;
  }
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, want);
  if (e != cudaSuccess && !tl_pool.free.empty()) {
    // give the cached blocks back and retry once
    cudaGetLastError();
    for (auto &kv : tl_pool.free) cudaFree(kv.second);
    tl_pool.free.clear();
    tl_pool.cached = 0;
    e = cudaMalloc(&p, want);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(BSE_ERR_OOM, "cudaMalloc of " + std::to_string(want) + " bytes failed");
  }
  *granted = want;
  return p;
}

void dev_release(void *p, size_t bytes) {
  if (!p) return;
  if (tl_pool_state != 1 || bytes > kPoolMaxBlock || tl_pool.cached + bytes > kPoolCap) {
    cudaFree(p);
    return;
  }
  tl_pool.free.emplace(bytes, p);
  tl_pool.cached += bytes;
}

Ctx::~Ctx() {
  // buffers go back to the thread's cache when the members are destroyed: let the stream drain
  if (stream) cudaStreamSynchronize(stream);
  for (auto &kv : graphs)
    if (kv.second) cudaGraphExecDestroy(kv.second);
  fft.destroy();
  if (own_stream && stream) cudaStreamDestroy(stream);
}

namespace {

thread_local std::string g_last_error = "no error";

using clk = std::chrono::steady_clock;

// BSE_VERBOSE=1 in the environment logs solver progress to stderr
bool verbose() {
  static const bool v = [] {
    const char *e = std::getenv("BSE_VERBOSE");
    return e && e[0] && e[0] != '0';
  }();
  return v;
}
double ms_since(clk::time_point t0) {
  return std::chrono::duration<double, std::milli>(clk::now() - t0).count();
}

void sync(Ctx &c) { BSE_CUDA(cudaStreamSynchronize(c.stream)); }

void h2d(void *d, const void *h, size_t bytes, Ctx &c) {
  BSE_CUDA(cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, c.stream));
  sync(c);
}
void d2h(void *h, const void *d, size_t bytes, Ctx &c) {
  BSE_CUDA(cudaMemcpyAsync(h, d, bytes, cudaMemcpyDeviceToHost, c.stream));
  sync(c);
}
void d2d(void *d, const void *s, size_t bytes, Ctx &c) {
  if (bytes) BSE_CUDA(cudaMemcpyAsync(d, s, bytes, cudaMemcpyDeviceToDevice, c.stream));
}

bool finite_all(const double *p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

// ---------------------------------------------------------------------------------
// spheres and static tables
void inv3(const double *a, double *o) {
  const double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                     a[2] * (a[3] * a[7] - a[4] * a[6]);
  BSE_REQUIRE(std::fabs(det) > 1e-12, "singular lattice");
  o[0] = (a[4] * a[8] - a[5] * a[7]) / det;
  o[1] = (a[2] * a[7] - a[1] * a[8]) / det;
  o[2] = (a[1] * a[5] - a[2] * a[4]) / det;
  o[3] = (a[5] * a[6] - a[3] * a[8]) / det;
  o[4] = (a[0] * a[8] - a[2] * a[6]) / det;
  o[5] = (a[2] * a[3] - a[0] * a[5]) / det;
  o[6] = (a[3] * a[7] - a[4] * a[6]) / det;
  o[7] = (a[1] * a[6] - a[0] * a[7]) / det;
  o[8] = (a[0] * a[4] - a[1] * a[3]) / det;
}

struct Miller {
  int n[3];
};

// Miller triples with |G|^2 <= gmax2, in ascending (n3, n2, n1) order
std::vector<Miller> sphere(const Ctx &c, double gmax2, std::vector<double> *g2out) {
  int nmax[3];
  for (int i = 0; i < 3; ++i) {
    const double len = std::sqrt(c.lat[3 * i] * c.lat[3 * i] + c.lat[3 * i + 1] * c.lat[3 * i + 1] +
                                 c.lat[3 * i + 2] * c.lat[3 * i + 2]);
    nmax[i] = (int)std::floor(std::sqrt(gmax2) * len / (2.0 * M_PI)) + 1;
  }
  std::vector<Miller> out;
  for (int n3 = -nmax[2]; n3 <= nmax[2]; ++n3)
    for (int n2 = -nmax[1]; n2 <= nmax[1]; ++n2)
      for (int n1 = -nmax[0]; n1 <= nmax[0]; ++n1) {
        double G[3];
        for (int a = 0; a < 3; ++a) G[a] = n1 * c.B[a] + n2 * c.B[3 + a] + n3 * c.B[6 + a];
        const double g2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
        if (g2 <= gmax2) {
          out.push_back({{n1, n2, n3}});
          if (g2out) g2out->push_back(g2);
        }
      }
  return out;
}

long grid_index(const Ctx &c, const int n[3]) {
  long j[3];
  for (int i = 0; i < 3; ++i) j[i] = ((n[i] % c.N[i]) + c.N[i]) % c.N[i];
  return j[0] + (long)c.N[0] * (j[1] + (long)c.N[1] * j[2]);
}

void build_tables(Ctx &c) {
  const bse_system_desc &d = c.desc;
  std::memcpy(c.lat, d.lattice, sizeof(c.lat));
  double inv[9];
  inv3(c.lat, inv);
  // b_i = 2 pi (inv^T)_i  (rows)
  for (int i = 0; i < 3; ++i)
    for (int a = 0; a < 3; ++a) c.B[3 * i + a] = 2.0 * M_PI * inv[3 * a + i];
  c.omega = std::fabs(c.lat[0] * (c.lat[4] * c.lat[8] - c.lat[5] * c.lat[7]) -
                      c.lat[1] * (c.lat[3] * c.lat[8] - c.lat[5] * c.lat[6]) +
                      c.lat[2] * (c.lat[3] * c.lat[7] - c.lat[4] * c.lat[6]));
  for (int i = 0; i < 3; ++i) c.N[i] = d.grid[i];
  c.nr = (long)c.N[0] * c.N[1] * c.N[2];
  std::vector<double> g2w, g2d;
  std::vector<Miller> wf = sphere(c, d.ecut, &g2w);
  std::vector<Miller> dn = sphere(c, 4.0 * d.ecut, &g2d);
  int kw[3] = {0, 0, 0}, kd[3] = {0, 0, 0};
  for (auto &m : wf)
    for (int i = 0; i < 3; ++i) kw[i] = std::max(kw[i], std::abs(m.n[i]));
  for (auto &m : dn)
    for (int i = 0; i < 3; ++i) kd[i] = std::max(kd[i], std::abs(m.n[i]));
  for (int i = 0; i < 3; ++i)
    BSE_REQUIRE(c.N[i] >= kd[i] + 2 * kw[i] + 1,
                "FFT grid too small: products of density- and wave-function-sphere functions alias");
  c.ndens = (int)dn.size();
  // half sphere in the documented order
  std::vector<int> gp{(int)0}, gm{(int)0};
  std::vector<double> kin{0.0};
  std::vector<int> miller_half{0, 0, 0};
  for (size_t i = 0; i < wf.size(); ++i) {
    const int *n = wf[i].n;
    const bool pos = n[2] > 0 || (n[2] == 0 && n[1] > 0) || (n[2] == 0 && n[1] == 0 && n[0] > 0);
    if (!pos) continue;
    int neg[3] = {-n[0], -n[1], -n[2]};
    miller_half.insert(miller_half.end(), {n[0], n[1], n[2]});
    gp.push_back((int)grid_index(c, n));
    gm.push_back((int)grid_index(c, neg));
    kin.push_back(0.5 * g2w[i]);
    kin.push_back(0.5 * g2w[i]);
  }
  c.nhalf = (int)gp.size() - 1;
  c.npw = 2 * c.nhalf + 1;
  BSE_REQUIRE((size_t)c.npw == wf.size(), "internal: sphere is not symmetric");
  c.kin_h = kin;
  c.gp.alloc(gp.size());
  c.gm.alloc(gm.size());
  c.kin.alloc(kin.size());
  h2d(c.gp.get(), gp.data(), gp.size() * sizeof(int), c);
  h2d(c.gm.get(), gm.data(), gm.size() * sizeof(int), c);
  h2d(c.kin.get(), kin.data(), kin.size() * sizeof(double), c);
  // Coulomb kernel on the grid: 4 pi/|G|^2 for 0 < |G|^2 <= 4 ecut
  std::vector<double> vcg(c.nr, 0.0);
  for (auto &m : dn) {
    double G[3];
    for (int a = 0; a < 3; ++a) G[a] = m.n[0] * c.B[a] + m.n[1] * c.B[3 + a] + m.n[2] * c.B[6 + a];
    const double g2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
    if (g2 > 0) vcg[grid_index(c, m.n)] = 4.0 * M_PI / g2;
  }
  c.g64.vcg.alloc(c.nr);
  h2d(c.g64.vcg.get(), vcg.data(), c.nr * sizeof(double), c);
  if (c.prec == 1) {
    c.g32.vcg.alloc(c.nr);
    k::convert(c.nr, c.g64.vcg.get(), c.g32.vcg.get(), c.stream);
    sync(c);
  }
  c.fft.init(c.N[0], c.N[1], c.N[2]);
  std::vector<int> dens_cols;
  for (auto &m : dn) dens_cols.insert(dens_cols.end(), {m.n[0], m.n[1]});
  sphere_fft_init(c, miller_half, dens_cols);
  c.sfft.disabled = (c.flags & BSE_FLAG_FULL_GRID_FFT) != 0;
}

void upload_pdep(Ctx &c) {
  const bse_system_desc &d = c.desc;
  c.npdep = d.n_pdep;
  if (c.npdep == 0) return;
  BSE_REQUIRE(d.pdep_coef && d.pdep_lambda, "pdep_coef and pdep_lambda are required when n_pdep > 0");
  BSE_REQUIRE(c.npdep <= c.npw - 1, "n_pdep exceeds the number of G != 0 basis functions");
  std::vector<double> cp(c.npdep);
  for (int a = 0; a < c.npdep; ++a) {
    const double l = d.pdep_lambda[a];
    BSE_REQUIRE(std::isfinite(l) && l < 0.0, "pdep_lambda must be finite and negative");
    cp[a] = l / (1.0 - l);
  }
  Grids<double> &g = c.g64;
  g.pdep.alloc((size_t)c.npdep * c.npw);
  const size_t bytes = (size_t)c.npdep * c.npw * sizeof(double);
  if (d.pdep_on_device) {
    BSE_CUDA(cudaMemcpyAsync(g.pdep.get(), d.pdep_coef, bytes, cudaMemcpyDeviceToDevice, c.stream));
  } else {
    BSE_REQUIRE(finite_all(d.pdep_coef, (size_t)c.npdep * c.npw), "non-finite pdep_coef");
    h2d(g.pdep.get(), d.pdep_coef, bytes, c);
  }
  // fold v_c^{1/2}(G) = sqrt(4 pi)/|G| into the rows (zero at G = 0)
  std::vector<double> s(c.npw);
  for (int i = 0; i < c.npw; ++i) s[i] = c.kin_h[i] > 0 ? std::sqrt(4.0 * M_PI / (2.0 * c.kin_h[i])) : 0.0;
  DevBuf<double> sd;
  sd.alloc(c.npw);
  h2d(sd.get(), s.data(), c.npw * sizeof(double), c);
  k::scale_cols<double>(c.npdep, c.npw, g.pdep.get(), sd.get(), c.stream);
  g.cpdep.alloc(c.npdep);
  h2d(g.cpdep.get(), cp.data(), c.npdep * sizeof(double), c);
  if (c.prec == 1) {
    c.g32.pdep.alloc((size_t)c.npdep * c.npw);
    c.g32.cpdep.alloc(c.npdep);
    k::convert((long)c.npdep * c.npw, g.pdep.get(), c.g32.pdep.get(), c.stream);
    k::convert(c.npdep, g.cpdep.get(), c.g32.cpdep.get(), c.stream);
    // tensor-core operands of the projection (rows) and back-projection (transpose), split once
    split_bf16(c.npdep, c.npw, c.g32.pdep.get(), c.npw, c.pdep_split, c.stream);
    DevBuf<float> tr;
    tr.alloc((size_t)c.npdep * c.npw);
    transpose_f32(c.npdep, c.npw, c.g32.pdep.get(), tr.get(), c.stream);
    split_bf16(c.npw, c.npdep, tr.get(), c.npdep, c.pdepT_split, c.stream);
    sync(c);
  }
  sync(c);
}

// typed GEMM dispatch for the pair pipelines
inline void gemm_r(char ta, char tb, int M, int N, int K, double alpha, const double *A, int lda, const double *B,
                   int ldb, double beta, double *C, int ldc, cudaStream_t s) {
  dgemm(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s);
}
inline void gemm_r(char ta, char tb, int M, int N, int K, double alpha, const float *A, int lda, const float *B,
                   int ldb, double beta, float *C, int ldc, cudaStream_t s) {
  sgemm(ta, tb, M, N, K, (float)alpha, A, lda, B, ldb, (float)beta, C, ldc, s);
}

// PDEP part of Eq. 3 for a batch of np density rows X [np][npw] (real-basis coefficients times
// v_c^{1/2}): Qm = X P^T, Qm *= lambda/(1-lambda), X = Qm P.  FP64 grids: FP64 GEMMs.  Mixed:
// split-BF16 tensor-core GEMMs with FP32 accumulation.
template <class R>
void pdep_gemms(Ctx &c, int np, R *X, R *Qm) {
  Grids<R> &g = c.grids<R>();
  if constexpr (std::is_same<R, float>::value) {
    split_bf16(np, c.npw, X, c.npw, c.gemm_a, c.stream);
    umma_gemm_nt(np, c.npdep, 1.f, c.gemm_a, c.pdep_split, 0.f, Qm, c.npdep, c.gemm_part, c.dev_err.get(), c.stream);
    k::scale_cols<float>(np, c.npdep, Qm, g.cpdep.get(), c.stream);
    split_bf16(np, c.npdep, Qm, c.npdep, c.gemm_a, c.stream);
    umma_gemm_nt(np, c.npw, 1.f, c.gemm_a, c.pdepT_split, 0.f, X, c.npw, c.gemm_part, c.dev_err.get(), c.stream);
  } else {
    gemm_r('N', 'T', np, c.npdep, c.npw, 1.0, X, c.npw, g.pdep.get(), c.npw, 0.0, Qm, c.npdep, c.stream);
    k::scale_cols<R>(np, c.npdep, Qm, g.cpdep.get(), c.stream);
    gemm_r('N', 'N', np, c.npw, c.npdep, 1.0, Qm, c.npdep, g.pdep.get(), c.npw, 0.0, X, c.npw, c.stream);
  }
}

// ---------------------------------------------------------------------------------
// timed launches of the profiled kernel classes
template <class C>
void fft_exec(Ctx &c, C *data, int batch, int dir) {
  cudaEvent_t stop;
  const double nr = (double)c.nr;
  c.prof.begin(c.stream, BSE_KERNEL_FFT, 2.0 * batch * nr * sizeof(C), 5.0 * batch * nr * std::log2(nr), &stop);
  c.fft.exec(data, batch, dir, c.stream);
  if (stop) BSE_CUDA(cudaEventRecord(stop, c.stream));
  if (c.prof.pending.size() > 512) c.prof.flush();
}

// sphere-pruned transforms, timed as one class.  Algorithmic bytes: the grid side written or read
// once (none for the fused H product) plus the sphere vectors; flops: 5 n log2 n per transformed line.
double sphere_flops(const Ctx &c, int nq) {
  const double n1 = c.N[0], n2 = c.N[1], n3 = c.N[2];
  return 5.0 * nq *
         (c.sfft.ncols * n3 * std::log2(n3) + n3 * (c.sfft.nxs * n2 * std::log2(n2) + n2 * n1 * std::log2(n1)));
}

template <class R>
void sphere_to_grid_exec(Ctx &c, int nf, const double *X, CT<R> *P, double scale, CT<R> *colbuf = nullptr) {
  cudaEvent_t stop;
  const int nq = (nf + 1) / 2;
  c.prof.begin(c.stream, BSE_KERNEL_SPHERE_FFT, (double)nq * c.nr * sizeof(CT<R>) + 8.0 * nf * c.npw,
               sphere_flops(c, nq), &stop);
  sphere_to_grid<R>(c, nf, X, P, scale, colbuf);
  if (stop) BSE_CUDA(cudaEventRecord(stop, c.stream));
  if (c.prof.pending.size() > 512) c.prof.flush();
}

template <class R>
void grid_to_sphere_exec(Ctx &c, int nf, CT<R> *P, double *Y, double scale, const double *Xd, const double *shift,
                         int period, double shift_const, CT<R> *colbuf = nullptr) {
  cudaEvent_t stop;
  const int nq = (nf + 1) / 2;
  c.prof.begin(c.stream, BSE_KERNEL_SPHERE_FFT,
               (double)nq * c.nr * sizeof(CT<R>) + 8.0 * nf * c.npw * (Xd ? 2 : 1), sphere_flops(c, nq), &stop);
  grid_to_sphere<R>(c, nf, P, Y, scale, Xd, shift, period, shift_const, colbuf);
  if (stop) BSE_CUDA(cudaEventRecord(stop, c.stream));
  if (c.prof.pending.size() > 512) c.prof.flush();
}

template <class R>
void sphere_h_exec(Ctx &c, int nf, const double *X, double *HX, const double *shift) {
  cudaEvent_t stop;
  const int nq = (nf + 1) / 2;
  c.prof.begin(c.stream, BSE_KERNEL_SPHERE_FFT, 8.0 * 3 * nf * c.npw + (double)c.nr * sizeof(R),
               2.0 * sphere_flops(c, nq) + 2.0 * nq * c.nr, &stop);
  sphere_h<R>(c, nf, X, HX, shift);
  if (stop) BSE_CUDA(cudaEventRecord(stop, c.stream));
  if (c.prof.pending.size() > 512) c.prof.flush();
}

template <class R>
void combine_exec(Ctx &c, int nb, const CT<R> *Pa, const CT<R> *Pvh, CT<R> *Py, bool k1e, bool k1d) {
  cudaEvent_t stop;
  Grids<R> &g = c.grids<R>();
  const double nr = (double)c.nr, no = (double)c.nocc, w = sizeof(R);
  const double bytes = (k1d ? (double)c.npairs * nr * w : 0.0) + 2.0 * nb * no * nr * w + no * nr * w +
                       nr * w * (1 + nb);
  const double flops = (k1d ? 2.0 * nb * no * no * nr : 0.0) + 4.0 * nb * no * nr;
  c.prof.begin(c.stream, BSE_KERNEL_K1D, bytes, flops, &stop);
  if constexpr (std::is_same<R, float>::value) {
    if (k1d && c.k1d.ready)
      k1d_tma(c, c.k1d, nb, g.phir.get(), g.vloc.get(), Pa, Pvh, Py, true, k1e);
    else
      k::combine_tau<R>(c, nb, g.phir.get(), g.vloc.get(), g.tau.get(), Pa, Pvh, Py, true, k1e, k1d);
  } else {
    k::combine_tau<R>(c, nb, g.phir.get(), g.vloc.get(), g.tau.get(), Pa, Pvh, Py, true, k1e, k1d);
  }
  if (stop) BSE_CUDA(cudaEventRecord(stop, c.stream));
}

// the wave-function-sphere transforms of the Liouville apply on their own (utility entry points):
// n real-basis rows -> packed real-space grids, and back
template <class R>
void sphere_to_grid_util(Ctx &c, int n, const double *X, CT<R> *P) {
  const int nq = (n + 1) / 2;
  if (sphere_fft_ok<R>(c)) {
    sphere_to_grid_exec<R>(c, n, X, P, 1.0 / std::sqrt(c.omega));
  } else {
    BSE_CUDA(cudaMemsetAsync(P, 0, (size_t)nq * c.nr * sizeof(CT<R>), c.stream));
    k::scatter_pairs<R, double>(c, n, X, P, 1.0 / std::sqrt(c.omega));
    fft_exec(c, P, nq, +1);
  }
}

template <class R>
void grid_to_sphere_util(Ctx &c, int n, CT<R> *P, double *Y) {
  const int nq = (n + 1) / 2;
  if (sphere_fft_ok<R>(c)) {
    grid_to_sphere_exec<R>(c, n, P, Y, std::sqrt(c.omega) / c.nr, nullptr, nullptr, c.nocc, 0.0);
  } else {
    fft_exec(c, P, nq, -1);
    k::gather_pairs<R, double>(c, n, P, Y, std::sqrt(c.omega) / c.nr);
  }
}

// a bounded device-side wait gave up: report it (the flag is cleared for the next call)
void check_device_flag(Ctx &c) {
  if (!c.dev_err.get()) return;
  int flag = 0;
  d2h(&flag, c.dev_err.get(), sizeof(int), c);
  if (flag) {
    BSE_CUDA(cudaMemsetAsync(c.dev_err.get(), 0, sizeof(int), c.stream));
    throw Error(BSE_ERR_TIMEOUT, "a device-side wait on the tau stream gave up");
  }
}

// ---------------------------------------------------------------------------------
// work buffers
template <class R>
int apply_block(const Ctx &c) {
  // trial vectors per pass of the Liouville operator, bounded by ~6 GB of packed grids
  const double per = (double)((c.nocc + 1) / 2) * c.nr * sizeof(CT<R>);
  int nb = (int)std::floor(6.0e9 / std::max(per, 1.0));
  return std::max(1, std::min(4, nb));
}
const int kPairBatch = 256;

template <class R>
void ensure_grids(Ctx &c) {
  Grids<R> &g = c.grids<R>();
  const long q_apply = (long)apply_block<R>(c) * c.nocc / 2 + 1;
  const long q_pairs = kPairBatch / 2 + 1;
  const long q = std::max(std::max(q_apply, q_pairs), (long)(c.nocc + 9) / 2 + 1);
  g.work.alloc((size_t)q * c.nr);
  g.work2.alloc((size_t)q * c.nr);
  g.sbuf.alloc((size_t)std::max(kPairBatch, c.nocc) * c.npw);
  g.qbuf.alloc((size_t)kPairBatch * std::max(1, c.npdep));
  // the Liouville apply's own buffers, sized once for its largest block (their addresses are
  // recorded by captured graphs)
  const int nbmax = apply_block<R>(c);
  g.vh.alloc((size_t)((nbmax + 1) / 2) * c.nr);
  g.colbuf_apply.alloc((size_t)((nbmax * c.nocc + 1) / 2) * c.N[2] * c.sfft.ncols_pad);
  if (std::is_same<R, float>::value) {
    c.pc32.alloc((size_t)nbmax * c.nocc * (c.npw + c.nocc));
    c.apply_s32.alloc((size_t)1 << 20);
  }
  c.apply_s64.alloc((size_t)1 << 20);
}

void ensure_work(Ctx &c) {
  if (c.prec == 0) {
    ensure_grids<double>(c);
  } else {
    // FP64 grids only for the ground state, phi(r) and the force densities
    c.g64.work.alloc((size_t)std::max<long>(32, (c.nocc + 9) / 2 + 1) * c.nr);
    if (c.hartree) {
      // the FP64 residual of the Z-vector refinement applies the coupled operator (apply op 2)
      // on FP64 grids, one vector at a time
      Grids<double> &g = c.g64;
      g.work2.alloc((size_t)((c.nocc + 1) / 2) * c.nr);
      g.vh.alloc(c.nr);
      g.colbuf_apply.alloc((size_t)((c.nocc + 1) / 2) * c.N[2] * c.sfft.ncols_pad);
    }
    ensure_grids<float>(c);
    c.dev_err.alloc(1);
    BSE_CUDA(cudaMemsetAsync(c.dev_err.get(), 0, sizeof(int), c.stream));
  }
  c.smat.alloc((size_t)std::max<long>(4L * c.nocc * c.nocc, 4096));
}

// ---------------------------------------------------------------------------------
// operators on real-basis vectors
// HX = H X for k functions [k][npw] on grids of type R; shift (device, period nocc) adds shift_v X
template <class R>
void apply_h(Ctx &c, int kf, const double *X, double *HX, const double *shift) {
  Grids<R> &g = c.grids<R>();
  long cap = (long)(g.work.n / c.nr) * 2;
  if (sphere_fft_ok<R>(c)) {
    // sphere-pruned: z pass, fused (inverse, V(r), forward) plane pass, z pass with the gather
    cap = shift ? std::max<long>(c.nocc, 512 / c.nocc * c.nocc) : 512;  // chunks start at orbital 0
    for (int f0 = 0; f0 < kf; f0 += (int)cap) {
      const int nf = (int)std::min<long>(cap, kf - f0);
      sphere_h_exec<R>(c, nf, X + (long)f0 * c.npw, HX + (long)f0 * c.npw, shift);
    }
    return;
  }
  if (shift && cap >= c.nocc) cap -= cap % c.nocc;  // chunks start on an orbital-0 boundary
  for (int f0 = 0; f0 < kf; f0 += (int)cap) {
    const int nf = (int)std::min<long>(cap, kf - f0);
    const int nq = (nf + 1) / 2;
    BSE_CUDA(cudaMemsetAsync(g.work.get(), 0, (size_t)nq * c.nr * sizeof(CT<R>), c.stream));
    k::scatter_pairs<R, double>(c, nf, X + (long)f0 * c.npw, g.work.get(), 1.0 / std::sqrt(c.omega));
    fft_exec(c, g.work.get(), nq, +1);
    k::mul_grid<R>(c.nr, nq, g.work.get(), g.vloc.get(), (R)1, c.stream);
    fft_exec(c, g.work.get(), nq, -1);
    k::gather_pairs<R, double>(c, nf, g.work.get(), HX + (long)f0 * c.npw, std::sqrt(c.omega) / c.nr,
                               X + (long)f0 * c.npw, shift ? shift : nullptr, c.nocc, 0.0);
  }
}

// P_c X for rows of `nf` functions with the occupied orbitals (nf = nvec * nocc); keeps S if asked
// (fixed: split-K scratch of fixed size, for the apply path whose launches may be captured)
void project_pc(Ctx &c, int nf, double *X, double *S_keep, DevBuf<double> *fixed = nullptr) {
  double *S = c.smat.get();
  DevBuf<double> big;
  if ((size_t)nf * c.nocc > c.smat.n) {
    big.alloc((size_t)nf * c.nocc);
    S = big.get();
  }
  dgemm('N', 'T', nf, c.nocc, c.npw, 1.0, X, c.npw, c.phi.get(), c.npw, 0.0, S, c.nocc, c.stream, fixed,
        c.gemm_split_pct);
  if (S_keep) d2d(S_keep, S, (size_t)nf * c.nocc * sizeof(double), c);
  dgemm('N', 'N', nf, c.npw, c.nocc, -1.0, S, c.nocc, c.phi.get(), c.npw, 1.0, X, c.npw, c.stream, fixed,
        c.gemm_split_pct);
}

// P_c X with FP32 overlaps (the FP32-grid operator of the mixed path): S = X phi^T and X -= S phi
// through FP32 copies; X itself stays FP64
void project_pc32(Ctx &c, int nf, double *X, DevBuf<float> *fixed = nullptr) {
  const long n = (long)nf * c.npw;
  c.pc32.alloc((size_t)n + (size_t)nf * c.nocc);
  float *Xf = c.pc32.get();
  float *Sf = Xf + n;
  k::convert(n, X, Xf, c.stream);
  sgemm('N', 'T', nf, c.nocc, c.npw, 1.0f, Xf, c.npw, c.phi32.get(), c.npw, 0.0f, Sf, c.nocc, c.stream, fixed,
        c.gemm_split_pct);
  sgemm('N', 'N', nf, c.npw, c.nocc, 1.0f, Sf, c.nocc, c.phi32.get(), c.npw, 0.0f, Xf, c.npw, c.stream, fixed,
        c.gemm_split_pct);
  k::sub_f32(n, X, Xf, c.stream);
}

// P_c in the precision of the grids R (the overlaps are kept only by the FP64 route); the
// Liouville apply passes its fixed-size scratch
template <class R>
void project_pc_t(Ctx &c, int nf, double *X, double *S_keep, bool apply_scratch = false) {
  if (std::is_same<R, float>::value && !S_keep) project_pc32(c, nf, X, apply_scratch ? &c.apply_s32 : nullptr);
  else project_pc(c, nf, X, S_keep, apply_scratch ? &c.apply_s64 : nullptr);
}

// project each block of nocc rows (a trial vector) on P_c
void project_vectors(Ctx &c, int nvec, double *X) { project_pc(c, nvec * c.nocc, X, nullptr); }

// L A for nvec trial vectors (op 0), P_c (H - eps_v) (op 1), or the Z-vector operator of the
// Hartree model (op 2: P_c (H - eps_v) Z_v + (2 K1e,KS + 2 K2e,KS) Z = ... + 4 P_c [v_c * sum_v'
// phi_v' Z_v'] phi_v, Eq. 7 with f_Hxc = v_c) with grids of type R
template <class R>
void apply_liouville_t(Ctx &c, int nvec, const double *A, double *LA, int op, double *S_keep, R *vh_keep,
                       const R *k1d_grid = nullptr) {
  const long vlen = (long)c.nocc * c.npw;
  if (op == 1) {
    apply_h<R>(c, nvec * c.nocc, A, LA, c.negeps.get());
    project_pc_t<R>(c, nvec * c.nocc, LA, nullptr, true);
    return;
  }
  Grids<R> &g = c.grids<R>();
  const bool zop = op == 2;
  const bool k1e = zop || ((c.spin == 0) && !(c.flags & BSE_FLAG_NO_K1E));
  // k1d_grid (one vector): -K1d a computed elsewhere on the grid, added instead of the cached tau
  const bool k1d = !zop && !(c.flags & BSE_FLAG_NO_K1D) && !k1d_grid;
  BSE_REQUIRE(!k1d_grid || nvec == 1, "internal: an external K1d grid serves one vector");
  BSE_REQUIRE(!k1d || !c.wan.on, "internal: the canonical tau is not cached under Wannier pair pruning");
  // the combine kernels add 2 v_H phi_v: the Z-vector operator's kernel is twice the BSE's
  const double vh_scale = zop ? 2.0 : 1.0;
  const double scissor = zop ? 0.0 : c.scissor;
  int nbmax = apply_block<R>(c);
  DevBuf<CT<R>> &vh = g.vh;  // sized at setup
  // the block may not exceed the buffers sized at setup (the FP64 grids of the mixed path hold one
  // vector)
  nbmax = std::min<long>(nbmax, std::min<long>(2 * (long)(vh.n / c.nr), (long)(g.work2.n / c.nr) * 2 / c.nocc));
  nbmax = std::min<long>(nbmax, std::min<long>((long)(g.work.n / c.nr) * 2 / c.nocc, std::max(1, nvec)));
  if (!(nbmax >= 1 && g.work.n >= (size_t)((nbmax * c.nocc + 1) / 2) * c.nr))
    throw Error(BSE_ERR_INVALID, "internal: Liouville apply buffers not allocated for this precision (grid bytes " +
                                     std::to_string(sizeof(R)) + ", op " + std::to_string(op) + ", block " +
                                     std::to_string(nbmax) + ", work " + std::to_string(g.work.n / c.nr) +
                                     ", work2 " + std::to_string(g.work2.n / c.nr) + ", vh " +
                                     std::to_string(g.vh.n / c.nr) + " grids)");
  BSE_REQUIRE(!sphere_fft_ok<R>(c) ||
                  g.colbuf_apply.n >= (size_t)((nbmax * c.nocc + 1) / 2) * c.N[2] * c.sfft.ncols_pad,
              "internal: column buffer of the Liouville apply too small");
  for (int b0 = 0; b0 < nvec; b0 += nbmax) {
    const int nb = std::min(nbmax, nvec - b0);
    const int nf = nb * c.nocc;
    const int nq = (nf + 1) / 2;
    const double *Ab = A + (long)b0 * vlen;
    double *LAb = LA + (long)b0 * vlen;
    if (sphere_fft_ok<R>(c)) {
      sphere_to_grid_exec<R>(c, nf, Ab, g.work.get(), 1.0 / std::sqrt(c.omega), g.colbuf_apply.get());
    } else {
      BSE_CUDA(cudaMemsetAsync(g.work.get(), 0, (size_t)nq * c.nr * sizeof(CT<R>), c.stream));
      k::scatter_pairs<R, double>(c, nf, Ab, g.work.get(), 1.0 / std::sqrt(c.omega));
      fft_exec(c, g.work.get(), nq, +1);
    }
    if (k1e) {
      // v_H = v_c * Delta rho (Eq. 2b)
      const int nqb = (nb + 1) / 2;
      k::drho<R>(c, nb, g.phir.get(), g.work.get(), vh.get());
      fft_exec(c, vh.get(), nqb, -1);
      k::mul_grid<R>(c.nr, nqb, vh.get(), g.vcg.get(), (R)(vh_scale / c.nr), c.stream);
      fft_exec(c, vh.get(), nqb, +1);
      if (vh_keep) k::unpack_real<R, R>(c.nr, 1, vh.get(), vh_keep, c.stream);
    }
    combine_exec<R>(c, nb, g.work.get(), vh.get(), g.work2.get(), k1e, k1d);
    if (k1d_grid) k::add_packed<R>(c.nr, nf, k1d_grid, g.work2.get(), c.stream);
    if (sphere_fft_ok<R>(c)) {
      grid_to_sphere_exec<R>(c, nf, g.work2.get(), LAb, std::sqrt(c.omega) / c.nr, Ab, c.negeps.get(), c.nocc,
                             scissor, g.colbuf_apply.get());
    } else {
      fft_exec(c, g.work2.get(), nq, -1);
      k::gather_pairs<R, double>(c, nf, g.work2.get(), LAb, std::sqrt(c.omega) / c.nr, Ab, c.negeps.get(),
                                 c.nocc, scissor);
    }
    project_pc_t<R>(c, nf, LAb, (S_keep && b0 == 0) ? S_keep : nullptr, true);
  }
  if (!zop) c.stats.n_applies += nvec;
}

// the Liouville operator in the context's precision (FP64 grids, or FP32 grids for mixed)
constexpr int kGraphMaxVec = 8;

// every device address a captured apply may have recorded
std::vector<const void *> apply_fingerprint(const Ctx &c) {
  std::vector<const void *> f = {c.gA.get(), c.gLA.get(), c.pc32.get(), c.smat.get(), c.apply_s64.get(),
                                 c.apply_s32.get(), c.phi.get(), c.phi32.get(), c.negeps.get(), c.kin.get(),
                                 c.k1d.tau, c.dev_err.get(), c.gp.get(), c.gm.get(), c.sfft.colpos.get(),
                                 c.sfft.xs.get(), c.sfft.ent.get(), c.sfft.ent_off.get()};
  for (int a = 0; a < 3; ++a) {
    f.push_back(c.fft.ax[a].tw);
    f.push_back(c.fft.ax[a].tw32);
  }
  auto grids = [&f](const auto &g) {
    for (const void *p : {(const void *)g.work.get(), (const void *)g.work2.get(), (const void *)g.vh.get(),
                          (const void *)g.colbuf_apply.get(), (const void *)g.tau.get(), (const void *)g.phir.get(),
                          (const void *)g.vloc.get(), (const void *)g.vcg.get()})
      f.push_back(p);
  };
  grids(c.g64);
  grids(c.g32);
  return f;
}

void drop_graphs(Ctx &c) {
  for (auto &kv : c.graphs)
    if (kv.second) cudaGraphExecDestroy(kv.second);
  c.graphs.clear();
  c.graph_kernels.clear();
}

template <class R>
void apply_graph(Ctx &c, int nvec, const double *A, double *LA) {
  const size_t len = (size_t)nvec * c.nocc * c.npw;
  const size_t cap = (size_t)kGraphMaxVec * c.nocc * c.npw;
  c.gA.alloc(cap);
  c.gLA.alloc(cap);
  d2d(c.gA.get(), A, len * sizeof(double), c);
  // a buffer that moved since the graphs were captured (a new geometry never moves them; this is
  // the safety net) invalidates them all
  if (!c.graphs.empty() && apply_fingerprint(c) != c.graph_fp) drop_graphs(c);
  auto it = c.graphs.find(nvec);
  if (it == c.graphs.end()) {
    // first block of this size: one plain run (every lazily sized buffer reaches its final size
    // and the result is used), then the same launch sequence is captured
    apply_liouville_t<R>(c, nvec, c.gA.get(), c.gLA.get(), 0, nullptr, nullptr);
    const long long n0 = launch_count_now();
    const long long a0 = tl_alloc_calls;
    cudaGraph_t graph = nullptr;
    BSE_CUDA(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeRelaxed));
    try {
      apply_liouville_t<R>(c, nvec, c.gA.get(), c.gLA.get(), 0, nullptr, nullptr);
    } catch (...) {
      cudaStreamEndCapture(c.stream, &graph);
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      throw;
    }
    BSE_CUDA(cudaStreamEndCapture(c.stream, &graph));
    c.stats.n_applies -= nvec;  // the captured sequence did not run
    const long long nk = launch_count_now() - n0;
    add_launches(-nk);
    if (tl_alloc_calls != a0) {
      // a buffer was allocated inside the sequence: its address would not outlive the call
      cudaGraphDestroy(graph);
      c.use_graphs = false;
      d2d(LA, c.gLA.get(), len * sizeof(double), c);
      return;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    BSE_CUDA(e);
    if (!c.graphs.empty() && apply_fingerprint(c) != c.graph_fp) drop_graphs(c);
    c.graphs[nvec] = exec;
    c.graph_kernels[nvec] = nk;
    c.graph_fp = apply_fingerprint(c);
  } else {
    BSE_CUDA(cudaGraphLaunch(it->second, c.stream));
    add_launches(c.graph_kernels[nvec]);
    c.stats.n_applies += nvec;
  }
  d2d(LA, c.gLA.get(), len * sizeof(double), c);
}

// ---- autotuner ----------------------------------------------------------------------------
// On a context's first Liouville apply: time every candidate launch shape (transform path; trial
// vectors per K1d pass on the TMA path) on the caller's block with CUDA events, keep the fastest.
// Choices are cached per problem shape for the process, so equal systems are tuned once.
struct TuneKey {
  int n1, n2, n3, nocc, npw, prec, flags;
  bool operator<(const TuneKey &o) const {
    return std::tie(n1, n2, n3, nocc, npw, prec, flags) < std::tie(o.n1, o.n2, o.n3, o.nocc, o.npw, o.prec, o.flags);
  }
};
struct TuneChoice {
  bool full_grid;
  int k1d_nb;
  int xy_threads = 0;       // plane-pass threads per CTA (0: the default)
  int gemm_split_pct = 100;  // split-K of the occupied-projection GEMMs, percent of the heuristic
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tune;

void apply_choice(Ctx &c, const TuneChoice &t) {
  c.sfft.disabled = t.full_grid;
  c.k1d_nb_cap = t.k1d_nb;
  c.xy_threads = t.xy_threads;
  c.gemm_split_pct = t.gemm_split_pct;
  c.stats.tuned = 1;
  c.stats.tuned_full_grid_fft = t.full_grid ? 1 : 0;
  c.stats.tuned_k1d_nb = t.k1d_nb;
  c.stats.tuned_xy_threads = t.xy_threads;
  c.stats.tuned_gemm_split_pct = t.gemm_split_pct;
}

template <class R>
void autotune(Ctx &c, int nvec, const double *A, double *LA) {
  const TuneKey key{c.N[0], c.N[1], c.N[2], c.nocc, c.npw, c.prec, c.flags};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      apply_choice(c, it->second);
      return;
    }
  }
  std::vector<bool> ffts{c.sfft.disabled};
  if (c.sfft.ready && (sizeof(R) == sizeof(double) ? c.sfft.ok64 : c.sfft.ok32)) ffts = {false, true};
  std::vector<int> nbs{0};
  if (std::is_same<R, float>::value && c.k1d.ready) {
    nbs.clear();
    for (int nb = 1; nb <= k1d_tma_max_nb(c.nocc); ++nb) nbs.push_back(nb);
  }
  cudaEvent_t e0, e1;
  BSE_CUDA(cudaEventCreate(&e0));
  BSE_CUDA(cudaEventCreate(&e1));
  TuneChoice best{c.sfft.disabled, 0};
  float best_ms = 1e30f;
  const long long n_applies = c.stats.n_applies;
  auto trial = [&](const TuneChoice &t, bool warm) {
    apply_choice(c, t);
    if (warm) apply_liouville_t<R>(c, nvec, A, LA, 0, nullptr, nullptr);
    BSE_CUDA(cudaEventRecord(e0, c.stream));
    apply_liouville_t<R>(c, nvec, A, LA, 0, nullptr, nullptr);
    BSE_CUDA(cudaEventRecord(e1, c.stream));
    BSE_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    BSE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best_ms) {
      best_ms = ms;
      best = t;
    }
  };
  // coordinate search: transform path x K1d width, then the plane-pass width of the sphere-pruned
  // transforms (FFT tile shape), then the split-K of the occupied-projection GEMMs (GEMM tile shape)
  // (a new transform path or K1d width gets a warm-up apply; the later knobs reuse every buffer)
  for (bool fg : ffts)
    for (int nb : nbs) trial(TuneChoice{fg, nb, 0, 100}, true);
  if (!best.full_grid) {
    TuneChoice t = best;
    t.xy_threads = 256;
    trial(t, false);
  }
  for (int pct : {50, 200}) {
    TuneChoice t = best;
    t.gemm_split_pct = pct;
    trial(t, false);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c.stats.n_applies = n_applies;  // tuning runs are not solver applies
  apply_choice(c, best);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[key] = best;
}

// L~ A~ for nvec trial vectors in the Wannier gauge with the K1d pairs pruned (grids of type R):
// (L~ A~)_i = P_c [H a~_i - sum_j eps~_ij a~_j + Delta a~_i + 2 v_H w_i - sum_{j kept} tau~_ji a~_j]
template <class R>
void apply_wannier_t(Ctx &c, int nvec, const double *A, double *LA) {
  Grids<R> &g = c.grids<R>();
  WannierPrune &W = c.wan;
  const long vlen = (long)c.nocc * c.npw;
  const bool k1e = (c.spin == 0) && !(c.flags & BSE_FLAG_NO_K1E);
  const bool k1d = !(c.flags & BSE_FLAG_NO_K1D);
  int nbmax = apply_block<R>(c);
  nbmax = std::min<long>(nbmax, std::min<long>(2 * (long)(g.vh.n / c.nr), (long)(g.work2.n / c.nr) * 2 / c.nocc));
  nbmax = std::min<long>(nbmax, std::min<long>((long)(g.work.n / c.nr) * 2 / c.nocc, std::max(1, nvec)));
  BSE_REQUIRE(nbmax >= 1, "internal: apply buffers not allocated");
  for (int b0 = 0; b0 < nvec; b0 += nbmax) {
    const int nb = std::min(nbmax, nvec - b0);
    const int nf = nb * c.nocc;
    const int nq = (nf + 1) / 2;
    const double *Ab = A + (long)b0 * vlen;
    double *LAb = LA + (long)b0 * vlen;
    if (sphere_fft_ok<R>(c)) {
      sphere_to_grid_exec<R>(c, nf, Ab, g.work.get(), 1.0 / std::sqrt(c.omega), g.colbuf_apply.get());
    } else {
      BSE_CUDA(cudaMemsetAsync(g.work.get(), 0, (size_t)nq * c.nr * sizeof(CT<R>), c.stream));
      k::scatter_pairs<R, double>(c, nf, Ab, g.work.get(), 1.0 / std::sqrt(c.omega));
      fft_exec(c, g.work.get(), nq, +1);
    }
    if (k1e) {
      const int nqb = (nb + 1) / 2;
      k::drho<R>(c, nb, g.wphir.get(), g.work.get(), g.vh.get());
      fft_exec(c, g.vh.get(), nqb, -1);
      k::mul_grid<R>(c.nr, nqb, g.vh.get(), g.vcg.get(), (R)(1.0 / c.nr), c.stream);
      fft_exec(c, g.vh.get(), nqb, +1);
    }
    {
      cudaEvent_t stop;
      const double bytes = (double)W.npairs * c.nr * sizeof(R) + 2.0 * nb * c.nocc * c.nr * sizeof(R);
      c.prof.begin(c.stream, BSE_KERNEL_K1D, bytes, 2.0 * nb * (2.0 * W.npairs - c.nocc) * c.nr, &stop);
      k::combine_pruned<R>(c, nb, g.wphir.get(), g.vloc.get(), g.wtau.get(), W.off.get(), W.nbr.get(), g.work.get(),
                           g.vh.get(), g.work2.get(), k1e, k1d);
      if (stop) BSE_CUDA(cudaEventRecord(stop, c.stream));
    }
    if (sphere_fft_ok<R>(c)) {
      grid_to_sphere_exec<R>(c, nf, g.work2.get(), LAb, std::sqrt(c.omega) / c.nr, Ab, nullptr, c.nocc, c.scissor,
                             g.colbuf_apply.get());
    } else {
      fft_exec(c, g.work2.get(), nq, -1);
      k::gather_pairs<R, double>(c, nf, g.work2.get(), LAb, std::sqrt(c.omega) / c.nr, Ab, nullptr, c.nocc,
                                 c.scissor);
    }
    // the D term's eps matrix in the Wannier gauge
    for (int b = 0; b < nb; ++b)
      dgemm('N', 'N', c.nocc, c.npw, c.nocc, -1.0, W.epst.get(), c.nocc, Ab + (long)b * vlen, c.npw, 1.0,
            LAb + (long)b * vlen, c.npw, c.stream);
    project_pc_t<R>(c, nf, LAb, nullptr, true);
  }
}

void apply_liouville(Ctx &c, int nvec, const double *A, double *LA, int op) {
  if (op == 0 && c.wan.on) {
    // the pruned operator in the canonical gauge: U L~ U^T
    WannierPrune &W = c.wan;
    const long vlen = (long)c.nocc * c.npw;
    W.rot.alloc((size_t)2 * nvec * vlen);
    double *At = W.rot.get(), *LAt = W.rot.get() + (size_t)nvec * vlen;
    for (int b = 0; b < nvec; ++b)
      dgemm('T', 'N', c.nocc, c.npw, c.nocc, 1.0, W.U.get(), c.nocc, A + (long)b * vlen, c.npw, 0.0,
            At + (long)b * vlen, c.npw, c.stream);
    if (c.prec == 0) apply_wannier_t<double>(c, nvec, At, LAt);
    else apply_wannier_t<float>(c, nvec, At, LAt);
    for (int b = 0; b < nvec; ++b)
      dgemm('N', 'N', c.nocc, c.npw, c.nocc, 1.0, W.U.get(), c.nocc, LAt + (long)b * vlen, c.npw, 0.0,
            LA + (long)b * vlen, c.npw, c.stream);
    c.stats.n_applies += nvec;
    return;
  }
  if (op == 0 && c.autotune && !c.stats.tuned) {
    if (c.prec == 0) autotune<double>(c, nvec, A, LA);
    else autotune<float>(c, nvec, A, LA);
  }
  const bool graph = c.use_graphs && op == 0 && !c.prof.on && nvec <= kGraphMaxVec && !c.wan.on;
  if (c.prec == 0) {
    if (graph) apply_graph<double>(c, nvec, A, LA);
    else apply_liouville_t<double>(c, nvec, A, LA, op, nullptr, nullptr);
  } else {
    if (graph) apply_graph<float>(c, nvec, A, LA);
    else apply_liouville_t<float>(c, nvec, A, LA, op, nullptr, nullptr);
    if (op == 0) check_device_flag(c);
  }
}

// ---------------------------------------------------------------------------------
// block Davidson with deflation against Q (device, orthonormal rows)
struct DavSpec {
  long n = 0;
  int nwant = 1, block = 1, maxsub = 8, maxit = 100;
  double tol = 1e-9;
  const double *Q = nullptr;
  int nq = 0;
  std::function<void(int, const double *, double *)> apply;
  std::function<void(int, double *, const double *)> precond;  // (k, T in/out, theta_dev)
  std::function<void(int, double *)> project;
  bool fp32 = false;  // subspace products in FP32 (FP32-level tolerances only)
  int keep = 0;       // Ritz vectors kept at a restart (0: block)
};
struct DavOut {
  std::vector<double> theta, res;
  int iters = 0;
  bool converged = false;
};

// C = alpha op(A) op(B) + beta C.  With fp32 the product is taken in FP32 (operands rounded,
// FP32 accumulation) and only the update is FP64: the subspace arithmetic of the ground-state
// chunks that are converged with the FP32-grid Hamiltonian to FP32-level tolerances.
void gemm_p(Ctx &c, bool fp32, char ta, char tb, int M, int N, int K, double alpha, const double *A, int lda,
            const double *B, int ldb, double beta, double *C, int ldc) {
  if (!fp32 || M <= 0 || N <= 0 || K <= 0) {
    dgemm(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, c.stream);
    return;
  }
  mgemm(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, c.stream);
}

// W = L^-1 for the Cholesky factor G = L L^T of a symmetric positive definite n x n matrix
// (row-major, lower triangle used); false when a pivot L_ii^2 falls below floor.  min_ratio (may
// be null): the smallest L_jj^2 / G_jj, the part of column j's squared norm outside the span of
// the columns before it
bool cholesky_inverse(int n, const std::vector<double> &G, double floor, std::vector<double> &W,
                      double *min_ratio = nullptr) {
  std::vector<double> L((size_t)n * n, 0.0);
  if (min_ratio) *min_ratio = 1.0;
  for (int j = 0; j < n; ++j) {
    double d = G[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
    if (!(d > floor)) return false;
    if (min_ratio && G[(size_t)j * n + j] > 0.0) *min_ratio = std::min(*min_ratio, d / G[(size_t)j * n + j]);
    const double ljj = std::sqrt(d);
    L[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double x = G[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) x -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      L[(size_t)i * n + j] = x / ljj;
    }
  }
  // forward substitution column by column: L W = I
  W.assign((size_t)n * n, 0.0);
  for (int col = 0; col < n; ++col) {
    for (int i = col; i < n; ++i) {
      double x = i == col ? 1.0 : 0.0;
      for (int k = col; k < i; ++k) x -= L[(size_t)i * n + k] * W[(size_t)k * n + col];
      W[(size_t)i * n + col] = x / L[(size_t)i * n + i];
    }
  }
  return true;
}

// orthonormalise k rows of T (device) against V (m rows) and Q (nq rows); returns the rank kept
int orthonormalize(Ctx &c, long n, double *T, int kk, const double *V, int m, const double *Q, int nq,
                   bool fp32 = false) {
  if (kk <= 0) return 0;
  std::vector<double> d0(kk);
  DevBuf<double> dd, C, tmp;
  dd.alloc(kk);
  rowdot(kk, n, T, T, dd.get(), c.stream);
  d2h(d0.data(), dd.get(), kk * sizeof(double), c);
  double ref = 0.0;
  for (double x : d0) ref = std::max(ref, x);
  if (!(ref > 0.0) || !std::isfinite(ref)) return 0;
  C.alloc((size_t)kk * std::max(std::max(m, nq), kk));
  tmp.alloc((size_t)kk * n);
  bool once = false;
  for (int pass = 0; pass < 2; ++pass) {
    // classical Gram-Schmidt against V and Q, then Cholesky QR of the block; a second pass only
    // when the first cancelled: "twice is enough" (Kahan-Parlett; Giraud, Langou and Rozloznik),
    // and once is enough when every vector kept at least half its squared norm through the
    // projection and through the Cholesky pivots (its loss of orthogonality is then a small
    // multiple of the rounding unit)
    if (m > 0) {
      gemm_p(c, fp32, 'N', 'T', kk, m, (int)n, 1.0, T, (int)n, V, (int)n, 0.0, C.get(), m);
      gemm_p(c, fp32, 'N', 'N', kk, (int)n, m, -1.0, C.get(), m, V, (int)n, 1.0, T, (int)n);
    }
    if (nq > 0) {
      gemm_p(c, fp32, 'N', 'T', kk, nq, (int)n, 1.0, T, (int)n, Q, (int)n, 0.0, C.get(), nq);
      gemm_p(c, fp32, 'N', 'N', kk, (int)n, nq, -1.0, C.get(), nq, Q, (int)n, 1.0, T, (int)n);
    }
    // symmetric orthonormalisation, dropping directions with relative norm below 1e-9 (1e-5 when
    // the Gram matrix is FP32: below that its eigenvectors are rounding noise)
    std::vector<double> G((size_t)kk * kk), w(kk), U((size_t)kk * kk);
    gemm_p(c, fp32, 'N', 'T', kk, kk, (int)n, 1.0, T, (int)n, T, (int)n, 0.0, C.get(), kk);
    d2h(G.data(), C.get(), G.size() * sizeof(double), c);
    std::vector<double> Wm;
    int kept = 0;
    {
      auto te = clk::now();
      // Cholesky QR when the block is well conditioned; otherwise the symmetric (Loewdin) form,
      // which can drop dependent directions
      double gmax = 0.0;
      for (int i = 0; i < kk; ++i) gmax = std::max(gmax, G[(size_t)i * kk + i]);
      double pivot_ratio = 0.0;
      if (cholesky_inverse(kk, G, (fp32 ? 1e-6 : 1e-12) * gmax, Wm, &pivot_ratio)) {
        kept = kk;
        if (pass == 0 && pivot_ratio >= 0.5) {
          once = true;
          for (int i = 0; i < kk; ++i)
            if (!(G[(size_t)i * kk + i] >= 0.5 * d0[i])) once = false;
        }
      } else {
        sym_eig(kk, G.data(), w.data(), U.data());
        Wm.clear();
        for (int j = kk - 1; j >= 0; --j) {
          if (!(w[j] > (fp32 ? 1e-10 : 1e-18) * ref)) continue;
          const double s = 1.0 / std::sqrt(w[j]);
          for (int i = 0; i < kk; ++i) Wm.push_back(U[(size_t)i * kk + j] * s);
          ++kept;
        }
      }
      c.stats.ms_host_eig += ms_since(te);
    }
    if (kept == 0) return 0;
    h2d(C.get(), Wm.data(), Wm.size() * sizeof(double), c);
    gemm_p(c, fp32, 'N', 'N', kept, (int)n, kk, 1.0, C.get(), kk, T, (int)n, 0.0, tmp.get(), (int)n);
    d2d(T, tmp.get(), (size_t)kept * n * sizeof(double), c);
    kk = kept;
    ref = 1.0;
    if (once) break;
  }
  return kk;
}

// Block Davidson with thick restarts.  The projected matrix H = V (A V)^T is kept on the host and
// grown by the rows of each new block only (k x m products instead of m x m per iteration); at a
// restart the `keep` lowest Ritz vectors (with their A images) become the new basis and H their
// Ritz values.
DavOut davidson(Ctx &c, const DavSpec &sp, const double *X0, int k0, double *Xout) {
  const long n = sp.n;
  const int S = sp.maxsub;
  const int keep = std::max(1, std::min(sp.keep > 0 ? sp.keep : sp.block, S / 2));
  DevBuf<double> V, AV, X, AX, T, th, rn, small, Xk, AXk;
  V.alloc((size_t)S * n);
  AV.alloc((size_t)S * n);
  X.alloc((size_t)sp.block * n);
  AX.alloc((size_t)sp.block * n);
  T.alloc((size_t)std::max(sp.block, k0) * n);
  th.alloc(sp.block);
  rn.alloc(sp.block);
  small.alloc((size_t)S * S);
  DavOut out;
  d2d(T.get(), X0, (size_t)k0 * n * sizeof(double), c);
  if (sp.project) sp.project(k0, T.get());
  int kk = orthonormalize(c, n, T.get(), k0, nullptr, 0, sp.Q, sp.nq, sp.fp32);
  BSE_REQUIRE(kk > 0, "Davidson: initial block has no component outside the deflated space");
  d2d(V.get(), T.get(), (size_t)kk * n * sizeof(double), c);
  sp.apply(kk, V.get(), AV.get());
  std::vector<double> H((size_t)S * S, 0.0), Hn;
  // rows [m0, m1) of H: V_i . (A V)_j for j < m1; the old-new entries are mirrored (A is
  // symmetric on the P_c space), the new-new block is symmetrised
  auto grow = [&](int m0, int m1) {
    const int k = m1 - m0;
    gemm_p(c, sp.fp32, 'N', 'T', k, m1, (int)n, 1.0, V.get() + (size_t)m0 * n, (int)n, AV.get(), (int)n, 0.0,
           small.get(), m1);
    Hn.resize((size_t)k * m1);
    d2h(Hn.data(), small.get(), Hn.size() * sizeof(double), c);
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < m1; ++j) {
        const int gi = m0 + i;
        const double v = Hn[(size_t)i * m1 + j];
        if (j < m0) {
          H[(size_t)gi * S + j] = v;
          H[(size_t)j * S + gi] = v;
        } else if (j >= gi) {
          const double u = Hn[(size_t)(j - m0) * m1 + gi];
          H[(size_t)gi * S + j] = H[(size_t)j * S + gi] = 0.5 * (v + u);
        }
      }
  };
  int m = kk;
  grow(0, m);
  std::vector<double> Hs, w, Y, Yb;
  for (int it = 1;; ++it) {
    out.iters = it;
    Hs.resize((size_t)m * m);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) Hs[(size_t)i * m + j] = H[(size_t)i * S + j];
    w.resize(m);
    Y.resize((size_t)m * m);
    {
      auto te = clk::now();
      // vectors only for the Ritz pairs this iteration can use: the corrected block, and the
      // `keep` lowest when the new directions could overflow the subspace (a thick restart)
      const bool may_restart = m + std::min(sp.block, m) > S;
      sym_eig_lowest(m, Hs.data(), std::min(m, may_restart ? std::max(sp.block, keep) : sp.block), w.data(),
                     Y.data(), false);
      c.stats.ms_host_eig += ms_since(te);
    }
    const int nb = std::min(sp.block, m);
    Yb.resize((size_t)m * nb);
    for (int j = 0; j < m; ++j)
      for (int r = 0; r < nb; ++r) Yb[(size_t)j * nb + r] = Y[(size_t)j * m + r];
    h2d(small.get(), Yb.data(), Yb.size() * sizeof(double), c);
    gemm_p(c, sp.fp32, 'T', 'N', nb, (int)n, m, 1.0, small.get(), nb, V.get(), (int)n, 0.0, X.get(), (int)n);
    gemm_p(c, sp.fp32, 'T', 'N', nb, (int)n, m, 1.0, small.get(), nb, AV.get(), (int)n, 0.0, AX.get(), (int)n);
    h2d(th.get(), w.data(), nb * sizeof(double), c);
    k::residual(nb, n, AX.get(), X.get(), th.get(), T.get(), c.stream);
    rowdot(nb, n, T.get(), T.get(), rn.get(), c.stream);
    std::vector<double> r2(nb);
    d2h(r2.data(), rn.get(), nb * sizeof(double), c);
    out.theta.assign(w.begin(), w.begin() + nb);
    out.res.resize(nb);
    if (verbose())
      std::fprintf(stderr, "[bse davidson] n=%ld it=%d m=%d theta0=%.12f res0=%.3e\n", n, it, m, w[0],
                   std::sqrt(std::max(0.0, r2[0])));
    bool conv = true;
    for (int r = 0; r < nb; ++r) {
      out.res[r] = std::sqrt(std::max(0.0, r2[r]));
      if (r < sp.nwant && !(out.res[r] <= sp.tol)) conv = false;
    }
    if (conv || it >= sp.maxit) {
      out.converged = conv;
      d2d(Xout, X.get(), (size_t)sp.nwant * n * sizeof(double), c);
      sync(c);
      return out;
    }
    // corrections for the unconverged Ritz vectors
    std::vector<double> thsel;
    int nsel = 0;
    for (int r = 0; r < nb; ++r) {
      if (out.res[r] <= sp.tol) continue;
      if (nsel != r) d2d(T.get() + (size_t)nsel * n, T.get() + (size_t)r * n, n * sizeof(double), c);
      thsel.push_back(w[r]);
      ++nsel;
    }
    h2d(th.get(), thsel.data(), nsel * sizeof(double), c);
    sp.precond(nsel, T.get(), th.get());
    if (sp.project) sp.project(nsel, T.get());
    if (m + nsel > S) {
      // thick restart on the `keep` lowest Ritz vectors
      const int nk = std::min(std::max(keep, nb), m);
      if (nk == nb) {
        d2d(V.get(), X.get(), (size_t)nb * n * sizeof(double), c);
        d2d(AV.get(), AX.get(), (size_t)nb * n * sizeof(double), c);
      } else {
        Xk.alloc((size_t)nk * n);
        AXk.alloc((size_t)nk * n);
        Yb.resize((size_t)m * nk);
        for (int j = 0; j < m; ++j)
          for (int r = 0; r < nk; ++r) Yb[(size_t)j * nk + r] = Y[(size_t)j * m + r];
        h2d(small.get(), Yb.data(), Yb.size() * sizeof(double), c);
        gemm_p(c, sp.fp32, 'T', 'N', nk, (int)n, m, 1.0, small.get(), nk, V.get(), (int)n, 0.0, Xk.get(), (int)n);
        gemm_p(c, sp.fp32, 'T', 'N', nk, (int)n, m, 1.0, small.get(), nk, AV.get(), (int)n, 0.0, AXk.get(),
               (int)n);
        d2d(V.get(), Xk.get(), (size_t)nk * n * sizeof(double), c);
        d2d(AV.get(), AXk.get(), (size_t)nk * n * sizeof(double), c);
      }
      std::fill(H.begin(), H.end(), 0.0);
      for (int r = 0; r < nk; ++r) H[(size_t)r * S + r] = w[r];
      m = nk;
    }
    int knew = orthonormalize(c, n, T.get(), nsel, V.get(), m, sp.Q, sp.nq, sp.fp32);
    knew = std::min(knew, S - m);
    if (knew <= 0) {
      out.converged = false;
      d2d(Xout, X.get(), (size_t)sp.nwant * n * sizeof(double), c);
      sync(c);
      return out;
    }
    d2d(V.get() + (size_t)m * n, T.get(), (size_t)knew * n * sizeof(double), c);
    sp.apply(knew, V.get() + (size_t)m * n, AV.get() + (size_t)m * n);
    grow(m, m + knew);
    m += knew;
  }
}

// ---------------------------------------------------------------------------------
// geometry stage: V, ground state, tau
// atom data on the device: positions, well depths, widths and (when given) ionic charges
struct AtomArgs {
  DevBuf<double> pd, zd, sd, qd;
  AtomArgs(Ctx &c) {
    pd.alloc(c.natoms * 3);
    zd.alloc(c.natoms);
    sd.alloc(c.natoms);
    h2d(pd.get(), c.pos.data(), c.natoms * 3 * sizeof(double), c);
    h2d(zd.get(), c.Z.data(), c.natoms * sizeof(double), c);
    h2d(sd.get(), c.sigma.data(), c.natoms * sizeof(double), c);
    if (!c.q.empty()) {
      qd.alloc(c.natoms);
      h2d(qd.get(), c.q.data(), c.natoms * sizeof(double), c);
    }
  }
  const double *q() const { return qd.n ? qd.get() : nullptr; }
};

// the local potential of H on the grids: V_ext, plus v_H when given (Hartree model)
void set_local_potential(Ctx &c, const double *vh) {
  Grids<double> &g = c.g64;
  g.vloc.alloc(c.nr);
  d2d(g.vloc.get(), c.vext.get(), c.nr * sizeof(double), c);
  if (vh) row_axpby(1, c.nr, nullptr, g.vloc.get(), nullptr, vh, c.stream);
  if (c.prec == 1) {
    c.g32.vloc.alloc(c.nr);
    k::convert(c.nr, g.vloc.get(), c.g32.vloc.get(), c.stream);
  }
}

void compute_vloc(Ctx &c) {
  AtomArgs at(c);
  Grids<double> &g = c.g64;
  k::vloc_G(c, at.pd.get(), at.zd.get(), at.sd.get(), at.q(), g.work.get());
  fft_exec(c, g.work.get(), 1, +1);
  c.vext.alloc(c.nr);
  k::unpack_real<double, double>(c.nr, 1, g.work.get(), c.vext.get(), c.stream);
  set_local_potential(c, nullptr);
  c.v0 = 0.0;
  for (int a = 0; a < c.natoms; ++a)
    c.v0 += -c.Z[a] * std::pow(2.0 * M_PI * c.sigma[a] * c.sigma[a], 1.5) / c.omega;
  sync(c);
}

// Empty states solved with the occupied ones: the first kTightEmpty to the ground-state
// tolerance (the LUMO, and the transitions near the gap in which the BSE preconditioner divides
// by small eps_c - eps_v - theta), up to kPrecEmpty more loosely; they span the low-energy part
// of the unoccupied space in which the BSE preconditioner is exact.
const int kTightEmpty = 4;
const int kPrecEmpty = 64;
const double kLooseTol = 1e-3;

int gs_nstates(const Ctx &c, bool with_empty) {
  const int n = c.npw;
  const int nwant_guard = std::min(c.nocc + kTightEmpty, n);
  return with_empty ? std::min(c.nocc + kPrecEmpty, std::max(nwant_guard, n / 2)) : c.nocc;
}

// Lowest states of the current H (local potential g.vloc) to residual norm gtol: the occupied
// ones, and with_empty kTightEmpty more plus the loosely solved empty states (without: the
// occupied states alone, as inside the Hartree SCF loop, where only the density is needed).
// init: ninit starting vectors for the lowest states, whose signs the result keeps; the other
// states start from unit vectors on the lowest kinetic energies.
void ground_state(Ctx &c, std::vector<double> &eps_all, DevBuf<double> &Qall, double gtol, const double *init,
                  int ninit, bool with_empty = true) {
  const int n = c.npw;
  const int nwant_tight = with_empty ? std::min(c.nocc + kTightEmpty, n) : c.nocc;
  const int nwant_total = gs_nstates(c, with_empty);
  Qall.alloc((size_t)nwant_total * n);
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return c.kin_h[a] < c.kin_h[b]; });
  // positive-definite kinetic preconditioner (1/2 |G|^2 + s)^-1; s = 1/2 Ha measured fastest over
  // 0.1-2 Ha on the 63-well cells (non-SCF and Hartree: a smaller shift weights the smooth
  // components of the occupied states more, too small a one over-corrects them)
  DevBuf<double> vsh;
  vsh.alloc(1);
  const double shift = 0.5;
  h2d(vsh.get(), &shift, sizeof(double), c);
  double maxres = 0.0;
  int its = 0;
  int guess_off = 0;
  int nchunks = 0;
  // Locked-chunk Davidson for states [from, to): each chunk of up to 44 states (36 buffer vectors)
  // is deflated against the states before it.  init (optional) holds starting vectors per state.
  // Chunk, buffer and subspace depths were chosen by timing on the 63-well cell, where the top of
  // the occupied states lies in a dense spectrum (chunk 48 / buffer 24 / FP32 subspace 2x: 462 ms
  // mixed, 601 ms FP64 per ground state; 44 / 36 / 2.5x: 370 and 568 ms).
  auto solve_chunks = [&](int from, int to, double tol, bool fp32, const double *init, int ninit_k, bool record) {
    int nq = from;
    // loosely converged states go in one chunk of up to 64
    const int maxchunk = tol >= kLooseTol ? 64 : 44;
    while (nq < to) {
      ++nchunks;
      // the chunk's states get corrections; 36 more Ritz vectors ride along in the basis (start
      // block and thick restarts) to separate the chunk's top from the states above it.  The
      // subspace is deeper when the applies are FP64 (they dominate), shallower in FP32 (where
      // the host Rayleigh-Ritz does)
      const int chunk = std::min(maxchunk, to - nq);
      const int block = std::min(chunk + 36, n - nq);
      const int maxsub = std::min(fp32 ? 5 * block / 2 : 3 * block, n - nq);
      DevBuf<double> X0;
      X0.alloc((size_t)block * n);
      const int from_init = init ? std::max(0, std::min(block, ninit_k - nq)) : 0;
      if (from_init > 0) d2d(X0.get(), init + (size_t)nq * n, (size_t)from_init * n * sizeof(double), c);
      if (from_init < block) {
        std::vector<double> x0((size_t)(block - from_init) * n, 0.0);
        for (int i = 0; i < block - from_init; ++i) x0[(size_t)i * n + order[(guess_off + i) % n]] = 1.0;
        guess_off += block - from_init;
        h2d(X0.get() + (size_t)from_init * n, x0.data(), x0.size() * sizeof(double), c);
      }
      DavSpec sp;
      sp.n = n;
      sp.nwant = chunk;
      sp.block = chunk;
      sp.keep = block;
      sp.maxsub = maxsub;
      sp.maxit = 400;
      sp.tol = tol;
      sp.Q = Qall.get();
      sp.nq = nq;
      sp.fp32 = fp32;
      if (fp32) sp.apply = [&](int kk, const double *X, double *AX) { apply_h<float>(c, kk, X, AX, nullptr); };
      else sp.apply = [&](int kk, const double *X, double *AX) { apply_h<double>(c, kk, X, AX, nullptr); };
      sp.precond = [&](int kk, double *T, const double *th) {
        k::precond_diag(kk, n, T, c.kin.get(), n, vsh.get(), 0.0, th, 0.1, T, c.stream);
      };
      DavOut r = davidson(c, sp, X0.get(), block, Qall.get() + (size_t)nq * n);
      its += r.iters;
      if (record)
        for (int i = 0; i < chunk; ++i) maxres = std::max(maxres, r.res[i]);
      if (!r.converged) throw Error(BSE_ERR_NOT_CONVERGED, "ground-state Davidson did not converge");
      nq += chunk;
    }
  };
  const double *warm = init;
  ninit = init ? std::min(ninit, nwant_total) : 0;
  if (c.prec == 0) {
    solve_chunks(0, nwant_tight, gtol, false, warm, ninit, true);
    solve_chunks(nwant_tight, nwant_total, std::max(gtol, kLooseTol), false, warm, ninit, false);
  } else {
    // mixed precision: the FP32-grid Hamiltonian carries the bulk of the convergence, then the
    // occupied states and the LUMO are refined with the FP64 Hamiltonian from those vectors.  A
    // tolerance at FP32 level (early Hartree SCF iterations) takes the FP32 phase alone; starting
    // vectors for all the occupied states inside the SCF loop (the previous iteration's, closer
    // than those of a previous geometry) go straight to the FP64 refinement.
    const bool fp32_only = gtol >= 1e-5;
    const bool from_init = !with_empty && init && ninit >= nwant_tight && !fp32_only;
    if (from_init) {
      // the tight states first (the loose ones are deflated against them)
      solve_chunks(0, nwant_tight, gtol, false, warm, ninit, true);
      solve_chunks(nwant_tight, nwant_total, std::max(gtol, kLooseTol), true, warm, ninit, false);
    } else {
      solve_chunks(0, nwant_tight, std::max(gtol, 1e-5), true, warm, ninit, fp32_only);
      solve_chunks(nwant_tight, nwant_total, std::max(gtol, kLooseTol), true, warm, ninit, false);
      if (!fp32_only) {
        DevBuf<double> Qinit;
        Qinit.alloc((size_t)nwant_total * n);
        d2d(Qinit.get(), Qall.get(), (size_t)nwant_total * n * sizeof(double), c);
        solve_chunks(0, nwant_tight, gtol, false, Qinit.get(), nwant_total, true);
      }
    }
    // keep the loosely solved empty states orthogonal to the refined ones
    const int ne = nwant_total - nwant_tight;
    if (ne > 0) {
      const int kept = orthonormalize(c, n, Qall.get() + (size_t)nwant_tight * n, ne, Qall.get(), nwant_tight,
                                      nullptr, 0);
      BSE_REQUIRE(kept == ne, "internal: empty states lost rank after refinement");
    }
  }
  const int nq_done = nwant_total;
  (void)nq_done;
  // final Rayleigh-Ritz over all solved states
  DevBuf<double> HQ, small, tmp;
  HQ.alloc((size_t)nwant_total * n);
  tmp.alloc((size_t)nwant_total * n);
  small.alloc((size_t)nwant_total * nwant_total);
  apply_h<double>(c, nwant_total, Qall.get(), HQ.get(), nullptr);
  std::vector<double> Hs((size_t)nwant_total * nwant_total), Y(Hs.size());
  eps_all.resize(nwant_total);
  dgemm('N', 'T', nwant_total, nwant_total, n, 1.0, Qall.get(), n, HQ.get(), n, 0.0, small.get(), nwant_total,
        c.stream);
  d2h(Hs.data(), small.get(), Hs.size() * sizeof(double), c);
  sym_eig(nwant_total, Hs.data(), eps_all.data(), Y.data());
  h2d(small.get(), Y.data(), Y.size() * sizeof(double), c);
  dgemm('T', 'N', nwant_total, n, nwant_total, 1.0, small.get(), nwant_total, Qall.get(), n, 0.0, tmp.get(), n,
        c.stream);
  d2d(Qall.get(), tmp.get(), (size_t)nwant_total * n * sizeof(double), c);
  sync(c);
  c.stats.gs_iterations += its;
  c.stats.gs_residual = maxres;
  c.stats.gs_chunks += nchunks;
  if (warm && ninit > 0) {
    // keep each state's sign from the starting block (the previous geometry's or SCF
    // iteration's states), so that orbital-indexed vectors built on them stay valid
    DevBuf<double> dots, sg;
    dots.alloc(ninit);
    rowdot(ninit, n, Qall.get(), warm, dots.get(), c.stream);
    std::vector<double> dh(ninit);
    d2h(dh.data(), dots.get(), ninit * sizeof(double), c);
    for (double &x : dh) x = x < 0 ? -1.0 : 1.0;
    sg.alloc(ninit);
    h2d(sg.get(), dh.data(), ninit * sizeof(double), c);
    row_axpby(ninit, n, sg.get(), Qall.get(), nullptr, nullptr, c.stream);
  }
}

// W * rho for np packed real pair densities rho on the grid P, in place (Eq. 2c with Eq. 3):
// the bare Coulomb part 4 pi/|G|^2 on the density sphere plus the PDEP part, a projection of
// v_c^{1/2} rho on the PDEP vectors, lambda/(1 - lambda), and the back-projection.  X, Qm:
// scratch for the PDEP coefficients.  The transforms are the density-sphere-pruned ones when
// they fit, else full-grid FFTs.
template <class R>
void pair_screen(Ctx &c, int np, CT<R> *P, R *X, R *Qm) {
  Grids<R> &g = c.grids<R>();
  const int nq = (np + 1) / 2;
  if (dens_fft_ok<R>(c)) {
    cudaEvent_t stop;
    const double n1 = c.N[0], n2 = c.N[1], n3 = c.N[2];
    const double fl = 5.0 * nq *
                      (c.dfft.ncols * n3 * std::log2(n3) + n3 * (c.dfft.nxs * n2 * std::log2(n2) + n2 * n1 * std::log2(n1)));
    c.prof.begin(c.stream, BSE_KERNEL_SPHERE_FFT, 2.0 * nq * c.nr * sizeof(CT<R>), 2.0 * fl, &stop);
    dens_forward<R>(c, np, P, c.npdep ? X : nullptr, 1.0 / c.nr, g.vcg.get(), (R)(1.0 / c.nr));
    if (c.npdep) pdep_gemms<R>(c, np, X, Qm);
    dens_inverse<R>(c, np, c.npdep ? X : nullptr, 1.0, P);
    if (stop) BSE_CUDA(cudaEventRecord(stop, c.stream));
    if (c.prof.pending.size() > 512) c.prof.flush();
    return;
  }
  fft_exec(c, P, nq, -1);
  if (c.npdep) k::gather_pairs<R, R>(c, np, P, X, 1.0 / c.nr);
  k::mul_grid<R>(c.nr, nq, P, g.vcg.get(), (R)(1.0 / c.nr), c.stream);
  if (c.npdep) {
    // PDEP part of Eq. 3: projection on v_c^{1/2} phi_a, times lambda/(1-lambda), back-projection
    pdep_gemms<R>(c, np, X, Qm);
    k::scatter_pairs<R, R>(c, np, X, P, 1.0, true);
  }
  fft_exec(c, P, nq, +1);
}

// tiled: tau in the tile-major layout of the bulk-copy K1d kernel (FP32 only)
template <class R>
void build_tau_t(Ctx &c, bool tiled = false) {
  const long npairs = c.npairs;
  Grids<R> &g = c.grids<R>();
  g.tau.alloc((size_t)npairs * c.nr);
  c.stats.bytes_tau = (double)npairs * c.nr * sizeof(R);
  const R *phir = g.phir.get();
  R *X = g.sbuf.get();
  R *Qm = g.qbuf.get();
  for (long p0 = 0; p0 < npairs; p0 += kPairBatch) {
    const int np = (int)std::min<long>(kPairBatch, npairs - p0);
    k::pair_products<R>(c.nr, np, c.pairs.get() + p0, phir, phir, g.work.get(), c.stream);
    pair_screen<R>(c, np, g.work.get(), X, Qm);
    if constexpr (std::is_same<R, float>::value) {
      if (tiled) {
        k1d_unpack_tiled(c, np, c.pairs.get() + p0, g.work.get(), g.tau.get());
        continue;
      }
    }
    k::unpack_real<R, R>(c.nr, np, g.work.get(), g.tau.get() + p0 * c.nr, c.stream);
  }
  sync(c);
}

// Gamma-point Wannier localisation of the occupied orbitals (maximising sum_k g_k sum_i
// |<w_i|e^{-i b_k.r}|w_i>|^2, g_k = |a_k|^2/(2 pi)^2, by Jacobi rotations jointly diagonalising the
// cos and sin position matrices; each pair's angle in Cardoso and Souloumiac's closed form), the
// pairs whose centres lie within the cutoff (minimum image), and tau~ for those pairs.
template <class R>
void wannier_tau(Ctx &c) {
  WannierPrune &W = c.wan;
  Grids<R> &g = c.grids<R>();
  const int np_all = W.npairs;
  g.wtau.alloc((size_t)np_all * c.nr);
  c.stats.bytes_tau = (double)np_all * c.nr * sizeof(R);
  const int2 *list = W.pairs.get();
  for (long p0 = 0; p0 < np_all; p0 += kPairBatch) {
    const int np = (int)std::min<long>(kPairBatch, np_all - p0);
    k::pair_products<R>(c.nr, np, list + p0, g.wphir.get(), g.wphir.get(), g.work.get(), c.stream);
    pair_screen<R>(c, np, g.work.get(), g.sbuf.get(), g.qbuf.get());
    k::unpack_real<R, R>(c.nr, np, g.work.get(), g.wtau.get() + p0 * c.nr, c.stream);
  }
  sync(c);
}

void wannier_setup(Ctx &c) {
  WannierPrune &W = c.wan;
  const int no = c.nocc;
  const long nr = c.nr;
  Grids<double> &g = c.g64;
  const double dv = c.omega / (double)nr;
  DevBuf<double> oc, os, mat;
  oc.alloc((size_t)no * nr);
  os.alloc((size_t)no * nr);
  mat.alloc((size_t)2 * no * no);
  // the six position matrices and their weights
  std::vector<std::vector<double>> Ms;
  std::vector<double> wts;
  for (int k = 0; k < 3; ++k) {
    k::phase_rows(c, k, g.phir.get(), oc.get(), os.get());
    dgemm('N', 'T', no, no, (int)nr, dv, oc.get(), (int)nr, g.phir.get(), (int)nr, 0.0, mat.get(), no, c.stream);
    dgemm('N', 'T', no, no, (int)nr, dv, os.get(), (int)nr, g.phir.get(), (int)nr, 0.0, mat.get() + (size_t)no * no,
          no, c.stream);
    std::vector<double> h((size_t)2 * no * no);
    d2h(h.data(), mat.get(), h.size() * sizeof(double), c);
    const double *a = c.lat + 3 * k;
    const double wk = (a[0] * a[0] + a[1] * a[1] + a[2] * a[2]) / (4.0 * M_PI * M_PI);
    for (int m = 0; m < 2; ++m) {
      std::vector<double> M((size_t)no * no);
      for (int i = 0; i < no; ++i)
        for (int j = 0; j < no; ++j)
          M[(size_t)i * no + j] = 0.5 * (h[(size_t)m * no * no + (size_t)i * no + j] + h[(size_t)m * no * no + (size_t)j * no + i]);
      Ms.push_back(M);
      wts.push_back(wk);
    }
  }
  // Jacobi sweeps
  std::vector<double> U((size_t)no * no, 0.0);
  for (int i = 0; i < no; ++i) U[(size_t)i * no + i] = 1.0;
  int sweep = 0;
  for (sweep = 1; sweep <= 200; ++sweep) {
    double biggest = 0.0;
    for (int p = 0; p < no - 1; ++p)
      for (int q = p + 1; q < no; ++q) {
        double G00 = 0, G01 = 0, G11 = 0;
        for (size_t m = 0; m < Ms.size(); ++m) {
          const std::vector<double> &M = Ms[m];
          const double h0 = M[(size_t)p * no + p] - M[(size_t)q * no + q], h1 = 2.0 * M[(size_t)p * no + q];
          G00 += wts[m] * h0 * h0;
          G01 += wts[m] * h0 * h1;
          G11 += wts[m] * h1 * h1;
        }
        // leading eigenvector (x, y) of [[G00, G01], [G01, G11]], x >= 0: (cos 2t, sin 2t)
        const double tr = 0.5 * (G00 + G11), dd = 0.5 * (G00 - G11);
        const double lam = tr + std::sqrt(dd * dd + G01 * G01);
        // two closed forms of the eigenvector; the longer one is the well-conditioned one
        double x = G01, y = lam - G00;
        if (std::hypot(lam - G11, G01) > std::hypot(x, y)) {
          x = lam - G11;
          y = G01;
        }
        const double nrm = std::hypot(x, y);
        if (!(nrm > 0)) continue;
        x /= nrm;
        y /= nrm;
        if (x < 0) {
          x = -x;
          y = -y;
        }
        const double t = 0.5 * std::atan2(y, x);
        if (std::fabs(t) < 1e-15) continue;
        biggest = std::max(biggest, std::fabs(t));
        const double cs = std::cos(t), sn = std::sin(t);
        // w_p = c phi_p + s phi_q, w_q = -s phi_p + c phi_q: columns, then rows, of every matrix
        for (std::vector<double> &M : Ms) {
          for (int i = 0; i < no; ++i) {
            const double mp = M[(size_t)i * no + p], mq = M[(size_t)i * no + q];
            M[(size_t)i * no + p] = cs * mp + sn * mq;
            M[(size_t)i * no + q] = -sn * mp + cs * mq;
          }
          for (int j = 0; j < no; ++j) {
            const double mp = M[(size_t)p * no + j], mq = M[(size_t)q * no + j];
            M[(size_t)p * no + j] = cs * mp + sn * mq;
            M[(size_t)q * no + j] = -sn * mp + cs * mq;
          }
        }
        for (int v = 0; v < no; ++v) {
          const double up = U[(size_t)v * no + p], uq = U[(size_t)v * no + q];
          U[(size_t)v * no + p] = cs * up + sn * uq;
          U[(size_t)v * no + q] = -sn * up + cs * uq;
        }
      }
    if (biggest < 1e-13) break;
  }
  W.sweeps = sweep;
  // centres: fractional s_k = arg(C_ii + i S_ii) / (2 pi) (the phase of <w|e^{-i b.r}|w> = C - i S, negated)
  std::vector<double> cen((size_t)no * 3, 0.0);
  double inv[9];
  inv3(c.lat, inv);
  for (int i = 0; i < no; ++i)
    for (int k = 0; k < 3; ++k) {
      double sk = std::atan2(Ms[2 * k + 1][(size_t)i * no + i], Ms[2 * k][(size_t)i * no + i]) / (2.0 * M_PI);
      sk -= std::floor(sk);
      for (int a = 0; a < 3; ++a) cen[(size_t)i * 3 + a] += sk * c.lat[3 * k + a];
    }
  // kept pairs (minimum image over the 27 neighbouring cells of the fractional difference)
  auto dist = [&](int i, int j) {
    double f[3];
    for (int a = 0; a < 3; ++a) {
      double d = 0.0;
      for (int b = 0; b < 3; ++b) d += (cen[(size_t)i * 3 + b] - cen[(size_t)j * 3 + b]) * inv[3 * b + a];
      f[a] = d - std::round(d);
    }
    double best = HUGE_VAL;
    for (int s0 = -1; s0 <= 1; ++s0)
      for (int s1 = -1; s1 <= 1; ++s1)
        for (int s2 = -1; s2 <= 1; ++s2) {
          const double g0 = f[0] + s0, g1 = f[1] + s1, g2 = f[2] + s2;
          double r2 = 0.0;
          for (int a = 0; a < 3; ++a) {
            const double x = g0 * c.lat[a] + g1 * c.lat[3 + a] + g2 * c.lat[6 + a];
            r2 += x * x;
          }
          best = std::min(best, std::sqrt(r2));
        }
    return best;
  };
  std::vector<int2> pairs;
  std::vector<int> pidx((size_t)no * no, -1);
  for (int j = 0; j < no; ++j)
    for (int i = 0; i <= j; ++i)
      if (i == j || dist(i, j) <= W.cutoff) {
        pidx[(size_t)i * no + j] = pidx[(size_t)j * no + i] = (int)pairs.size();
        pairs.push_back(make_int2(i, j));
      }
  std::vector<int> off(no + 1, 0);
  std::vector<int2> nbr;
  for (int i = 0; i < no; ++i) {
    for (int j = 0; j < no; ++j)
      if (pidx[(size_t)i * no + j] >= 0) nbr.push_back(make_int2(j, pidx[(size_t)i * no + j]));
    off[i + 1] = (int)nbr.size();
  }
  W.npairs = (int)pairs.size();
  W.pairs.alloc(pairs.size());
  h2d(W.pairs.get(), pairs.data(), pairs.size() * sizeof(int2), c);
  W.off.alloc(off.size());
  h2d(W.off.get(), off.data(), off.size() * sizeof(int), c);
  W.nbr.alloc(nbr.size());
  h2d(W.nbr.get(), nbr.data(), nbr.size() * sizeof(int2), c);
  // U, eps~ = U^T diag(eps) U, w(r) = U^T phi(r)
  W.U_h = U;
  W.U.alloc((size_t)no * no);
  h2d(W.U.get(), U.data(), U.size() * sizeof(double), c);
  std::vector<double> et((size_t)no * no, 0.0);
  for (int i = 0; i < no; ++i)
    for (int j = 0; j < no; ++j) {
      double t = 0.0;
      for (int v = 0; v < no; ++v) t += U[(size_t)v * no + i] * c.eps_h[v] * U[(size_t)v * no + j];
      et[(size_t)i * no + j] = t;
    }
  W.epst.alloc(et.size());
  h2d(W.epst.get(), et.data(), et.size() * sizeof(double), c);
  g.wphir.alloc((size_t)no * nr);
  dgemm('T', 'N', no, (int)nr, no, 1.0, W.U.get(), no, g.phir.get(), (int)nr, 0.0, g.wphir.get(), (int)nr, c.stream);
  c.stats.wannier_pairs = W.npairs;
  c.stats.wannier_sweeps = W.sweeps;
  if (c.prec == 1) {
    c.g32.wphir.alloc((size_t)no * nr);
    k::convert((long)no * nr, g.wphir.get(), c.g32.wphir.get(), c.stream);
  }
  if (c.flags & BSE_FLAG_NO_K1D) {
    c.stats.bytes_tau = 0;
  } else if (c.prec == 0) {
    wannier_tau<double>(c);
  } else {
    wannier_tau<float>(c);
  }
}

void build_tau(Ctx &c) {
  c.npairs = (long)c.nocc * (c.nocc + 1) / 2;
  c.k1d.ready = false;
  if (c.wan.on) {
    wannier_setup(c);
    c.stats.k1d_tma = 0;
    return;
  }
  if (!(c.flags & BSE_FLAG_NO_K1D)) {
    if (c.prec == 0) {
      build_tau_t<double>(c);
    } else {
      const bool tiled = k1d_tma_supported(c.nocc, c.nr);
      build_tau_t<float>(c, tiled);
      check_device_flag(c);
      if (tiled) k1d_tma_init(c.k1d, c.g32.tau.get(), c.npairs, c.nr, c.dev_err.get());
    }
  } else {
    c.stats.bytes_tau = 0;
  }
  c.stats.k1d_tma = c.k1d.ready ? 1 : 0;
}

// phi_v(r) on the FP64 grids (g64.phir) for the first nocc rows of Q
void orbitals_to_grid(Ctx &c, const double *Q) {
  Grids<double> &g = c.g64;
  g.phir.alloc((size_t)c.nocc * c.nr);
  const long capf = (long)(g.work.n / c.nr) * 2;
  for (int f0 = 0; f0 < c.nocc; f0 += (int)capf) {
    const int nf = (int)std::min<long>(capf, c.nocc - f0);
    const int nq = (nf + 1) / 2;
    if (sphere_fft_ok<double>(c)) {
      sphere_to_grid_exec<double>(c, nf, Q + (long)f0 * c.npw, g.work.get(), 1.0 / std::sqrt(c.omega));
    } else {
      BSE_CUDA(cudaMemsetAsync(g.work.get(), 0, (size_t)nq * c.nr * sizeof(double2), c.stream));
      k::scatter_pairs<double, double>(c, nf, Q + (long)f0 * c.npw, g.work.get(), 1.0 / std::sqrt(c.omega));
      fft_exec(c, g.work.get(), nq, +1);
    }
    k::unpack_real<double, double>(c.nr, nf, g.work.get(), g.phir.get() + (long)f0 * c.nr, c.stream);
  }
}

// v_c * rho for a real density on the grids of type R (4 pi/|G|^2 on the density sphere, G = 0
// dropped), in place
template <class R>
void coulomb_grid(Ctx &c, R *rho) {
  Grids<R> &g = c.grids<R>();
  k::pack_real<R>(c.nr, 1, rho, g.work.get(), c.stream);
  fft_exec(c, g.work.get(), 1, -1);
  k::mul_grid<R>(c.nr, 1, g.work.get(), g.vcg.get(), (R)(1.0 / c.nr), c.stream);
  fft_exec(c, g.work.get(), 1, +1);
  k::unpack_real<R, R>(c.nr, 1, g.work.get(), rho, c.stream);
}

// Hartree-SCF ground state (f_Hxc = v_c): phi_v the lowest n_occ states of
// H_ext + v_c * rho_in, rho_out = 2 sum_v phi_v^2, iterated until the density residual
// (int |rho_out - rho_in|^2)^{1/2} <= scf_tol.  The fixed point is reached by Anderson mixing
// (history 8, damping 1/2) on the host; each iteration's ground-state Davidson starts from the
// previous iteration's states and is converged to a tolerance that tightens with the residual,
// reaching gs_tol before convergence is accepted.  Only the occupied states (and the LUMO
// guard set) are solved inside the loop; the empty states follow once at the converged
// potential.  Leaves the potential of rho_in (the density that built H) in the grids and
// rho_in in c.rho_gs.
void scf_ground_state(Ctx &c, std::vector<double> &eps_all, DevBuf<double> &Qall, const double *warm,
                      int nwarm) {
  const long nr = c.nr;
  const double dv = c.omega / (double)nr;
  const int kMaxIter = 200, kDepth = 8;
  const int kSlots = kDepth - 1;  // differences of the last kDepth iterates
  const double kBeta = 0.5;
  // Anderson mixing on the device: the input density x (rin), its residual f = rho_out - x, and a
  // ring of the last kSlots differences dX_i = x_k - x_{k-1}, dF_i = f_k - f_{k-1}.  Each
  // iteration adds one difference and its row of the Gram matrix dF_i . dF_j (one small product
  // over the grid) and the right-hand side dF_i . f; the normal equations of
  // min || f - sum_i gamma_i dF_i || are solved on the host, and
  // x <- x + beta f - sum_i gamma_i (dX_i + beta dF_i)  (the same update, oldest difference first).
  DevBuf<double> rin, vh, Qprev, f, xprev, fprev, dX, dF, dots, coef, m1;
  rin.alloc(nr);
  vh.alloc(nr);
  f.alloc(nr);
  xprev.alloc(nr);
  fprev.alloc(nr);
  dX.alloc((size_t)kSlots * nr);
  dF.alloc((size_t)kSlots * nr);
  dots.alloc(2 * kSlots + 1);
  coef.alloc(2 * kSlots + 1);
  m1.alloc(1);
  BSE_CUDA(cudaMemsetAsync(dX.get(), 0, (size_t)kSlots * nr * sizeof(double), c.stream));
  BSE_CUDA(cudaMemsetAsync(dF.get(), 0, (size_t)kSlots * nr * sizeof(double), c.stream));
  {
    const double minus_one = -1.0;
    h2d(m1.get(), &minus_one, sizeof(double), c);
  }
  if ((c.flags & BSE_FLAG_WARM_START) && c.have_warm_rho) d2d(rin.get(), c.warm_rho.get(), nr * sizeof(double), c);
  else BSE_CUDA(cudaMemsetAsync(rin.get(), 0, nr * sizeof(double), c.stream));
  std::vector<int> order;                                    // active slots, oldest first
  std::vector<double> G((size_t)kSlots * kSlots, 0.0), hd(2 * kSlots + 1);
  bool have_prev = false;
  const double *init = warm;
  int ninit = warm ? nwarm : 0;
  double res = HUGE_VAL;
  int it = 0;
  for (;; ++it) {
    if (it >= kMaxIter) throw Error(BSE_ERR_NOT_CONVERGED, "Hartree SCF did not reach scf_tol");
    d2d(vh.get(), rin.get(), nr * sizeof(double), c);
    coulomb_grid<double>(c, vh.get());
    set_local_potential(c, vh.get());
    const double gtol = std::max(c.gs_tol, std::min(1e-4, 1e-2 * res));
    ground_state(c, eps_all, Qall, gtol, init, ninit, false);
    const int nst = (int)eps_all.size();
    Qprev.alloc((size_t)nst * c.npw);
    d2d(Qprev.get(), Qall.get(), (size_t)nst * c.npw * sizeof(double), c);
    init = Qprev.get();
    ninit = nst;
    orbitals_to_grid(c, Qall.get());
    k::density_sum(nr, c.nocc, c.g64.phir.get(), 2.0, f.get(), c.stream);
    row_axpby(1, nr, nullptr, f.get(), m1.get(), rin.get(), c.stream);  // f = rho_out - x
    rowdot(1, nr, f.get(), f.get(), dots.get() + 2 * kSlots, c.stream);
    double s2 = 0.0;
    d2h(&s2, dots.get() + 2 * kSlots, sizeof(double), c);
    res = std::sqrt(std::max(0.0, s2) * dv);
    if (verbose()) std::fprintf(stderr, "[bse scf] it=%d density residual=%.3e gs_tol=%.1e\n", it, res, gtol);
    if (res <= c.scf_tol && gtol <= c.gs_tol) break;
    if (have_prev) {
      // the slot of the new difference: a free one, or the oldest
      int slot = (int)order.size();
      if ((int)order.size() == kSlots) {
        slot = order.front();
        order.erase(order.begin());
      }
      double *dxs = dX.get() + (size_t)slot * nr, *dfs = dF.get() + (size_t)slot * nr;
      d2d(dxs, rin.get(), nr * sizeof(double), c);
      row_axpby(1, nr, nullptr, dxs, m1.get(), xprev.get(), c.stream);
      d2d(dfs, f.get(), nr * sizeof(double), c);
      row_axpby(1, nr, nullptr, dfs, m1.get(), fprev.get(), c.stream);
      order.push_back(slot);
      // dF_j . dF_new and dF_j . f for every slot (inactive slots are ignored)
      dgemm('N', 'T', kSlots, 1, (int)nr, 1.0, dF.get(), (int)nr, dfs, (int)nr, 0.0, dots.get(), 1, c.stream);
      dgemm('N', 'T', kSlots, 1, (int)nr, 1.0, dF.get(), (int)nr, f.get(), (int)nr, 0.0, dots.get() + kSlots, 1,
            c.stream);
      d2h(hd.data(), dots.get(), 2 * kSlots * sizeof(double), c);
      for (int j : order) G[(size_t)slot * kSlots + j] = G[(size_t)j * kSlots + slot] = hd[j];
    }
    d2d(xprev.get(), rin.get(), nr * sizeof(double), c);
    d2d(fprev.get(), f.get(), nr * sizeof(double), c);
    have_prev = true;
    const int m = (int)order.size();
    std::vector<double> gam(m, 0.0);
    if (m > 0) {
      std::vector<double> A((size_t)m * m), bv(m);
      for (int i = 0; i < m; ++i) {
        for (int j = 0; j < m; ++j) A[(size_t)i * m + j] = G[(size_t)order[i] * kSlots + order[j]];
        bv[i] = hd[kSlots + order[i]];
      }
      for (int i = 0; i < m; ++i) A[(size_t)i * m + i] *= 1.0 + 1e-12;
      // Gaussian elimination with partial pivoting on the small normal equations
      for (int col = 0; col < m; ++col) {
        int piv = col;
        for (int r = col + 1; r < m; ++r)
          if (std::fabs(A[(size_t)r * m + col]) > std::fabs(A[(size_t)piv * m + col])) piv = r;
        if (A[(size_t)piv * m + col] == 0.0) continue;
        if (piv != col) {
          for (int j = 0; j < m; ++j) std::swap(A[(size_t)col * m + j], A[(size_t)piv * m + j]);
          std::swap(bv[col], bv[piv]);
        }
        for (int r = col + 1; r < m; ++r) {
          const double t = A[(size_t)r * m + col] / A[(size_t)col * m + col];
          for (int j = col; j < m; ++j) A[(size_t)r * m + j] -= t * A[(size_t)col * m + j];
          bv[r] -= t * bv[col];
        }
      }
      for (int i = m - 1; i >= 0; --i) {
        double t = bv[i];
        for (int j = i + 1; j < m; ++j) t -= A[(size_t)i * m + j] * gam[j];
        gam[i] = A[(size_t)i * m + i] != 0.0 ? t / A[(size_t)i * m + i] : 0.0;
      }
    }
    // x <- x + beta f - sum_i gamma_i (dX_i + beta dF_i)
    std::vector<double> cf(1 + 2 * m);
    cf[0] = kBeta;
    for (int i = 0; i < m; ++i) {
      cf[1 + 2 * i] = -gam[i];
      cf[2 + 2 * i] = -kBeta * gam[i];
    }
    h2d(coef.get(), cf.data(), cf.size() * sizeof(double), c);
    row_axpby(1, nr, nullptr, rin.get(), coef.get(), f.get(), c.stream);
    for (int i = 0; i < m; ++i) {
      row_axpby(1, nr, nullptr, rin.get(), coef.get() + 1 + 2 * i, dX.get() + (size_t)order[i] * nr, c.stream);
      row_axpby(1, nr, nullptr, rin.get(), coef.get() + 2 + 2 * i, dF.get() + (size_t)order[i] * nr, c.stream);
    }
  }
  c.stats.scf_iterations = it + 1;
  c.stats.scf_residual = res;
  // the empty states of the converged Hamiltonian (same potential), occupied states as the start
  ground_state(c, eps_all, Qall, c.gs_tol, Qprev.get(), ninit, true);
  c.rho_gs.alloc(nr);
  d2d(c.rho_gs.get(), rin.get(), nr * sizeof(double), c);
  if (c.flags & BSE_FLAG_WARM_START) {
    c.warm_rho.alloc(nr);
    d2d(c.warm_rho.get(), rin.get(), nr * sizeof(double), c);
    c.have_warm_rho = true;
  }
}

void geometry_stage(Ctx &c) {
  auto t0 = clk::now();
  c.stats.ms_host_eig = 0.0;
  c.stats.gs_iterations = 0;
  c.stats.gs_chunks = 0;
  c.stats.scf_iterations = 0;
  c.stats.scf_residual = 0.0;
  c.have_gs = false;
  c.warm_roots = (c.flags & BSE_FLAG_WARM_START) ? c.nroots : 0;  // roots stay in c.roots
  c.nroots = 0;
  c.z_root = -1;
  c.have_rho = false;
  compute_vloc(c);
  std::vector<double> eps_all;
  DevBuf<double> Qall;
  // warm start: the previous geometry's states as the starting blocks
  const double *warm = (c.flags & BSE_FLAG_WARM_START) && c.warm_nstates > 0 ? c.warm_states.get() : nullptr;
  const int nwarm = warm ? c.warm_nstates : 0;
  if (c.hartree) scf_ground_state(c, eps_all, Qall, warm, nwarm);
  else ground_state(c, eps_all, Qall, c.gs_tol, warm, nwarm, true);
  if (c.flags & BSE_FLAG_WARM_START) {
    const int nst = (int)eps_all.size();
    c.warm_states.alloc((size_t)nst * c.npw);
    d2d(c.warm_states.get(), Qall.get(), (size_t)nst * c.npw * sizeof(double), c);
    c.warm_nstates = nst;
  }
  c.phi.alloc((size_t)c.nocc * c.npw);
  d2d(c.phi.get(), Qall.get(), (size_t)c.nocc * c.npw * sizeof(double), c);
  c.eps_h.assign(eps_all.begin(), eps_all.begin() + c.nocc);
  c.eps.alloc(c.nocc);
  h2d(c.eps.get(), c.eps_h.data(), c.nocc * sizeof(double), c);
  {
    std::vector<double> ne(c.nocc);
    for (int v = 0; v < c.nocc; ++v) ne[v] = -c.eps_h[v];
    c.negeps.alloc(c.nocc);
    h2d(c.negeps.get(), ne.data(), c.nocc * sizeof(double), c);
  }
  // extra empty states kept as Davidson guesses in sbuf
  const int nextra = (int)eps_all.size() - c.nocc;
  c.stats.homo_lumo_gap = nextra > 0 ? eps_all[c.nocc] - eps_all[c.nocc - 1] : 0.0;
  c.empty.alloc((size_t)std::max(1, nextra) * c.npw);
  if (nextra > 0)
    d2d(c.empty.get(), Qall.get() + (size_t)c.nocc * c.npw, (size_t)nextra * c.npw * sizeof(double), c);
  c.eps_empty.assign(eps_all.begin() + c.nocc, eps_all.end());
  c.eps_empty_d.alloc(std::max(1, nextra));
  if (nextra > 0) h2d(c.eps_empty_d.get(), c.eps_empty.data(), nextra * sizeof(double), c);
  // phi_v(r) in FP64 (and rounded to FP32 for the mixed-precision operator)
  Grids<double> &g = c.g64;
  orbitals_to_grid(c, c.phi.get());
  if (!c.hartree) {
    c.rho_gs.alloc(c.nr);
    k::density_sum(c.nr, c.nocc, g.phir.get(), 2.0, c.rho_gs.get(), c.stream);
  }
  if (c.prec == 1) {
    c.phi32.alloc((size_t)c.nocc * c.npw);
    k::convert((long)c.nocc * c.npw, c.phi.get(), c.phi32.get(), c.stream);
    c.g32.phir.alloc((size_t)c.nocc * c.nr);
    k::convert((long)c.nocc * c.nr, g.phir.get(), c.g32.phir.get(), c.stream);
  }
  sync(c);
  c.stats.ms_ground_state = ms_since(t0);
  auto t1 = clk::now();
  build_tau(c);
  c.stats.ms_tau = ms_since(t1);
  c.have_gs = true;
  if (nextra > 0 && !(c.stats.homo_lumo_gap >= 1e-6))
    throw Error(BSE_ERR_DEGENERATE, "HOMO-LUMO gap below 1e-6 Ha");
}

void init_pairs(Ctx &c) {
  std::vector<int2> list;
  for (int v = 0; v < c.nocc; ++v)
    for (int vp = 0; vp <= v; ++vp) list.push_back(make_int2(vp, v));
  c.pairs.alloc(list.size());
  h2d(c.pairs.get(), list.data(), list.size() * sizeof(int2), c);
}

// ---------------------------------------------------------------------------------
// BSE Davidson (Eq. 1)
// Start block of the excitation solves: nwarm previous roots (c.roots), then the lowest single
// transitions v -> c among the solved empty states, then smooth deterministic vectors
void transition_start(Ctx &c, int k0, double *X0, int nwarm) {
  const long n = (long)c.nocc * c.npw;
  const int nextra = (int)c.eps_empty.size();
  const std::vector<double> &emp = c.eps_empty;  // empty energies from the ground-state solve
  struct Tr { double de; int v, e; };
  std::vector<Tr> tr;
  for (int v = std::max(0, c.nocc - 4); v < c.nocc; ++v)
    for (int e = 0; e < nextra; ++e) tr.push_back({emp[e] - c.eps_h[v], v, e});
  std::sort(tr.begin(), tr.end(), [](const Tr &a, const Tr &b) { return a.de < b.de; });
  BSE_CUDA(cudaMemsetAsync(X0, 0, (size_t)k0 * n * sizeof(double), c.stream));
  std::vector<double> seed((size_t)c.npw);
  if (nwarm > 0) d2d(X0, c.roots.get(), (size_t)nwarm * n * sizeof(double), c);
  for (int j = nwarm; j < k0; ++j) {
    double *dst = X0 + (size_t)j * n;
    const int jt = j - nwarm;  // transitions fill the rest of the start block
    if (jt < (int)tr.size()) {
      d2d(dst + (size_t)tr[jt].v * c.npw, c.empty.get() + (size_t)tr[jt].e * c.npw, c.npw * sizeof(double), c);
    } else {
      // deterministic fallback: a smooth function times the HOMO index
      for (int i = 0; i < c.npw; ++i) seed[i] = std::cos(0.37 * (i + 1) * (j + 1)) / (1.0 + c.kin_h[i]);
      h2d(dst + (size_t)(c.nocc - 1 - (j % c.nocc)) * c.npw, seed.data(), c.npw * sizeof(double), c);
    }
  }
}

// Two-level preconditioner for the correction equation (D - theta) t = r on P_c, rows of kk
// trial vectors (kk <= maxvec): exact denominators eps_c - eps_v + Delta - theta in the span E
// of the solved empty states, (1/2 |G|^2 + 1)^-1 on the rest.
struct PairPrecond {
  Ctx &c;
  int ne;
  DevBuf<double> Cb, Ckb, one;
  PairPrecond(Ctx &c_, int maxvec) : c(c_), ne((int)c_.eps_empty.size()) {
    Cb.alloc((size_t)maxvec * c.nocc * std::max(1, ne));
    Ckb.alloc((size_t)maxvec * c.nocc * std::max(1, ne));
    std::vector<double> v(c.nocc, 1.0);
    one.alloc(c.nocc);
    h2d(one.get(), v.data(), c.nocc * sizeof(double), c);
  }
  // the products with the empty states run in FP32 in the mixed form (a preconditioner only
  // changes the convergence rate, not the converged root; its FP64 products cost a quarter of a
  // mixed Davidson iteration)
  void operator()(int kk, double *T, const double *th) {
    const long n = (long)c.nocc * c.npw;
    const int rows = kk * c.nocc;
    const bool fp32 = c.prec == 1;
    if (ne > 0)
      gemm_p(c, fp32, 'N', 'T', rows, ne, c.npw, 1.0, T, c.npw, c.empty.get(), c.npw, 0.0, Cb.get(), ne);
    k::precond_diag(kk, n, T, c.kin.get(), c.npw, one.get(), 0.0, th, 1e-3, T, c.stream);
    if (ne > 0) {
      gemm_p(c, fp32, 'N', 'T', rows, ne, c.npw, 1.0, T, c.npw, c.empty.get(), c.npw, 0.0, Ckb.get(), ne);
      k::subspace_den(rows, ne, c.nocc, Cb.get(), Ckb.get(), c.eps_empty_d.get(), c.eps.get(), c.scissor, th,
                      1e-6, Cb.get(), c.stream);
      gemm_p(c, fp32, 'N', 'N', rows, c.npw, ne, 1.0, Cb.get(), ne, c.empty.get(), c.npw, 1.0, T, c.npw);
    }
  }
};

void bse_davidson_impl(Ctx &c, int nroots, double tol, int maxit, double *omega_host, double *A_dev) {
  BSE_REQUIRE(c.have_gs, "no ground state");
  BSE_REQUIRE(nroots >= 1 && nroots <= 64, "n_roots must be in 1..64");
  BSE_REQUIRE(tol > 0 && std::isfinite(tol), "tol must be positive");
  auto t0 = clk::now();
  const long n = (long)c.nocc * c.npw;
  // corrections for the wanted roots and, in mixed precision, for one more Ritz vector (a
  // two-vector FP32 apply costs little more than a one-vector one, and the extra direction
  // almost halves the iterations: 67 -> 41 on the 63-atom cell, 0.33 -> 0.29 s; an FP64 apply
  // costs in proportion to its vectors, so FP64 corrects the wanted roots only); a deep subspace
  // with thick restarts; the start block holds two more transitions than roots
  const int block = nroots + (c.prec == 1 ? 1 : 0);
  const int k0 = nroots + 2;
  DevBuf<double> X0;
  X0.alloc((size_t)k0 * n);
  const int nwarm = std::min(c.warm_roots, k0);
  transition_start(c, k0, X0.get(), nwarm);
  DavSpec sp;
  sp.n = n;
  sp.nwant = nroots;
  sp.block = block;
  sp.maxsub = std::max(24 * block, 96);
  sp.keep = std::max(12, 3 * block);
  sp.maxit = maxit;
  sp.tol = tol;
  sp.apply = [&](int kk, const double *X, double *AX) { apply_liouville(c, kk, X, AX, 0); };
  PairPrecond pre(c, block);
  sp.precond = [&](int kk, double *T, const double *th) { pre(kk, T, th); };
  // the new directions go back to the P_c space in the operator's precision (the mixed form's
  // applies already project their outputs with FP32 overlaps)
  sp.project = [&](int kk, double *X) {
    if (c.prec == 1) project_pc32(c, kk * c.nocc, X);
    else project_vectors(c, kk, X);
  };
  DevBuf<double> Xout;
  Xout.alloc((size_t)nroots * n);
  DavOut r = davidson(c, sp, X0.get(), k0, Xout.get());
  // the returned roots exactly in the P_c space (FP64 overlaps): the mixed form's FP32 projections
  // leave occupied components of FP32 size, which the U vector and the FP64 Z-vector refinement
  // would otherwise carry
  if (c.prec == 1) project_vectors(c, nroots, Xout.get());
  c.stats.davidson_iterations = r.iters;
  double mr = 0.0;
  for (int i = 0; i < nroots; ++i) mr = std::max(mr, r.res[i]);
  c.stats.davidson_residual = mr;
  c.roots.alloc((size_t)nroots * n);
  d2d(c.roots.get(), Xout.get(), (size_t)nroots * n * sizeof(double), c);
  c.nroots = nroots;
  c.omega_h.assign(r.theta.begin(), r.theta.begin() + nroots);
  c.z_root = -1;
  c.have_rho = false;
  if (A_dev) d2d(A_dev, Xout.get(), (size_t)nroots * n * sizeof(double), c);
  if (omega_host) std::memcpy(omega_host, r.theta.data(), nroots * sizeof(double));
  sync(c);
  c.stats.ms_davidson = ms_since(t0);
  if (!r.converged) throw Error(BSE_ERR_NOT_CONVERGED, "Davidson reached max_iter");
}

// ---------------------------------------------------------------------------------
// BSE beyond the TDA (Sec. SI)

// B A for nvec trial vectors with grids of type R: the coupling block, real orbitals,
// (2 K2e - K2d) A (singlet) or -K2d A (triplet), switched like K1e/K1d by the flags.
// K2e A = P_c [v_c * sum_v' a_v' phi_v'] phi_v (the density of K1e);
// K2d A = P_c sum_v' [W * (a_v' phi_v)] phi_v' over all ordered pairs: the pair densities depend
// on A, so W is applied to N_occ^2 of them per vector (the pair pipeline of the tau build).
template <class R>
void apply_b_t(Ctx &c, int nvec, const double *A, double *BA) {
  Grids<R> &g = c.grids<R>();
  const bool k2e = (c.spin == 0) && !(c.flags & BSE_FLAG_NO_K1E);
  const bool k2d = !(c.flags & BSE_FLAG_NO_K1D);
  const int no = c.nocc;
  const long vlen = (long)no * c.npw;
  if (!c.pairs_full.get()) {
    std::vector<int2> list;
    for (int v = 0; v < no; ++v)
      for (int vp = 0; vp < no; ++vp) list.push_back(make_int2(vp, v));
    c.pairs_full.alloc(list.size());
    h2d(c.pairs_full.get(), list.data(), list.size() * sizeof(int2), c);
  }
  const long nfull = (long)no * no;
  g.bar.alloc((size_t)no * c.nr);
  g.bt.alloc((size_t)no * c.nr);
  DevBuf<R> vx;
  vx.alloc(c.nr);
  const long capf = (long)(g.work.n / c.nr) * 2;
  for (int b = 0; b < nvec; ++b) {
    const double *a = A + (long)b * vlen;
    double *out = BA + (long)b * vlen;
    for (int f0 = 0; f0 < no; f0 += (int)capf) {
      const int nf = (int)std::min<long>(capf, no - f0);
      const int nq = (nf + 1) / 2;
      BSE_CUDA(cudaMemsetAsync(g.work.get(), 0, (size_t)nq * c.nr * sizeof(CT<R>), c.stream));
      k::scatter_pairs<R, double>(c, nf, a + (long)f0 * c.npw, g.work.get(), 1.0 / std::sqrt(c.omega));
      fft_exec(c, g.work.get(), nq, +1);
      k::unpack_real<R, R>(c.nr, nf, g.work.get(), g.bar.get() + (long)f0 * c.nr, c.stream);
    }
    BSE_CUDA(cudaMemsetAsync(g.bt.get(), 0, (size_t)no * c.nr * sizeof(R), c.stream));
    if (k2e) {
      k::pair_sum<R>(c.nr, no, g.bar.get(), g.phir.get(), vx.get(), c.stream);
      coulomb_grid<R>(c, vx.get());
      k::add_product<R>(c.nr, no, vx.get(), g.phir.get(), (R)2, g.bt.get(), c.stream);
    }
    if (k2d) {
      R *X = g.sbuf.get();
      R *Qm = g.qbuf.get();
      for (long p0 = 0; p0 < nfull; p0 += kPairBatch) {
        const int np = (int)std::min<long>(kPairBatch, nfull - p0);
        // pair (v', v): a_v' phi_v; T_v -= [W * (a_v' phi_v)] phi_v'
        k::pair_products<R>(c.nr, np, c.pairs_full.get() + p0, g.bar.get(), g.phir.get(), g.work.get(), c.stream);
        pair_screen<R>(c, np, g.work.get(), X, Qm);
        k::sigma_contract<R>(c, np, c.pairs_full.get() + p0, g.work.get(), g.phir.get(), g.bt.get(), false);
      }
    }
    for (int f0 = 0; f0 < no; f0 += (int)capf) {
      const int nf = (int)std::min<long>(capf, no - f0);
      const int nq = (nf + 1) / 2;
      k::pack_real<R>(c.nr, nf, g.bt.get() + (long)f0 * c.nr, g.work.get(), c.stream);
      fft_exec(c, g.work.get(), nq, -1);
      k::gather_pairs<R, double>(c, nf, g.work.get(), out + (long)f0 * c.npw, std::sqrt(c.omega) / c.nr);
    }
    project_pc(c, no, out, nullptr);
  }
}

void apply_b(Ctx &c, int nvec, const double *A, double *BA) {
  if (c.prec == 0) {
    apply_b_t<double>(c, nvec, A, BA);
  } else {
    apply_b_t<float>(c, nvec, A, BA);
    check_device_flag(c);
  }
}

// lower Cholesky factor of the symmetric positive-definite m x m matrix A (row-major); false if
// a pivot is not positive
bool host_cholesky(int m, const double *A, std::vector<double> &L) {
  L.assign((size_t)m * m, 0.0);
  for (int j = 0; j < m; ++j) {
    double d = A[(size_t)j * m + j];
    for (int k = 0; k < j; ++k) d -= L[(size_t)j * m + k] * L[(size_t)j * m + k];
    if (!(d > 0.0)) return false;
    const double ljj = std::sqrt(d);
    L[(size_t)j * m + j] = ljj;
    for (int i = j + 1; i < m; ++i) {
      double t = A[(size_t)i * m + j];
      for (int k = 0; k < j; ++k) t -= L[(size_t)i * m + k] * L[(size_t)j * m + k];
      L[(size_t)i * m + j] = t / ljj;
    }
  }
  return true;
}

// Lowest roots of the BSE beyond the TDA, (A B; B A)(X; Y) = omega (X; -Y) for real orbitals,
// i.e. (A - B)(A + B)(X + Y) = omega^2 (X + Y).  Davidson on one subspace V for X + Y and X - Y
// (the symmetric-pair scheme of Stratmann, Scuseria and Frisch, J. Chem. Phys. 109, 8218 (1998)):
// with P = V^T (A + B) V and M = V^T (A - B) V, the projected problem M P u = omega^2 u is solved
// through M = L L^T and the symmetric L^T P L s = omega^2 s, u = L s (X + Y = V u),
// w = P u / omega (X - Y = V w), scaled to (X + Y).(X - Y) = 1.  Both residuals
// (A + B)(X + Y) - omega (X - Y) and (A - B)(X - Y) - omega (X + Y) get a correction from the
// TDA's two-level preconditioner at theta = omega.  Needs A - B and A + B positive definite
// (else BSE_ERR_DEGENERATE: no real spectrum).
void bse_davidson_full_impl(Ctx &c, int nroots, double tol, int maxit, double *omega_host, double *X_dev,
                            double *Y_dev) {
  BSE_REQUIRE(c.have_gs, "no ground state");
  BSE_REQUIRE(nroots >= 1 && nroots <= 32, "n_roots must be in 1..32");
  BSE_REQUIRE(tol > 0 && std::isfinite(tol), "tol must be positive");
  auto t0 = clk::now();
  const long n = (long)c.nocc * c.npw;
  const int k0 = nroots + 2;
  const int S = std::max(24 * nroots, 96);
  const int keep = std::max(4, 2 * nroots);   // roots whose X + Y and X - Y survive a restart
  const int nbuf = std::max(std::max(2 * nroots, k0), 2 * keep);
  DevBuf<double> V, PV, MV, T, LA, BV, Xp, Xm, R1, R2, small, rn, th, m1, Vt;
  V.alloc((size_t)S * n);
  PV.alloc((size_t)S * n);
  MV.alloc((size_t)S * n);
  T.alloc((size_t)nbuf * n);
  LA.alloc((size_t)nbuf * n);
  BV.alloc((size_t)nbuf * n);
  Xp.alloc((size_t)keep * n);
  Xm.alloc((size_t)keep * n);
  R1.alloc((size_t)nroots * n);
  R2.alloc((size_t)nroots * n);
  Vt.alloc((size_t)nbuf * n);
  small.alloc((size_t)S * std::max(S, nbuf));
  rn.alloc(std::max(nbuf, S));
  th.alloc(std::max(nbuf, S));
  {
    std::vector<double> v(std::max(nbuf, S), -1.0);
    m1.alloc(v.size());
    h2d(m1.get(), v.data(), v.size() * sizeof(double), c);
  }
  PairPrecond pre(c, 2 * nroots);
  // start: the lowest transitions
  transition_start(c, k0, T.get(), 0);
  project_vectors(c, k0, T.get());
  int m = orthonormalize(c, n, T.get(), k0, nullptr, 0, nullptr, 0);
  BSE_REQUIRE(m > 0, "full-BSE Davidson: empty start block");
  d2d(V.get(), T.get(), (size_t)m * n * sizeof(double), c);
  std::vector<double> Pm((size_t)S * S, 0.0), Mm((size_t)S * S, 0.0), Hn;
  // (A + B) and (A - B) on rows [m0, m0 + k) of V
  auto apply_pm = [&](int m0, int k) {
    apply_liouville(c, k, V.get() + (size_t)m0 * n, LA.get(), 0);
    apply_b(c, k, V.get() + (size_t)m0 * n, BV.get());
    d2d(PV.get() + (size_t)m0 * n, LA.get(), (size_t)k * n * sizeof(double), c);
    row_axpby(k, n, nullptr, PV.get() + (size_t)m0 * n, nullptr, BV.get(), c.stream);
    d2d(MV.get() + (size_t)m0 * n, LA.get(), (size_t)k * n * sizeof(double), c);
    row_axpby(k, n, nullptr, MV.get() + (size_t)m0 * n, m1.get(), BV.get(), c.stream);
  };
  // rows [m0, m1) of P and M (old-new entries mirrored, new-new symmetrised)
  auto grow = [&](int r0, int r1) {
    const int k = r1 - r0;
    for (int which = 0; which < 2; ++which) {
      std::vector<double> &H = which == 0 ? Pm : Mm;
      dgemm('N', 'T', k, r1, (int)n, 1.0, V.get() + (size_t)r0 * n, (int)n, (which == 0 ? PV : MV).get(), (int)n,
            0.0, small.get(), r1, c.stream);
      Hn.resize((size_t)k * r1);
      d2h(Hn.data(), small.get(), Hn.size() * sizeof(double), c);
      for (int i = 0; i < k; ++i)
        for (int j = 0; j < r1; ++j) {
          const int gi = r0 + i;
          const double v = Hn[(size_t)i * r1 + j];
          if (j < r0) {
            H[(size_t)gi * S + j] = H[(size_t)j * S + gi] = v;
          } else if (j >= gi) {
            const double u = Hn[(size_t)(j - r0) * r1 + gi];
            H[(size_t)gi * S + j] = H[(size_t)j * S + gi] = 0.5 * (v + u);
          }
        }
    }
  };
  apply_pm(0, m);
  grow(0, m);
  std::vector<double> L, Pp, w, Ys, Uc, Wc, om, res(nroots, 0.0);
  int it = 0;
  bool conv = false;
  for (it = 1;; ++it) {
    // projected problem
    std::vector<double> Ms((size_t)m * m), Ps((size_t)m * m);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        Ms[(size_t)i * m + j] = Mm[(size_t)i * S + j];
        Ps[(size_t)i * m + j] = Pm[(size_t)i * S + j];
      }
    if (!host_cholesky(m, Ms.data(), L))
      throw Error(BSE_ERR_DEGENERATE, "A - B is not positive definite: the full BSE has no real spectrum here");
    // Pp = L^T P L
    std::vector<double> PL((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i)
      for (int k = 0; k < m; ++k) {
        const double p = Ps[(size_t)i * m + k];
        if (p == 0.0) continue;
        for (int j = 0; j <= k; ++j) PL[(size_t)i * m + j] += p * L[(size_t)k * m + j];
      }
    Pp.assign((size_t)m * m, 0.0);
    for (int k = 0; k < m; ++k)
      for (int i = 0; i <= k; ++i) {
        const double l = L[(size_t)k * m + i];
        if (l == 0.0) continue;
        for (int j = 0; j < m; ++j) Pp[(size_t)i * m + j] += l * PL[(size_t)k * m + j];
      }
    const int kk = std::min(m, std::max(nroots, keep));
    w.resize(m);
    Ys.resize((size_t)m * m);
    {
      auto te = clk::now();
      sym_eig_lowest(m, Pp.data(), kk, w.data(), Ys.data(), false);
      c.stats.ms_host_eig += ms_since(te);
    }
    // u = L s, w = P u / omega, scaled to u.w = 1
    Uc.assign((size_t)m * kk, 0.0);
    Wc.assign((size_t)m * kk, 0.0);
    om.resize(kk);
    for (int r = 0; r < kk; ++r) {
      if (!(w[r] > 0.0))
        throw Error(BSE_ERR_DEGENERATE, "A + B is not positive definite: the full BSE has no real spectrum here");
      om[r] = std::sqrt(w[r]);
      for (int i = 0; i < m; ++i) {
        double t = 0.0;
        for (int j = 0; j <= i; ++j) t += L[(size_t)i * m + j] * Ys[(size_t)j * m + r];
        Uc[(size_t)i * kk + r] = t;
      }
      double uw = 0.0;
      for (int i = 0; i < m; ++i) {
        double t = 0.0;
        for (int j = 0; j < m; ++j) t += Ps[(size_t)i * m + j] * Uc[(size_t)j * kk + r];
        Wc[(size_t)i * kk + r] = t / om[r];
        uw += Uc[(size_t)i * kk + r] * Wc[(size_t)i * kk + r];
      }
      const double f = 1.0 / std::sqrt(uw);
      for (int i = 0; i < m; ++i) {
        Uc[(size_t)i * kk + r] *= f;
        Wc[(size_t)i * kk + r] *= f;
      }
    }
    const int nb = std::min(nroots, kk);
    // Ritz vectors X + Y, X - Y and the residuals of the wanted roots
    auto combine = [&](const std::vector<double> &C, int cols, const double *Src, double *Dst) {
      h2d(small.get(), C.data(), (size_t)m * cols * sizeof(double), c);
      dgemm('T', 'N', cols, (int)n, m, 1.0, small.get(), cols, Src, (int)n, 0.0, Dst, (int)n, c.stream);
    };
    combine(Uc, kk, V.get(), Xp.get());
    combine(Wc, kk, V.get(), Xm.get());
    h2d(th.get(), om.data(), nb * sizeof(double), c);
    std::vector<double> Ub((size_t)m * nb), Wb((size_t)m * nb);
    for (int i = 0; i < m; ++i)
      for (int r = 0; r < nb; ++r) {
        Ub[(size_t)i * nb + r] = Uc[(size_t)i * kk + r];
        Wb[(size_t)i * nb + r] = Wc[(size_t)i * kk + r];
      }
    combine(Ub, nb, PV.get(), LA.get());
    k::residual(nb, n, LA.get(), Xm.get(), th.get(), R1.get(), c.stream);
    combine(Wb, nb, MV.get(), LA.get());
    k::residual(nb, n, LA.get(), Xp.get(), th.get(), R2.get(), c.stream);
    std::vector<double> r1(nb), r2(nb);
    rowdot(nb, n, R1.get(), R1.get(), rn.get(), c.stream);
    d2h(r1.data(), rn.get(), nb * sizeof(double), c);
    rowdot(nb, n, R2.get(), R2.get(), rn.get(), c.stream);
    d2h(r2.data(), rn.get(), nb * sizeof(double), c);
    conv = true;
    for (int r = 0; r < nb; ++r) {
      res[r] = std::sqrt(std::max(0.0, r1[r]) + std::max(0.0, r2[r]));
      if (!(res[r] <= tol)) conv = false;
    }
    if (verbose())
      std::fprintf(stderr, "[bse full davidson] it=%d m=%d omega0=%.12f res0=%.3e\n", it, m, om[0], res[0]);
    if (conv || it >= maxit) break;
    // corrections for the unconverged roots, from both residuals
    int nsel = 0;
    std::vector<double> thsel;
    for (int r = 0; r < nb; ++r) {
      if (res[r] <= tol) continue;
      d2d(T.get() + (size_t)nsel * n, R1.get() + (size_t)r * n, n * sizeof(double), c);
      d2d(T.get() + (size_t)(nsel + 1) * n, R2.get() + (size_t)r * n, n * sizeof(double), c);
      thsel.push_back(om[r]);
      thsel.push_back(om[r]);
      nsel += 2;
    }
    h2d(th.get(), thsel.data(), nsel * sizeof(double), c);
    pre(nsel, T.get(), th.get());
    project_vectors(c, nsel, T.get());
    if (m + nsel > S) {
      // thick restart on X + Y and X - Y of the kk lowest roots, orthonormalised in coefficient
      // space (V is orthonormal): C = [U | W], Gram-Schmidt on the host, V <- V C, and the
      // projected matrices C^T P C, C^T M C
      std::vector<double> C((size_t)m * 2 * kk);
      for (int i = 0; i < m; ++i)
        for (int r = 0; r < kk; ++r) {
          C[(size_t)i * 2 * kk + r] = Uc[(size_t)i * kk + r];
          C[(size_t)i * 2 * kk + kk + r] = Wc[(size_t)i * kk + r];
        }
      std::vector<double> Q;
      int q = 0;
      for (int col = 0; col < 2 * kk; ++col) {
        std::vector<double> x(m);
        for (int i = 0; i < m; ++i) x[i] = C[(size_t)i * 2 * kk + col];
        const double n0 = std::sqrt(std::inner_product(x.begin(), x.end(), x.begin(), 0.0));
        for (int pass = 0; pass < 2; ++pass)
          for (int j = 0; j < q; ++j) {
            double d = 0.0;
            for (int i = 0; i < m; ++i) d += Q[(size_t)i * nbuf + j] * x[i];
            for (int i = 0; i < m; ++i) x[i] -= d * Q[(size_t)i * nbuf + j];
          }
        const double nx = std::sqrt(std::inner_product(x.begin(), x.end(), x.begin(), 0.0));
        if (!(nx > 1e-8 * n0) || q >= nbuf) continue;
        Q.resize((size_t)m * nbuf, 0.0);
        for (int i = 0; i < m; ++i) Q[(size_t)i * nbuf + q] = x[i] / nx;
        ++q;
      }
      std::vector<double> Qc((size_t)m * q);
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < q; ++j) Qc[(size_t)i * q + j] = Q[(size_t)i * nbuf + j];
      for (DevBuf<double> *B : {&V, &PV, &MV}) {
        combine(Qc, q, B->get(), Vt.get());
        d2d(B->get(), Vt.get(), (size_t)q * n * sizeof(double), c);
      }
      for (std::vector<double> *H : {&Pm, &Mm}) {
        std::vector<double> HQ((size_t)m * q, 0.0), Hnew((size_t)S * S, 0.0);
        for (int i = 0; i < m; ++i)
          for (int k = 0; k < m; ++k) {
            const double h = (*H)[(size_t)i * S + k];
            for (int j = 0; j < q; ++j) HQ[(size_t)i * q + j] += h * Qc[(size_t)k * q + j];
          }
        for (int a = 0; a < q; ++a)
          for (int b2 = 0; b2 < q; ++b2) {
            double t = 0.0;
            for (int i = 0; i < m; ++i) t += Qc[(size_t)i * q + a] * HQ[(size_t)i * q + b2];
            Hnew[(size_t)a * S + b2] = t;
          }
        for (int a = 0; a < q; ++a)
          for (int b2 = 0; b2 < a; ++b2)
            Hnew[(size_t)a * S + b2] = Hnew[(size_t)b2 * S + a] = 0.5 * (Hnew[(size_t)a * S + b2] + Hnew[(size_t)b2 * S + a]);
        *H = Hnew;
      }
      m = q;
    }
    int knew = orthonormalize(c, n, T.get(), nsel, V.get(), m, nullptr, 0);
    knew = std::min(knew, S - m);
    if (knew <= 0) break;
    d2d(V.get() + (size_t)m * n, T.get(), (size_t)knew * n * sizeof(double), c);
    apply_pm(m, knew);
    grow(m, m + knew);
    m += knew;
  }
  c.stats.davidson_iterations = it;
  double mr = 0.0;
  for (int r = 0; r < nroots; ++r) mr = std::max(mr, res[r]);
  c.stats.davidson_residual = mr;
  // X = (X+Y + X-Y)/2, Y = (X+Y - X-Y)/2
  std::vector<double> half(nroots, 0.5), mhalf(nroots, -0.5);
  DevBuf<double> hb, mhb;
  hb.alloc(nroots);
  mhb.alloc(nroots);
  h2d(hb.get(), half.data(), nroots * sizeof(double), c);
  h2d(mhb.get(), mhalf.data(), nroots * sizeof(double), c);
  if (X_dev) {
    d2d(X_dev, Xp.get(), (size_t)nroots * n * sizeof(double), c);
    row_axpby(nroots, n, hb.get(), X_dev, hb.get(), Xm.get(), c.stream);
  }
  if (Y_dev) {
    d2d(Y_dev, Xp.get(), (size_t)nroots * n * sizeof(double), c);
    row_axpby(nroots, n, hb.get(), Y_dev, mhb.get(), Xm.get(), c.stream);
  }
  if (omega_host) std::memcpy(omega_host, om.data(), nroots * sizeof(double));
  sync(c);
  c.stats.ms_davidson = ms_since(t0);
  if (!conv) throw Error(BSE_ERR_NOT_CONVERGED, "full-BSE Davidson reached max_iter");
}

// U vector (Sec. SI, non-SCF reading) with grids of type R
template <class R>
void uvector_t(Ctx &c, int root, double *U) {
  Grids<R> &g = c.grids<R>();
  const double *A = c.roots.get() + (size_t)root * c.nocc * c.npw;
  const bool k1e = (c.spin == 0) && !(c.flags & BSE_FLAG_NO_K1E);
  const bool k1d = !(c.flags & BSE_FLAG_NO_K1D);
  DevBuf<double> LA, S;
  DevBuf<R> vh, ar, T;
  LA.alloc((size_t)c.nocc * c.npw);
  S.alloc((size_t)c.nocc * c.nocc);
  vh.alloc(c.nr);
  ar.alloc((size_t)c.nocc * c.nr);
  T.alloc((size_t)c.nocc * c.nr);
  // a_v(r)
  const long capf = (long)(g.work.n / c.nr) * 2;
  for (int f0 = 0; f0 < c.nocc; f0 += (int)capf) {
    const int nf = (int)std::min<long>(capf, c.nocc - f0);
    const int nq = (nf + 1) / 2;
    BSE_CUDA(cudaMemsetAsync(g.work.get(), 0, (size_t)nq * c.nr * sizeof(CT<R>), c.stream));
    k::scatter_pairs<R, double>(c, nf, A + (long)f0 * c.npw, g.work.get(), 1.0 / std::sqrt(c.omega));
    fft_exec(c, g.work.get(), nq, +1);
    k::unpack_real<R, R>(c.nr, nf, g.work.get(), ar.get() + (long)f0 * c.nr, c.stream);
  }
  if (c.wan.on && k1d) {
    // under pair pruning the canonical tau is not cached: -sum_v' tau_v'v a_v' on the fly for
    // this one vector (all pairs v' <= v through W, contracted with a), so U is the exact one
    BSE_CUDA(cudaMemsetAsync(T.get(), 0, (size_t)c.nocc * c.nr * sizeof(R), c.stream));
    for (long p0 = 0; p0 < c.npairs; p0 += kPairBatch) {
      const int np = (int)std::min<long>(kPairBatch, c.npairs - p0);
      k::pair_products<R>(c.nr, np, c.pairs.get() + p0, g.phir.get(), g.phir.get(), g.work.get(), c.stream);
      pair_screen<R>(c, np, g.work.get(), g.sbuf.get(), g.qbuf.get());
      k::sigma_contract<R>(c, np, c.pairs.get() + p0, g.work.get(), ar.get(), T.get(), true);
    }
    apply_liouville_t<R>(c, 1, A, LA.get(), 0, S.get(), vh.get(), T.get());  // S[v][w] = <phi_w|(M A)_v>
  } else {
    apply_liouville_t<R>(c, 1, A, LA.get(), 0, S.get(), vh.get());  // S[v][w] = <phi_w|(M A)_v>
  }
  BSE_CUDA(cudaMemsetAsync(T.get(), 0, (size_t)c.nocc * c.nr * sizeof(R), c.stream));
  if (k1e) {
    // T_w = 2 [v_c * Delta rho] a_w  (first term of the K1e contribution, Sec. SI)
    for (int f0 = 0; f0 < c.nocc; f0 += (int)capf) {
      const int nf = (int)std::min<long>(capf, c.nocc - f0);
      const int nq = (nf + 1) / 2;
      k::pack_real<R>(c.nr, nf, ar.get() + (long)f0 * c.nr, g.work.get(), c.stream);
      k::mul_grid<R>(c.nr, nq, g.work.get(), vh.get(), (R)2, c.stream);
      k::unpack_real<R, R>(c.nr, nf, g.work.get(), T.get() + (long)f0 * c.nr, c.stream);
    }
  }
  if (c.hartree) {
    // T_w += 2 [v_c * Delta rho^(x)] phi_w: the f_Hxc = v_c term of the D contribution (Sec. SI),
    // 2 the closed-shell factor of rho; Delta rho^(x) = sum_v a_v^2 - phi_v (O phi)_v (Eq. 5)
    DevBuf<double> O;
    DevBuf<R> Or, psi, rx;
    O.alloc((size_t)c.nocc * c.nocc);
    psi.alloc((size_t)c.nocc * c.nr);
    rx.alloc(c.nr);
    dgemm('N', 'T', c.nocc, c.nocc, c.npw, 1.0, A, c.npw, A, c.npw, 0.0, O.get(), c.nocc, c.stream);
    if constexpr (std::is_same<R, float>::value) {
      Or.alloc((size_t)c.nocc * c.nocc);
      k::convert((long)c.nocc * c.nocc, O.get(), Or.get(), c.stream);
      sgemm('N', 'N', c.nocc, (int)c.nr, c.nocc, 1.0f, Or.get(), c.nocc, g.phir.get(), (int)c.nr, 0.0f, psi.get(),
            (int)c.nr, c.stream);
    } else {
      dgemm('N', 'N', c.nocc, (int)c.nr, c.nocc, 1.0, O.get(), c.nocc, g.phir.get(), (int)c.nr, 0.0, psi.get(),
            (int)c.nr, c.stream);
    }
    k::xdensity<R>(c.nr, c.nocc, g.phir.get(), ar.get(), psi.get(), rx.get(), c.stream);
    coulomb_grid<R>(c, rx.get());
    k::add_product<R>(c.nr, c.nocc, rx.get(), g.phir.get(), (R)2, T.get(), c.stream);
  }
  if (k1d) {
    // T_w -= sum_v [W * (a_v a_w)] phi_v  (first term of the K1d contribution, Sec. SI)
    R *X = g.sbuf.get();
    R *Qm = g.qbuf.get();
    for (long p0 = 0; p0 < c.npairs; p0 += kPairBatch) {
      const int np = (int)std::min<long>(kPairBatch, c.npairs - p0);
      k::pair_products<R>(c.nr, np, c.pairs.get() + p0, ar.get(), ar.get(), g.work.get(), c.stream);
      pair_screen<R>(c, np, g.work.get(), X, Qm);
      k::sigma_contract<R>(c, np, c.pairs.get() + p0, g.work.get(), g.phir.get(), T.get());
    }
  }
  // to the sphere, P_c, and the S term
  for (int f0 = 0; f0 < c.nocc; f0 += (int)capf) {
    const int nf = (int)std::min<long>(capf, c.nocc - f0);
    const int nq = (nf + 1) / 2;
    k::pack_real<R>(c.nr, nf, T.get() + (long)f0 * c.nr, g.work.get(), c.stream);
    fft_exec(c, g.work.get(), nq, -1);
    k::gather_pairs<R, double>(c, nf, g.work.get(), U + (long)f0 * c.npw, std::sqrt(c.omega) / c.nr);
  }
  project_pc(c, c.nocc, U, nullptr);
  // u_w -= sum_v S_wv a_v with S_wv = S[v][w]
  dgemm('T', 'N', c.nocc, c.npw, c.nocc, -1.0, S.get(), c.nocc, A, c.npw, 1.0, U, c.npw, c.stream);
  sync(c);
}

void uvector_impl(Ctx &c, int root, double *U) {
  if (c.prec == 0) {
    uvector_t<double>(c, root, U);
  } else {
    uvector_t<float>(c, root, U);
    check_device_flag(c);
  }
}

// Batched preconditioned CG for P_c (H - eps_v) x_v = b_v on P_c, all orbitals at once, with the
// operator on grids of type R; x starts at zero.  Stops when every ||r_v|| <= tol * ||b_v||.
// Returns the iterations; relmax receives the largest relative residual.
// ---- the Z-vector conjugate gradients ----------------------------------------------------------
// The scalars of the iteration live on the device, so that an iteration is a fixed sequence of
// launches: the step lengths (per orbital row, or for the coupled operator from block sums), the
// residual norms and the decision to go on.  That sequence is captured once per context as the
// body of a WHILE conditional graph node; one launch of the graph then runs the whole solve and
// the host reads the outcome once.
namespace {
constexpr int kCgThreads = 256;

// block sums (coupled) or per-row values: thread 0's s1/s2 hold the sums after the call
__device__ void block_sum2(double *s1, double *s2) {
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      s1[threadIdx.x] += s1[threadIdx.x + h];
      s2[threadIdx.x] += s2[threadIdx.x + h];
    }
    __syncthreads();
  }
}

// alpha = rz / pAp (per row; coupled: sum rz / sum pAp for every row); al = alpha, aln = -alpha
__global__ void __launch_bounds__(kCgThreads) cg_alpha_kernel(int no, int coupled, const double *__restrict__ rz,
                                                              const double *__restrict__ pap, double *__restrict__ al,
                                                              double *__restrict__ aln) {
  __shared__ double s1[kCgThreads], s2[kCgThreads];
  if (coupled) {
    double x = 0.0, y = 0.0;
    for (int v = threadIdx.x; v < no; v += blockDim.x) {
      x += rz[v];
      y += pap[v];
    }
    s1[threadIdx.x] = x;
    s2[threadIdx.x] = y;
    block_sum2(s1, s2);
    const double a = (s2[0] > 0 && s1[0] > 0) ? s1[0] / s2[0] : 0.0;
    for (int v = threadIdx.x; v < no; v += blockDim.x) {
      al[v] = a;
      aln[v] = -a;
    }
  } else {
    for (int v = threadIdx.x; v < no; v += blockDim.x) {
      const double a = (pap[v] > 0 && rz[v] > 0) ? rz[v] / pap[v] : 0.0;
      al[v] = a;
      aln[v] = -a;
    }
  }
}

// beta = rz_new / rz (per row; coupled: block sums), then rz = rz_new
__global__ void __launch_bounds__(kCgThreads) cg_beta_kernel(int no, int coupled, double *__restrict__ rz,
                                                             const double *__restrict__ rzn, double *__restrict__ be) {
  __shared__ double s1[kCgThreads], s2[kCgThreads];
  if (coupled) {
    double x = 0.0, y = 0.0;
    for (int v = threadIdx.x; v < no; v += blockDim.x) {
      x += rz[v];
      y += rzn[v];
    }
    s1[threadIdx.x] = x;
    s2[threadIdx.x] = y;
    block_sum2(s1, s2);
    const double b = s1[0] > 0 ? s2[0] / s1[0] : 0.0;
    for (int v = threadIdx.x; v < no; v += blockDim.x) {
      be[v] = b;
      rz[v] = rzn[v];
    }
  } else {
    for (int v = threadIdx.x; v < no; v += blockDim.x) {
      be[v] = rz[v] > 0 ? rzn[v] / rz[v] : 0.0;
      rz[v] = rzn[v];
    }
  }
}

// the relative residual (largest per row, or of the block), the iteration count and the stop rule:
// converged, max_iter reached, or (stall > 0) no fall below 0.7 of the best value for `stall`
// iterations.  Inside the captured loop it also sets the WHILE node's condition.
__global__ void __launch_bounds__(kCgThreads) cg_control_kernel(int no, int coupled, const double *__restrict__ rr,
                                                                const double *__restrict__ r0, CgState *st,
                                                                cudaGraphConditionalHandle handle, int graphed) {
  __shared__ double s1[kCgThreads], s2[kCgThreads];
  double x = 0.0, y = 0.0;
  for (int v = threadIdx.x; v < no; v += blockDim.x) {
    if (coupled) {
      x += rr[v];
      y += r0[v];
    } else {
      x = fmax(x, r0[v] > 0 ? sqrt(fmax(0.0, rr[v]) / r0[v]) : 0.0);
    }
  }
  s1[threadIdx.x] = x;
  s2[threadIdx.x] = y;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      s1[threadIdx.x] = coupled ? s1[threadIdx.x] + s1[threadIdx.x + h] : fmax(s1[threadIdx.x], s1[threadIdx.x + h]);
      s2[threadIdx.x] += s2[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double relmax = coupled ? (s2[0] > 0 ? sqrt(fmax(0.0, s1[0]) / s2[0]) : 0.0) : s1[0];
  CgState &S = *st;
  S.it += 1;
  S.relmax = relmax;
  int done = relmax <= S.tol || S.it >= S.maxit;
  if (!done && S.stall > 0) {
    if (relmax < 0.7 * S.best) {
      S.best = relmax;
      S.best_it = S.it;
    } else if (S.it - S.best_it >= S.stall) {
      done = 1;
    }
  }
  S.done = done;
  if (graphed) cudaGraphSetConditional(handle, done ? 0u : 1u);
}
}  // namespace

// every device address the captured conjugate-gradient loop records
std::vector<const void *> cg_fingerprint(const Ctx &c, const double *x) {
  std::vector<const void *> f = apply_fingerprint(c);
  const CgWork &w = c.cg;
  for (const void *p : {(const void *)w.Rr.get(), (const void *)w.Zr.get(), (const void *)w.P.get(),
                        (const void *)w.AP.get(), (const void *)w.dots.get(), (const void *)w.rz.get(),
                        (const void *)w.rr.get(), (const void *)w.r0.get(), (const void *)w.al.get(),
                        (const void *)w.aln.get(), (const void *)w.be.get(), (const void *)w.Cb.get(),
                        (const void *)w.Ck.get(), (const void *)w.zth.get(), (const void *)w.vsh.get(),
                        (const void *)w.part.get(), (const void *)w.s64.get(), (const void *)w.st.get(),
                        (const void *)x, (const void *)c.empty.get(), (const void *)c.eps_empty_d.get(),
                        (const void *)c.eps.get(), (const void *)c.g64.colbuf.get(), (const void *)c.g32.colbuf.get()})
    f.push_back(p);
  return f;
}

// Run the iteration `body` (handle, graphed) until the control kernel stops it, through the
// context's captured WHILE graph for this key (made on first use, remade when a recorded address
// moved).  False when no graph can serve (profiling on, graphs switched off, the first solve on
// this context, or a capture that failed or allocated): the caller then loops on the host.
bool run_cg_graph(Ctx &c, int key, const double *x, const std::function<void(cudaGraphConditionalHandle, int)> &body,
                  CgState &out) {
  CgWork &w = c.cg;
  if (w.failed[key] || c.prof.on || (c.flags & BSE_FLAG_NO_GRAPHS) || w.plain_runs[key] == 0) return false;
  auto it = w.graphs.find(key);
  if (it != w.graphs.end() && w.fp[key] != cg_fingerprint(c, x)) {
    if (verbose()) {
      const std::vector<const void *> now = cg_fingerprint(c, x);
      size_t i = 0;
      while (i < now.size() && i < w.fp[key].size() && now[i] == w.fp[key][i]) ++i;
      std::fprintf(stderr, "[bse zvector] captured loop %d rebuilt: recorded address %zu moved\n", key, i);
    }
    cudaGraphExecDestroy(it->second);
    w.graphs.erase(it);
    it = w.graphs.end();
  }
  if (it == w.graphs.end()) {
    const auto tc = clk::now();
    cudaGraph_t graph = nullptr;
    auto give_up = [&]() {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      w.failed[key] = true;
      return false;
    };
    if (cudaGraphCreate(&graph, 0) != cudaSuccess) return give_up();
    cudaGraphConditionalHandle handle;
    if (cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault) != cudaSuccess)
      return give_up();
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = handle;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np) != cudaSuccess) return give_up();
    cudaGraph_t bodyg = np.conditional.phGraph_out[0];
    const long long n0 = launch_count_now();
    const long long a0 = tl_alloc_calls;
    if (cudaStreamBeginCaptureToGraph(c.stream, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
        cudaSuccess)
      return give_up();
    bool ok = true;
    try {
      body(handle, 1);
    } catch (...) {
      ok = false;
    }
    cudaGraph_t captured = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(c.stream, &captured);
    const long long nk = launch_count_now() - n0;
    add_launches(-nk);  // nothing ran
    if (!ok || ec != cudaSuccess || tl_alloc_calls != a0) return give_up();
    cudaGraphExec_t exec = nullptr;
    if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) return give_up();
    cudaGraphDestroy(graph);
    w.graphs[key] = exec;
    w.body_kernels[key] = nk;
    w.fp[key] = cg_fingerprint(c, x);
    it = w.graphs.find(key);
    if (verbose())
      std::fprintf(stderr, "[bse zvector] captured loop %d: %lld kernels per iteration, %.2f ms to capture\n", key,
                   nk, ms_since(tc));
  }
  BSE_CUDA(cudaGraphLaunch(it->second, c.stream));
  d2h(&out, w.st.get(), sizeof(CgState), c);
  add_launches((long long)out.it * w.body_kernels[key]);
  return true;
}

template <class R>
// stall > 0: stop once the largest relative residual has not fallen below 0.7 of its best value
// for `stall` iterations (an inner solve of the refinement at the FP32 operator's rounding floor).
// coupled: the Hartree model's operator (apply op 2), which couples the orbitals: one CG over the
// whole block (step lengths from block inner products), converged on the block's relative residual.
// x must keep its address from one call to the next for the captured loop to be reused.
int pcg_t(Ctx &c, const double *b, double *x, double tol, int maxit, double &relmax, int stall = 0,
          bool coupled = false) {
  const int no = c.nocc;
  const long n = (long)c.npw;
  const size_t vec = (size_t)no * n;
  CgWork &w = c.cg;
  w.Rr.alloc(vec);
  w.Zr.alloc(vec);
  w.P.alloc(vec);
  w.AP.alloc(vec);
  for (DevBuf<double> *d : {&w.dots, &w.rz, &w.rr, &w.r0, &w.al, &w.aln, &w.be, &w.vsh}) d->alloc(no);
  // Symmetric positive-definite two-level preconditioner for P_c (H - eps_v) on P_c:
  //   M^-1 r = sum_{c in E} phi_c <phi_c|r> / (eps_c - eps_v) + Q K Q r,
  // E the solved empty states, Q = 1 - P_E, K = (1/2 |G|^2 + 1)^-1; then P_c.
  const int ne = (int)c.eps_empty.size();
  w.Cb.alloc((size_t)no * std::max(1, ne));
  w.Ck.alloc((size_t)no * std::max(1, ne));
  w.zth.alloc(1);
  w.s64.alloc((size_t)1 << 20);
  w.st.alloc(1);
  {
    std::vector<double> v(no, 1.0);
    h2d(w.vsh.get(), v.data(), no * sizeof(double), c);
    const double zero = 0.0;
    h2d(w.zth.get(), &zero, sizeof(double), c);
  }
  auto precond = [&](double *dst, const double *src) {
    if (ne > 0) {
      dgemm('N', 'T', no, ne, c.npw, 1.0, src, c.npw, c.empty.get(), c.npw, 0.0, w.Cb.get(), ne, c.stream, &w.s64);
      d2d(dst, src, vec * sizeof(double), c);
      dgemm('N', 'N', no, c.npw, ne, -1.0, w.Cb.get(), ne, c.empty.get(), c.npw, 1.0, dst, c.npw, c.stream, &w.s64);
      k::precond_diag(no, n, dst, c.kin.get(), c.npw, w.vsh.get(), 0.0, nullptr, 1e-3, dst, c.stream);
      dgemm('N', 'T', no, ne, c.npw, 1.0, dst, c.npw, c.empty.get(), c.npw, 0.0, w.Ck.get(), ne, c.stream, &w.s64);
      // Cb / (eps_c - eps_v) - Ck   (theta = 0, one row per orbital)
      k::subspace_den(no, ne, no, w.Cb.get(), w.Ck.get(), c.eps_empty_d.get(), c.eps.get(), 0.0, w.zth.get(), 1e-8,
                      w.Cb.get(), c.stream);
      dgemm('N', 'N', no, c.npw, ne, 1.0, w.Cb.get(), ne, c.empty.get(), c.npw, 1.0, dst, c.npw, c.stream, &w.s64);
    } else {
      k::precond_diag(no, n, src, c.kin.get(), c.npw, w.vsh.get(), 0.0, nullptr, 1e-3, dst, c.stream);
    }
    project_pc(c, no, dst, nullptr, &w.s64);
  };
  BSE_CUDA(cudaMemsetAsync(x, 0, vec * sizeof(double), c.stream));
  d2d(w.Rr.get(), b, vec * sizeof(double), c);
  precond(w.Zr.get(), w.Rr.get());
  d2d(w.P.get(), w.Zr.get(), vec * sizeof(double), c);
  rowdot(no, n, w.Rr.get(), w.Zr.get(), w.rz.get(), c.stream, &w.part);
  rowdot(no, n, w.Rr.get(), w.Rr.get(), w.r0.get(), c.stream, &w.part);
  std::vector<double> r0(no);
  d2h(r0.data(), w.r0.get(), no * sizeof(double), c);
  relmax = 0.0;
  for (int v = 0; v < no; ++v) relmax = std::max(relmax, r0[v] > 0 ? 1.0 : 0.0);
  if (relmax == 0.0) return 0;
  const CgState s0 = {tol, 1.0, 0.0, maxit, stall, 0, 0, 0};
  h2d(w.st.get(), &s0, sizeof(CgState), c);
  // one iteration: the operator on the search direction, step, residual, preconditioned residual,
  // new direction, stop decision
  auto body = [&](cudaGraphConditionalHandle handle, int graphed) {
    apply_liouville_t<R>(c, 1, w.P.get(), w.AP.get(), coupled ? 2 : 1, nullptr, nullptr);
    rowdot(no, n, w.P.get(), w.AP.get(), w.dots.get(), c.stream, &w.part);
    cg_alpha_kernel<<<1, kCgThreads, 0, c.stream>>>(no, coupled ? 1 : 0, w.rz.get(), w.dots.get(), w.al.get(),
                                                    w.aln.get());
    BSE_CHECK_LAUNCH();
    row_axpby(no, n, nullptr, x, w.al.get(), w.P.get(), c.stream);
    row_axpby(no, n, nullptr, w.Rr.get(), w.aln.get(), w.AP.get(), c.stream);
    rowdot(no, n, w.Rr.get(), w.Rr.get(), w.rr.get(), c.stream, &w.part);
    precond(w.Zr.get(), w.Rr.get());
    rowdot(no, n, w.Rr.get(), w.Zr.get(), w.dots.get(), c.stream, &w.part);
    cg_beta_kernel<<<1, kCgThreads, 0, c.stream>>>(no, coupled ? 1 : 0, w.rz.get(), w.dots.get(), w.be.get());
    BSE_CHECK_LAUNCH();
    row_axpby(no, n, w.be.get(), w.P.get(), nullptr, w.Zr.get(), c.stream);
    cg_control_kernel<<<1, kCgThreads, 0, c.stream>>>(no, coupled ? 1 : 0, w.rr.get(), w.r0.get(), w.st.get(),
                                                      handle, graphed);
    BSE_CHECK_LAUNCH();
  };
  const int key = (std::is_same<R, float>::value ? 2 : 0) + (coupled ? 1 : 0);
  CgState fin{};
  const bool graphed = run_cg_graph(c, key, x, body, fin);
  c.stats.zvector_graphed = graphed ? 1 : 0;
  if (!graphed) {
    // host loop: one read of the stop decision per iteration
    for (;;) {
      body(0, 0);
      d2h(&fin, w.st.get(), sizeof(CgState), c);
      if (verbose() && (fin.it % 10 == 0))
        std::fprintf(stderr, "[bse zvector] it=%d max relative residual=%.3e\n", fin.it, fin.relmax);
      if (fin.done) break;
    }
    ++w.plain_runs[key];
  }
  relmax = fin.relmax;
  project_pc(c, no, x, nullptr);
  sync(c);
  return std::min(fin.it, maxit);
}

// Z-vector (Eq. 7): P_c (H - eps_v) Z_v = -u_v (non-SCF model), or with the Hartree kernel terms
// 2 K1e,KS + 2 K2e,KS (Hartree-SCF model; one coupled system).  FP64: one PCG.  Mixed: FP64
// iterative refinement, r = -U - A Z with the FP64 operator, around FP32-operator PCG corrections.
void zvector_impl(Ctx &c, int root, double tol, int maxit) {
  BSE_REQUIRE(c.nroots > 0, "bse_zvector needs bse_davidson first");
  BSE_REQUIRE(root >= 0 && root < c.nroots, "root out of range");
  BSE_REQUIRE(tol > 0 && std::isfinite(tol), "tol must be positive");
  const int no = c.nocc;
  const long n = (long)c.npw;
  auto t0 = clk::now();
  c.uvec.alloc((size_t)no * n);
  c.zvec.alloc((size_t)no * n);
  uvector_impl(c, root, c.uvec.get());
  c.stats.ms_uvec = ms_since(t0);
  auto t1 = clk::now();
  DevBuf<double> rhs, minus1;
  rhs.alloc(no * n);
  minus1.alloc(no);
  {
    std::vector<double> m1(no, -1.0);
    h2d(minus1.get(), m1.data(), no * sizeof(double), c);
  }
  d2d(rhs.get(), c.uvec.get(), no * n * sizeof(double), c);
  row_axpby(no, n, minus1.get(), rhs.get(), nullptr, nullptr, c.stream);  // rhs = -U
  double relmax = 0.0;
  int its = 0;
  bool conv = false;
  const bool coupled = c.hartree;
  if (c.prec == 0) {
    its = pcg_t<double>(c, rhs.get(), c.zvec.get(), tol, maxit, relmax, 0, coupled);
    conv = relmax <= tol;
  } else {
    DevBuf<double> r, AZ, dots;
    DevBuf<double> &dz = c.cg.dz;  // fixed address: the inner solves' captured loop records it
    r.alloc(no * n);
    AZ.alloc(no * n);
    dz.alloc(no * n);
    dots.alloc(no);
    std::vector<double> b2(no), r2(no);
    rowdot(no, n, rhs.get(), rhs.get(), dots.get(), c.stream);
    d2h(b2.data(), dots.get(), no * sizeof(double), c);
    BSE_CUDA(cudaMemsetAsync(c.zvec.get(), 0, no * n * sizeof(double), c.stream));
    d2d(r.get(), rhs.get(), no * n * sizeof(double), c);
    // each FP32 correction only needs to gain a few digits: the FP32 operator's rounding
    // (~1e-7 of ||A||) times the condition number of the smallest-gap orbital bounds how far
    // an inner solve can go, and the FP64 residual recovers the rest
    for (int outer = 0; outer < 20 && its < maxit; ++outer) {
      double inner_rel = 0.0;
      its += pcg_t<float>(c, r.get(), dz.get(), 1e-3, std::min(60, maxit - its), inner_rel, 10, coupled);
      row_axpby(no, n, nullptr, c.zvec.get(), nullptr, dz.get(), c.stream);
      // FP64 residual of the accumulated solution
      apply_liouville_t<double>(c, 1, c.zvec.get(), AZ.get(), coupled ? 2 : 1, nullptr, nullptr);
      d2d(r.get(), rhs.get(), no * n * sizeof(double), c);
      row_axpby(no, n, nullptr, r.get(), minus1.get(), AZ.get(), c.stream);
      rowdot(no, n, r.get(), r.get(), dots.get(), c.stream);
      d2h(r2.data(), dots.get(), no * sizeof(double), c);
      relmax = 0.0;
      if (coupled) {
        double sr = 0.0, sb = 0.0;
        for (int v = 0; v < no; ++v) sr += std::max(0.0, r2[v]), sb += b2[v];
        relmax = sb > 0 ? std::sqrt(sr / sb) : 0.0;
      } else {
        for (int v = 0; v < no; ++v)
          relmax = std::max(relmax, b2[v] > 0 ? std::sqrt(std::max(0.0, r2[v]) / b2[v]) : 0.0);
      }
      if (verbose())
        std::fprintf(stderr, "[bse zvector] refinement %d: FP64 relative residual %.3e\n", outer, relmax);
      if (relmax <= tol) {
        conv = true;
        break;
      }
    }
    project_pc(c, no, c.zvec.get(), nullptr);
    sync(c);
  }
  c.stats.zvector_iterations = its;
  c.stats.zvector_residual = relmax;
  c.stats.ms_zvector = ms_since(t1);
  c.z_root = root;
  if (!conv) throw Error(BSE_ERR_NOT_CONVERGED, "Z-vector solve reached max_iter");
}

void forces_impl(Ctx &c, int root, double *F_host) {
  BSE_REQUIRE(c.nroots > 0, "bse_forces needs bse_davidson first");
  BSE_REQUIRE(root >= 0 && root < c.nroots, "root out of range");
  if (c.z_root != root) zvector_impl(c, root, 1e-10, 1000);
  auto t0 = clk::now();
  const int no = c.nocc;
  const double *A = c.roots.get() + (size_t)root * no * c.npw;
  DevBuf<double> ar, zr, psi, O, part, dw;
  ar.alloc((size_t)no * c.nr);
  zr.alloc((size_t)no * c.nr);
  psi.alloc((size_t)no * c.nr);
  O.alloc((size_t)no * no);
  Grids<double> &g = c.g64;  // the force densities and the contraction are FP64 in both modes
  const long capf = (long)(g.work.n / c.nr) * 2;
  auto to_grid = [&](const double *X, double *R) {
    for (int f0 = 0; f0 < no; f0 += (int)capf) {
      const int nf = (int)std::min<long>(capf, no - f0);
      const int nq = (nf + 1) / 2;
      BSE_CUDA(cudaMemsetAsync(g.work.get(), 0, (size_t)nq * c.nr * sizeof(double2), c.stream));
      k::scatter_pairs<double, double>(c, nf, X + (long)f0 * c.npw, g.work.get(), 1.0 / std::sqrt(c.omega));
      fft_exec(c, g.work.get(), nq, +1);
      k::unpack_real<double, double>(c.nr, nf, g.work.get(), R + (long)f0 * c.nr, c.stream);
    }
  };
  to_grid(A, ar.get());
  to_grid(c.zvec.get(), zr.get());
  // O[v'][v] = <a_v'|a_v>, Psi = O phi(r)  (Eq. 5 second term)
  dgemm('N', 'T', no, no, c.npw, 1.0, A, c.npw, A, c.npw, 0.0, O.get(), no, c.stream);
  dgemm('N', 'N', no, (int)c.nr, no, 1.0, O.get(), no, g.phir.get(), (int)c.nr, 0.0, psi.get(), (int)c.nr,
        c.stream);
  c.rho_x.alloc(c.nr);
  c.rho_z.alloc(c.nr);
  k::rel_density(c, g.phir.get(), ar.get(), psi.get(), zr.get(), c.rho_x.get(), c.rho_z.get());
  // rho_rel in G space
  d2d(psi.get(), c.rho_x.get(), c.nr * sizeof(double), c);
  row_axpby(1, c.nr, nullptr, psi.get(), nullptr, c.rho_z.get(), c.stream);
  k::fill_real_grid(c.nr, g.work.get(), psi.get(), c.stream);
  fft_exec(c, g.work.get(), 1, -1);
  AtomArgs at(c);
  const int nchunk = (int)std::max<long>(1, std::min<long>(64, c.nr / 8192));
  part.alloc((size_t)c.natoms * nchunk * 3);
  dw.alloc(c.natoms * 3);
  k::force_reduce(c, g.work.get(), at.pd.get(), at.zd.get(), at.sd.get(), at.q(), part.get(), nchunk, dw.get());
  std::vector<double> h(c.natoms * 3);
  d2h(h.data(), dw.get(), h.size() * sizeof(double), c);
  for (int i = 0; i < c.natoms * 3; ++i) F_host[i] = -h[i];
  c.have_rho = true;
  c.stats.ms_forces = ms_since(t0);
}

}  // namespace
}  // namespace bse

// ---------------------------------------------------------------------------------
// Excited-state relaxation
namespace bse {
namespace {
// FIRE (Bitzek et al., PRL 97, 170201 (2006)) with unit masses: semi-implicit Euler steps in
// which the velocity is mixed toward the force direction while the power F.v stays positive
// (after kMinUp such steps the time step grows and the mixing decays), and zeroed, with the
// time step halved, when it turns negative.  Returns the number of force evaluations.
struct FireOut {
  int evals = 0;
  double energy = 0.0;
  bool converged = false;
};
FireOut fire(int n, double *x, const std::function<int(const double *, double &, double *)> &grad, double fmax,
             int max_evals, double dt, double dt_max, double max_move) {
  const int kMinUp = 5;
  const double kInc = 1.1, kDec = 0.5, kAlpha0 = 0.1, kAlphaDecay = 0.99;
  std::vector<double> v(n, 0.0), F(n);
  double alpha = kAlpha0;
  int nup = 0;
  FireOut out;
  while (out.evals < max_evals) {
    double E = 0.0;
    if (grad(x, E, F.data()) != 0) throw Error(BSE_ERR_INVALID, "energy callback failed");
    ++out.evals;
    out.energy = E;
    BSE_REQUIRE(std::isfinite(E), "non-finite energy");
    double fm = 0.0, f2 = 0.0, v2 = 0.0, P = 0.0;
    for (int i = 0; i < n; ++i) {
      BSE_REQUIRE(std::isfinite(F[i]), "non-finite force");
      fm = std::max(fm, std::fabs(F[i]));
      f2 += F[i] * F[i];
      v2 += v[i] * v[i];
      P += F[i] * v[i];
    }
    if (fm <= fmax) {
      out.converged = true;
      return out;
    }
    if (P > 0.0) {
      const double fn = std::sqrt(f2), vn = std::sqrt(v2);
      for (int i = 0; i < n; ++i) v[i] = (1.0 - alpha) * v[i] + alpha * vn * F[i] / fn;
      if (nup > kMinUp) {
        dt = std::min(dt * kInc, dt_max);
        alpha *= kAlphaDecay;
      }
      ++nup;
    } else {
      std::fill(v.begin(), v.end(), 0.0);
      alpha = kAlpha0;
      dt *= kDec;
      nup = 0;
    }
    double dmax = 0.0;
    for (int i = 0; i < n; ++i) {
      v[i] += dt * F[i];
      dmax = std::max(dmax, std::fabs(dt * v[i]));
    }
    const double sc = dmax > max_move ? max_move / dmax : 1.0;
    for (int i = 0; i < n; ++i) x[i] += sc * dt * v[i];
  }
  return out;
}

struct RelaxResult {
  double energy = 0.0, omega = 0.0;
  int evals = 0;
};

// FIRE on E = E_gs + omega for one context (see bse_relax)
RelaxResult relax_impl(Ctx &c, const bse_relax_opts &o, bse_gs_energy_fn gs, void *user, int system, double *pos) {
  const double fmax = o.fmax, dav_tol = o.davidson_tol > 0 ? o.davidson_tol : 1e-8;
  const double z_tol = o.zvector_tol > 0 ? o.zvector_tol : 1e-10;
  BSE_REQUIRE(fmax > 0 && std::isfinite(fmax), "fmax must be positive");
  BSE_REQUIRE(o.max_steps >= 1, "max_steps must be >= 1");
  BSE_REQUIRE(o.root >= 0 && o.root < 64, "root out of range");
  BSE_REQUIRE(gs, "a ground-state energy callback is required");
  const double dt = o.dt > 0 ? o.dt : 0.1, dt_max = o.dt_max > 0 ? o.dt_max : 0.5;
  const double max_move = o.max_move > 0 ? o.max_move : 0.1;
  const int n = 3 * c.natoms;
  struct FlagGuard {
    Ctx &c;
    int saved;
    ~FlagGuard() { c.flags = saved; }
  } guard{c, c.flags};
  c.flags |= BSE_FLAG_WARM_START;
  std::vector<double> Fw(n), Fg(n), w(o.root + 1);
  double fcur = HUGE_VAL;
  bool tight = !o.inexact;
  RelaxResult res;
  auto grad = [&](const double *x, double &E, double *F) -> int {
    // inexact solves: tolerances in proportion to the largest force of the previous step
    double dtol = dav_tol, ztol = z_tol;
    if (!tight) {
      dtol = std::max(dav_tol, std::min(1e-4, 1e-2 * fcur));
      ztol = std::max(z_tol, std::min(1e-3, 1e-1 * fcur));
    }
    c.pos.assign(x, x + n);
    geometry_stage(c);
    bse_davidson_impl(c, o.root + 1, dtol, 500, w.data(), nullptr);
    zvector_impl(c, o.root, ztol, 3000);
    forces_impl(c, o.root, Fw.data());
    double Eg = 0.0;
    if (gs(system, c.natoms, x, &Eg, Fg.data(), user) != 0) return 1;
    E = Eg + w[o.root];
    fcur = 0.0;
    for (int i = 0; i < n; ++i) {
      F[i] = Fw[i] + Fg[i];
      fcur = std::max(fcur, std::fabs(F[i]));
    }
    res.omega = w[o.root];
    return 0;
  };
  FireOut r = fire(n, pos, grad, fmax, o.max_steps, dt, dt_max, max_move);
  res.evals = r.evals;
  if (r.converged && !tight) {
    // confirm with the tight tolerances (and continue from there if the forces disagree)
    tight = true;
    FireOut r2 = fire(n, pos, grad, fmax, std::max(1, o.max_steps - res.evals), dt, dt_max, max_move);
    res.evals += r2.evals;
    r = r2;
  }
  res.energy = r.energy;
  if (!r.converged) throw Error(BSE_ERR_NOT_CONVERGED, "relaxation reached max_steps");
  return res;
}
}  // namespace
}  // namespace bse

// =====================================================================================
// C ABI
struct bse_ctx {
  bse::Ctx c;
};

namespace {
void set_err(bse_ctx *ctx, const std::string &m) {
  bse::g_last_error = m;
  if (ctx) ctx->c.last_error = m;
}
}  // namespace

#define BSE_API_BEGIN try {
#define BSE_API_END(ctx)                                       \
  if (ctx) ctx->c.prof.flush();                                \
  }                                                            \
  catch (const bse::Error &e) {                                \
    set_err(ctx, e.what());                                    \
    return e.status;                                           \
  }                                                            \
  catch (const std::exception &e) {                            \
    set_err(ctx, e.what());                                    \
    return BSE_ERR_CUDA;                                       \
  }                                                            \
  return BSE_OK;

extern "C" {

bse_status bse_setup(const bse_system_desc *desc, bse_ctx **out) {
  bse_ctx *ctx = nullptr;
  BSE_API_BEGIN
  BSE_REQUIRE(desc && out, "desc and out are required");
  *out = nullptr;
  const bse_system_desc &d = *desc;
  BSE_REQUIRE(bse::finite_all(d.lattice, 9) && std::isfinite(d.ecut) && d.ecut > 0, "bad lattice or ecut");
  BSE_REQUIRE(d.n_atoms >= 1 && d.pos && d.Z && d.sigma, "atoms are required");
  BSE_REQUIRE(bse::finite_all(d.pos, 3 * (size_t)d.n_atoms) && bse::finite_all(d.Z, d.n_atoms) &&
                  bse::finite_all(d.sigma, d.n_atoms),
              "non-finite atom data");
  for (int a = 0; a < d.n_atoms; ++a) BSE_REQUIRE(d.sigma[a] > 0, "sigma must be positive");
  BSE_REQUIRE(d.n_occ >= 1 && d.n_pdep >= 0, "n_occ >= 1 and n_pdep >= 0 required");
  BSE_REQUIRE(d.spin == 0 || d.spin == 1, "spin must be 0 or 1");
  BSE_REQUIRE(d.precision == 0 || d.precision == 1, "precision must be 0 (FP64) or 1 (mixed)");
  BSE_REQUIRE(std::isfinite(d.scissor), "non-finite scissor");
  ctx = new bse_ctx();
  bse::Ctx &c = ctx->c;
  auto t0 = bse::clk::now();
  c.desc = d;
  c.prec = d.precision;
  c.natoms = d.n_atoms;
  c.nocc = d.n_occ;
  c.spin = d.spin;
  c.flags = d.flags;
  c.autotune = (d.flags & BSE_FLAG_AUTOTUNE) != 0;
  c.scissor = d.scissor;
  BSE_REQUIRE(std::isfinite(d.gs_tol) && d.gs_tol >= 0, "gs_tol must be >= 0");
  c.gs_tol = d.gs_tol > 0 ? d.gs_tol : 1e-11;
  c.pos.assign(d.pos, d.pos + 3 * d.n_atoms);
  c.Z.assign(d.Z, d.Z + d.n_atoms);
  c.sigma.assign(d.sigma, d.sigma + d.n_atoms);
  if (d.q_ion) {
    BSE_REQUIRE(bse::finite_all(d.q_ion, d.n_atoms), "non-finite ionic charges");
    c.q.assign(d.q_ion, d.q_ion + d.n_atoms);
  }
  c.hartree = (d.flags & BSE_FLAG_HARTREE_SCF) != 0;
  c.wan.on = (d.flags & BSE_FLAG_WANNIER_PRUNE) != 0;
  if (c.wan.on) {
    BSE_REQUIRE(std::isfinite(d.pair_cutoff) && d.pair_cutoff > 0, "pair_cutoff must be positive");
    c.wan.cutoff = d.pair_cutoff;
    c.autotune = false;  // the pruned apply has one launch shape
  }
  BSE_REQUIRE(std::isfinite(d.scf_tol) && d.scf_tol >= 0, "scf_tol must be >= 0");
  c.scf_tol = d.scf_tol > 0 ? d.scf_tol : (d.precision == 0 ? 1e-10 : 1e-9);
  if (d.stream) {
    c.stream = (cudaStream_t)d.stream;
  } else {
    BSE_CUDA(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking));
    c.own_stream = true;
  }
  bse::build_tables(c);
  BSE_REQUIRE(c.nocc + 1 <= c.npw, "n_occ must be below the number of plane waves");
  bse::upload_pdep(c);
  bse::ensure_work(c);
  bse::init_pairs(c);
  c.desc.pos = nullptr;
  c.desc.Z = nullptr;
  c.desc.sigma = nullptr;
  c.desc.q_ion = nullptr;
  c.desc.pdep_coef = nullptr;
  c.desc.pdep_lambda = nullptr;
  *out = ctx;
  try {
    bse::geometry_stage(c);
  } catch (const bse::Error &e) {
    if (e.status != BSE_ERR_DEGENERATE) {
      *out = nullptr;
      set_err(nullptr, e.what());
      delete ctx;
      return e.status;
    }
    set_err(ctx, e.what());
    c.stats.ms_setup = bse::ms_since(t0);
    return e.status;
  }
  c.stats.ms_setup = bse::ms_since(t0);
  }
  catch (const bse::Error &e) {
    set_err(nullptr, e.what());
    if (out) *out = nullptr;
    delete ctx;
    return e.status;
  }
  catch (const std::exception &e) {
    set_err(nullptr, e.what());
    if (out) *out = nullptr;
    delete ctx;
    return BSE_ERR_CUDA;
  }
  return BSE_OK;
}

bse_status bse_set_positions(bse_ctx *ctx, const double *pos) {
  BSE_API_BEGIN
  BSE_REQUIRE(ctx && pos, "ctx and pos are required");
  bse::Ctx &c = ctx->c;
  BSE_REQUIRE(bse::finite_all(pos, 3 * (size_t)c.natoms), "non-finite positions");
  c.pos.assign(pos, pos + 3 * c.natoms);
  bse::geometry_stage(c);
  BSE_API_END(ctx)
}

bse_status bse_get_dims(const bse_ctx *ctx, int *dims) {
  if (!ctx || !dims) return BSE_ERR_INVALID;
  const bse::Ctx &c = ctx->c;
  dims[0] = c.npw;
  dims[1] = c.nocc;
  dims[2] = c.npdep;
  dims[3] = c.natoms;
  dims[4] = c.N[0];
  dims[5] = c.N[1];
  dims[6] = c.N[2];
  dims[7] = c.ndens;
  return BSE_OK;
}


bse_status bse_get_ground_state(bse_ctx *ctx, double *eps_host, double *phi_dev) {
  BSE_API_BEGIN
  BSE_REQUIRE(ctx, "ctx is required");
  bse::Ctx &c = ctx->c;
  if (!c.have_gs) throw bse::Error(BSE_ERR_STATE, "no ground state");
  if (eps_host) std::memcpy(eps_host, c.eps_h.data(), c.nocc * sizeof(double));
  if (phi_dev) {
    bse::d2d(phi_dev, c.phi.get(), (size_t)c.nocc * c.npw * sizeof(double), c);
    bse::sync(c);
  }
  BSE_API_END(ctx)
}

bse_status bse_get_empty_states(bse_ctx *ctx, int max_states, int *n_empty, double *eps_host, double *phi_dev) {
  BSE_API_BEGIN
  BSE_REQUIRE(ctx && n_empty && max_states >= 0, "ctx and n_empty are required, max_states >= 0");
  bse::Ctx &c = ctx->c;
  if (!c.have_gs) throw bse::Error(BSE_ERR_STATE, "no ground state");
  const int ne = (int)c.eps_empty.size();
  *n_empty = ne;
  const int k = std::min(ne, max_states);
  if (eps_host && k > 0) std::memcpy(eps_host, c.eps_empty.data(), k * sizeof(double));
  if (phi_dev && k > 0) {
    bse::d2d(phi_dev, c.empty.get(), (size_t)k * c.npw * sizeof(double), c);
    bse::sync(c);
  }
  BSE_API_END(ctx)
}

bse_status bse_apply_liouville(bse_ctx *ctx, int n_vec, const double *A_dev, double *LA_dev, int op) {
  BSE_API_BEGIN
  BSE_REQUIRE(ctx && A_dev && LA_dev, "ctx, A and LA are required");
  BSE_REQUIRE(n_vec >= 0, "n_vec must be >= 0");
  BSE_REQUIRE(op >= 0 && op <= 3, "op must be 0, 1, 2 or 3");
  bse::Ctx &c = ctx->c;
  if (!c.have_gs) throw bse::Error(BSE_ERR_STATE, "no ground state");
  if (op == 2 && !c.hartree) op = 1;
  const size_t bytes = (size_t)n_vec * c.nocc * c.npw * sizeof(double);
  const char *a0 = (const char *)A_dev, *l0 = (const char *)LA_dev;
  BSE_REQUIRE(a0 + bytes <= l0 || l0 + bytes <= a0, "A and LA overlap");
  if (n_vec > 0) {
    if (op == 3) bse::apply_b(c, n_vec, A_dev, LA_dev);
    else bse::apply_liouville(c, n_vec, A_dev, LA_dev, op);
  }
  bse::sync(c);
  BSE_API_END(ctx)
}

bse_status bse_davidson(bse_ctx *ctx, int n_roots, double tol, int max_iter, double *omega_host,
                        double *A_dev) {
  BSE_API_BEGIN
  BSE_REQUIRE(ctx, "ctx is required");
  BSE_REQUIRE(max_iter >= 1, "max_iter must be >= 1");
  bse::Ctx &c = ctx->c;
  if (!c.have_gs) throw bse::Error(BSE_ERR_STATE, "no ground state");
  bse::bse_davidson_impl(c, n_roots, tol, max_iter, omega_host, A_dev);
  for (int r = 0; r + 1 < n_roots; ++r)
    if (r == 0 && !(c.omega_h[1] - c.omega_h[0] >= 1e-6))
      throw bse::Error(BSE_ERR_DEGENERATE, "lowest two roots closer than 1e-6 Ha");
  BSE_API_END(ctx)
}

bse_status bse_davidson_full(bse_ctx *ctx, int n_roots, double tol, int max_iter, double *omega_host,
                             double *X_dev, double *Y_dev) {
  BSE_API_BEGIN
  BSE_REQUIRE(ctx && omega_host, "ctx and omega are required");
  BSE_REQUIRE(max_iter >= 1, "max_iter must be >= 1");
  bse::bse_davidson_full_impl(ctx->c, n_roots, tol, max_iter, omega_host, X_dev, Y_dev);
  BSE_API_END(ctx)
}

bse_status bse_fire_minimize(int n, double *x, bse_grad_fn fn, void *user, double fmax, int max_steps, double dt,
                             double dt_max, double max_move, int *steps_out, double *energy_out) {
  bse_ctx *ctx = nullptr;
  BSE_API_BEGIN
  BSE_REQUIRE(n >= 1 && x && fn, "n, x and fn are required");
  BSE_REQUIRE(fmax > 0 && max_steps >= 1 && dt > 0 && dt_max >= dt && max_move > 0, "bad FIRE parameters");
  auto grad = [&](const double *xx, double &E, double *F) { return fn(n, xx, &E, F, user); };
  bse::FireOut r = bse::fire(n, x, grad, fmax, max_steps, dt, dt_max, max_move);
  if (steps_out) *steps_out = r.evals;
  if (energy_out) *energy_out = r.energy;
  if (!r.converged) throw bse::Error(BSE_ERR_NOT_CONVERGED, "FIRE reached max_steps");
  BSE_API_END(ctx)
}

namespace {
// bse_relax for the system index passed to the callback (0 alone, its batch index in a batch)
bse_status relax_system(bse_ctx *ctx, const bse_relax_opts *opts, bse_gs_energy_fn gs, void *user, int system,
                        double *pos_inout, double *energy_out, double *omega_out, int *steps_out) {
  BSE_API_BEGIN
  BSE_REQUIRE(ctx && opts && pos_inout, "ctx, opts and pos are required");
  BSE_REQUIRE(bse::finite_all(pos_inout, 3 * (size_t)ctx->c.natoms), "non-finite positions");
  bse::RelaxResult r = bse::relax_impl(ctx->c, *opts, gs, user, system, pos_inout);
  if (energy_out) *energy_out = r.energy;
  if (omega_out) *omega_out = r.omega;
  if (steps_out) *steps_out = r.evals;
  BSE_API_END(ctx)
}
}  // namespace

bse_status bse_relax(bse_ctx *ctx, const bse_relax_opts *opts, bse_gs_energy_fn gs, void *user, double *pos_inout,
                     double *energy_out, double *omega_out, int *steps_out) {
  return relax_system(ctx, opts, gs, user, 0, pos_inout, energy_out, omega_out, steps_out);
}

bse_status bse_zvector(bse_ctx *ctx, int root, double tol, int max_iter, double *Z_dev, double *U_dev) {
  BSE_API_BEGIN
  BSE_REQUIRE(ctx, "ctx is required");
  BSE_REQUIRE(max_iter >= 1, "max_iter must be >= 1");
  bse::Ctx &c = ctx->c;
  if (c.nroots == 0) throw bse::Error(BSE_ERR_STATE, "bse_zvector needs bse_davidson first");
  c.have_rho = false;
  bse_status st = BSE_OK;
  std::string msg;
  try {
    bse::zvector_impl(c, root, tol, max_iter);
  } catch (const bse::Error &e) {
    if (e.status != BSE_ERR_NOT_CONVERGED) throw;
    st = e.status;
    msg = e.what();
  }
  const size_t bytes = (size_t)c.nocc * c.npw * sizeof(double);
  if (Z_dev) bse::d2d(Z_dev, c.zvec.get(), bytes, c);
  if (U_dev) bse::d2d(U_dev, c.uvec.get(), bytes, c);
  bse::sync(c);
  if (st != BSE_OK) throw bse::Error(st, msg);
  BSE_API_END(ctx)
}

bse_status bse_forces(bse_ctx *ctx, int root, double *F_host) {
  BSE_API_BEGIN
  BSE_REQUIRE(ctx && F_host, "ctx and F are required");
  bse::Ctx &c = ctx->c;
  if (c.nroots == 0) throw bse::Error(BSE_ERR_STATE, "bse_forces needs bse_davidson first");
  bse::forces_impl(c, root, F_host);
  BSE_API_END(ctx)
}

bse_status bse_get_density(bse_ctx *ctx, int which, double *rho_host) {
  BSE_API_BEGIN
  BSE_REQUIRE(ctx && rho_host, "ctx and rho are required");
  BSE_REQUIRE(which >= 0 && which <= 2, "which must be 0, 1 or 2");
  bse::Ctx &c = ctx->c;
  if (which == 2) {
    if (!c.have_gs) throw bse::Error(BSE_ERR_STATE, "no ground state");
    bse::d2h(rho_host, c.rho_gs.get(), c.nr * sizeof(double), c);
  } else {
    if (!c.have_rho) throw bse::Error(BSE_ERR_STATE, "no densities: call bse_forces first");
    bse::d2h(rho_host, which == 0 ? c.rho_x.get() : c.rho_z.get(), c.nr * sizeof(double), c);
  }
  BSE_API_END(ctx)
}

bse_status bse_sphere_to_grid(bse_ctx *ctx, int n, const double *X_dev, void *P_dev) {
  BSE_API_BEGIN
  BSE_REQUIRE(ctx && n >= 0 && (n == 0 || (X_dev && P_dev)), "ctx, n >= 0, X and P are required");
  bse::Ctx &c = ctx->c;
  if (n > 0) {
    if (c.prec == 0) bse::sphere_to_grid_util<double>(c, n, X_dev, (double2 *)P_dev);
    else bse::sphere_to_grid_util<float>(c, n, X_dev, (float2 *)P_dev);
  }
  bse::sync(c);
  BSE_API_END(ctx)
}

bse_status bse_grid_to_sphere(bse_ctx *ctx, int n, void *P_dev, double *Y_dev) {
  BSE_API_BEGIN
  BSE_REQUIRE(ctx && n >= 0 && (n == 0 || (Y_dev && P_dev)), "ctx, n >= 0, P and Y are required");
  bse::Ctx &c = ctx->c;
  if (n > 0) {
    if (c.prec == 0) bse::grid_to_sphere_util<double>(c, n, (double2 *)P_dev, Y_dev);
    else bse::grid_to_sphere_util<float>(c, n, (float2 *)P_dev, Y_dev);
  }
  bse::sync(c);
  BSE_API_END(ctx)
}

bse_status bse_get_stats(const bse_ctx *ctx, bse_stats *out) {
  if (!ctx || !out) return BSE_ERR_INVALID;
  *out = ctx->c.stats;
  return BSE_OK;
}

bse_status bse_fft3d(int n1, int n2, int n3, int batch, double *data_dev, int direction, void *stream) {
  bse_ctx *ctx = nullptr;
  BSE_API_BEGIN
  BSE_REQUIRE(data_dev && batch >= 0, "data and batch >= 0 are required");
  BSE_REQUIRE(direction == -1 || direction == 1, "direction must be -1 or +1");
  bse::FFTPlan plan;
  try {
    plan.init(n1, n2, n3);
    plan.exec((double2 *)data_dev, batch, direction, (cudaStream_t)stream);
    BSE_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  } catch (...) {
    plan.destroy();
    throw;
  }
  plan.destroy();
  BSE_API_END(ctx)
}

bse_status bse_profile(bse_ctx *ctx, int enable) {
  BSE_API_BEGIN
  BSE_REQUIRE(ctx, "ctx is required");
  bse::Ctx &c = ctx->c;
  c.prof.flush();
  c.prof.on = enable != 0;
  if (enable)
    for (int k = 0; k < BSE_KERNEL_COUNT; ++k) {
      c.prof.launches[k] = 0;
      c.prof.ms[k] = c.prof.bytes[k] = c.prof.flops[k] = 0.0;
    }
  BSE_API_END(ctx)
}

bse_status bse_get_kernel_timing(const bse_ctx *ctx, int kernel, long long *launches, double *total_ms,
                                 double *alg_bytes, double *alg_flops) {
  if (!ctx || kernel < 0 || kernel >= BSE_KERNEL_COUNT) return BSE_ERR_INVALID;
  const bse::KernelProf &p = ctx->c.prof;
  if (launches) *launches = p.launches[kernel];
  if (total_ms) *total_ms = p.ms[kernel];
  if (alg_bytes) *alg_bytes = p.bytes[kernel];
  if (alg_flops) *alg_flops = p.flops[kernel];
  return BSE_OK;
}

long long bse_launch_count(void) { return bse::g_launches.load(); }

bse_status bse_gemm(char ta, char tb, int M, int N, int K, double alpha, const double *A, int lda,
                    const double *B, int ldb, double beta, double *C, int ldc, void *stream) {
  bse_ctx *ctx = nullptr;
  BSE_API_BEGIN
  BSE_REQUIRE((ta == 'N' || ta == 'T') && (tb == 'N' || tb == 'T'), "ta and tb must be 'N' or 'T'");
  BSE_REQUIRE(M >= 0 && N >= 0 && K >= 0 && C, "bad sizes");
  BSE_REQUIRE(K == 0 || (A && B), "A and B are required");
  bse::dgemm(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, (cudaStream_t)stream);
  BSE_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  BSE_API_END(ctx)
}

bse_status bse_gemm_bf16x3(int M, int N, int K, float alpha, const float *A, int lda, const float *B, int ldb,
                           float beta, float *C, int ldc, void *stream) {
  bse_ctx *ctx = nullptr;
  BSE_API_BEGIN
  BSE_REQUIRE(M >= 0 && N >= 0 && K >= 1 && A && B && C, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  bse::SplitBF16 a, b;
  bse::DevBuf<float> part;
  bse::DevBuf<int> err;
  err.alloc(1);
  BSE_CUDA(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
  bse::split_bf16(M, K, A, lda, a, s);
  bse::split_bf16(N, K, B, ldb, b, s);
  bse::umma_gemm_nt(M, N, alpha, a, b, beta, C, ldc, part, err.get(), s);
  int flag = 0;
  BSE_CUDA(cudaMemcpyAsync(&flag, err.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
  BSE_CUDA(cudaStreamSynchronize(s));
  if (flag) throw bse::Error(BSE_ERR_TIMEOUT, "tensor-core GEMM: a bounded wait gave up");
  BSE_API_END(ctx)
}

bse_status bse_host_sym_eig_lowest(int n, const double *A, int k, double *w, double *V) {
  bse_ctx *ctx = nullptr;
  BSE_API_BEGIN
  BSE_REQUIRE(n >= 0 && k >= 0 && k <= n && (n == 0 || (A && w && V)), "bad arguments");
  BSE_REQUIRE(bse::finite_all(A, (size_t)n * n), "non-finite matrix");
  bse::sym_eig_lowest(n, A, k, w, V);
  BSE_API_END(ctx)
}

bse_status bse_host_sym_eig_k(int n, const double *A, int k, double *w, double *V) {
  bse_ctx *ctx = nullptr;
  BSE_API_BEGIN
  BSE_REQUIRE(n >= 0 && k >= 0 && k <= n && (n == 0 || (A && w && V)), "bad arguments");
  BSE_REQUIRE(bse::finite_all(A, (size_t)n * n), "non-finite matrix");
  bse::sym_eig_lowest(n, A, k, w, V, false);
  BSE_API_END(ctx)
}

bse_status bse_selftest_bounded_wait(void *stream) {
  bse_ctx *ctx = nullptr;
  BSE_API_BEGIN
  cudaStream_t s = (cudaStream_t)stream;
  bse::DevBuf<int> flag;
  flag.alloc(1);
  BSE_CUDA(cudaMemsetAsync(flag.get(), 0, sizeof(int), s));
  bse::wait_selftest(s, flag.get());
  int h = 0;
  BSE_CUDA(cudaMemcpyAsync(&h, flag.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
  BSE_CUDA(cudaStreamSynchronize(s));
  if (h) throw bse::Error(BSE_ERR_TIMEOUT, "the bounded wait gave up as designed");
  throw bse::Error(BSE_ERR_CUDA, "the bounded wait did not give up");
  BSE_API_END(ctx)
}

bse_status bse_selftest_k1d_stall(bse_ctx *ctx) {
  BSE_API_BEGIN
  BSE_REQUIRE(ctx, "ctx is required");
  bse::Ctx &c = ctx->c;
  if (!c.have_gs || !c.k1d.ready)
    throw bse::Error(BSE_ERR_STATE, "no tiled FP32 K1d pipeline (mixed precision, n_occ a multiple of 16)");
  bse::Grids<float> &g = c.g32;
  const int nb = bse::k1d_tma_max_nb(c.nocc);
  const size_t need = (size_t)((nb * c.nocc + 1) / 2) * c.nr;
  BSE_REQUIRE(g.work.n >= need && g.work2.n >= need && g.vh.n >= (size_t)((nb + 1) / 2) * c.nr,
              "work grids smaller than one K1d block");
  bse::k1d_tma_stall_test(c, c.k1d, g.phir.get(), g.vloc.get(), g.work.get(), g.vh.get(), g.work2.get());
  bse::sync(c);
  bse::check_device_flag(c);  // BSE_ERR_TIMEOUT when the waits gave up
  throw bse::Error(BSE_ERR_CUDA, "the K1d pipeline's bounded waits did not give up");
  BSE_API_END(ctx)
}

bse_status bse_host_sym_eig(int n, const double *A, double *w, double *V) {
  bse_ctx *ctx = nullptr;
  BSE_API_BEGIN
  BSE_REQUIRE(n >= 0 && (n == 0 || (A && w && V)), "bad arguments");
  BSE_REQUIRE(bse::finite_all(A, (size_t)n * n), "non-finite matrix");
  bse::sym_eig(n, A, w, V);
  BSE_API_END(ctx)
}

bse_status bse_fft3d_noalloc(int n1, int n2, int n3, int batch, double *data_dev, int direction,
                             void *stream) {
  bse_ctx *ctx = nullptr;
  BSE_API_BEGIN
  BSE_REQUIRE(data_dev && batch >= 0, "data and batch >= 0 are required");
  BSE_REQUIRE(direction == -1 || direction == 1, "direction must be -1 or +1");
  bse::fft3d_noalloc(n1, n2, n3, batch, (double2 *)data_dev, direction, (cudaStream_t)stream);
  BSE_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  BSE_API_END(ctx)
}

}  // extern "C"

struct bse_batch {
  int n = 0, nworkers = 0;
  std::vector<bse_ctx *> sys;
  std::vector<bse_status> status;
  std::vector<int> atom_off;           // offsets into the concatenated [3 n_atoms] arrays
  std::vector<std::vector<int>> work;  // systems of each worker, in order
  std::vector<cudaStream_t> streams;
  double setup_ms = 0.0, solve_ms = 0.0;  // device spans of the last setup and solve (CUDA events)
};

namespace {
// run fn(i) for every system on its worker thread (worker w's CUDA stream), all workers at once;
// span_ms (optional): the device time from the first worker's start to the last worker's end,
// from CUDA events recorded on the workers' streams around their systems
template <class F>
void batch_run(bse_batch *b, F fn, double *span_ms = nullptr) {
  int dev = 0;
  cudaGetDevice(&dev);
  const int nw = b->nworkers;
  std::vector<cudaEvent_t> ev0(nw, nullptr), ev1(nw, nullptr);
  bool timed = span_ms != nullptr;
  for (int w = 0; timed && w < nw; ++w)
    timed = cudaEventCreate(&ev0[w]) == cudaSuccess && cudaEventCreate(&ev1[w]) == cudaSuccess;
  std::vector<std::thread> th;
  for (int w = 0; w < nw; ++w)
    th.emplace_back([b, w, dev, &fn, &ev0, &ev1, timed] {
      cudaSetDevice(dev);
      if (timed) cudaEventRecord(ev0[w], b->streams[w]);
      for (int i : b->work[w]) fn(i, w);
      if (timed) cudaEventRecord(ev1[w], b->streams[w]);
    });
  for (auto &t : th) t.join();
  if (timed) {
    double lo = 0.0, hi = 0.0;
    for (int w = 0; w < nw; ++w) {
      float a = 0.f, z = 0.f;
      cudaEventSynchronize(ev1[w]);
      cudaEventElapsedTime(&a, ev0[0], ev0[w]);
      cudaEventElapsedTime(&z, ev0[0], ev1[w]);
      lo = std::min(lo, (double)a);
      hi = std::max(hi, (double)z);
    }
    *span_ms = hi - lo;
  }
  for (int w = 0; w < nw; ++w) {
    if (ev0[w]) cudaEventDestroy(ev0[w]);
    if (ev1[w]) cudaEventDestroy(ev1[w]);
  }
  cudaGetLastError();
}

bse_status first_failure(const bse_batch *b) {
  for (bse_status st : b->status)
    if (st != BSE_OK) return st;
  return BSE_OK;
}
}  // namespace

extern "C" {

bse_status bse_setup_batch(int n, const bse_system_desc *descs, int n_workers, bse_batch **out) {
  if (!out || n < 1 || !descs || n_workers < 1) {
    bse::g_last_error = "bse_setup_batch: n >= 1, descs, n_workers >= 1 and out are required";
    return BSE_ERR_INVALID;
  }
  *out = nullptr;
  bse_batch *b = new bse_batch();
  b->n = n;
  b->nworkers = std::min(n_workers, n);
  b->sys.assign(n, nullptr);
  b->status.assign(n, BSE_OK);
  b->atom_off.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) b->atom_off[i + 1] = b->atom_off[i] + 3 * std::max(0, descs[i].n_atoms);
  // largest estimated cost first (grid points x N_occ^2: the K1d stream and the pair build),
  // each to the least loaded worker
  std::vector<double> cost(n);
  for (int i = 0; i < n; ++i)
    cost[i] = (double)descs[i].grid[0] * descs[i].grid[1] * descs[i].grid[2] *
              ((double)descs[i].n_occ * descs[i].n_occ + 64.0);
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  b->work.assign(b->nworkers, {});
  std::vector<double> load(b->nworkers, 0.0);
  for (int i : order) {
    const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->work[w].push_back(i);
    load[w] += cost[i];
  }
  b->streams.assign(b->nworkers, nullptr);
  for (int w = 0; w < b->nworkers; ++w) {
    if (cudaStreamCreateWithFlags(&b->streams[w], cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      bse::g_last_error = "bse_setup_batch: cudaStreamCreate failed";
      bse_destroy_batch(b);
      return BSE_ERR_CUDA;
    }
  }
  batch_run(b, [&](int i, int w) {
    bse_system_desc d = descs[i];
    d.stream = b->streams[w];
    bse_ctx *ctx = nullptr;
    b->status[i] = bse_setup(&d, &ctx);
    if (ctx && b->status[i] != BSE_OK) {
      bse_destroy(ctx);
      ctx = nullptr;
    }
    if (ctx) {
      ctx->c.use_graphs = !(d.flags & BSE_FLAG_NO_GRAPHS);
      ctx->c.autotune = true;
    }
    b->sys[i] = ctx;
  }, &b->setup_ms);
  *out = b;
  return first_failure(b);
}

bse_status bse_batch_timing(const bse_batch *b, double *setup_ms, double *solve_ms) {
  if (!b) return BSE_ERR_INVALID;
  if (setup_ms) *setup_ms = b->setup_ms;
  if (solve_ms) *solve_ms = b->solve_ms;
  return BSE_OK;
}

bse_status bse_solve_batch(bse_batch *b, double davidson_tol, double zvector_tol, int max_iter, double *omega_host,
                           double *F_host) {
  if (!b || max_iter < 1) return BSE_ERR_INVALID;
  batch_run(b, [&](int i, int) {
    const int na = (b->atom_off[i + 1] - b->atom_off[i]) / 3;
    double w = std::nan("");
    std::vector<double> F(3 * (size_t)na, std::nan(""));
    bse_ctx *ctx = b->sys[i];
    if (ctx) {
      bse_status st = bse_davidson(ctx, 1, davidson_tol, max_iter, &w, nullptr);
      if (st == BSE_OK) st = bse_zvector(ctx, 0, zvector_tol, 10 * max_iter, nullptr, nullptr);
      if (st == BSE_OK) st = bse_forces(ctx, 0, F.data());
      b->status[i] = st;
      if (st != BSE_OK) {
        w = std::nan("");
        std::fill(F.begin(), F.end(), std::nan(""));
      }
    }
    if (omega_host) omega_host[i] = w;
    if (F_host) std::copy(F.begin(), F.end(), F_host + b->atom_off[i]);
  }, &b->solve_ms);
  return first_failure(b);
}

bse_status bse_relax_batch(bse_batch *b, const bse_relax_opts *opts, bse_gs_energy_fn gs, void *user,
                           double *pos_all_inout, double *energy_out, double *omega_out, int *steps_out) {
  if (!b || !opts || !gs || !pos_all_inout) return BSE_ERR_INVALID;
  batch_run(b, [&](int i, int) {
    bse_ctx *ctx = b->sys[i];
    double E = std::nan(""), w = std::nan("");
    int steps = 0;
    if (ctx) {
      b->status[i] = relax_system(ctx, opts, gs, user, i, pos_all_inout + b->atom_off[i], &E, &w, &steps);
    }
    if (energy_out) energy_out[i] = E;
    if (omega_out) omega_out[i] = w;
    if (steps_out) steps_out[i] = steps;
  });
  return first_failure(b);
}

bse_status bse_batch_set_positions(bse_batch *b, const double *pos_all) {
  if (!b || !pos_all) return BSE_ERR_INVALID;
  batch_run(b, [&](int i, int) {
    if (b->sys[i]) b->status[i] = bse_set_positions(b->sys[i], pos_all + b->atom_off[i]);
  });
  return first_failure(b);
}

int bse_batch_size(const bse_batch *b) { return b ? b->n : 0; }

bse_status bse_batch_status(const bse_batch *b, int i) {
  if (!b || i < 0 || i >= b->n) return BSE_ERR_INVALID;
  return b->status[i];
}

bse_ctx *bse_batch_system(bse_batch *b, int i) {
  if (!b || i < 0 || i >= b->n) return nullptr;
  return b->sys[i];
}

void bse_destroy_batch(bse_batch *b) {
  if (!b) return;
  for (auto *ctx : b->sys) bse_destroy(ctx);
  for (auto s : b->streams)
    if (s) cudaStreamDestroy(s);
  delete b;
}

const char *bse_last_error(const bse_ctx *ctx) {
  if (ctx) return ctx->c.last_error.empty() ? "no error" : ctx->c.last_error.c_str();
  return bse::g_last_error.c_str();
}

void bse_destroy(bse_ctx *ctx) { delete ctx; }

}  // extern "C"
