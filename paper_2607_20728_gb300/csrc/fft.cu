// Batched 3D complex FFT for the real-space products of the Liouville operator (Eq. 2).
//
// One kernel per axis.  A CTA stages T lines of length N in shared memory, runs a
// self-sorting (Stockham) mixed-radix 2/3/4/5/8/9 transform out of place between two
// shared buffers, and writes the lines back.  Along the strided axes the T lines of a
// CTA are consecutive in the fastest grid index, so every global load and store of a
// line element moves T contiguous complex numbers.  Twiddles exp(-2 pi i k/N) are
// tabulated on the host in FP64.
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>

#include "fft_codelets.cuh"
#include "internal.cuh"

namespace bse {

namespace {
using namespace fftc;

template <int AXIS, class C>
__global__ void __launch_bounds__(256) fft_axis_kernel(C *__restrict__ data, int n1, int n2, int n3, long nr,
                                                       int batch, AxisArgs<C> ax, int T,
                                                       typename RealOf<C>::T sg) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C *sm = reinterpret_cast<C *>(sm_raw);
  const int N = ax.n;
  C *bufA = sm;
  C *bufB = sm + (size_t)T * N;
  const long g = blockIdx.x;
  long base, stride, tstride;
  int tvalid;
  if (AXIS == 0) {
    const long nl = (long)n2 * n3 * batch;
    const long l0 = g * T;
    tvalid = (int)min((long)T, nl - l0);
    base = l0 * n1;
    tstride = n1;
    stride = 1;
  } else if (AXIS == 1) {
    const int ntile = n1 / T;
    const long rest = g / ntile;
    const int xt = (int)(g % ntile);
    const int z = (int)(rest % n3);
    const long b = rest / n3;
    base = b * nr + (long)z * n1 * n2 + (long)xt * T;
    tstride = 1;
    stride = n1;
    tvalid = T;
  } else {
    const int ntile = n1 / T;
    const long rest = g / ntile;
    const int xt = (int)(g % ntile);
    const int y = (int)(rest % n2);
    const long b = rest / n2;
    base = b * nr + (long)y * n1 + (long)xt * T;
    tstride = 1;
    stride = (long)n1 * n2;
    tvalid = T;
  }
  const int tot = T * N;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    int t, j;
    if (AXIS == 0) {
      t = e / N;
      j = e - t * N;
    } else {
      j = e / T;
      t = e - j * T;
    }
    C v = mkc<C>(0, 0);
    if (t < tvalid) v = data[base + t * tstride + j * stride];
    bufA[t * N + j] = v;
  }
  __syncthreads();
  C *in = bufA, *out = bufB;
  int Ns = 1;
  for (int s = 0; s < ax.nstage; ++s) {
    const int R = ax.radix[s];
    const int nb = N / R;
    const int work = T * nb;
    for (int e = threadIdx.x; e < work; e += blockDim.x) {
      const int t = e / nb;
      const int j = e - t * nb;
      const C *src = in + t * N;
      C *dst = out + t * N;
      stage_bfly_any<C>(R, src, dst, j, N, Ns, ax.tw, sg);
    }
    __syncthreads();
    C *tmp = in;
    in = out;
    out = tmp;
    Ns *= R;
  }
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    int t, j;
    if (AXIS == 0) {
      t = e / N;
      j = e - t * N;
    } else {
      j = e / T;
      t = e - j * T;
    }
    if (t < tvalid) data[base + t * tstride + j * stride] = in[t * N + j];
  }
}

int largest_divisor_le(int n, int cap) {
  for (int t = cap; t >= 1; --t)
    if (n % t == 0) return t;
  return 1;
}

const int kMaxSmem = 160 * 1024;

// the dynamic shared-memory limit is a per-device function attribute: set it once per device
void set_smem_attrs() {
  static std::mutex mu;
  static std::map<int, bool> done;
  int dev = 0;
  BSE_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return;
  BSE_CUDA(cudaFuncSetAttribute(fft_axis_kernel<0, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
  BSE_CUDA(cudaFuncSetAttribute(fft_axis_kernel<1, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
  BSE_CUDA(cudaFuncSetAttribute(fft_axis_kernel<2, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
  BSE_CUDA(cudaFuncSetAttribute(fft_axis_kernel<0, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
  BSE_CUDA(cudaFuncSetAttribute(fft_axis_kernel<1, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
  BSE_CUDA(cudaFuncSetAttribute(fft_axis_kernel<2, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem));
  done[dev] = true;
}

}  // namespace

bool fft_size_ok(int n) {
  if (n < 2 || n > 512) return false;
  int m = n;
  for (int p : {2, 3, 5})
    while (m % p == 0) m /= p;
  return m == 1;
}

namespace {
void factor_axis(FFTAxis &x, int n) {
  x.n = n;
  x.nstage = 0;
  int m = n;
  // large radices first: every stage is one pass over the line in shared memory
  while (m % 8 == 0) { x.radix[x.nstage++] = 8; m /= 8; }
  while (m % 9 == 0) { x.radix[x.nstage++] = 9; m /= 9; }
  while (m % 4 == 0) { x.radix[x.nstage++] = 4; m /= 4; }
  while (m % 2 == 0) { x.radix[x.nstage++] = 2; m /= 2; }
  while (m % 3 == 0) { x.radix[x.nstage++] = 3; m /= 3; }
  while (m % 5 == 0) { x.radix[x.nstage++] = 5; m /= 5; }
}

// exp(-2 pi i k/n), k < n, in FP64 on the host
void twiddles(int n, double2 *out) {
  for (int k = 0; k < n; ++k) {
    const double ang = -2.0 * M_PI * (double)k / (double)n;
    out[k] = make_double2(std::cos(ang), std::sin(ang));
  }
}
}  // namespace

void FFTPlan::init(int n1, int n2, int n3) {
  destroy();
  n[0] = n1;
  n[1] = n2;
  n[2] = n3;
  nr = (long)n1 * n2 * n3;
  for (int a = 0; a < 3; ++a) {
    BSE_REQUIRE(fft_size_ok(n[a]), "FFT sizes must be 2..512 with prime factors 2, 3, 5");
    FFTAxis &x = ax[a];
    factor_axis(x, n[a]);
    std::vector<double2> tw(n[a]);
    twiddles(n[a], tw.data());
    std::vector<float2> tw32(n[a]);
    for (int k = 0; k < n[a]; ++k) tw32[k] = make_float2((float)tw[k].x, (float)tw[k].y);
    void *p = nullptr;
    BSE_CUDA(cudaMalloc(&p, sizeof(double2) * n[a]));
    owned.push_back(p);
    BSE_CUDA(cudaMemcpy(p, tw.data(), sizeof(double2) * n[a], cudaMemcpyHostToDevice));
    x.tw = (double2 *)p;
    void *p32 = nullptr;
    BSE_CUDA(cudaMalloc(&p32, sizeof(float2) * n[a]));
    owned.push_back(p32);
    BSE_CUDA(cudaMemcpy(p32, tw32.data(), sizeof(float2) * n[a], cudaMemcpyHostToDevice));
    x.tw32 = (float2 *)p32;
  }
  set_smem_attrs();
}

void FFTPlan::destroy() {
  for (void *p : owned) cudaFree(p);
  owned.clear();
}

namespace {
using namespace fftc;
template <class C>
void exec_axes(const FFTPlan &p, C *data, int batch, int dir, cudaStream_t s) {
  if (batch <= 0) return;
  using T = typename RealOf<C>::T;
  const T sg = dir < 0 ? (T)-1 : (T)1;
  const int n1 = p.n[0], n2 = p.n[1], n3 = p.n[2];
  for (int a = 0; a < 3; ++a) {
    const FFTAxis &x = p.ax[a];
    AxisArgs<C> args;
    args.n = x.n;
    args.nstage = x.nstage;
    std::memcpy(args.radix, x.radix, sizeof(args.radix));
    if constexpr (sizeof(C) == sizeof(double2)) args.tw = reinterpret_cast<const C *>(x.tw);
    else args.tw = reinterpret_cast<const C *>(x.tw32);
    int T;
    long nblk;
    if (a == 0) {
      T = std::max(1, std::min(32, (int)(32768 / sizeof(C)) / x.n));
      const long nl = (long)n2 * n3 * batch;
      nblk = (nl + T - 1) / T;
    } else {
      T = largest_divisor_le(n1, 16);
      while (T > 1 && (long)T * x.n * 2 * (long)sizeof(C) > kMaxSmem) T = largest_divisor_le(n1, T - 1);
      nblk = (long)(n1 / T) * (a == 1 ? n3 : n2) * batch;
    }
    const size_t smem = (size_t)2 * T * x.n * sizeof(C);
    if (a == 0)
      fft_axis_kernel<0, C><<<nblk, 256, smem, s>>>(data, n1, n2, n3, p.nr, batch, args, T, sg);
    else if (a == 1)
      fft_axis_kernel<1, C><<<nblk, 256, smem, s>>>(data, n1, n2, n3, p.nr, batch, args, T, sg);
    else
      fft_axis_kernel<2, C><<<nblk, 256, smem, s>>>(data, n1, n2, n3, p.nr, batch, args, T, sg);
    BSE_CHECK_LAUNCH();
  }
}
}  // namespace

void FFTPlan::exec(double2 *data, int batch, int dir, cudaStream_t s) const { exec_axes(*this, data, batch, dir, s); }
void FFTPlan::exec(float2 *data, int batch, int dir, cudaStream_t s) const { exec_axes(*this, data, batch, dir, s); }

// ---------------------------------------------------------------------------------
// Allocation-free variant of the batched 3D FFT.  Its only global memory beyond the
// caller's data is the twiddle tables, kept in one file-scope device array shared by
// every call on a device (3 axes x 512 entries = 24 KB per GPU that loads the library).
namespace {
constexpr int kNoAllocMaxN = 512;
__device__ __align__(256) double2 g_noalloc_twiddle[3 * kNoAllocMaxN];

std::mutex g_noalloc_mu;
std::map<int, double2 *> g_noalloc_addr;  // device ordinal -> device address of the table

// Device address of the table for the current device, looked up once per device.
double2 *noalloc_table() {
  int dev = 0;
  BSE_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  auto it = g_noalloc_addr.find(dev);
  if (it != g_noalloc_addr.end()) return it->second;
  double2 *p = nullptr;
  BSE_CUDA(cudaGetSymbolAddress((void **)&p, g_noalloc_twiddle));
  g_noalloc_addr[dev] = p;
  return p;
}
}  // namespace

void fft3d_noalloc(int n1, int n2, int n3, int batch, double2 *data, int dir, cudaStream_t s) {
  const int n[3] = {n1, n2, n3};
  for (int a = 0; a < 3; ++a)
    BSE_REQUIRE(fft_size_ok(n[a]) && n[a] <= kNoAllocMaxN,
                "bse_fft3d_noalloc: sizes must be 2..512 with prime factors 2, 3, 5");
  double2 *table = noalloc_table();
  // every entry the transform reads is overwritten here, so nothing needs clearing
  std::vector<double2> h((size_t)3 * kNoAllocMaxN, make_double2(0.0, 0.0));
  FFTPlan plan;  // describes the axes only: its twiddle pointers point into the shared table
  plan.n[0] = n1;
  plan.n[1] = n2;
  plan.n[2] = n3;
  plan.nr = (long)n1 * n2 * n3;
  for (int a = 0; a < 3; ++a) {
    factor_axis(plan.ax[a], n[a]);
    twiddles(n[a], h.data() + (size_t)a * kNoAllocMaxN);
    plan.ax[a].tw = table + (size_t)a * kNoAllocMaxN;
  }
  set_smem_attrs();
  BSE_CUDA(cudaMemcpyAsync(table, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
  plan.exec(data, batch, dir, s);
}

}  // namespace bse
