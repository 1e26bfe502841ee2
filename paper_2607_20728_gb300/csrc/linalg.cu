// FP64 dense linear algebra for the plain path: tiled SIMT GEMM (occupied overlaps of
// P_c, PDEP projection and back-projection of Eq. 3, Davidson subspace products),
// deterministic row reductions, and the host eigensolver for Rayleigh-Ritz matrices.
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>
#include <type_traits>
#include <vector>

#include "internal.cuh"

namespace bse {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

// C = alpha op(A) op(B) + beta C over k in [kz * kchunk, min(K, (kz + 1) kchunk)), kz = blockIdx.z.
// With split-K (gridDim.z > 1) each slice writes its own partial matrix C + kz * M * ldc.
// T: the arithmetic type of the products and sums; TI: the operands' type in memory (rounded to
// T as the tiles are staged); TO: the output's type (alpha and beta applied in TO)
template <bool TA, bool TB, class T, class TI = T, class TO = T>
__global__ void __launch_bounds__(256) dgemm_kernel(int M, int N, int K, int kchunk, TO alpha,
                                                    const TI *__restrict__ A, int lda,
                                                    const TI *__restrict__ B, int ldb,
                                                    TO beta, TO *__restrict__ C, int ldc) {
  __shared__ T As[BK][BM + 2];
  __shared__ T Bs[BK][BN + 2];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  if (gridDim.z > 1) C += (long)blockIdx.z * M * ldc;
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = tid + i * 256;
      int m, k;
      if (!TA) { k = e % BK; m = e / BK; } else { m = e % BM; k = e / BM; }
      const int gm = m0 + m, gk = k0 + k;
      T v = 0;
      if (gm < M && gk < kend) v = (T)(TA ? A[(long)gk * lda + gm] : A[(long)gm * lda + gk]);
      As[k][m] = v;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = tid + i * 256;
      int n, k;
      if (!TB) { n = e % BN; k = e / BN; } else { k = e % BK; n = e / BK; }
      const int gn = n0 + n, gk = k0 + k;
      T v = 0;
      if (gn < N && gk < kend) v = (T)(TB ? B[(long)gn * ldb + gk] : B[(long)gk * ldb + gn]);
      Bs[k][n] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      TO *c = C + (long)gm * ldc + gn;
      const TO v = (TO)acc[i][j];
      *c = beta == (TO)0 ? alpha * v : alpha * v + beta * (*c);
    }
  }
}

// Small-output NT product: C[i][j] = sum_k A[i][k] B[j][k] for M*N <= 4096 outputs and long K.
// Each CTA stages K-chunks of the M + N rows in shared memory; every output is owned by a group
// of tpo adjacent lanes (tpo a power of two <= 32, so that small outputs still occupy the CTA)
// which accumulate interleaved k in registers over the CTA's chunks and are summed by shuffles;
// part[cta][M][N] is reduced afterwards.
constexpr int kSmallOut = 4096;
constexpr int kSmallPerThread = kSmallOut / 256;

// Skinny inner products for at most four rows of A: part[z][i][j] = sum over the z-th K slice of
// A[i][k] B[j][k] for i < MM and the kSkinnyRows rows j of B this block takes.  Threads stream
// consecutive k (coalesced loads of every row; VEC: pairs of k as one 16-byte load, rows and slices
// 16-byte aligned), keep the MM x kSkinnyRows products in registers, and reduce them through warp
// shuffles and shared memory at the end: every element of B is read once, and the FP64 pipe bounds
// the launch.
constexpr int kSkinnyRows = 8;
template <int MM, bool VEC>
__global__ void __launch_bounds__(256) gemm_nt_skinny_kernel(int N, int K, int kchunk, const double *__restrict__ A,
                                                             int lda, const double *__restrict__ B, int ldb,
                                                             double *__restrict__ part) {
  __shared__ double red[8][MM * kSkinnyRows];
  const int j0 = blockIdx.x * kSkinnyRows;
  const int nj = min(kSkinnyRows, N - j0);
  const long k0 = (long)blockIdx.y * kchunk;
  const long k1 = min((long)K, k0 + kchunk);
  double acc[MM][kSkinnyRows];
#pragma unroll
  for (int i = 0; i < MM; ++i)
#pragma unroll
    for (int r = 0; r < kSkinnyRows; ++r) acc[i][r] = 0.0;
  auto step = [&](long k) {
    double a[MM];
#pragma unroll
    for (int i = 0; i < MM; ++i) a[i] = __ldg(&A[(long)i * lda + k]);
#pragma unroll
    for (int r = 0; r < kSkinnyRows; ++r) {
      if (r < nj) {
        const double b = __ldg(&B[(long)(j0 + r) * ldb + k]);
#pragma unroll
        for (int i = 0; i < MM; ++i) acc[i][r] = fma(a[i], b, acc[i][r]);
      }
    }
  };
  if constexpr (VEC) {
    // k0 is even; pairs (k, k + 1) with k + 1 < k1, then the odd last element of the matrix
    for (long k = k0 + 2 * threadIdx.x; k + 1 < k1; k += 2 * blockDim.x) {
      double2 a[MM];
#pragma unroll
      for (int i = 0; i < MM; ++i) a[i] = __ldg(reinterpret_cast<const double2 *>(&A[(long)i * lda + k]));
#pragma unroll
      for (int r = 0; r < kSkinnyRows; ++r) {
        if (r < nj) {
          const double2 b = __ldg(reinterpret_cast<const double2 *>(&B[(long)(j0 + r) * ldb + k]));
#pragma unroll
          for (int i = 0; i < MM; ++i) acc[i][r] = fma(a[i].y, b.y, fma(a[i].x, b.x, acc[i][r]));
        }
      }
    }
    if (((k1 - k0) & 1) && threadIdx.x == 0) step(k1 - 1);
  } else {
    for (long k = k0 + threadIdx.x; k < k1; k += blockDim.x) step(k);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < MM; ++i)
#pragma unroll
    for (int r = 0; r < kSkinnyRows; ++r) {
      double v = acc[i][r];
#pragma unroll
      for (int w = 16; w > 0; w >>= 1) v += __shfl_xor_sync(0xffffffffu, v, w);
      if (lane == 0) red[warp][i * kSkinnyRows + r] = v;
    }
  __syncthreads();
  if ((int)threadIdx.x < MM * kSkinnyRows) {
    const int i = threadIdx.x / kSkinnyRows, r = threadIdx.x % kSkinnyRows;
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][threadIdx.x];
    if (r < nj) part[((long)blockIdx.y * MM + i) * N + j0 + r] = v;
  }
}

__global__ void __launch_bounds__(256) gemm_nt_small_kernel(int M, int N, int K, int L, int tpo,
                                                            const double *__restrict__ A, int lda,
                                                            const double *__restrict__ B, int ldb,
                                                            double *__restrict__ part) {
  extern __shared__ double sh[];
  const int Lp = L + 1;  // padded row stride against bank conflicts
  double *As = sh;
  double *Bs = sh + (size_t)M * Lp;
  const int MN = M * N;
  const int slots = MN * tpo;
  const int j = threadIdx.x & (tpo - 1);
  double acc[kSmallPerThread];
#pragma unroll
  for (int q = 0; q < kSmallPerThread; ++q) acc[q] = 0.0;
  const int nchunk = (K + L - 1) / L;
  for (int ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
    const int k0 = ch * L;
    const int len = min(L, K - k0);
    for (int e = threadIdx.x; e < (M + N) * L; e += blockDim.x) {
      const int row = e / L, l = e - row * L;
      double v = 0.0;
      if (l < len) v = row < M ? A[(long)row * lda + k0 + l] : B[(long)(row - M) * ldb + k0 + l];
      sh[(size_t)row * Lp + l] = v;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kSmallPerThread; ++q) {
      const int idx = threadIdx.x + q * 256;
      if (idx < slots) {
        const int o = idx / tpo;
        const int i = o / N, jj = o - i * N;
        const double *a = As + (size_t)i * Lp;
        const double *b = Bs + (size_t)jj * Lp;
        double s = acc[q];
        for (int l = j; l < len; l += tpo) s = fma(a[l], b[l], s);
        acc[q] = s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < kSmallPerThread; ++q) {
    const int idx = threadIdx.x + q * 256;
    if ((idx & ~31) >= slots) break;  // warp-uniform: every lane of the warp takes the shuffles
    double s = acc[q];                  // zero for slots past the end (whole groups of tpo lanes)
    for (int w = 1; w < tpo; w <<= 1) s += __shfl_xor_sync(0xffffffffu, s, w);
    if (j == 0 && idx < slots) part[(long)blockIdx.x * MN + idx / tpo] = s;
  }
}

// Small-M product C = alpha op(A) B + beta C, op(A) M x K with M <= 16, K <= 1024, B [K][N]:
// op(A) in shared memory, one output column per thread, B read once with eight rows in flight
// per thread (the product is a stream over B).  MT is M at compile time (0: run-time M).
constexpr int kSmallM = 16;

template <bool TA, int MT>
__global__ void __launch_bounds__(256) gemm_smallm_kernel(int M_, int N, int K, double alpha,
                                                          const double *__restrict__ A, int lda,
                                                          const double *__restrict__ B, int ldb,
                                                          double beta, double *__restrict__ C, int ldc) {
  const int M = MT > 0 ? MT : M_;
  constexpr int MM = MT > 0 ? MT : kSmallM;
  extern __shared__ double sa[];  // [K][M]
  for (int e = threadIdx.x; e < M * K; e += blockDim.x) {
    const int k = e / M, m = e - k * M;
    sa[e] = TA ? A[(long)k * lda + m] : A[(long)m * lda + k];
  }
  __syncthreads();
  const long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (n >= N) return;
  double acc[MM];
#pragma unroll
  for (int m = 0; m < MM; ++m) acc[m] = 0.0;
  constexpr int U = 8;
  int k = 0;
  for (; k + U <= K; k += U) {
    double b[U];
#pragma unroll
    for (int u = 0; u < U; ++u) b[u] = __ldg(&B[(long)(k + u) * ldb + n]);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const double *a = sa + (size_t)(k + u) * M;
#pragma unroll
      for (int m = 0; m < MM; ++m)
        if (MT > 0 || m < M) acc[m] = fma(a[m], b[u], acc[m]);
    }
  }
  for (; k < K; ++k) {
    const double b = __ldg(&B[(long)k * ldb + n]);
    const double *a = sa + (size_t)k * M;
#pragma unroll
    for (int m = 0; m < MM; ++m)
      if (MT > 0 || m < M) acc[m] = fma(a[m], b, acc[m]);
  }
#pragma unroll
  for (int m = 0; m < MM; ++m) {
    if (m >= M) break;
    double *c = C + (long)m * ldc + n;
    *c = beta == 0.0 ? alpha * acc[m] : alpha * acc[m] + beta * (*c);
  }
}

// C = alpha sum_z part[z] + beta C; the partial sums (type TP) are added in the output's type T
template <class T, class TP = T>
__global__ void splitk_reduce(int M, int N, int nsplit, const TP *__restrict__ part, T alpha, T beta,
                              T *__restrict__ C, int ldc) {
  const long total = (long)M * N;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    T s = 0;
    for (int z = 0; z < nsplit; ++z) s += (T)part[(long)z * total + i];
    T *c = C + (i / N) * ldc + (i % N);
    *c = beta == (T)0 ? alpha * s : alpha * s + beta * (*c);
  }
}

__global__ void rowdot_partial(int rows, long len, int nchunk, const double *__restrict__ X,
                               const double *__restrict__ Y, double *__restrict__ part) {
  const int row = blockIdx.y;
  const int ch = blockIdx.x;
  const long per = (len + nchunk - 1) / nchunk;
  const long j0 = (long)ch * per, j1 = min(len, j0 + per);
  const double *x = X + (long)row * len;
  const double *y = Y + (long)row * len;
  double s = 0.0;
  for (long j = j0 + threadIdx.x; j < j1; j += blockDim.x) s = fma(x[j], y[j], s);
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(long)row * nchunk + ch] = red[0];
}

__global__ void rowdot_final(int rows, int nchunk, const double *__restrict__ part, double *out) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= rows) return;
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += part[(long)row * nchunk + c];
  out[row] = s;
}

__global__ void row_axpby_kernel(int rows, long len, const double *__restrict__ a, double *X,
                                 const double *__restrict__ b, const double *__restrict__ Y) {
  const long total = (long)rows * len;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total;
       i += (long)gridDim.x * blockDim.x) {
    const int r = (int)(i / len);
    const double av = a ? a[r] : 1.0;
    const double bv = b ? b[r] : 1.0;
    X[i] = av * X[i] + (Y ? bv * Y[i] : 0.0);
  }
}

__global__ void scale_rows_kernel(int M, int N, int ldc, double beta, double *C) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < (long)M * N;
       i += (long)gridDim.x * blockDim.x) {
    double *c = C + (i / N) * ldc + (i % N);
    *c = beta == 0.0 ? 0.0 : beta * (*c);
  }
}

// Scratch of the reductions and split-K partials: one per host thread.  Every library call
// synchronises its stream before returning, so a thread never has two of its calls' kernels
// in flight on one scratch buffer; worker threads of a batch each own one.
DevBuf<double> &part_buf() {
  thread_local DevBuf<double> p;
  return p;
}

DevBuf<double> &splitk_buf() {
  thread_local DevBuf<double> p;
  return p;
}

DevBuf<float> &splitk_buf32() {
  thread_local DevBuf<float> p;
  return p;
}

// Number of K slices for a tiled product with `tiles` output tiles.  One 256-thread CTA already
// saturates an SM's FP64 pipe, so the time of a launch is about the largest number of CTAs that
// any of the 152 SMs receives times (the K length of one CTA + a fixed per-CTA cost of about
// 8 K steps for the prologue and the partial-tile store); the split minimises that.
int split_for(long tiles, int K) {
  constexpr int kSMs = 152;
  if (K < 2 * 64 || tiles >= 8 * kSMs) return 1;
  const int maxs = std::max(1, std::min(256, K / 64));
  int best = 1;
  double best_cost = 1e300;
  for (int ns = 1; ns <= maxs; ++ns) {
    int kc = (K + ns - 1) / ns;
    kc = (kc + BK - 1) / BK * BK;
    const int nsr = (K + kc - 1) / kc;
    const long waves = (tiles * nsr + kSMs - 1) / kSMs;
    const double cost = (double)waves * (kc + 8) + 0.05 * nsr;
    if (cost < best_cost * 0.999) {
      best_cost = cost;
      best = nsr;
    }
  }
  return best;
}

// tiled path shared by the FP64 and FP32 GEMMs (split-K when the output has few tiles)
// fixed: `scratch` keeps its size (its address is recorded in captured graphs); the split is
// clamped to what fits, down to no split at all
template <class T>
void gemm_tiled(char ta, char tb, int M, int N, int K, T alpha, const T *A, int lda, const T *B, int ldb, T beta,
                T *C, int ldc, cudaStream_t s, DevBuf<T> &scratch, bool fixed = false, int split_pct = 100) {
  const long tiles = (long)((N + BN - 1) / BN) * ((M + BM - 1) / BM);
  int nsplit0 = split_for(tiles, K);
  if (split_pct != 100) nsplit0 = std::max(1, std::min(K / BK, nsplit0 * split_pct / 100));
  if (fixed && (size_t)nsplit0 * M * N > scratch.n) nsplit0 = (int)std::max<size_t>(1, scratch.n / ((size_t)M * N));
  int kchunk = (K + nsplit0 - 1) / nsplit0;
  kchunk = (kchunk + BK - 1) / BK * BK;
  const int nsplit = (K + kchunk - 1) / kchunk;
  T *Cout = C;
  int ldo = ldc;
  T a = alpha, b = beta;
  if (nsplit > 1) {
    if (!fixed) scratch.alloc((size_t)nsplit * M * N);
    Cout = scratch.get();
    ldo = N;
    a = 1;
    b = 0;
  }
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, nsplit);
  const bool TA = (ta == 'T'), TB = (tb == 'T');
  if (!TA && !TB) dgemm_kernel<false, false, T><<<grid, 256, 0, s>>>(M, N, K, kchunk, a, A, lda, B, ldb, b, Cout, ldo);
  else if (!TA && TB) dgemm_kernel<false, true, T><<<grid, 256, 0, s>>>(M, N, K, kchunk, a, A, lda, B, ldb, b, Cout, ldo);
  else if (TA && !TB) dgemm_kernel<true, false, T><<<grid, 256, 0, s>>>(M, N, K, kchunk, a, A, lda, B, ldb, b, Cout, ldo);
  else dgemm_kernel<true, true, T><<<grid, 256, 0, s>>>(M, N, K, kchunk, a, A, lda, B, ldb, b, Cout, ldo);
  BSE_CHECK_LAUNCH();
  if (nsplit > 1) {
    const long total = (long)M * N;
    splitk_reduce<T><<<(int)std::min<long>(4096, (total + 255) / 256), 256, 0, s>>>(M, N, nsplit, Cout, alpha, beta,
                                                                                     C, ldc);
    BSE_CHECK_LAUNCH();
  }
}

// FP64 operands and output, FP32 products and sums: the tiles are rounded to FP32 as they are
// staged, each split-K slice writes FP32 partial sums, and alpha, beta and the sum over slices are
// applied in FP64 (one launch, or two with a split over K)
void gemm_tiled_mixed(char ta, char tb, int M, int N, int K, double alpha, const double *A, int lda, const double *B,
                      int ldb, double beta, double *C, int ldc, cudaStream_t s, DevBuf<float> &scratch,
                      int split_pct) {
  const long tiles = (long)((N + BN - 1) / BN) * ((M + BM - 1) / BM);
  int nsplit0 = split_for(tiles, K);
  if (split_pct != 100) nsplit0 = std::max(1, std::min(K / BK, nsplit0 * split_pct / 100));
  int kchunk = (K + nsplit0 - 1) / nsplit0;
  kchunk = (kchunk + BK - 1) / BK * BK;
  const int nsplit = (K + kchunk - 1) / kchunk;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, nsplit);
  const bool TA = (ta == 'T'), TB = (tb == 'T');
  auto go = [&](auto out, auto a, auto b, int ldo) {
    using TO = std::remove_pointer_t<decltype(out)>;
    if (!TA && !TB)
      dgemm_kernel<false, false, float, double, TO><<<grid, 256, 0, s>>>(M, N, K, kchunk, a, A, lda, B, ldb, b, out, ldo);
    else if (!TA && TB)
      dgemm_kernel<false, true, float, double, TO><<<grid, 256, 0, s>>>(M, N, K, kchunk, a, A, lda, B, ldb, b, out, ldo);
    else if (TA && !TB)
      dgemm_kernel<true, false, float, double, TO><<<grid, 256, 0, s>>>(M, N, K, kchunk, a, A, lda, B, ldb, b, out, ldo);
    else
      dgemm_kernel<true, true, float, double, TO><<<grid, 256, 0, s>>>(M, N, K, kchunk, a, A, lda, B, ldb, b, out, ldo);
    BSE_CHECK_LAUNCH();
  };
  if (nsplit == 1) {
    go(C, alpha, beta, ldc);
    return;
  }
  scratch.alloc((size_t)nsplit * M * N);
  go(scratch.get(), 1.0f, 0.0f, N);
  const long total = (long)M * N;
  splitk_reduce<double, float><<<(int)std::min<long>(4096, (total + 255) / 256), 256, 0, s>>>(
      M, N, nsplit, scratch.get(), alpha, beta, C, ldc);
  BSE_CHECK_LAUNCH();
}

}  // namespace

namespace {
// one full wave of skinny CTAs: resident CTAs per SM for this instantiation
template <int MM, bool VEC>
int skinny_slots() {
  // computed once (thread-safe static initialisation: the batch's worker threads share it)
  static const int slots = [] {
    int per_sm = 0;
    BSE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gemm_nt_skinny_kernel<MM, VEC>, 256, 0));
    int dev = 0, sms = 0;
    BSE_CUDA(cudaGetDevice(&dev));
    BSE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    return std::max(1, per_sm) * std::max(1, sms);
  }();
  return slots;
}

template <int MM, bool VEC>
void skinny_launch(int N, int K, const double *A, int lda, const double *B, int ldb, double alpha, double beta,
                   double *C, int ldc, cudaStream_t s, DevBuf<double> *fixed, DevBuf<double> &scratch) {
  const int nb = (N + kSkinnyRows - 1) / kSkinnyRows;
  int nsplit = std::max(1, std::min(K / 2048, skinny_slots<MM, VEC>() / nb));
  if (fixed) nsplit = (int)std::max<size_t>(1, std::min<size_t>(nsplit, fixed->n / ((size_t)MM * N)));
  int kchunk = (K + nsplit - 1) / nsplit;
  kchunk += kchunk & 1;  // even slice starts keep the 16-byte loads aligned
  nsplit = (K + kchunk - 1) / kchunk;
  DevBuf<double> &p = fixed ? *fixed : scratch;
  if (!fixed) p.alloc((size_t)nsplit * MM * N);
  gemm_nt_skinny_kernel<MM, VEC><<<dim3((unsigned)nb, (unsigned)nsplit), 256, 0, s>>>(N, K, kchunk, A, lda, B, ldb,
                                                                                    p.get());
  BSE_CHECK_LAUNCH();
  const long total = (long)MM * N;
  splitk_reduce<double><<<(int)std::min<long>(4096, (total + 255) / 256), 256, 0, s>>>(MM, N, nsplit, p.get(), alpha,
                                                                                        beta, C, ldc);
  BSE_CHECK_LAUNCH();
}

}  // namespace

void dgemm(char ta, char tb, int M, int N, int K, double alpha, const double *A, int lda,
           const double *B, int ldb, double beta, double *C, int ldc, cudaStream_t s, DevBuf<double> *fixed,
           int split_pct) {
  if (M <= 0 || N <= 0) return;
  if (K <= 0) {
    if (beta != 1.0) {
      scale_rows_kernel<<<(int)std::min<long>(4096, ((long)M * N + 255) / 256), 256, 0, s>>>(
          M, N, ldc, beta, C);
      BSE_CHECK_LAUNCH();
    }
    return;
  }
  // at most four rows of A against any number of rows of B over a very long K (the Davidson
  // subspace products of trial vectors): register-blocked streaming, split over K
  if (ta == 'N' && tb == 'T' && M <= 4 && K >= 65536 && (!fixed || fixed->n >= (size_t)M * N * 8)) {
    const bool vec = ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15) == 0 &&
                     (lda % 2) == 0 && (ldb % 2) == 0;
    auto go = [&](auto mm_c) {
      constexpr int MM = decltype(mm_c)::value;
      if (vec) skinny_launch<MM, true>(N, K, A, lda, B, ldb, alpha, beta, C, ldc, s, fixed, splitk_buf());
      else skinny_launch<MM, false>(N, K, A, lda, B, ldb, alpha, beta, C, ldc, s, fixed, splitk_buf());
    };
    switch (M) {
      case 1: go(std::integral_constant<int, 1>()); break;
      case 2: go(std::integral_constant<int, 2>()); break;
      case 3: go(std::integral_constant<int, 3>()); break;
      default: go(std::integral_constant<int, 4>()); break;
    }
    return;
  }
  // tall-skinny inner products: every output of a small M x N block over a long K
  if (ta == 'N' && tb == 'T' && (long)M * N <= kSmallOut && M + N <= 1024 && K >= 4096 &&
      (!fixed || fixed->n >= (size_t)M * N)) {
    // chunks of L k-values: about two CTAs per SM when K allows, at most 96 KB of staging
    int tpo = 1;
    while (tpo < 32 && (long)M * N * tpo * 2 <= 256) tpo *= 2;
    const int lmax = std::min(256, (int)(96 * 1024 / ((M + N) * sizeof(double))) - 1) / 8 * 8;
    int L = (int)std::min<long>(lmax, std::max<long>(8, ((K + 2 * 152 - 1) / (2 * 152) + 7) / 8 * 8));
    L = std::max(L, 8);
    const int nchunk = (K + L - 1) / L;
    int nct = std::min(nchunk, 2 * 152);
    DevBuf<double> &p = fixed ? *fixed : splitk_buf();
    if (fixed) nct = (int)std::min<size_t>(nct, fixed->n / ((size_t)M * N));
    else p.alloc((size_t)nct * M * N);
    const size_t smem = (size_t)(M + N) * (L + 1) * sizeof(double);
    BSE_CUDA(cudaFuncSetAttribute(gemm_nt_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
    gemm_nt_small_kernel<<<nct, 256, smem, s>>>(M, N, K, L, tpo, A, lda, B, ldb, p.get());
    BSE_CHECK_LAUNCH();
    const long total = (long)M * N;
    splitk_reduce<double><<<(int)std::min<long>(4096, (total + 255) / 256), 256, 0, s>>>(M, N, nct, p.get(), alpha,
                                                                                          beta, C, ldc);
    BSE_CHECK_LAUNCH();
    return;
  }
  // few output rows, short K, long N: one column per thread
  if (tb == 'N' && M <= kSmallM && K <= 1024 && N >= 4096) {
    const size_t smem = (size_t)M * K * sizeof(double);
    const int grid = (N + 255) / 256;
    auto go = [&](auto ta_c, auto mt_c) {
      constexpr bool TA = decltype(ta_c)::value;
      constexpr int MT = decltype(mt_c)::value;
      BSE_CUDA(cudaFuncSetAttribute(gemm_smallm_kernel<TA, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    130 * 1024));
      gemm_smallm_kernel<TA, MT><<<grid, 256, smem, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    };
    auto by_m = [&](auto ta_c) {
      switch (M) {
        case 1: go(ta_c, std::integral_constant<int, 1>()); break;
        case 2: go(ta_c, std::integral_constant<int, 2>()); break;
        case 3: go(ta_c, std::integral_constant<int, 3>()); break;
        case 4: go(ta_c, std::integral_constant<int, 4>()); break;
        default: go(ta_c, std::integral_constant<int, 0>()); break;
      }
    };
    if (ta == 'T') by_m(std::true_type());
    else by_m(std::false_type());
    BSE_CHECK_LAUNCH();
    return;
  }
  if (fixed) gemm_tiled<double>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s, *fixed, true, split_pct);
  else gemm_tiled<double>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s, splitk_buf(), false, split_pct);
}

void mgemm(char ta, char tb, int M, int N, int K, double alpha, const double *A, int lda, const double *B, int ldb,
           double beta, double *C, int ldc, cudaStream_t s, int split_pct) {
  if (M <= 0 || N <= 0) return;
  if (K <= 0) {
    dgemm(ta, tb, M, N, 0, alpha, A, lda, B, ldb, beta, C, ldc, s);
    return;
  }
  gemm_tiled_mixed(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s, splitk_buf32(), split_pct);
}

void sgemm(char ta, char tb, int M, int N, int K, float alpha, const float *A, int lda, const float *B, int ldb,
           float beta, float *C, int ldc, cudaStream_t s, DevBuf<float> *fixed, int split_pct) {
  if (M <= 0 || N <= 0 || K <= 0) return;
  if (fixed) gemm_tiled<float>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s, *fixed, true, split_pct);
  else gemm_tiled<float>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, s, splitk_buf32(), false, split_pct);
}

void rowdot(int rows, long len, const double *X, const double *Y, double *out, cudaStream_t s,
            DevBuf<double> *part) {
  if (rows <= 0) return;
  int nchunk = (int)std::min<long>(64, std::max<long>(1, len / 4096));
  DevBuf<double> &p = part ? *part : part_buf();
  p.alloc((size_t)rows * nchunk);
  rowdot_partial<<<dim3(nchunk, rows), 256, 0, s>>>(rows, len, nchunk, X, Y, p.get());
  BSE_CHECK_LAUNCH();
  rowdot_final<<<(rows + 127) / 128, 128, 0, s>>>(rows, nchunk, p.get(), out);
  BSE_CHECK_LAUNCH();
}

void row_axpby(int rows, long len, const double *a, double *X, const double *b, const double *Y,
               cudaStream_t s) {
  const long total = (long)rows * len;
  if (total <= 0) return;
  const int grid = (int)std::min<long>(152 * 16, (total + 255) / 256);
  row_axpby_kernel<<<grid, 256, 0, s>>>(rows, len, a, X, b, Y);
  BSE_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------------
// Persistent host worker threads for the O(n^3) loops of the Rayleigh-Ritz eigensolver.  One
// caller at a time uses them (a try-lock: other callers, e.g. the worker threads of a batch, run
// their solve serially), so concurrent solvers do not oversubscribe the cores.  Idle workers spin
// for 2 ms after a job (the Davidson solvers call the eigensolver every few ms) and then sleep
// on a condition variable.  A process forked after the pool was made runs serially (its copy of
// the pool has no threads).
namespace {
class HostPool {
 public:
  static HostPool &instance() {
    static HostPool pool;
    return pool;
  }
  int threads() const { return nt_; }
  // f(tid, nt) on the caller (tid 0) and the nt - 1 workers; false (nothing run) when the pool is
  // busy or has no workers
  bool run(const std::function<void(int, int)> &f) {
    if (nt_ <= 1 || getpid() != pid_ || !use_.try_lock()) return false;
    job_ = &f;
    done_.store(0, std::memory_order_relaxed);
    {
      std::lock_guard<std::mutex> lk(mu_);
      gen_.fetch_add(1, std::memory_order_release);
    }
    cv_.notify_all();
    f(0, nt_);
    while (done_.load(std::memory_order_acquire) < nt_ - 1) {
    }
    job_ = nullptr;
    use_.unlock();
    return true;
  }
  // all nt threads of the current job
  void barrier() {
    const long g = bar_gen_.load(std::memory_order_acquire);
    if (bar_count_.fetch_add(1, std::memory_order_acq_rel) == nt_ - 1) {
      bar_count_.store(0, std::memory_order_relaxed);
      bar_gen_.fetch_add(1, std::memory_order_release);
    } else {
      while (bar_gen_.load(std::memory_order_acquire) == g) {
      }
    }
  }
  ~HostPool() {
    if (getpid() != pid_) return;
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_.store(true);
    }
    cv_.notify_all();
    for (auto &t : th_) t.join();
  }

 private:
  HostPool() {
    pid_ = getpid();
    const unsigned hw = std::thread::hardware_concurrency();
    nt_ = (int)std::max(1u, std::min(8u, hw / 2));
    for (int t = 1; t < nt_; ++t) th_.emplace_back([this, t] { worker(t); });
  }
  void worker(int tid) {
    long seen = 0;
    for (;;) {
      auto t0 = std::chrono::steady_clock::now();
      long spins = 0;
      long g;
      while ((g = gen_.load(std::memory_order_acquire)) == seen) {
        if (stop_.load(std::memory_order_relaxed)) return;
        if ((++spins & 1023) == 0 && std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(2)) {
          std::unique_lock<std::mutex> lk(mu_);
          cv_.wait(lk, [&] { return gen_.load(std::memory_order_acquire) != seen || stop_.load(); });
          if (stop_.load()) return;
          t0 = std::chrono::steady_clock::now();
        }
      }
      seen = g;
      (*job_)(tid, nt_);
      done_.fetch_add(1, std::memory_order_release);
    }
  }
  std::vector<std::thread> th_;
  int nt_ = 1;
  pid_t pid_ = 0;
  std::mutex use_, mu_;
  std::condition_variable cv_;
  std::atomic<long> gen_{0};
  std::atomic<int> done_{0};
  std::atomic<bool> stop_{false};
  const std::function<void(int, int)> *job_ = nullptr;
  // the arrival counter and the generation the waiters spin on sit on separate cache lines
  alignas(64) std::atomic<int> bar_count_{0};
  alignas(64) std::atomic<long> bar_gen_{0};
};
// the eigensolver takes the pool from this size on (below it the barriers cost more than the
// split saves)
constexpr int kParallelEigMin = 64;
}  // namespace

// Host symmetric eigensolver.  Householder reduction to tridiagonal form followed by
// the implicit symmetric QR iteration with Wilkinson shifts (Golub & Van Loan,
// Matrix Computations, Algorithms 8.3.1 and 8.3.2), accumulating the orthogonal
// transformations.  Used for Rayleigh-Ritz matrices of a few hundred rows at most.
namespace {
// Householder tridiagonalisation of the symmetrised A (Golub-Van Loan 8.3.1): T = Q^T A Q with
// diagonal d and off-diagonal e (e[i] couples i, i+1); Qt = Q^T row-major (row k = column k of Q).
// With refl != nullptr the reflectors are kept instead (row k of refl: v of step k, placed at
// columns k+1..n-1; refl_beta[k]: its beta, 0 for a skipped step) and Qt is left empty.
void tridiagonalise(int n, const double *Ain, std::vector<double> &d, std::vector<double> &e,
                    std::vector<double> &Qt, std::vector<double> *refl = nullptr,
                    std::vector<double> *refl_beta = nullptr) {
  std::vector<double> A(Ain, Ain + (size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) {
      const double m = 0.5 * (A[(size_t)i * n + j] + A[(size_t)j * n + i]);
      A[(size_t)i * n + j] = A[(size_t)j * n + i] = m;
    }
  if (refl) {
    refl->assign((size_t)n * n, 0.0);
    refl_beta->assign(n, 0.0);
    Qt.clear();
  } else {
    Qt.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Qt[(size_t)i * n + i] = 1.0;
  }
  std::vector<double> srow(n), v(n), p(n), wv(n);
  auto a = [&](int i, int j) -> double & { return A[(size_t)i * n + j]; };
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    // the full symmetric matrix is kept, so column k is row k and every inner loop below is a
    // contiguous axpy (no reductions in the O(m^2) work: they vectorise)
    const double *rowk = &A[(size_t)k * n + k + 1];
    double sigma = 0.0;
    for (int i = 0; i < m; ++i) sigma += rowk[i] * rowk[i];
    sigma = std::sqrt(sigma);
    if (sigma == 0.0) continue;
    const double x0 = rowk[0];
    const double alpha = x0 >= 0 ? -sigma : sigma;
    for (int i = 0; i < m; ++i) v[i] = rowk[i];
    v[0] -= alpha;
    double vtv = 0.0;
    for (int i = 0; i < m; ++i) vtv += v[i] * v[i];
    if (vtv == 0.0) continue;
    const double beta = 2.0 / vtv;
    // p = beta A22 v as a sum of rows; A22 <- A22 - v w^T - w v^T on full rows (exactly symmetric:
    // the two products of an entry and of its mirror are the same)
    for (int i = 0; i < m; ++i) p[i] = 0.0;
    for (int i = 0; i < m; ++i) {
      const double *ai = &A[(size_t)(k + 1 + i) * n + k + 1];
      const double vi = v[i];
      for (int j = 0; j < m; ++j) p[j] += ai[j] * vi;
    }
    for (int i = 0; i < m; ++i) p[i] *= beta;
    double pv = 0.0;
    for (int i = 0; i < m; ++i) pv += p[i] * v[i];
    const double half = 0.5 * beta * pv;
    for (int i = 0; i < m; ++i) wv[i] = p[i] - half * v[i];
    for (int i = 0; i < m; ++i) {
      double *ai = &A[(size_t)(k + 1 + i) * n + k + 1];
      const double vi = v[i], wi = wv[i];
      for (int j = 0; j < m; ++j) ai[j] -= vi * wv[j] + wi * v[j];
    }
    a(k + 1, k) = alpha;
    a(k, k + 1) = alpha;
    if (refl) {
      for (int j = 0; j < m; ++j) (*refl)[(size_t)k * n + k + 1 + j] = v[j];
      (*refl_beta)[k] = beta;
      continue;
    }
    for (int r = 0; r < n; ++r) srow[r] = 0.0;
    for (int j = 0; j < m; ++j) {
      const double *qj = &Qt[(size_t)(k + 1 + j) * n];
      const double vj = v[j];
      for (int r = 0; r < n; ++r) srow[r] += qj[r] * vj;
    }
    for (int j = 0; j < m; ++j) {
      double *qj = &Qt[(size_t)(k + 1 + j) * n];
      const double bv = beta * v[j];
      for (int r = 0; r < n; ++r) qj[r] -= bv * srow[r];
    }
  }
  d.assign(n, 0.0);
  e.assign(std::max(1, n - 1), 0.0);
  for (int i = 0; i < n; ++i) d[i] = a(i, i);
  for (int i = 0; i + 1 < n; ++i) e[i] = a(i + 1, i);
}

// tridiagonalise with the reflectors kept (refl, refl_beta as above), on the pool's threads, one
// barrier per step.  Rows are owned in blocks of 8 dealt out cyclically (row j by thread
// (j / 8) mod nt, one cache line of p per owner) for the whole reduction.
// At step k every thread forms w = p - (beta/2)(p.v) v from the complete p, updates its own rows
// j >= k + 2 by the rank-2 term, and computes row k + 1 after the update privately (that row is
// read by all and written by none during the step), from which it forms the next reflector; it
// then takes its rows' share of the next p = beta' A22' v' on the rows it has just updated.  The
// two p buffers alternate, so the next p is written while no thread reads it.  False when the
// pool was busy (nothing done).
bool tridiagonalise_par(int n, const double *Ain, std::vector<double> &d, std::vector<double> &e,
                        std::vector<double> &refl, std::vector<double> &refl_beta) {
  HostPool &pool = HostPool::instance();
  if (pool.threads() <= 1 || n < 3) return false;
  std::vector<double> A(Ain, Ain + (size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) {
      const double m = 0.5 * (A[(size_t)i * n + j] + A[(size_t)j * n + i]);
      A[(size_t)i * n + j] = A[(size_t)j * n + i] = m;
    }
  refl.assign((size_t)n * n, 0.0);
  refl_beta.assign(n, 0.0);
  d.assign(n, 0.0);
  e.assign(n - 1, 0.0);
  std::vector<double> pbuf[2] = {std::vector<double>(n, 0.0), std::vector<double>(n, 0.0)};
  // Householder vector of x[0..m): v = x - alpha e_0 with alpha = -sign(x_0) |x|, beta = 2/(v.v);
  // beta = 0 (no reflection) for x = 0
  auto reflector = [](const double *x, int m, double *v, double &beta, double &alpha) {
    double sigma = 0.0;
    for (int i = 0; i < m; ++i) sigma += x[i] * x[i];
    sigma = std::sqrt(sigma);
    beta = 0.0;
    alpha = 0.0;
    if (sigma == 0.0) return;
    alpha = x[0] >= 0 ? -sigma : sigma;
    double vtv = 0.0;
    for (int i = 0; i < m; ++i) {
      v[i] = x[i];
      if (i == 0) v[0] -= alpha;
      vtv += v[i] * v[i];
    }
    if (vtv > 0.0) beta = 2.0 / vtv;
  };
  // beta A[j][c0 .. c0 + m) . v for one row (four partial sums)
  auto rowdot4 = [](const double *aj, const double *v, int m) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int i = 0;
    for (; i + 3 < m; i += 4) {
      s0 += aj[i] * v[i];
      s1 += aj[i + 1] * v[i + 1];
      s2 += aj[i + 2] * v[i + 2];
      s3 += aj[i + 3] * v[i + 3];
    }
    for (; i < m; ++i) s0 += aj[i] * v[i];
    return (s0 + s1) + (s2 + s3);
  };
  const bool ran = pool.run([&](int tid, int nt) {
    std::vector<double> v(n), vn(n), w(n), row(n);
    double beta = 0.0, alpha = 0.0;
    // step 0: the reflector of row 0, p on the rows 1 .. n-1
    reflector(&A[1], n - 1, v.data(), beta, alpha);
    if (beta != 0.0)
      for (int j = 1; j < n; ++j)
        if (((j >> 3) % nt) == tid) pbuf[0][j] = beta * rowdot4(&A[(size_t)j * n + 1], v.data(), n - 1);
    if (tid == 0) d[0] = A[0];
    pool.barrier();
    for (int k = 0; k + 2 < n; ++k) {
      const int m = n - k - 1;  // trailing rows k + 1 .. n - 1
      const double *P = pbuf[k & 1].data() + k + 1;
      const double *ak1 = &A[(size_t)(k + 1) * n + k + 1];
      if (beta != 0.0) {
        double pv = 0.0;
        for (int i = 0; i < m; ++i) pv += P[i] * v[i];
        const double half = 0.5 * beta * pv;
        for (int i = 0; i < m; ++i) w[i] = P[i] - half * v[i];
        // row k + 1 after the update (private), then this thread's rows
        for (int i = 0; i < m; ++i) row[i] = ak1[i] - (v[0] * w[i] + w[0] * v[i]);
        for (int j = k + 2; j < n; ++j) {
          if (((j >> 3) % nt) != tid) continue;
          double *aj = &A[(size_t)j * n + k + 2];
          const double vj = v[j - k - 1], wj = w[j - k - 1];
          for (int i = 1; i < m; ++i) aj[i - 1] -= vj * w[i] + wj * v[i];
        }
      } else {
        for (int i = 0; i < m; ++i) row[i] = ak1[i];
      }
      if (tid == 0) {
        e[k] = alpha;
        d[k + 1] = row[0];
        refl_beta[k] = beta;
        for (int i = 0; i < m; ++i) refl[(size_t)k * n + k + 1 + i] = beta != 0.0 ? v[i] : 0.0;
      }
      // the next reflector from row k + 1 (columns k + 2 .. n - 1), p on the rows k + 2 .. n - 1
      double beta_n = 0.0, alpha_n = 0.0;
      reflector(row.data() + 1, m - 1, vn.data(), beta_n, alpha_n);
      if (k + 3 < n && beta_n != 0.0) {
        double *Pn = pbuf[(k + 1) & 1].data();
        for (int j = k + 2; j < n; ++j)
          if (((j >> 3) % nt) == tid) Pn[j] = beta_n * rowdot4(&A[(size_t)j * n + k + 2], vn.data(), m - 1);
      }
      pool.barrier();
      if (k + 3 == n && tid == 0) {
        // the last 2 x 2 block: row n - 2 (private, updated) and the diagonal of row n - 1
        e[n - 2] = row[1];
        d[n - 1] = A[(size_t)(n - 1) * n + n - 1];
      }
      v.swap(vn);
      beta = beta_n;
      alpha = alpha_n;
    }
  });
  return ran;
}

// eigenvalues of the symmetric tridiagonal (d, e) by the implicit QR iteration with Wilkinson
// shifts (Golub-Van Loan 8.3.2), no vectors; ascending
// sqrt(x^2 + z^2); the overflow-safe std::hypot only for operands far from 1 (the plain form is
// several times faster, and these rotations see O(||T||) values)
inline double rot_norm(double x, double z) {
  const double ax = std::fabs(x), az = std::fabs(z);
  const double m = ax > az ? ax : az;
  if (m < 1e-150 || m > 1e150) return std::hypot(x, z);
  return std::sqrt(x * x + z * z);
}

void tridiag_eigenvalues(std::vector<double> d, std::vector<double> e, double *w) {
  // root-free form (Pal, Walker and Kahan; Parlett, The Symmetric Eigenvalue Problem, Sec. 8-15):
  // the sweep carries the squared off-diagonals E_k = e_k^2 and the squared rotation cosines and
  // sines C, S, so that no rotation needs a square root; a block [lo, hi] splits off its bottom
  // row once E_{hi-1} <= eps^2 (|d_{hi-1}| + |d_hi|)^2
  const int n = (int)d.size();
  const double eps = 2.220446049250313e-16, eps2 = eps * eps;
  std::vector<double> E(std::max(1, n - 1), 0.0);
  for (int i = 0; i + 1 < n; ++i) E[i] = e[i] * e[i];
  auto small = [&](int k) {
    const double s = std::fabs(d[k]) + std::fabs(d[k + 1]);
    return E[k] <= eps2 * s * s;
  };
  int hi = n - 1, guard = 0;
  while (hi > 0) {
    if (++guard > 60 * n) break;
    if (small(hi - 1)) {
      E[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && !small(lo - 1)) --lo;
    // Wilkinson shift: the eigenvalue of the bottom 2 x 2 block nearer d_hi
    const double dl = 0.5 * (d[hi - 1] - d[hi]);
    const double b2 = E[hi - 1];
    const double rt = std::sqrt(dl * dl + b2);
    const double sigma = d[hi] - b2 / (dl + (dl >= 0 ? rt : -rt));
    // one implicit QR sweep over [lo, hi]: gam is the shifted diagonal entry carried down the
    // sweep, p = gam^2 / C the squared length the next rotation combines with E_k
    double C = 1.0, S = 0.0;
    double gam = d[lo] - sigma;
    double p = gam * gam;
    for (int k = lo; k < hi; ++k) {
      const double bb = E[k];
      const double r = p + bb;
      if (k > lo) E[k - 1] = S * r;
      const double oldC = C;
      C = p / r;
      S = bb / r;
      const double oldgam = gam;
      const double alpha = d[k + 1] - sigma;
      gam = C * alpha - S * oldgam;
      d[k] = oldgam + (alpha - gam) + sigma;
      p = C != 0.0 ? gam * gam / C : oldC * bb;
    }
    E[hi - 1] = S * p;
    d[hi] = gam + sigma;
  }
  std::sort(d.begin(), d.end());
  for (int i = 0; i < n; ++i) w[i] = d[i];
}

// The k lowest eigenvalues w[0..k) (ascending) of the symmetric tridiagonal (d, e) by bisection
// on the Sturm count: the number of eigenvalues below x is the number of negative pivots of the
// LDL^T factorisation of T - x (q_0 = d_0 - x, q_i = d_i - x - e_{i-1}^2 / q_{i-1}; Golub-Van
// Loan Sec. 8.4.1; a pivot that vanishes is replaced by -pmin).  Each eigenvalue starts from the
// Gershgorin interval and is bisected until the interval is below 2 eps max(|lo|, |hi|) + pmin.
// Eigenvalues [j0, j1) are found four at a time (independent recurrences in one pass over T, so
// that their divisions overlap).
void tridiag_lowest_range(const std::vector<double> &d, const std::vector<double> &E, double gl, double gu,
                          double pmin, int j0, int j1, double *w) {
  const int n = (int)d.size();
  const double eps = 2.220446049250313e-16;
  for (int j = j0; j < j1; j += 4) {
    const int nj = std::min(4, j1 - j);
    double lo[4], hi[4];
    bool done[4];
    for (int q = 0; q < 4; ++q) {
      lo[q] = gl;
      hi[q] = gu;
      done[q] = q >= nj;
    }
    for (int step = 0; step < 256; ++step) {
      double x[4], qv[4];
      int cnt[4] = {0, 0, 0, 0};
      bool all = true;
      for (int q = 0; q < 4; ++q) {
        if (!done[q] && hi[q] - lo[q] <= 2.0 * eps * std::max(std::fabs(lo[q]), std::fabs(hi[q])) + pmin)
          done[q] = true;
        all = all && done[q];
        x[q] = 0.5 * (lo[q] + hi[q]);
        qv[q] = d[0] - x[q];
        if (std::fabs(qv[q]) < pmin) qv[q] = -pmin;
        cnt[q] += qv[q] < 0.0;
      }
      if (all) break;
      for (int i = 1; i < n; ++i) {
        const double Ei = E[i - 1], di = d[i];
#pragma GCC unroll 4
        for (int q = 0; q < 4; ++q) {
          double t = (di - x[q]) - Ei / qv[q];
          if (std::fabs(t) < pmin) t = -pmin;
          qv[q] = t;
          cnt[q] += t < 0.0;
        }
      }
      for (int q = 0; q < 4; ++q) {
        if (done[q]) continue;
        if (cnt[q] >= j + q + 1) hi[q] = x[q];  // at least j + q + 1 eigenvalues below x
        else lo[q] = x[q];
      }
    }
    for (int q = 0; q < nj; ++q) w[j + q] = 0.5 * (lo[q] + hi[q]);
  }
}

// LU of T - lambda for the tridiagonal T = (d, e) by Gaussian elimination with partial pivoting
// (the factor of a tridiagonal matrix has two super-diagonals); zero pivots become `tiny`.
// Factored once per shift, solved for every inverse-iteration step.
struct TridiagLU {
  int n = 0;
  std::vector<double> dd, dl, du, du2;
  std::vector<char> swp;
  void factor(const std::vector<double> &d, const std::vector<double> &e, double lambda, double tiny) {
    n = (int)d.size();
    dd.assign(n, 0.0);
    dl.assign(std::max(1, n - 1), 0.0);
    du.assign(std::max(1, n - 1), 0.0);
    du2.assign(std::max(1, n - 2), 0.0);
    swp.assign(std::max(1, n - 1), 0);
    for (int i = 0; i < n; ++i) dd[i] = d[i] - lambda;
    for (int i = 0; i + 1 < n; ++i) dl[i] = du[i] = e[i];
    for (int i = 0; i + 1 < n; ++i) {
      if (std::fabs(dd[i]) >= std::fabs(dl[i])) {
        if (dd[i] == 0.0) dd[i] = tiny;
        const double f = dl[i] / dd[i];
        dl[i] = f;
        dd[i + 1] -= f * du[i];
      } else {
        // rows i and i + 1 exchanged
        const double f = dd[i] / dl[i];
        dd[i] = dl[i];
        dl[i] = f;
        const double t = du[i];
        du[i] = dd[i + 1];
        dd[i + 1] = t - f * dd[i + 1];
        if (i + 2 < n) {
          du2[i] = du[i + 1];
          du[i + 1] = -f * du[i + 1];
        }
        swp[i] = 1;
      }
    }
    if (dd[n - 1] == 0.0) dd[n - 1] = tiny;
  }
  void solve(std::vector<double> &x) const {
    for (int i = 0; i + 1 < n; ++i) {
      if (swp[i]) std::swap(x[i], x[i + 1]);
      x[i + 1] -= dl[i] * x[i];
    }
    x[n - 1] /= dd[n - 1];
    if (n > 1) x[n - 2] = (x[n - 2] - du[n - 2] * x[n - 1]) / dd[n - 2];
    for (int i = n - 3; i >= 0; --i) x[i] = (x[i] - du[i] * x[i + 1] - du2[i] * x[i + 2]) / dd[i];
  }
};

}  // namespace

// All eigenvalues w[n] (ascending) and the eigenvectors of the k lowest (columns 0..k-1 of V,
// row-major [n][n]; other columns untouched): tridiagonalisation, eigenvalues by QR without
// vectors, vectors by inverse iteration on the tridiagonal with Gram-Schmidt inside clusters of
// close eigenvalues (as in LAPACK's stein), back-transformed with Q.  For Rayleigh-Ritz steps
// that need a few vectors of a matrix of up to a few hundred rows; from kParallelEigMin rows on,
// the reduction, the inverse iteration (cluster by cluster) and the back-transform (column range
// by column range) run on the host pool.
void sym_eig_lowest(int n, const double *A, int k, double *w, double *V, bool all_values) {
  if (n <= 0) return;
  k = std::max(0, std::min(k, n));
  if (n < 3 || (k > n / 2 + 8 && n < kParallelEigMin)) {
    std::vector<double> Vall((size_t)n * n);
    sym_eig(n, A, w, Vall.data());
    for (int r = 0; r < n; ++r)
      for (int j = 0; j < k; ++j) V[(size_t)r * n + j] = Vall[(size_t)r * n + j];
    return;
  }
  HostPool &pool = HostPool::instance();
  std::vector<double> d, e, Qt, refl, rbeta;
  const bool par = n >= kParallelEigMin && tridiagonalise_par(n, A, d, e, refl, rbeta);
  if (!par) tridiagonalise(n, A, d, e, Qt, &refl, &rbeta);
  if (all_values || !par || k == 0) {
    tridiag_eigenvalues(d, e, w);
  } else {
    // the k lowest by bisection on the pool (thread t: eigenvalues [k t/nt, k (t+1)/nt))
    std::vector<double> E(std::max(1, n - 1), 0.0);
    double gl = d[0], gu = d[0], emax = 0.0;
    for (int i = 0; i + 1 < n; ++i) {
      E[i] = e[i] * e[i];
      emax = std::max(emax, E[i]);
    }
    for (int i = 0; i < n; ++i) {
      const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(e[i]) : 0.0);
      gl = std::min(gl, d[i] - r);
      gu = std::max(gu, d[i] + r);
    }
    const double span = std::max(gu - gl, 1e-300);
    gl -= 4.0 * 2.220446049250313e-16 * span * n;
    gu += 4.0 * 2.220446049250313e-16 * span * n;
    const double pmin = 1e-290 * std::max(1.0, emax);
    if (!pool.run([&](int tid, int nt) {
          tridiag_lowest_range(d, E, gl, gu, pmin, (int)((long)k * tid / nt), (int)((long)k * (tid + 1) / nt), w);
        }))
      tridiag_lowest_range(d, E, gl, gu, pmin, 0, k, w);
  }
  double tnorm = 0.0;
  for (int i = 0; i < n; ++i)
    tnorm = std::max(tnorm, std::fabs(d[i]) + (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(e[i]) : 0.0));
  const double eps = 2.220446049250313e-16;
  const double tiny = std::max(eps * tnorm, 1e-300);
  const double ortol = 1e-3 * tnorm;  // eigenvalues closer than this form a cluster
  std::vector<int> cstart(std::max(1, k), 0);
  for (int j = 1; j < k; ++j) cstart[j] = w[j] - w[j - 1] > ortol ? j : cstart[j - 1];
  std::vector<std::vector<double>> X(k, std::vector<double>(n));
  // eigenvectors j0 <= j < j1 (j0 a cluster start)
  auto inverse_iteration = [&](int j0, int j1) {
    TridiagLU lu;
    for (int j = j0; j < j1; ++j) {
      const int cs = cstart[j];
      // shift slightly apart from an equal predecessor so that the solves differ
      double lam = w[j];
      if (j > cs) lam = std::max(lam, w[j - 1] + 10.0 * eps * std::max(1.0, std::fabs(w[j])));
      std::vector<double> &x = X[j];
      // deterministic quasi-random start: fractional parts of (i + 1)(j + 1) times the golden ratio
      for (int i = 0; i < n; ++i) {
        const double t = 0.6180339887498949 * (double)((long)(i + 1) * (j + 1));
        x[i] = 0.5 + (t - std::floor(t));
      }
      lu.factor(d, e, lam, tiny);
      for (int it = 0; it < 4; ++it) {
        double s = 0.0;
        for (double xi : x) s += xi * xi;
        s = 1.0 / std::sqrt(s);
        for (double &xi : x) xi *= s;
        lu.solve(x);
        for (int q = cs; q < j; ++q) {  // orthogonalise inside the cluster
          double dot = 0.0;
          for (int i = 0; i < n; ++i) dot += X[q][i] * x[i];
          for (int i = 0; i < n; ++i) x[i] -= dot * X[q][i];
        }
      }
      double s = 0.0;
      for (double xi : x) s += xi * xi;
      s = 1.0 / std::sqrt(s);
      for (double &xi : x) xi *= s;
    }
  };
  // thread t takes the clusters that start in [k t/nt, k (t+1)/nt)
  auto cluster_range = [&](int tid, int nt, int &j0, int &j1) {
    auto first_start_at_or_after = [&](int j) {
      while (j < k && cstart[j] != j) ++j;
      return j;
    };
    j0 = first_start_at_or_after((int)((long)k * tid / nt));
    j1 = first_start_at_or_after((int)((long)k * (tid + 1) / nt));
  };
  if (!(par && pool.run([&](int tid, int nt) {
        int j0, j1;
        cluster_range(tid, nt, j0, j1);
        inverse_iteration(j0, j1);
      })))
    inverse_iteration(0, k);
  // V[:, j] = Q x_j, Q = H_0 H_1 ... H_{n-3}: the reflectors applied to the columns j0 <= j < j1,
  // last one first, on a private [component][vector] copy (contiguous axpys over the vectors;
  // threads own disjoint column ranges and share no cache lines while they work)
  auto back = [&](int j0, int j1) {
    const int kc = j1 - j0;
    if (kc <= 0) return;
    std::vector<double> Xt((size_t)n * kc), dot(kc);
    for (int j = 0; j < kc; ++j)
      for (int r = 0; r < n; ++r) Xt[(size_t)r * kc + j] = X[j0 + j][r];
    for (int kk = n - 3; kk >= 0; --kk) {
      const double beta = rbeta[kk];
      if (beta == 0.0) continue;
      const double *vk = &refl[(size_t)kk * n];
      std::fill(dot.begin(), dot.end(), 0.0);
      for (int r = kk + 1; r < n; ++r) {
        const double vr = vk[r];
        const double *xr = &Xt[(size_t)r * kc];
        for (int j = 0; j < kc; ++j) dot[j] += vr * xr[j];
      }
      for (int j = 0; j < kc; ++j) dot[j] *= beta;
      for (int r = kk + 1; r < n; ++r) {
        const double vr = vk[r];
        double *xr = &Xt[(size_t)r * kc];
        for (int j = 0; j < kc; ++j) xr[j] -= dot[j] * vr;
      }
    }
    for (int r = 0; r < n; ++r)
      for (int j = 0; j < kc; ++j) V[(size_t)r * n + j0 + j] = Xt[(size_t)r * kc + j];
  };
  if (!(par && pool.run([&](int tid, int nt) { back(k * tid / nt, k * (tid + 1) / nt); }))) back(0, k);
}

void sym_eig(int n, const double *Ain, double *w, double *Vout) {
  if (n <= 0) return;
  // Householder reduction with the accumulated orthogonal factor, stored transposed (Qt[k][r] =
  // Q[r][k]) so that both the reflector updates and the plane rotations stream over contiguous rows
  std::vector<double> d, e, Qt;
  tridiagonalise(n, Ain, d, e, Qt);
  e.resize(std::max(1, n - 1));
  // implicit QR on the tridiagonal (d, e), e[i] couples i and i+1
  const double eps = 2.220446049250313e-16;
  int hi = n - 1;
  int guard = 0;
  while (hi > 0) {
    if (++guard > 60 * n) break;
    if (std::fabs(e[hi - 1]) <= eps * (std::fabs(d[hi - 1]) + std::fabs(d[hi]))) {
      e[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && std::fabs(e[lo - 1]) > eps * (std::fabs(d[lo - 1]) + std::fabs(d[lo]))) --lo;
    // Wilkinson shift from the trailing 2x2 block
    const double dl = 0.5 * (d[hi - 1] - d[hi]);
    const double bb = e[hi - 1];
    const double den = dl + (dl >= 0 ? 1.0 : -1.0) * rot_norm(dl, bb);
    const double mu = d[hi] - bb * bb / den;
    double x = d[lo] - mu, z = e[lo];
    double bulge = 0.0;
    for (int k = lo; k < hi; ++k) {
      const double r = rot_norm(x, z);
      const double c = r == 0.0 ? 1.0 : x / r;
      const double s = r == 0.0 ? 0.0 : z / r;
      if (k > lo) e[k - 1] = r;  // column k-1 after eliminating the bulge
      const double pk = d[k], qk = e[k], tk = d[k + 1];
      d[k] = c * c * pk + 2 * c * s * qk + s * s * tk;
      d[k + 1] = s * s * pk - 2 * c * s * qk + c * c * tk;
      e[k] = c * s * (tk - pk) + (c * c - s * s) * qk;
      if (k + 1 < hi) {
        bulge = s * e[k + 1];
        e[k + 1] = c * e[k + 1];
      }
      double *q0r = &Qt[(size_t)k * n];
      double *q1r = &Qt[(size_t)(k + 1) * n];
      for (int r2 = 0; r2 < n; ++r2) {
        const double q0 = q0r[r2], q1 = q1r[r2];
        q0r[r2] = c * q0 + s * q1;
        q1r[r2] = -s * q0 + c * q1;
      }
      x = e[k];
      z = bulge;
    }
  }
  // sort ascending
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int i, int j) { return d[i] < d[j]; });
  for (int j = 0; j < n; ++j) {
    w[j] = d[idx[j]];
    const double *qj = &Qt[(size_t)idx[j] * n];
    for (int r = 0; r < n; ++r) Vout[(size_t)r * n + j] = qj[r];
  }
}

}  // namespace bse
