// Split-BF16 tensor-core GEMM for the PDEP projection and back-projection of Eq. 3 (mixed
// precision):  C = alpha A B^T + beta C,  A [M][K], B [N][K] FP32 row-major, C [M][N] FP32.
//
// Each FP32 operand is split once into x = hi + lo with hi = bf16(x), lo = bf16(x - hi); the
// product is accumulated as A_hi B_hi + A_hi B_lo + A_lo B_hi in FP32 (the dropped lo*lo term is
// ~2^-16 of each product).  The kernel is written for the 5th-generation tensor cores:
//   - TMA (cp.async.bulk.tensor.2d, 128-byte swizzle) streams 128 x 64 tiles of A_hi, A_lo,
//     B_hi, B_lo into a ring of shared-memory stages (full/empty mbarriers);
//   - one thread issues tcgen05.mma.cta_group::1.kind::f16 (BF16 x BF16 -> FP32, M = 128,
//     N = 128, K = 16) into a TMEM accumulator and releases stages with tcgen05.commit;
//   - four warps read the accumulator back with tcgen05.ld.32x32b and store FP32 partials.
// K is split over CTAs (gridDim.z) because the PDEP shapes are small M x N with long K; a
// second kernel sums the partials.  All waits are bounded by time and report through a flag.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cstring>

#include "internal.cuh"

namespace bse {
namespace {

constexpr int BM = 128, BN = 128, BK = 64;     // BK bf16 = 128 bytes: one swizzle row
constexpr int kStages = 3;
constexpr int kTileBytes = BM * BK * 2;        // 16 KB for a 128 x 64 bf16 tile (BM == BN)
constexpr int kStageBytes = 4 * kTileBytes;    // A_hi, A_lo, B_hi, B_lo
constexpr int kThreads = 128;
constexpr long long kSpinLimit = 1LL << 26;

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(unsigned addr, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned addr, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(addr), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned addr, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(unsigned addr, unsigned parity) {
  if (mbar_try_wait(addr, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (long long spin = 0; spin < kSpinLimit; ++spin) {
    if (mbar_try_wait(addr, parity)) return true;
    if ((spin & 63) == 0 && global_ns() - t0 > 1000000000ull) return false;
  }
  return false;
}
__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap *map, int x, int y, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// shared-memory matrix descriptor: K-major tile, 128-byte swizzle, 8-row atoms 1024 bytes apart
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr) {
  unsigned long long d = 0;
  d |= (unsigned long long)((addr >> 4) & 0x3FFF);       // start address
  d |= (unsigned long long)1 << 16;                       // leading byte offset (unused when swizzled)
  d |= (unsigned long long)(1024 >> 4) << 32;             // stride byte offset: next 8-row atom
  d |= (unsigned long long)1 << 46;                       // descriptor version
  d |= (unsigned long long)2 << 61;                       // layout: 128-byte swizzle
  return d;
}

// instruction descriptor of kind::f16: FP32 accumulate, A and B BF16, both K-major, M = 128, N = 128
constexpr unsigned kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(BN >> 3) << 17) |
                            ((unsigned)(BM >> 4) << 24);

__device__ __forceinline__ void umma_bf16(unsigned tmem_d, unsigned long long adesc, unsigned long long bdesc,
                                          unsigned accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(unsigned bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__global__ void __launch_bounds__(kThreads) umma_gemm_kernel(
    const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
    const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl, int M, int N, int ktiles,
    int kt_per_split, float *__restrict__ part, int *__restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  // 1024-byte alignment for the swizzle atoms
  const unsigned base = smem_u32(smem_raw);
  const unsigned pad = (1024u - (base & 1023u)) & 1023u;
  unsigned char *smem = smem_raw + pad;
  const unsigned sbase = base + pad;
  const unsigned bars = sbase + kStages * kStageBytes;   // full[S], empty[S], done
  const unsigned full0 = bars, empty0 = bars + 8 * kStages, done = bars + 16 * kStages;
  unsigned *tmem_slot = reinterpret_cast<unsigned *>(smem + kStages * kStageBytes + 16 * kStages + 8);
  int *fail_s = reinterpret_cast<int *>(smem + kStages * kStageBytes + 16 * kStages + 16);
  int *issued_s = fail_s + 1;    // tiles whose copies were issued
  int *consumed_s = fail_s + 2;  // tiles whose copies the MMA thread saw complete

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kt0 = blockIdx.z * kt_per_split;
  const int kt1 = min(ktiles, kt0 + kt_per_split);
  const int nk = kt1 - kt0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    *fail_s = 0;
    *issued_s = 0;
    *consumed_s = 0;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = *tmem_slot;

  if (warp == 0 && lane == 0 && nk > 0) {
    // TMA producer
    for (int i = 0; i < nk; ++i) {
      const int s = i % kStages;
      if (i >= kStages && !mbar_wait(empty0 + 8 * s, (unsigned)(((i / kStages) - 1) & 1))) {
        atomicExch(fail_s, 1);
        break;
      }
      const unsigned st = sbase + s * kStageBytes;
      const int kx = (kt0 + i) * BK;
      mbar_expect_tx(full0 + 8 * s, kStageBytes);
      tma_load_2d(st, &mAh, kx, m0, full0 + 8 * s);
      tma_load_2d(st + kTileBytes, &mAl, kx, m0, full0 + 8 * s);
      tma_load_2d(st + 2 * kTileBytes, &mBh, kx, n0, full0 + 8 * s);
      tma_load_2d(st + 3 * kTileBytes, &mBl, kx, n0, full0 + 8 * s);
      *issued_s = i + 1;
    }
  } else if (warp == 1 && lane == 0 && nk > 0) {
    // MMA issuer
    bool ok = true;
    for (int i = 0; i < nk && ok; ++i) {
      const int s = i % kStages;
      if (!mbar_wait(full0 + 8 * s, (unsigned)((i / kStages) & 1))) {
        atomicExch(fail_s, 1);
        ok = false;
        break;
      }
      *consumed_s = i + 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned st = sbase + s * kStageBytes;
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const unsigned off = kk * 32;  // 16 bf16 along K inside the 128-byte swizzled row
        const unsigned long long ah = smem_desc(st + off), al = smem_desc(st + kTileBytes + off);
        const unsigned long long bh = smem_desc(st + 2 * kTileBytes + off);
        const unsigned long long bl = smem_desc(st + 3 * kTileBytes + off);
        umma_bf16(tmem, ah, bh, (i > 0 || kk > 0) ? 1u : 0u);
        umma_bf16(tmem, ah, bl, 1u);
        umma_bf16(tmem, al, bh, 1u);
      }
      umma_commit(empty0 + 8 * s);  // frees the stage once these MMAs have read it
    }
    umma_commit(done);              // the accumulator is complete after every MMA issued so far
  }
  __syncwarp();

  // epilogue: all four warps; warp w reads TMEM lanes 32w .. 32w + 31 (rows of the tile)
  bool ok = nk > 0 && mbar_wait(done, 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  ok = ok && (*fail_s == 0);
  const int row = m0 + warp * 32 + lane;
  float *dst = part + (long)blockIdx.z * M * N;
  for (int c0 = 0; c0 < BN; c0 += 32) {
    unsigned r[32];
    const unsigned taddr = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (ok && row < M) {
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int col = n0 + c0 + j;
        if (col < N) dst[(long)row * N + col] = __uint_as_float(r[j]);
      }
    } else if (row < M) {
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int col = n0 + c0 + j;
        if (col < N) dst[(long)row * N + col] = 0.f;  // empty K slice or failure: contributes nothing
      }
    }
  }
  if (!ok && nk > 0 && threadIdx.x == 0) {
    atomicExch(err, 1);
    // copies issued but never seen complete must land (bounded) before the CTA exits
    for (int i = *consumed_s; i < *issued_s; ++i) mbar_wait(full0 + 8 * (i % kStages), (unsigned)((i / kStages) & 1));
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 2) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
  }
}

// x = hi + lo, hi = bf16(x), lo = bf16(x - hi), rows padded with zeros to kp columns
__global__ void split_bf16_kernel(int rows, int k, int kp, const float *__restrict__ X, int ldx,
                                  __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ lo) {
  const long total = (long)rows * kp;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int r = (int)(i / kp), c = (int)(i % kp);
    const float x = c < k ? X[(long)r * ldx + c] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[i] = h;
    lo[i] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}

__global__ void splitk_sum_kernel(int M, int N, int nsplit, const float *__restrict__ part, float alpha,
                                  float beta, float *__restrict__ C, int ldc) {
  const long total = (long)M * N;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < nsplit; ++z) s += part[(long)z * total + i];
    float *c = C + (i / N) * ldc + (i % N);
    *c = beta == 0.f ? alpha * s : alpha * s + beta * (*c);
  }
}

// Y [cols][rows] = X [rows][cols]^T
__global__ void transpose_kernel(int rows, int cols, const float *__restrict__ X, float *__restrict__ Y) {
  const long total = (long)rows * cols;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int r = (int)(i / cols), c = (int)(i % cols);
    Y[(long)c * rows + r] = X[i];
  }
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled lookup_encode_fn() {
  void *p = nullptr;
  cudaDriverEntryPointQueryResult q;
  BSE_CUDA(cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q));
  if (q != cudaDriverEntryPointSuccess || !p) throw Error(BSE_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  return reinterpret_cast<EncodeTiled>(p);
}

EncodeTiled encode_fn() {
  static const EncodeTiled fn = lookup_encode_fn();  // thread-safe one-time lookup
  return fn;
}

// tensor map of a bf16 [rows][kp] operand, box 64 (K) x 128 (rows), 128-byte swizzle
void make_map(CUtensorMap *map, const __nv_bfloat16 *p, int rows, int kp) {
  std::memset(map, 0, sizeof(*map));
  const cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
  const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)BM};
  const cuuint32_t es[2] = {1, 1};
  CUresult r = encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(p), dims, strides,
                           box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(BSE_ERR_CUDA, "cuTensorMapEncodeTiled failed for a GEMM operand");
}

}  // namespace

size_t umma_smem_bytes() { return (size_t)kStages * kStageBytes + 16 * kStages + 64 + 1024; }

void transpose_f32(int rows, int cols, const float *X, float *Y, cudaStream_t s) {
  transpose_kernel<<<(int)std::min<long>(152 * 16, ((long)rows * cols + 255) / 256), 256, 0, s>>>(rows, cols, X, Y);
  BSE_CHECK_LAUNCH();
}

void split_bf16(int rows, int k, const float *X, int ldx, SplitBF16 &out, cudaStream_t s) {
  const int kp = (k + BK - 1) / BK * BK;
  out.rows = rows;
  out.k = k;
  out.kp = kp;
  out.hi.alloc((size_t)rows * kp);
  out.lo.alloc((size_t)rows * kp);
  const long total = (long)rows * kp;
  const int grid = (int)std::min<long>(152 * 16, (total + 255) / 256);
  split_bf16_kernel<<<grid, 256, 0, s>>>(rows, k, kp, X, ldx, reinterpret_cast<__nv_bfloat16 *>(out.hi.get()),
                                         reinterpret_cast<__nv_bfloat16 *>(out.lo.get()));
  BSE_CHECK_LAUNCH();
}

void umma_gemm_nt(int M, int N, float alpha, const SplitBF16 &A, const SplitBF16 &B, float beta, float *C, int ldc,
                  DevBuf<float> &partial, int *err, cudaStream_t s) {
  BSE_REQUIRE(A.kp == B.kp && A.k == B.k, "split operands with different K");
  BSE_REQUIRE(A.rows >= M && B.rows >= N, "split operands too small");
  if (M <= 0 || N <= 0) return;
  CUtensorMap mAh, mAl, mBh, mBl;
  make_map(&mAh, reinterpret_cast<const __nv_bfloat16 *>(A.hi.get()), A.rows, A.kp);
  make_map(&mAl, reinterpret_cast<const __nv_bfloat16 *>(A.lo.get()), A.rows, A.kp);
  make_map(&mBh, reinterpret_cast<const __nv_bfloat16 *>(B.hi.get()), B.rows, B.kp);
  make_map(&mBl, reinterpret_cast<const __nv_bfloat16 *>(B.lo.get()), B.rows, B.kp);
  const int ktiles = A.kp / BK;
  const int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
  int nsplit = std::max(1, std::min(ktiles, (2 * 152) / std::max(1, tiles)));
  const int per = (ktiles + nsplit - 1) / nsplit;
  nsplit = (ktiles + per - 1) / per;
  partial.alloc((size_t)nsplit * M * N);
  const size_t smem = umma_smem_bytes();
  BSE_CUDA(cudaFuncSetAttribute(umma_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, nsplit);
  umma_gemm_kernel<<<grid, kThreads, smem, s>>>(mAh, mAl, mBh, mBl, M, N, ktiles, per, partial.get(), err);
  BSE_CHECK_LAUNCH();
  const long total = (long)M * N;
  splitk_sum_kernel<<<(int)std::min<long>(4096, (total + 255) / 256), 256, 0, s>>>(M, N, nsplit, partial.get(), alpha,
                                                                                   beta, C, ldc);
  BSE_CHECK_LAUNCH();
}

}  // namespace bse
