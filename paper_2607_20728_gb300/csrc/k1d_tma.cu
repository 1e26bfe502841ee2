// FP32 K1d contraction fused with the grid terms of the Liouville operator (Eq. 2):
//   Y_{b,v}(r) = V(r) a_{b,v}(r) + 2 v_H,b(r) phi_v(r) - sum_v' tau_{v'v}(r) a_{b,v'}(r)
// with tau_{v'v} = W * (phi_v' phi_v) stored once per unordered pair, [pair][r] (FP32).
//
// The kernel is HBM-bound on the tau stream, so it reads every tau element once: a CTA owns
// 32 grid points, walks the 16 x 16 orbital blocks (I <= J) of the packed symmetric tau, and
// uses each staged block for both Y_J (tau^T a_I) and Y_I (tau a_J).  Blocks arrive by TMA
// (cp.async.bulk.tensor.2d: 16 boxes of 16 pairs x 32 points, one per v in J, because the pairs
// (v', v) with v' in I are consecutive rows) into a ring of shared-memory stages guarded by
// mbarriers.  a and the accumulators Y live in shared memory for the whole pass.
#include <cuda.h>

#include <cstring>

#include "internal.cuh"

namespace bse {
namespace {

constexpr int kR = 32;        // grid points per CTA (one per lane)
constexpr int kB = 16;        // orbital block
constexpr int kStages = 2;
constexpr int kThreads = 256;
constexpr int kStageFloats = kB * kB * kR;                  // 8192 floats = 32 KB
constexpr unsigned kStageBytes = kStageFloats * sizeof(float);
constexpr long long kSpinLimit = 1LL << 26;                 // bounded mbarrier waits

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// true when the phase with parity `parity` has completed
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tma_load_2d(float *dst, const CUtensorMap *map, int x, int y,
                                            unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// issue the 16 boxes of block q (pairs (v', v), v' in block I, v in block J) into stage s
__device__ __forceinline__ void issue_block(const CUtensorMap *map, float *stage, unsigned long long *bar, int I,
                                            int J, int r0) {
  mbar_expect_tx(bar, kStageBytes);
  for (int jj = 0; jj < kB; ++jj) {
    const int v = J * kB + jj;
    const int y = v * (v + 1) / 2 + I * kB;
    tma_load_2d(stage + jj * kB * kR, map, r0, y, bar);
  }
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// bounded wait: false when one second (or the iteration cap) ran out
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (long long spin = 0; spin < kSpinLimit; ++spin) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((spin & 63) == 0 && global_ns() - t0 > 1000000000ull) return false;
  }
  return false;
}

__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// Warp-specialised pipeline: warp 8 is the TMA producer, warps 0-7 consume.  Stage s has a
// "full" barrier (producer's expect_tx, completed by the copy bytes) and an "empty" barrier
// (one arrival per consumer warp).  Consumer warp w owns the Y rows 16 X + 2w and 16 X + 2w + 1
// of every orbital block X, so warps never share accumulator rows and need no CTA barrier.
template <int NB, int S>
__global__ void __launch_bounds__(kThreads + 32) k1d_tma_kernel(
    const __grid_constant__ CUtensorMap tmap, long nr, int nocc, int nb_total, int b0,
    const float *__restrict__ phir, const float *__restrict__ vloc, const float2 *__restrict__ Pa,
    const float2 *__restrict__ Pvh, float2 *__restrict__ Py, int use_vloc, int use_k1e, int *__restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  float *tau_s = reinterpret_cast<float *>(smem);                       // [S][16][16][32]
  float *a_s = tau_s + S * kStageFloats;                                // [NB][nocc][32]
  float *y_s = a_s + (size_t)NB * nocc * kR;                            // [NB][nocc][32]
  unsigned long long *full = reinterpret_cast<unsigned long long *>(y_s + (size_t)NB * nocc * kR);
  unsigned long long *empty = full + S;

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const long r0 = (long)blockIdx.x * kR;
  const int nblk = nocc / kB;
  const int nq = nblk * (nblk + 1) / 2;

  auto block_ij = [&](int q, int &I, int &J) {
    int i = 0, rem = q;
    while (rem >= nblk - i) {
      rem -= nblk - i;
      ++i;
    }
    I = i;
    J = i + rem;
  };

  if (tid == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], kThreads / 32);
    }
    fence_async_shared();
  }
  __syncthreads();

  if (warp == kThreads / 32) {
    // ---- producer ----
    if (lane == 0) {
      int issued = 0;
      bool ok = true;
      for (int q = 0; q < nq; ++q) {
        const int st = q % S;
        if (q >= S && !mbar_wait(&empty[st], (unsigned)(((q / S) - 1) & 1))) {
          atomicExch(err, 1);
          ok = false;
          break;
        }
        int I, J;
        block_ij(q, I, J);
        fence_async_shared();
        issue_block(&tmap, tau_s + st * kStageFloats, &full[st], I, J, (int)r0);
        ++issued;
      }
      if (!ok) {
        // let the copies already issued land (bounded) before the CTA can exit
        for (int q = (issued > S ? issued - S : 0); q < issued; ++q) mbar_wait(&full[q % S], (unsigned)((q / S) & 1));
      }
    }
    return;
  }

  // ---- consumers ----
  const float2 *Pa2 = Pa;
  for (int e = tid; e < NB * (nocc / 2) * kR; e += kThreads) {
    const int b = e / ((nocc / 2) * kR);
    const int vp2 = (e / kR) % (nocc / 2);
    const int l = e % kR;
    const long rr = r0 + l;
    const int bb = b0 + b;
    float2 val = make_float2(0.f, 0.f);
    if (rr < nr && bb < nb_total) {
      const long f = (long)bb * nocc + 2 * vp2;  // even: (a_f, a_{f+1}) share one packed grid
      val = Pa2[(f >> 1) * nr + rr];
    }
    a_s[((size_t)b * nocc + 2 * vp2) * kR + l] = val.x;
    a_s[((size_t)b * nocc + 2 * vp2 + 1) * kR + l] = val.y;
    y_s[((size_t)b * nocc + 2 * vp2) * kR + l] = 0.f;
    y_s[((size_t)b * nocc + 2 * vp2 + 1) * kR + l] = 0.f;
  }
  consumer_sync();

  bool ok = true;
  const int j0 = warp * 2, j1 = j0 + 1;
  for (int q = 0; q < nq; ++q) {
    const int st = q % S;
    if (ok && !mbar_wait(&full[st], (unsigned)((q / S) & 1))) {
      ok = false;
      if (lane == 0) atomicExch(err, 1);
    }
    if (ok) {
      int I, J;
      block_ij(q, I, J);
      const float *T = tau_s + st * kStageFloats;  // T[jj][ii][l] = tau_{I16+ii, J16+jj}(r0 + l)
      {
        // Y_J[v] += sum_{v' in I} tau_{v'v} a_{v'}, v = J16 + j0, J16 + j1
        float acc0[NB], acc1[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) acc0[b] = acc1[b] = 0.f;
#pragma unroll 4
        for (int ii = 0; ii < kB; ++ii) {
          float t0, t1;
          if (I != J) {
            t0 = T[(j0 * kB + ii) * kR + lane];
            t1 = T[(j1 * kB + ii) * kR + lane];
          } else {
            // diagonal block: stored entries are ii <= jj; the others are the mirror T[ii][jj]
            t0 = ii <= j0 ? T[(j0 * kB + ii) * kR + lane] : T[(ii * kB + j0) * kR + lane];
            t1 = ii <= j1 ? T[(j1 * kB + ii) * kR + lane] : T[(ii * kB + j1) * kR + lane];
          }
          const int vp = I * kB + ii;
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            const float a = a_s[((size_t)b * nocc + vp) * kR + lane];
            acc0[b] = fmaf(t0, a, acc0[b]);
            acc1[b] = fmaf(t1, a, acc1[b]);
          }
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          y_s[((size_t)b * nocc + J * kB + j0) * kR + lane] += acc0[b];
          y_s[((size_t)b * nocc + J * kB + j1) * kR + lane] += acc1[b];
        }
      }
      if (I != J) {
        // Y_I[v'] += sum_{v in J} tau_{v'v} a_v, v' = I16 + j0, I16 + j1
        float acc0[NB], acc1[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) acc0[b] = acc1[b] = 0.f;
#pragma unroll 4
        for (int jj = 0; jj < kB; ++jj) {
          const float t0 = T[(jj * kB + j0) * kR + lane];
          const float t1 = T[(jj * kB + j1) * kR + lane];
          const int v = J * kB + jj;
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            const float a = a_s[((size_t)b * nocc + v) * kR + lane];
            acc0[b] = fmaf(t0, a, acc0[b]);
            acc1[b] = fmaf(t1, a, acc1[b]);
          }
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          y_s[((size_t)b * nocc + I * kB + j0) * kR + lane] += acc0[b];
          y_s[((size_t)b * nocc + I * kB + j1) * kR + lane] += acc1[b];
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);  // release the stage (also after a failure)
  }
  if (!ok) return;
  // epilogue for this warp's rows: Y = V a + 2 v_H phi - (tau a), written as packed pairs
  const float *Pv_f = reinterpret_cast<const float *>(Pvh);
  const long rr = r0 + lane;
  if (rr >= nr) return;
  const float V = use_vloc ? vloc[rr] : 0.f;
  for (int b = 0; b < NB; ++b) {
    const int bb = b0 + b;
    if (bb >= nb_total) break;
    const float vh2 = use_k1e ? 2.f * Pv_f[2 * ((long)(bb >> 1) * nr + rr) + (bb & 1)] : 0.f;
    for (int X = 0; X < nblk; ++X) {
      const int v = X * kB + j0;  // rows v (even) and v + 1 share one packed grid
      const size_t e0 = ((size_t)b * nocc + v) * kR + lane, e1 = e0 + kR;
      float y0 = -y_s[e0], y1 = -y_s[e1];
      y0 = fmaf(V, a_s[e0], y0);
      y1 = fmaf(V, a_s[e1], y1);
      if (use_k1e) {
        y0 = fmaf(vh2, phir[(long)v * nr + rr], y0);
        y1 = fmaf(vh2, phir[(long)(v + 1) * nr + rr], y1);
      }
      const long f = (long)bb * nocc + v;
      Py[(f >> 1) * nr + rr] = make_float2(y0, y1);
    }
  }
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    BSE_CUDA(cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) throw Error(BSE_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    fn = reinterpret_cast<EncodeTiled>(p);
  }
  return fn;
}

constexpr size_t kSmemCap = 227 * 1024;

size_t smem_bytes(int nb, int stages, int nocc) {
  return (size_t)stages * kStageBytes + 2 * (size_t)nb * nocc * kR * sizeof(float) + 2 * stages * 8;
}

// deepest ring (2..4 stages) that fits beside the a and Y tiles of nb vectors; 0 if none
int stages_for(int nb, int nocc) {
  for (int st = 4; st >= 2; --st)
    if (smem_bytes(nb, st, nocc) <= kSmemCap) return st;
  return 0;
}

template <int NB, int S>
void launch_s(const Ctx &c, const K1dTma &t, int nb, int b0, const float *phir, const float *vloc,
              const float2 *Pa, const float2 *Pvh, float2 *Py, bool use_vloc, bool use_k1e) {
  const size_t smem = smem_bytes(NB, S, c.nocc);
  BSE_CUDA(cudaFuncSetAttribute(k1d_tma_kernel<NB, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned grid = (unsigned)((c.nr + kR - 1) / kR);
  k1d_tma_kernel<NB, S><<<grid, kThreads + 32, smem, c.stream>>>(*reinterpret_cast<const CUtensorMap *>(t.map),
                                                                  c.nr, c.nocc, nb, b0, phir, vloc, Pa, Pvh, Py,
                                                                  use_vloc, use_k1e, t.err);
  BSE_CHECK_LAUNCH();
}

template <int NB>
void launch(const Ctx &c, const K1dTma &t, int nb, int b0, const float *phir, const float *vloc, const float2 *Pa,
            const float2 *Pvh, float2 *Py, bool use_vloc, bool use_k1e) {
  const int st = stages_for(NB, c.nocc);
  if (st >= 4) launch_s<NB, 4>(c, t, nb, b0, phir, vloc, Pa, Pvh, Py, use_vloc, use_k1e);
  else if (st == 3) launch_s<NB, 3>(c, t, nb, b0, phir, vloc, Pa, Pvh, Py, use_vloc, use_k1e);
  else launch_s<NB, 2>(c, t, nb, b0, phir, vloc, Pa, Pvh, Py, use_vloc, use_k1e);
}

}  // namespace

// largest number of trial vectors per launch whose a and Y tiles fit beside the stages (0: none)
int k1d_tma_max_nb(int nocc) {
  for (int nb = 4; nb >= 1; --nb)
    if (stages_for(nb, nocc) >= 2) return nb;
  return 0;
}

bool k1d_tma_supported(int nocc, long nr) {
  // 16-orbital blocks; the pair stride nr * 4 bytes must be a multiple of 16 for the tensor map
  return nocc >= kB && nocc % kB == 0 && nr % 4 == 0 && k1d_tma_max_nb(nocc) > 0;
}

void k1d_tma_init(K1dTma &t, const float *tau, long npairs, long nr, int *err) {
  static_assert(sizeof(CUtensorMap) <= sizeof(t.map), "tensor map storage too small");
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  const cuuint64_t dims[2] = {(cuuint64_t)nr, (cuuint64_t)npairs};
  const cuuint64_t strides[1] = {(cuuint64_t)nr * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kR, (cuuint32_t)kB};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(tau), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(BSE_ERR_CUDA, "cuTensorMapEncodeTiled failed for the tau stream");
  std::memcpy(t.map, &map, sizeof(map));
  t.err = err;
  t.ready = true;
}

void k1d_tma(const Ctx &c, const K1dTma &t, int nb, const float *phir, const float *vloc, const float2 *Pa,
             const float2 *Pvh, float2 *Py, bool use_vloc, bool use_k1e) {
  const int cap = k1d_tma_max_nb(c.nocc);
  int b0 = 0;
  while (b0 < nb) {
    const int left = std::min(nb - b0, cap);
    if (left >= 4) { launch<4>(c, t, nb, b0, phir, vloc, Pa, Pvh, Py, use_vloc, use_k1e); b0 += 4; }
    else if (left == 3) { launch<3>(c, t, nb, b0, phir, vloc, Pa, Pvh, Py, use_vloc, use_k1e); b0 += 3; }
    else if (left == 2) { launch<2>(c, t, nb, b0, phir, vloc, Pa, Pvh, Py, use_vloc, use_k1e); b0 += 2; }
    else { launch<1>(c, t, nb, b0, phir, vloc, Pa, Pvh, Py, use_vloc, use_k1e); b0 += 1; }
  }
}

}  // namespace bse
