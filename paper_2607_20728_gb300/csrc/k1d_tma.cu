// FP32 K1d contraction fused with the grid terms of the Liouville operator (Eq. 2):
//   Y_{b,v}(r) = V(r) a_{b,v}(r) + 2 v_H,b(r) phi_v(r) - sum_v' tau_{v'v}(r) a_{b,v'}(r)
// with tau_{v'v} = W * (phi_v' phi_v) stored once per unordered pair (FP32).
//
// The kernel is HBM-bound on the tau stream, so it reads every tau element once: a CTA owns
// 32 grid points, walks the 16 x 16 orbital blocks (I <= J) of the packed symmetric tau, and
// uses each staged block for both Y_J (tau^T a_I) and Y_I (tau a_J).  tau is stored tile-major
// (all pairs of one 32-point tile contiguous, block after block), so each block is one
// contiguous chunk (32 KB, or 17 KB for a packed diagonal block) that arrives by a 1D bulk copy
// (cp.async.bulk) into a ring of shared-memory stages guarded by mbarriers, and a CTA streams
// one contiguous 1 MB region.  a and the accumulators Y live in shared memory for the whole pass.
#include <algorithm>
#include <cstring>
#include <type_traits>

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

// 1D bulk copy global -> shared completing on an mbarrier (16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void bulk_load(float *dst, const float *src, unsigned bytes, unsigned long long *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

constexpr int kTri = kB * (kB + 1) / 2;  // pairs of a diagonal block

// pair (ii, jj) of a staged diagonal block, packed triangle with the smaller index first
__device__ __forceinline__ int tri(int a, int b) { return a <= b ? b * (b + 1) / 2 + a : a * (a + 1) / 2 + b; }

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

// Warp-specialised persistent pipeline: one CTA per SM walks 32-point tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ...  Warp 8 is the producer: it streams the blocks of tile after tile
// through the ring without pausing at tile boundaries.  Stage s has a "full" barrier (producer's
// expect_tx, completed by the copy bytes) and an "empty" barrier (one arrival per consumer warp).
//
// The blocks of a tile are consumed column by column: column J holds the blocks (I, J), I < J,
// then the diagonal block (J, J).  Block (I, J) contributes Y_J += tau^T a_I ("role A") and
// Y_I += tau a_J ("role B").  Consumer warps 0-3 take role A, warps 4-7 role B, each for 4 of the
// 16 rows of the block, so every staged tau element is read from shared memory once per role
// and every staged a value feeds 4 rows.  Role-A warps keep their 4 rows of Y_J in registers for
// the whole column (the diagonal block is theirs too) and add them to Y in shared memory at the
// column's end; role-B warps add their rows of Y_I after each block.  Within a column no two warps
// write the same rows of Y, and a named barrier separates the columns.
//
// a and Y live in shared memory for the whole tile.  Rows of a arrive one column block ahead:
// while column J is consumed, every consumer thread holds the next column's a values (and phi) of
// its point in registers and stores them at the column's end, so the global-load latency overlaps
// the tau stream.  Y starts as the grid terms V a + 2 v_H phi and the K1d sums are subtracted, so
// the epilogue only stores.
//
// A consumer warp whose bounded wait gives up sets the CTA's fail flag; from then on no consumer
// waits, computes or releases a stage (so the producer's own bounded wait runs out and it drains
// its copies), but every consumer warp still passes the same named barriers up to the next tile's
// first one, where all of them leave.  hold != 0 (failure-detection self-test only): the producer
// issues no copies, so every consumer wait runs out.
template <int NB, int S>
__global__ void __launch_bounds__(kThreads + 32, 1) k1d_tma_kernel(
    const float *__restrict__ tau, long npairs, long nr, int nocc, int nb_total, int b0,
    const float *__restrict__ phir, const float *__restrict__ vloc, const float2 *__restrict__ Pa,
    const float2 *__restrict__ Pvh, float2 *__restrict__ Py, int use_vloc, int use_k1e, int *__restrict__ err,
    int hold) {
  extern __shared__ __align__(128) unsigned char smem[];
  float *tau_s = reinterpret_cast<float *>(smem);                       // [S][16][16][32]
  float *a_s = tau_s + S * kStageFloats;                                // [NB][nocc][32]
  float *y_s = a_s + (size_t)NB * nocc * kR;                            // [NB][nocc][32]
  unsigned long long *full = reinterpret_cast<unsigned long long *>(y_s + (size_t)NB * nocc * kR);
  unsigned long long *empty = full + S;
  volatile int *fail = reinterpret_cast<volatile int *>(empty + S);  // CTA-wide: a consumer gave up

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int nblk = nocc / kB;
  const long ntiles = nr / kR;

  if (tid == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], kThreads / 32);
    }
    *fail = 0;
    fence_async_shared();
  }
  __syncthreads();

  if (warp == kThreads / 32) {
    // ---- producer: the blocks of each tile in column order, which is their order in memory ----
    if (lane == 0 && !hold) {
      long g = 0;  // blocks issued so far (all tiles)
      bool ok = true;
      for (long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const float *src = tau + (size_t)t * npairs * kR;  // this tile's contiguous region
        for (int J = 0; J < nblk && ok; ++J) {
          for (int I = 0; I <= J; ++I, ++g) {
            const int st = (int)(g % S);
            if (g >= S && !mbar_wait(&empty[st], (unsigned)(((g / S) - 1) & 1))) {
              atomicExch(err, 1);
              ok = false;
              break;
            }
            const unsigned bytes = (unsigned)((I == J ? kTri : kB * kB) * kR * sizeof(float));
            fence_async_shared();
            mbar_expect_tx(&full[st], bytes);
            bulk_load(tau_s + st * kStageFloats, src, bytes, &full[st]);
            src += bytes / sizeof(float);
          }
        }
      }
      // the copies still in flight land (bounded) before the CTA can exit; after a normal run
      // their barriers have completed already
      for (long q = (g > S ? g - S : 0); q < g; ++q) mbar_wait(&full[q % S], (unsigned)((q / S) & 1));
    }
    return;
  }
  // ---- consumers ----
  // a and Y: with an even number of vectors they are stored as pairs of vectors,
  // [v][NB/2][32 points][2], so that one float2 load feeds one packed FP32x2 multiply-add for two
  // vectors; otherwise [NB][v][32 points].  idx(b, v) is the float offset of (vector b, row v,
  // lane 0) and LS the lane stride.
  constexpr bool PAIR = (NB % 2) == 0;
  constexpr int NBH = PAIR ? NB / 2 : NB;
  constexpr int LS = PAIR ? 2 : 1;
  auto idx = [&](int b, int v) -> size_t {
    return PAIR ? ((size_t)v * NBH + (b >> 1)) * (kR * 2) + (b & 1) : ((size_t)b * nocc + v) * kR;
  };
  const bool roleA = warp < 4;
  const int r4 = (warp & 3) * 4;  // first of the 4 block rows this warp accumulates
  const int p2 = warp * 2;        // rows p2, p2 + 1 of every block: this warp's loads and stores
  const float *Pv_f = reinterpret_cast<const float *>(Pvh);
  // acc[k][*]: Y row r4 + k of the block being accumulated, one entry per vector (or vector pair)
  using Acc = typename std::conditional<PAIR, float2, float>::type;
  Acc acc[4][NBH];
  auto zero_acc = [&]() {
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int b = 0; b < NBH; ++b) acc[k][b] = Acc{};
  };
  // acc[k] += sum_m tau(slot(k, m)) a(16 C + m) over the 16 columns m of a staged block
  auto mac4 = [&](const float *T, int C, auto slot) {
#pragma unroll
    for (int m = 0; m < kB; ++m) {
      float t[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) t[k] = T[slot(k, m) * kR + lane];
#pragma unroll
      for (int b = 0; b < NBH; ++b) {
        if constexpr (PAIR) {
          const float2 a = *reinterpret_cast<const float2 *>(&a_s[idx(2 * b, C * kB + m) + 2 * lane]);
#pragma unroll
          for (int k = 0; k < 4; ++k) acc[k][b] = __ffma2_rn(make_float2(t[k], t[k]), a, acc[k][b]);
        } else {
          const float a = a_s[idx(b, C * kB + m) + lane];
#pragma unroll
          for (int k = 0; k < 4; ++k) acc[k][b] = fmaf(t[k], a, acc[k][b]);
        }
      }
    }
  };
  // Y rows X*16 + r4 + k -= acc[k]
  auto flush = [&](int X) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int b = 0; b < NBH; ++b) {
        if constexpr (PAIR) {
          float2 *y = reinterpret_cast<float2 *>(&y_s[idx(2 * b, X * kB + r4 + k) + 2 * lane]);
          const float2 o = *y;
          *y = make_float2(o.x - acc[k][b].x, o.y - acc[k][b].y);
        } else {
          y_s[idx(b, X * kB + r4 + k) + lane] -= acc[k][b];
        }
      }
  };

  long g = 0;
  bool ok = true;  // false once the CTA has given up (uniform within the warp)
  for (long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const long rr = t * kR + lane;
    consumer_sync();  // the previous tile's epilogue has read Y
    // a give-up recorded before this barrier is seen by every consumer warp: all leave together
    if (*fail) break;
    const float V = use_vloc ? vloc[rr] : 0.f;
    float vh2[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int bb = b0 + b;
      vh2[b] = (use_k1e && bb < nb_total) ? 2.f * Pv_f[2 * ((long)(bb >> 1) * nr + rr) + (bb & 1)] : 0.f;
    }
    // rows p2, p2 + 1 of column block J at this thread's point: a (one packed grid holds both
    // rows) and phi, held in registers until place() stores them with Y = V a + 2 v_H phi.  Two
    // register sets alternate between even and odd columns, so the rows of column J + 2 are
    // loaded while columns J and J + 1 are consumed
    struct Rows {
      float2 pa[NB];
      float ph0, ph1;
    };
    Rows ra, rb;
    auto fetch = [&](Rows &d, int J) {
      const int v = J * kB + p2;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int bb = b0 + b;
        d.pa[b] = bb < nb_total ? Pa[(((long)bb * nocc + v) >> 1) * nr + rr] : make_float2(0.f, 0.f);
      }
      d.ph0 = use_k1e ? phir[(long)v * nr + rr] : 0.f;
      d.ph1 = use_k1e ? phir[(long)(v + 1) * nr + rr] : 0.f;
    };
    auto place = [&](const Rows &d, int J) {
      const int v = J * kB + p2;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const size_t o0 = idx(b, v) + (size_t)lane * LS, o1 = idx(b, v + 1) + (size_t)lane * LS;
        a_s[o0] = d.pa[b].x;
        a_s[o1] = d.pa[b].y;
        y_s[o0] = fmaf(V, d.pa[b].x, vh2[b] * d.ph0);
        y_s[o1] = fmaf(V, d.pa[b].y, vh2[b] * d.ph1);
      }
    };
    // column J: its blocks, then role A's rows of Y_J, then the rows of column J + 1 (from `next`)
    auto column = [&](int J, Rows &next) {
      zero_acc();
      for (int I = 0; I <= J; ++I, ++g) {
        const int st = (int)(g % S);
        if (ok) {
          if (*fail) {
            ok = false;  // another warp gave up: wait no more
          } else if (!mbar_wait(&full[st], (unsigned)((g / S) & 1))) {
            ok = false;
            if (lane == 0) {
              atomicExch(err, 1);
              *fail = 1;
              __threadfence_block();
            }
          }
          ok = __all_sync(0xffffffffu, ok);  // warp-uniform outcome
        }
        if (!ok) continue;  // no compute and no release after a give-up
        const float *T = tau_s + st * kStageFloats;  // [jj][ii][32] (I < J) or packed triangle (I = J)
        if (I < J) {
          if (roleA) {
            // Y_J[jj] += sum_ii tau(ii, jj) a_I[ii], rows jj = r4 + k
            mac4(T, I, [&](int k, int m) { return (r4 + k) * kB + m; });
          } else {
            // Y_I[ii] += sum_jj tau(ii, jj) a_J[jj], rows ii = r4 + k
            zero_acc();
            mac4(T, J, [&](int k, int m) { return m * kB + r4 + k; });
            flush(I);
          }
        } else if (roleA) {
          // diagonal block: packed triangle of the symmetric 16 x 16 block, rows r4 + k of Y_J
          mac4(T, J, [&](int k, int m) { return tri(m, r4 + k); });
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);  // release the stage
      }
      if (ok && roleA) flush(J);
      if (J + 1 < nblk) place(next, J + 1);
      consumer_sync();  // column J done: Y rows of J final for role A, rows of J + 1 stored
    };
    fetch(ra, 0);
    if (nblk > 1) fetch(rb, 1);
    place(ra, 0);
    consumer_sync();
    for (int J = 0; J < nblk; J += 2) {
      if (J + 2 < nblk) fetch(ra, J + 2);  // lands while columns J and J + 1 are consumed
      column(J, rb);
      if (J + 1 < nblk) {
        if (J + 3 < nblk) fetch(rb, J + 3);
        column(J + 1, ra);
      }
    }
    if (!ok) continue;  // after a give-up: no epilogue; the next tile's first barrier ends the CTA
    // epilogue: Y = V a + 2 v_H phi - (tau a), rows p2, p2 + 1 of every block as packed pairs
#pragma unroll 2
    for (int X = 0; X < nblk; ++X) {
      const int v = X * kB + p2;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int bb = b0 + b;
        if (bb >= nb_total) break;
        const size_t e0 = idx(b, v) + (size_t)lane * LS, e1 = idx(b, v + 1) + (size_t)lane * LS;
        const long f = (long)bb * nocc + v;
        Py[(f >> 1) * nr + rr] = make_float2(y_s[e0], y_s[e1]);
      }
    }
  }
}

constexpr size_t kSmemCap = 227 * 1024;

size_t smem_bytes(int nb, int stages, int nocc) {
  return (size_t)stages * kStageBytes + 2 * (size_t)nb * nocc * kR * sizeof(float) + 2 * stages * 8 + 16;
}

// deepest ring (2..4 stages) that fits beside the a and Y tiles of nb vectors; 0 if none
int stages_for(int nb, int nocc) {
  for (int st = 4; st >= 2; --st)
    if (smem_bytes(nb, st, nocc) <= kSmemCap) return st;
  return 0;
}

template <int NB, int S>
void launch_s(const Ctx &c, const K1dTma &t, int nb, int b0, const float *phir, const float *vloc,
              const float2 *Pa, const float2 *Pvh, float2 *Py, bool use_vloc, bool use_k1e, int hold = 0) {
  const size_t smem = smem_bytes(NB, S, c.nocc);
  BSE_CUDA(cudaFuncSetAttribute(k1d_tma_kernel<NB, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // persistent: one CTA per SM (the ring and the a/Y tiles take most of the shared memory)
  int dev = 0, nsm = 0;
  BSE_CUDA(cudaGetDevice(&dev));
  BSE_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const unsigned grid = (unsigned)std::min<long>(c.nr / kR, std::max(1, nsm));
  k1d_tma_kernel<NB, S><<<grid, kThreads + 32, smem, c.stream>>>(t.tau, t.npairs, c.nr, c.nocc, nb, b0, phir, vloc,
                                                                  Pa, Pvh, Py, use_vloc, use_k1e, t.err, hold);
  BSE_CHECK_LAUNCH();
}

template <int NB>
void launch(const Ctx &c, const K1dTma &t, int nb, int b0, const float *phir, const float *vloc, const float2 *Pa,
            const float2 *Pvh, float2 *Py, bool use_vloc, bool use_k1e, int hold = 0) {
  const int st = stages_for(NB, c.nocc);
  if (st >= 4) launch_s<NB, 4>(c, t, nb, b0, phir, vloc, Pa, Pvh, Py, use_vloc, use_k1e, hold);
  else if (st == 3) launch_s<NB, 3>(c, t, nb, b0, phir, vloc, Pa, Pvh, Py, use_vloc, use_k1e, hold);
  else launch_s<NB, 2>(c, t, nb, b0, phir, vloc, Pa, Pvh, Py, use_vloc, use_k1e, hold);
}

}  // namespace

// largest number of trial vectors per launch whose a and Y tiles fit beside the stages (0: none)
int k1d_tma_max_nb(int nocc) {
  for (int nb = 4; nb >= 1; --nb)
    if (stages_for(nb, nocc) >= 2) return nb;
  return 0;
}

// Failure-detection self-test of the pipeline's bounded wait: one thread waits on an mbarrier
// that nothing arrives at; mbar_wait must give up (one second of %globaltimer, or its iteration
// cap), and the kernel records the device error flag and returns, as the K1d pipeline does.
__global__ void wait_selftest_kernel(int *err) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    if (!mbar_wait(&bar, 0)) atomicExch(err, 1);
  }
}

void wait_selftest(cudaStream_t s, int *err) {
  wait_selftest_kernel<<<1, 32, 0, s>>>(err);
  BSE_CHECK_LAUNCH();
}

bool k1d_tma_supported(int nocc, long nr) {
  // 16-orbital blocks; whole 32-point tiles
  return nocc >= kB && nocc % kB == 0 && nr % kR == 0 && k1d_tma_max_nb(nocc) > 0;
}

void k1d_tma_init(K1dTma &t, const float *tau, long npairs, long nr, int *err) {
  BSE_REQUIRE(nr % kR == 0, "internal: tile-major tau needs whole 32-point tiles");
  t.tau = tau;
  t.npairs = npairs;
  t.err = err;
  t.ready = true;
}

namespace {
__global__ void unpack_tiled_kernel(long nr, int np, int nocc, long npairs, const int2 *__restrict__ pairs,
                                    const float2 *__restrict__ P, float *__restrict__ tau) {
  const long total = nr * np;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int k = (int)(i / nr);
    const long r = i - (long)k * nr;
    const float2 v = P[(long)(k >> 1) * nr + r];
    const int2 pr = pairs[k];  // (v', v), v' <= v
    const long slot = k1d_tile_slot(pr.x, pr.y, nocc);
    tau[((r / kR) * npairs + slot) * kR + (r % kR)] = (k & 1) ? v.y : v.x;
  }
}
}  // namespace

void k1d_unpack_tiled(const Ctx &c, int np, const int2 *pairs, const float2 *P, float *tau) {
  const long total = c.nr * np;
  const int grid = (int)std::min<long>(152L * 64, (total + 255) / 256);
  unpack_tiled_kernel<<<grid, 256, 0, c.stream>>>(c.nr, np, c.nocc, (long)c.nocc * (c.nocc + 1) / 2, pairs, P, tau);
  BSE_CHECK_LAUNCH();
}

// Failure-detection self-test of the whole pipeline: one launch over every tile with the widest
// block the context supports, in which the producer issues no copies, so that every consumer
// wait runs out; the launch must end with the error flag set and nothing written to Py.
void k1d_tma_stall_test(const Ctx &c, const K1dTma &t, const float *phir, const float *vloc, const float2 *Pa,
                        const float2 *Pvh, float2 *Py) {
  const int nb = k1d_tma_max_nb(c.nocc);
  if (nb >= 4) launch<4>(c, t, nb, 0, phir, vloc, Pa, Pvh, Py, true, true, 1);
  else if (nb == 3) launch<3>(c, t, nb, 0, phir, vloc, Pa, Pvh, Py, true, true, 1);
  else if (nb == 2) launch<2>(c, t, nb, 0, phir, vloc, Pa, Pvh, Py, true, true, 1);
  else launch<1>(c, t, nb, 0, phir, vloc, Pa, Pvh, Py, true, true, 1);
}

void k1d_tma(const Ctx &c, const K1dTma &t, int nb, const float *phir, const float *vloc, const float2 *Pa,
             const float2 *Pvh, float2 *Py, bool use_vloc, bool use_k1e) {
  int cap = k1d_tma_max_nb(c.nocc);
  if (c.k1d_nb_cap > 0) cap = std::min(cap, c.k1d_nb_cap);
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
