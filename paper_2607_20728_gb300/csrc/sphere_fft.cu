// Sphere-pruned transforms between wave-function-sphere vectors and real-space grids.
//
// A function on the wave-function sphere |G|^2 <= Ecut occupies only the columns (n1, n2) of
// the grid whose disk the sphere projects onto, and within a z plane only the y lines of the
// n1 it reaches.  The transforms therefore run as two passes:
//   inverse (sphere -> grid):  z pass over the occupied columns, scattering the real-basis
//     coefficients of two functions (packed as re + i im, Gamma-point symmetry) straight into
//     shared memory; then one xy pass per z plane that places the column results, transforms
//     the occupied y lines and all x lines, and writes the plane once;
//   forward (grid -> sphere):  the mirror image, with the gather to real-basis coefficients
//     (and the diagonal D term of Eq. 2a when asked) fused into the z pass.
// Between the passes only the occupied columns travel through global memory ("column
// buffer", [q][z][column]).  The local-potential product H X = (-1/2 lap + V) X also has a
// fused form whose xy pass transforms, multiplies by V(r) and transforms back in shared
// memory, so the full grid never reaches global memory.
// Columns are ordered as mirror pairs (n1, n2), (-n1, -n2) followed by (0, 0); a z-pass CTA
// takes an even number of columns, so both +G and -G of every coefficient are in its shared
// memory.
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "fft_codelets.cuh"
#include "internal.cuh"

namespace bse {

namespace {
using namespace fftc;

constexpr double kRs2 = 0.70710678118654752440;  // 1/sqrt(2)
constexpr int kThreads = 256;
constexpr int kXYThreads = 512;  // plane passes: more warps to hide the latency of the FP64 pipe
constexpr size_t kSmemCap = 200 * 1024;

template <class C>
struct SphArgs {
  int N1, N2, N3, N3p, ncols_pad, CG, nxs;
  long nr;
  const int *colpos;  // [ncols_pad] j1 + N1 j2, -1 for padding
  const int *xs;      // [nxs] x indices with occupied y lines
  const int4 *ent;    // per group: (kk, slot_p N3p + j3_p, slot_m N3p + j3_m, 0)
  const int *ent_off; // [ngroups + 1]
  AxisArgs<C> ax[3];
};

struct StrideBase {
  int s;
  __device__ __forceinline__ int operator()(int t) const { return t * s; }
};
struct ListBase {
  const int *xs;
  __device__ __forceinline__ int operator()(int t) const { return __ldg(&xs[t]); }
};

// L lines of an axis in shared memory, ping-ponging between `in` and `out`; returns the buffer
// holding the result.  LINE_FAST maps consecutive threads to consecutive lines, otherwise to
// consecutive butterflies of one line.  SG is the sign of the exponent (+1 inverse, -1 forward),
// a compile-time constant so that the twiddle conjugation and the factors +-i of the codelets
// fold into additions.  The caller has synchronised the input; the result is synchronised on
// return.
template <class C, bool LINE_FAST, int SG, class Base>
__device__ C *lines_fft(C *in, C *out, int L, Base base, int es, const AxisArgs<C> &ax) {
  const typename RealOf<C>::T sg = (typename RealOf<C>::T)SG;
  const int N = ax.n;
  int Ns = 1;
  for (int s = 0; s < ax.nstage; ++s) {
    const int R = ax.radix[s];
    const int nb = N / R;
    const int work = L * nb;
    // e = threadIdx.x + k blockDim.x split as (slow, fast) = divmod(e, F), advanced without
    // divisions: F = L (line fastest) or nb (butterfly fastest)
    const int F = LINE_FAST ? L : nb;
    int slow = threadIdx.x / F, fast = threadIdx.x - (threadIdx.x / F) * F;
    const int dslow = blockDim.x / F, dfast = blockDim.x - dslow * F;
    for (int e = threadIdx.x; e < work; e += blockDim.x) {
      const int t = LINE_FAST ? fast : slow;
      const int j = LINE_FAST ? slow : fast;
      const int b0 = base(t);
      stage_bfly_any<C>(R, in + b0, out + b0, j, N, Ns, ax.tw, sg, es);
      fast += dfast;
      slow += dslow;
      if (fast >= F) {
        fast -= F;
        ++slow;
      }
    }
    __syncthreads();
    C *tmp = in;
    in = out;
    out = tmp;
    Ns *= R;
  }
  return in;
}

// ---- z passes -------------------------------------------------------------------------------
// inverse: real-basis rows X[2q], X[2q+1] -> packed columns of group g -> z transform -> colbuf
template <class C>
__global__ void __launch_bounds__(kThreads) sph_z_inv(SphArgs<C> a, int nf, int npw, const double *__restrict__ X,
                                                      double scale, C *__restrict__ colbuf) {
  using T = typename RealOf<C>::T;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C *A = reinterpret_cast<C *>(sm_raw);
  C *B = A + (size_t)a.CG * a.N3p;
  const int g = blockIdx.x, q = blockIdx.y;
  const int nline = a.CG * a.N3p;
  for (int e = threadIdx.x; e < nline; e += blockDim.x) A[e] = mkc<C>(0, 0);
  __syncthreads();
  const double *f = X + (long)(2 * q) * npw;
  const bool hasg = (2 * q + 1) < nf;
  const double *h = X + (long)(2 * q + 1) * npw;
  const int e0 = a.ent_off[g], e1 = a.ent_off[g + 1];
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int4 en = __ldg(&a.ent[e]);
    const int kk = en.x;
    if (kk == 0) {
      A[en.y] = mkc<C>((T)(f[0] * scale), (T)(hasg ? h[0] * scale : 0.0));
      continue;
    }
    const double r2 = kRs2 * scale;
    const double fc = f[2 * kk - 1] * r2, fs = f[2 * kk] * r2;
    const double gc = hasg ? h[2 * kk - 1] * r2 : 0.0, gs = hasg ? h[2 * kk] * r2 : 0.0;
    A[en.y] = mkc<C>((T)(fc - gs), (T)(fs + gc));  // c_f + i c_g at +G
    A[en.z] = mkc<C>((T)(fc + gs), (T)(gc - fs));  // conj(c_f) + i conj(c_g) at -G
  }
  __syncthreads();
  C *F = lines_fft<C, false, 1>(A, B, a.CG, StrideBase{a.N3p}, 1, a.ax[2]);
  C *dst = colbuf + (long)q * a.N3 * a.ncols_pad + (long)g * a.CG;
  for (int e = threadIdx.x; e < a.CG * a.N3; e += blockDim.x) {
    const int slot = e % a.CG, z = e / a.CG;
    dst[(long)z * a.ncols_pad + slot] = F[slot * a.N3p + z];
  }
}

// forward: colbuf -> z transform -> gather to real-basis rows (plus the D term when Xd is given)
template <class C>
__global__ void __launch_bounds__(kThreads) sph_z_fwd(SphArgs<C> a, int nf, int npw, const C *__restrict__ colbuf,
                                                      double *__restrict__ Y, double scale,
                                                      const double *__restrict__ Xd,
                                                      const double *__restrict__ kin,
                                                      const double *__restrict__ shift, int period,
                                                      double shift_const) {
  using T = typename RealOf<C>::T;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C *A = reinterpret_cast<C *>(sm_raw);
  C *B = A + (size_t)a.CG * a.N3p;
  const int g = blockIdx.x, q = blockIdx.y;
  const C *src = colbuf + (long)q * a.N3 * a.ncols_pad + (long)g * a.CG;
  for (int e = threadIdx.x; e < a.CG * a.N3; e += blockDim.x) {
    const int slot = e % a.CG, z = e / a.CG;
    A[slot * a.N3p + z] = src[(long)z * a.ncols_pad + slot];
  }
  __syncthreads();
  const C *F = lines_fft<C, false, -1>(A, B, a.CG, StrideBase{a.N3p}, 1, a.ax[2]);
  const int f0 = 2 * q, f1 = 2 * q + 1;
  const bool hasg = f1 < nf;
  const double sh0 = (shift ? shift[f0 % period] : 0.0) + shift_const;
  const double sh1 = (shift ? shift[f1 % period] : 0.0) + shift_const;
  const int e0 = a.ent_off[g], e1 = a.ent_off[g + 1];
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int4 en = __ldg(&a.ent[e]);
    const int kk = en.x;
    double a0, a1 = 0.0, b0, b1 = 0.0;
    int i0, i1;
    if (kk == 0) {
      const C v = F[en.y];
      i0 = 0;
      i1 = -1;
      a0 = (double)v.x * scale;
      b0 = (double)v.y * scale;
    } else {
      const C Fp = F[en.y], Fm = F[en.z];
      const double s = kRs2 * scale;
      i0 = 2 * kk - 1;
      i1 = 2 * kk;
      a0 = ((double)Fp.x + (double)Fm.x) * s;
      a1 = ((double)Fp.y - (double)Fm.y) * s;
      b0 = ((double)Fp.y + (double)Fm.y) * s;
      b1 = ((double)Fm.x - (double)Fp.x) * s;
    }
    if (Xd) {
      a0 += (kin[i0] + sh0) * Xd[(long)f0 * npw + i0];
      if (i1 >= 0) a1 += (kin[i1] + sh0) * Xd[(long)f0 * npw + i1];
      if (hasg) {
        b0 += (kin[i0] + sh1) * Xd[(long)f1 * npw + i0];
        if (i1 >= 0) b1 += (kin[i1] + sh1) * Xd[(long)f1 * npw + i1];
      }
    }
    Y[(long)f0 * npw + i0] = a0;
    if (i1 >= 0) Y[(long)f0 * npw + i1] = a1;
    if (hasg) {
      Y[(long)f1 * npw + i0] = b0;
      if (i1 >= 0) Y[(long)f1 * npw + i1] = b1;
    }
  }
}

// ---- xy passes (one CTA per plane z of grid q) ---------------------------------------------
// MODE 0: colbuf -> inverse y (occupied lines) and x -> grid plane
// MODE 1: grid plane -> forward x and y (occupied lines) -> colbuf
// MODE 2: colbuf -> inverse -> times V(r) -> forward -> colbuf (in place)
// The plane sits in shared memory with rows padded to N1 + 1 elements and consecutive threads on
// consecutive lines in both passes (x lines one padded row apart, y lines one x apart), so the
// strided butterfly loads and stores of every stage fall in distinct banks.
template <class C, int MODE>
__global__ void __launch_bounds__(kXYThreads) sph_xy(SphArgs<C> a, C *__restrict__ colbuf, C *__restrict__ P,
                                                     const typename RealOf<C>::T *__restrict__ vloc) {
  using T = typename RealOf<C>::T;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int N1 = a.N1, N1p = a.N1 + 1;
  const int np = N1 * a.N2, npp = N1p * a.N2;
  C *A = reinterpret_cast<C *>(sm_raw);
  C *B = A + npp;
  const int z = blockIdx.x, q = blockIdx.y;
  C *crow = colbuf + ((long)q * a.N3 + z) * a.ncols_pad;
  C *plane = P ? P + (long)q * a.nr + (long)z * np : nullptr;
  // the padded index of element e = y N1 + x of the plane is e + y; (y, x) stepped without divisions
  const int y0 = threadIdx.x / N1, x0 = threadIdx.x - y0 * N1;
  const int dy = blockDim.x / N1, dx = blockDim.x - dy * N1;
  auto for_plane = [&](auto body) {
    int y = y0, x = x0;
    for (int e = threadIdx.x; e < np; e += blockDim.x) {
      body(e, e + y);
      x += dx;
      y += dy;
      if (x >= N1) {
        x -= N1;
        ++y;
      }
    }
  };
  C *F;
  if (MODE == 0 || MODE == 2) {
    // the y pass transforms the occupied lines only, so the buffer its result lands in must hold
    // zeros on the others: A with an even number of stages (B is then fully overwritten by the x
    // pass before it is read), B with an odd number
    const bool zero_b = (a.ax[1].nstage & 1) != 0;
    for (int e = threadIdx.x; e < npp; e += blockDim.x) {
      A[e] = mkc<C>(0, 0);
      if (zero_b) B[e] = mkc<C>(0, 0);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < a.ncols_pad; c += blockDim.x) {
      const int pos = __ldg(&a.colpos[c]);
      if (pos >= 0) A[pos + pos / N1] = crow[c];
    }
    __syncthreads();
    F = lines_fft<C, true, 1>(A, B, a.nxs, ListBase{a.xs}, N1p, a.ax[1]);
    C *O = F == A ? B : A;
    F = lines_fft<C, true, 1>(F, O, a.N2, StrideBase{N1p}, 1, a.ax[0]);
    if (MODE == 0) {
      for_plane([&](int e, int ep) { plane[e] = F[ep]; });
      return;
    }
    const T *v = vloc + (long)z * np;
    for_plane([&](int e, int ep) {
      const T w = v[e];
      const C u = F[ep];
      F[ep] = mkc<C>(u.x * w, u.y * w);
    });
    __syncthreads();
  } else {
    for_plane([&](int e, int ep) { A[ep] = plane[e]; });
    __syncthreads();
    F = A;
  }
  C *O = F == A ? B : A;
  F = lines_fft<C, true, -1>(F, O, a.N2, StrideBase{N1p}, 1, a.ax[0]);
  O = F == A ? B : A;
  F = lines_fft<C, true, -1>(F, O, a.nxs, ListBase{a.xs}, N1p, a.ax[1]);
  for (int c = threadIdx.x; c < a.ncols_pad; c += blockDim.x) {
    const int pos = __ldg(&a.colpos[c]);
    crow[c] = pos >= 0 ? F[pos + pos / N1] : mkc<C>(0, 0);
  }
}

// ---- pair pipelines on the density sphere (tau build, U vector; Eq. 2c and Eq. 3) ----------
// forward z pass: z lines of the occupied density columns, then the wave-function-sphere
// coefficients of the two packed pair densities into X (real basis, type R, times `scale`) for
// the PDEP projection, and every column element times v_c(G) * cscale (zero outside the density
// sphere) written back
template <class C, class R>
__global__ void __launch_bounds__(kThreads) dsph_z_fwd(SphArgs<C> a, int np, int npw, C *__restrict__ colbuf,
                                                       R *__restrict__ X, double scale,
                                                       const R *__restrict__ vcg, R cscale) {
  using T = typename RealOf<C>::T;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C *A = reinterpret_cast<C *>(sm_raw);
  C *B = A + (size_t)a.CG * a.N3p;
  const int g = blockIdx.x, q = blockIdx.y;
  C *col = colbuf + (long)q * a.N3 * a.ncols_pad + (long)g * a.CG;
  for (int e = threadIdx.x; e < a.CG * a.N3; e += blockDim.x) {
    const int slot = e % a.CG, z = e / a.CG;
    A[slot * a.N3p + z] = col[(long)z * a.ncols_pad + slot];
  }
  __syncthreads();
  C *F = lines_fft<C, false, -1>(A, B, a.CG, StrideBase{a.N3p}, 1, a.ax[2]);
  if (X) {
    const int f0 = 2 * q, f1 = 2 * q + 1;
    const bool hasg = f1 < np;
    for (int e = a.ent_off[g] + threadIdx.x; e < a.ent_off[g + 1]; e += blockDim.x) {
      const int4 en = __ldg(&a.ent[e]);
      const int kk = en.x;
      if (kk == 0) {
        const C v = F[en.y];
        X[(long)f0 * npw] = (R)((double)v.x * scale);
        if (hasg) X[(long)f1 * npw] = (R)((double)v.y * scale);
        continue;
      }
      const C Fp = F[en.y], Fm = F[en.z];
      const double sc = kRs2 * scale;
      X[(long)f0 * npw + 2 * kk - 1] = (R)(((double)Fp.x + (double)Fm.x) * sc);
      X[(long)f0 * npw + 2 * kk] = (R)(((double)Fp.y - (double)Fm.y) * sc);
      if (hasg) {
        X[(long)f1 * npw + 2 * kk - 1] = (R)(((double)Fp.y + (double)Fm.y) * sc);
        X[(long)f1 * npw + 2 * kk] = (R)(((double)Fm.x - (double)Fp.x) * sc);
      }
    }
  }
  const long np2 = (long)a.N1 * a.N2;
  for (int e = threadIdx.x; e < a.CG * a.N3; e += blockDim.x) {
    const int slot = e % a.CG, z = e / a.CG;
    const int pos = __ldg(&a.colpos[g * a.CG + slot]);
    const T w = pos >= 0 ? (T)(vcg[(long)z * np2 + pos] * cscale) : (T)0;
    const C v = F[slot * a.N3p + z];
    col[(long)z * a.ncols_pad + slot] = mkc<C>(v.x * w, v.y * w);
  }
}

// inverse z pass: the PDEP back-projection X (real basis, type R, times `scale`) added at the
// wave-function-sphere coefficients of the two packed pairs, then z lines of the columns
template <class C, class R>
__global__ void __launch_bounds__(kThreads) dsph_z_inv(SphArgs<C> a, int np, int npw, const R *__restrict__ X,
                                                       double scale, C *__restrict__ colbuf) {
  using T = typename RealOf<C>::T;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C *A = reinterpret_cast<C *>(sm_raw);
  C *B = A + (size_t)a.CG * a.N3p;
  const int g = blockIdx.x, q = blockIdx.y;
  C *col = colbuf + (long)q * a.N3 * a.ncols_pad + (long)g * a.CG;
  for (int e = threadIdx.x; e < a.CG * a.N3; e += blockDim.x) {
    const int slot = e % a.CG, z = e / a.CG;
    A[slot * a.N3p + z] = col[(long)z * a.ncols_pad + slot];
  }
  __syncthreads();
  if (X) {
    const R *f = X + (long)(2 * q) * npw;
    const bool hasg = (2 * q + 1) < np;
    const R *h = X + (long)(2 * q + 1) * npw;
    for (int e = a.ent_off[g] + threadIdx.x; e < a.ent_off[g + 1]; e += blockDim.x) {
      const int4 en = __ldg(&a.ent[e]);
      const int kk = en.x;
      if (kk == 0) {
        C &t = A[en.y];
        t = mkc<C>(t.x + (T)((double)f[0] * scale), t.y + (T)(hasg ? (double)h[0] * scale : 0.0));
        continue;
      }
      const double r2 = kRs2 * scale;
      const double fc = (double)f[2 * kk - 1] * r2, fs = (double)f[2 * kk] * r2;
      const double gc = hasg ? (double)h[2 * kk - 1] * r2 : 0.0, gs = hasg ? (double)h[2 * kk] * r2 : 0.0;
      C &tp = A[en.y];
      tp = mkc<C>(tp.x + (T)(fc - gs), tp.y + (T)(fs + gc));
      C &tm = A[en.z];
      tm = mkc<C>(tm.x + (T)(fc + gs), tm.y + (T)(gc - fs));
    }
  }
  __syncthreads();
  C *F = lines_fft<C, false, 1>(A, B, a.CG, StrideBase{a.N3p}, 1, a.ax[2]);
  for (int e = threadIdx.x; e < a.CG * a.N3; e += blockDim.x) {
    const int slot = e % a.CG, z = e / a.CG;
    col[(long)z * a.ncols_pad + slot] = F[slot * a.N3p + z];
  }
}

template <class C>
SphArgs<C> make_args(const Ctx &c, const SphereFFT &s) {
  SphArgs<C> a;
  a.N1 = c.N[0];
  a.N2 = c.N[1];
  a.N3 = c.N[2];
  a.N3p = c.N[2] + 1;
  a.ncols_pad = s.ncols_pad;
  a.CG = s.cg;
  a.nxs = s.nxs;
  a.nr = c.nr;
  a.colpos = s.colpos.get();
  a.xs = s.xs.get();
  a.ent = s.ent.get();
  a.ent_off = s.ent_off.get();
  for (int i = 0; i < 3; ++i) {
    const FFTAxis &x = c.fft.ax[i];
    a.ax[i].n = x.n;
    a.ax[i].nstage = x.nstage;
    for (int r = 0; r < 12; ++r) a.ax[i].radix[r] = x.radix[r];
    if constexpr (sizeof(C) == sizeof(double2)) a.ax[i].tw = reinterpret_cast<const C *>(x.tw);
    else a.ax[i].tw = reinterpret_cast<const C *>(x.tw32);
  }
  return a;
}

template <class C>
size_t z_smem(const Ctx &c, const SphereFFT &s) { return (size_t)2 * s.cg * (c.N[2] + 1) * sizeof(C); }
template <class C>
size_t z_smem(const Ctx &c) { return z_smem<C>(c, c.sfft); }
template <class C>
size_t xy_smem(const Ctx &c) { return (size_t)2 * (c.N[0] + 1) * c.N[1] * sizeof(C); }

// dynamic shared-memory limits are per-device function attributes: set once per device
template <class C>
void set_attrs() {
  static std::mutex mu;
  static std::map<int, bool> done;
  int dev = 0;
  BSE_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return;
  const int cap = (int)kSmemCap;
  BSE_CUDA(cudaFuncSetAttribute(sph_z_inv<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
  BSE_CUDA(cudaFuncSetAttribute(sph_z_fwd<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
  BSE_CUDA(cudaFuncSetAttribute(sph_xy<C, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
  BSE_CUDA(cudaFuncSetAttribute(sph_xy<C, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
  BSE_CUDA(cudaFuncSetAttribute(sph_xy<C, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
  using R = typename RealOf<C>::T;
  BSE_CUDA(cudaFuncSetAttribute(dsph_z_fwd<C, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
  BSE_CUDA(cudaFuncSetAttribute(dsph_z_inv<C, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
  done[dev] = true;
}

// threads per plane-pass CTA: the autotuner's choice, else kXYThreads
int xy_threads(const Ctx &c) { return c.xy_threads > 0 ? std::min(c.xy_threads, kXYThreads) : kXYThreads; }

template <class R>
CT<R> *colbuf_for(Ctx &c, int nq) {
  Grids<R> &g = c.grids<R>();
  g.colbuf.alloc((size_t)nq * c.N[2] * c.sfft.ncols_pad);
  return g.colbuf.get();
}

}  // namespace

// ---- plan ----------------------------------------------------------------------------------
namespace {
// Column tables of one sphere: the columns of `col_millers` ((n1, n2) pairs, closed under
// negation) as mirror pairs then (0, 0); the coefficient entries of the wave-function half
// sphere (miller_half) placed in that column layout.
void build_tables(Ctx &c, SphereFFT &s, const std::vector<std::pair<int, int>> &col_millers,
                  const std::vector<int> &miller_half) {
  s.ready = s.ok64 = s.ok32 = false;
  const int N1 = c.N[0], N2 = c.N[1], N3 = c.N[2];
  const int nh = (int)miller_half.size() / 3;  // entries kk = 0..nhalf (kk = 0 is G = 0)
  auto md = [](int v, int n) { return ((v % n) + n) % n; };
  std::map<std::pair<int, int>, int> col;
  std::vector<std::pair<int, int>> order;
  for (const auto &cm : col_millers) {
    const int n1 = cm.first, n2 = cm.second;
    const bool pos = n2 > 0 || (n2 == 0 && n1 > 0);
    if (!pos || col.count({n1, n2})) continue;
    col[{n1, n2}] = -1;
    order.push_back({n1, n2});
  }
  std::sort(order.begin(), order.end(), [](const std::pair<int, int> &x, const std::pair<int, int> &y) {
    return x.second != y.second ? x.second < y.second : x.first < y.first;
  });
  std::vector<std::pair<int, int>> cols;
  for (auto &p : order) {
    cols.push_back(p);
    cols.push_back({-p.first, -p.second});
  }
  cols.push_back({0, 0});
  col.clear();
  for (size_t i = 0; i < cols.size(); ++i) col[cols[i]] = (int)i;
  // columns per z-pass CTA: even, so that mirror pairs stay together; shared memory bounded
  // for FP64 lines
  int cg = 32;
  while (cg > 2 && (size_t)2 * cg * (N3 + 1) * sizeof(double2) > kSmemCap) cg -= 2;
  s.cg = cg;
  s.ncols = (int)cols.size();
  s.ngroups = (s.ncols + cg - 1) / cg;
  s.ncols_pad = s.ngroups * cg;
  std::vector<int> colpos(s.ncols_pad, -1);
  std::vector<int> xs_all;
  for (int i = 0; i < s.ncols; ++i) {
    const int j1 = md(cols[i].first, N1), j2 = md(cols[i].second, N2);
    colpos[i] = j1 + N1 * j2;
    xs_all.push_back(j1);
  }
  std::sort(xs_all.begin(), xs_all.end());
  xs_all.erase(std::unique(xs_all.begin(), xs_all.end()), xs_all.end());
  s.nxs = (int)xs_all.size();
  // entries grouped by the z-pass CTA that owns both of their columns
  std::vector<std::vector<int4>> per(s.ngroups);
  const int N3p = N3 + 1;
  for (int kk = 0; kk < nh; ++kk) {
    const int n1 = miller_half[3 * kk], n2 = miller_half[3 * kk + 1], n3 = miller_half[3 * kk + 2];
    const int cp = col.at({n1, n2}), cm = col.at({-n1, -n2});
    const int gp_ = cp / cg;
    BSE_REQUIRE(cm / cg == gp_, "internal: mirror columns split across z-pass groups");
    int4 e;
    e.x = kk;
    e.y = (cp % cg) * N3p + md(n3, N3);
    e.z = (cm % cg) * N3p + md(-n3, N3);
    e.w = 0;
    per[gp_].push_back(e);
  }
  std::vector<int4> ent;
  std::vector<int> off{0};
  for (auto &v : per) {
    ent.insert(ent.end(), v.begin(), v.end());
    off.push_back((int)ent.size());
  }
  s.colpos.alloc(colpos.size());
  s.xs.alloc(xs_all.size());
  s.ent.alloc(ent.size());
  s.ent_off.alloc(off.size());
  BSE_CUDA(cudaMemcpy(s.colpos.get(), colpos.data(), colpos.size() * sizeof(int), cudaMemcpyHostToDevice));
  BSE_CUDA(cudaMemcpy(s.xs.get(), xs_all.data(), xs_all.size() * sizeof(int), cudaMemcpyHostToDevice));
  BSE_CUDA(cudaMemcpy(s.ent.get(), ent.data(), ent.size() * sizeof(int4), cudaMemcpyHostToDevice));
  BSE_CUDA(cudaMemcpy(s.ent_off.get(), off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice));
  s.ok64 = z_smem<double2>(c, s) <= kSmemCap && xy_smem<double2>(c) <= kSmemCap;
  s.ok32 = z_smem<float2>(c, s) <= kSmemCap && xy_smem<float2>(c) <= kSmemCap;
  s.ready = true;
}
}  // namespace

void sphere_fft_init(Ctx &c, const std::vector<int> &miller_half, const std::vector<int> &dens_cols) {
  std::vector<std::pair<int, int>> wcols;
  for (size_t kk = 1; kk < miller_half.size() / 3; ++kk)
    for (int sgn : {1, -1}) wcols.push_back({sgn * miller_half[3 * kk], sgn * miller_half[3 * kk + 1]});
  build_tables(c, c.sfft, wcols, miller_half);
  std::vector<std::pair<int, int>> dcols;
  for (size_t i = 0; i + 1 < dens_cols.size(); i += 2) dcols.push_back({dens_cols[i], dens_cols[i + 1]});
  build_tables(c, c.dfft, dcols, miller_half);
}

template <class R>
bool dens_fft_ok(const Ctx &c) {
  return c.dfft.ready && (sizeof(R) == sizeof(double) ? c.dfft.ok64 : c.dfft.ok32) && !c.sfft.disabled;
}

// forward half of the pair pipeline: packed pair grids P -> density columns (Coulomb applied,
// scaled by cscale) and the wave-function-sphere coefficients X (times scale) for the PDEP part
template <class R>
void dens_forward(Ctx &c, int np, CT<R> *P, R *X, double scale, const R *vcg, R cscale) {
  using C = CT<R>;
  const int nq = (np + 1) / 2;
  set_attrs<C>();
  SphArgs<C> a = make_args<C>(c, c.dfft);
  Grids<R> &g = c.grids<R>();
  g.colbuf_dens.alloc((size_t)nq * c.N[2] * c.dfft.ncols_pad);
  C *cb = g.colbuf_dens.get();
  sph_xy<C, 1><<<dim3(c.N[2], nq), xy_threads(c), xy_smem<C>(c), c.stream>>>(a, cb, P, nullptr);
  BSE_CHECK_LAUNCH();
  dsph_z_fwd<C, R><<<dim3(c.dfft.ngroups, nq), kThreads, z_smem<C>(c, c.dfft), c.stream>>>(a, np, c.npw, cb, X,
                                                                                         scale, vcg, cscale);
  BSE_CHECK_LAUNCH();
}

// inverse half: PDEP back-projection X (times scale) added in the columns, then to the grid P
template <class R>
void dens_inverse(Ctx &c, int np, const R *X, double scale, CT<R> *P) {
  using C = CT<R>;
  const int nq = (np + 1) / 2;
  set_attrs<C>();
  SphArgs<C> a = make_args<C>(c, c.dfft);
  C *cb = c.grids<R>().colbuf_dens.get();
  dsph_z_inv<C, R><<<dim3(c.dfft.ngroups, nq), kThreads, z_smem<C>(c, c.dfft), c.stream>>>(a, np, c.npw, X, scale,
                                                                                         cb);
  BSE_CHECK_LAUNCH();
  sph_xy<C, 0><<<dim3(c.N[2], nq), xy_threads(c), xy_smem<C>(c), c.stream>>>(a, cb, P, nullptr);
  BSE_CHECK_LAUNCH();
}

template bool dens_fft_ok<double>(const Ctx &);
template bool dens_fft_ok<float>(const Ctx &);
template void dens_forward<double>(Ctx &, int, double2 *, double *, double, const double *, double);
template void dens_forward<float>(Ctx &, int, float2 *, float *, double, const float *, float);
template void dens_inverse<double>(Ctx &, int, const double *, double, double2 *);
template void dens_inverse<float>(Ctx &, int, const float *, double, float2 *);

template <class R>
bool sphere_fft_ok(const Ctx &c) {
  return c.sfft.ready && (sizeof(R) == sizeof(double) ? c.sfft.ok64 : c.sfft.ok32) && !c.sfft.disabled;
}

template <class R>
void sphere_to_grid(Ctx &c, int nf, const double *X, CT<R> *P, double scale, CT<R> *colbuf) {
  using C = CT<R>;
  if (nf <= 0) return;
  const int nq = (nf + 1) / 2;
  set_attrs<C>();
  SphArgs<C> a = make_args<C>(c, c.sfft);
  C *cb = colbuf ? colbuf : colbuf_for<R>(c, nq);
  sph_z_inv<C><<<dim3(c.sfft.ngroups, nq), kThreads, z_smem<C>(c), c.stream>>>(a, nf, c.npw, X, scale, cb);
  BSE_CHECK_LAUNCH();
  sph_xy<C, 0><<<dim3(c.N[2], nq), xy_threads(c), xy_smem<C>(c), c.stream>>>(a, cb, P, nullptr);
  BSE_CHECK_LAUNCH();
}

template <class R>
void grid_to_sphere(Ctx &c, int nf, CT<R> *P, double *Y, double scale, const double *Xd, const double *shift,
                    int period, double shift_const, CT<R> *colbuf) {
  using C = CT<R>;
  if (nf <= 0) return;
  const int nq = (nf + 1) / 2;
  set_attrs<C>();
  SphArgs<C> a = make_args<C>(c, c.sfft);
  C *cb = colbuf ? colbuf : colbuf_for<R>(c, nq);
  sph_xy<C, 1><<<dim3(c.N[2], nq), xy_threads(c), xy_smem<C>(c), c.stream>>>(a, cb, P, nullptr);
  BSE_CHECK_LAUNCH();
  sph_z_fwd<C><<<dim3(c.sfft.ngroups, nq), kThreads, z_smem<C>(c), c.stream>>>(
      a, nf, c.npw, cb, Y, scale, Xd, c.kin.get(), shift, period > 0 ? period : 1, shift_const);
  BSE_CHECK_LAUNCH();
}

template <class R>
void sphere_h(Ctx &c, int nf, const double *X, double *HX, const double *shift) {
  using C = CT<R>;
  if (nf <= 0) return;
  const int nq = (nf + 1) / 2;
  set_attrs<C>();
  SphArgs<C> a = make_args<C>(c, c.sfft);
  C *cb = colbuf_for<R>(c, nq);
  const double s_in = 1.0 / std::sqrt(c.omega), s_out = std::sqrt(c.omega) / (double)c.nr;
  sph_z_inv<C><<<dim3(c.sfft.ngroups, nq), kThreads, z_smem<C>(c), c.stream>>>(a, nf, c.npw, X, s_in, cb);
  BSE_CHECK_LAUNCH();
  sph_xy<C, 2><<<dim3(c.N[2], nq), xy_threads(c), xy_smem<C>(c), c.stream>>>(a, cb, nullptr,
                                                                            c.grids<R>().vloc.get());
  BSE_CHECK_LAUNCH();
  sph_z_fwd<C><<<dim3(c.sfft.ngroups, nq), kThreads, z_smem<C>(c), c.stream>>>(
      a, nf, c.npw, cb, HX, s_out, X, c.kin.get(), shift, shift ? c.nocc : 1, 0.0);
  BSE_CHECK_LAUNCH();
}

template bool sphere_fft_ok<double>(const Ctx &);
template bool sphere_fft_ok<float>(const Ctx &);
template void sphere_to_grid<double>(Ctx &, int, const double *, double2 *, double, double2 *);
template void sphere_to_grid<float>(Ctx &, int, const double *, float2 *, double, float2 *);
template void grid_to_sphere<double>(Ctx &, int, double2 *, double *, double, const double *, const double *, int,
                                     double, double2 *);
template void grid_to_sphere<float>(Ctx &, int, float2 *, double *, double, const double *, const double *, int,
                                    double, float2 *);
template void sphere_h<double>(Ctx &, int, const double *, double *, const double *);
template void sphere_h<float>(Ctx &, int, const double *, double *, const double *);

}  // namespace bse
