// Grid and sphere kernels of the Liouville operator (Eq. 2), the screened interaction
// (Eq. 3), the densities (Eqs. 5-6) and the force contraction (Eq. 4).
//
// Gamma-point functions are real in r, so two of them share one complex FFT: a packed
// grid P holds f + i g.  Sphere coefficients use the real basis of the public header.
#include <cmath>

#include "internal.cuh"

namespace bse {
namespace k {

namespace {

constexpr double kRsqrt2 = 0.70710678118654752440;

template <class R> struct Cx;
template <> struct Cx<double> { using T = double2; };
template <> struct Cx<float> { using T = float2; };
template <class R>
__device__ __forceinline__ typename Cx<R>::T mk(R x, R y) {
  typename Cx<R>::T v;
  v.x = x;
  v.y = y;
  return v;
}

inline int nblocks(long n, int bs, int cap = 152 * 64) {
  long b = (n + bs - 1) / bs;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// ---- sphere <-> packed grids --------------------------------------------------------
template <class R, class I>
__global__ void scatter_pairs_kernel(int nf, int npw, int nhalf, long nr, const int *__restrict__ gp,
                                     const int *__restrict__ gm, const I *__restrict__ X,
                                     typename Cx<R>::T *__restrict__ P, double scale, int accumulate) {
  using C = typename Cx<R>::T;
  const int nq = (nf + 1) / 2;
  const long total = (long)nq * (nhalf + 1);
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total;
       idx += (long)gridDim.x * blockDim.x) {
    const int q = (int)(idx / (nhalf + 1));
    const int kk = (int)(idx - (long)q * (nhalf + 1));
    const I *f = X + (long)(2 * q) * npw;
    const bool hasg = (2 * q + 1) < nf;
    const I *g = X + (long)(2 * q + 1) * npw;
    C *Pq = P + (long)q * nr;
    if (kk == 0) {
      double vx = (double)f[0] * scale, vy = hasg ? (double)g[0] * scale : 0.0;
      const int i0 = gp[0];
      if (accumulate) { vx += Pq[i0].x; vy += Pq[i0].y; }
      Pq[i0] = mk<R>((R)vx, (R)vy);
      continue;
    }
    const double r2 = kRsqrt2 * scale;
    const double fc = (double)f[2 * kk - 1] * r2, fs = (double)f[2 * kk] * r2;
    const double gc = hasg ? (double)g[2 * kk - 1] * r2 : 0.0, gs = hasg ? (double)g[2 * kk] * r2 : 0.0;
    double px = fc - gs, py = fs + gc;   // c_f + i c_g at +G
    double mx = fc + gs, my = gc - fs;   // conj(c_f) + i conj(c_g) at -G
    const int ip = gp[kk], im = gm[kk];
    if (accumulate) {
      const C a = Pq[ip], b = Pq[im];
      px += a.x; py += a.y; mx += b.x; my += b.y;
    }
    Pq[ip] = mk<R>((R)px, (R)py);
    Pq[im] = mk<R>((R)mx, (R)my);
  }
}

template <class R, class O>
__global__ void gather_pairs_kernel(int nf, int npw, int nhalf, long nr, const int *__restrict__ gp,
                                    const int *__restrict__ gm, const typename Cx<R>::T *__restrict__ P,
                                    O *__restrict__ Y, double scale,
                                    const double *__restrict__ Xd, const double *__restrict__ kin,
                                    const double *__restrict__ shift, int period,
                                    double shift_const) {
  const int nq = (nf + 1) / 2;
  const long total = (long)nq * (nhalf + 1);
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total;
       idx += (long)gridDim.x * blockDim.x) {
    const int q = (int)(idx / (nhalf + 1));
    const int kk = (int)(idx - (long)q * (nhalf + 1));
    const typename Cx<R>::T *Pq = P + (long)q * nr;
    const int f0 = 2 * q, f1 = 2 * q + 1;
    const bool hasg = f1 < nf;
    double a0, a1, b0, b1;  // f[i0], f[i1], g[i0], g[i1]
    int i0, i1;
    if (kk == 0) {
      const typename Cx<R>::T F = Pq[gp[0]];
      i0 = 0; i1 = -1;
      a0 = (double)F.x * scale; b0 = (double)F.y * scale; a1 = b1 = 0.0;
    } else {
      const typename Cx<R>::T Fp = Pq[gp[kk]], Fm = Pq[gm[kk]];
      const double s = kRsqrt2 * scale;
      i0 = 2 * kk - 1; i1 = 2 * kk;
      a0 = ((double)Fp.x + (double)Fm.x) * s; a1 = ((double)Fp.y - (double)Fm.y) * s;
      b0 = ((double)Fp.y + (double)Fm.y) * s; b1 = ((double)Fm.x - (double)Fp.x) * s;
    }
    if (Xd) {
      const double sh0 = (shift ? shift[f0 % period] : 0.0) + shift_const;
      const double sh1 = (shift ? shift[f1 % period] : 0.0) + shift_const;
      a0 += (kin[i0] + sh0) * Xd[(long)f0 * npw + i0];
      if (i1 >= 0) a1 += (kin[i1] + sh0) * Xd[(long)f0 * npw + i1];
      if (hasg) {
        b0 += (kin[i0] + sh1) * Xd[(long)f1 * npw + i0];
        if (i1 >= 0) b1 += (kin[i1] + sh1) * Xd[(long)f1 * npw + i1];
      }
    }
    Y[(long)f0 * npw + i0] = (O)a0;
    if (i1 >= 0) Y[(long)f0 * npw + i1] = (O)a1;
    if (hasg) {
      Y[(long)f1 * npw + i0] = (O)b0;
      if (i1 >= 0) Y[(long)f1 * npw + i1] = (O)b1;
    }
  }
}

template <class R>
__global__ void mul_grid_kernel(long nr, int nq, typename Cx<R>::T *__restrict__ P, const R *__restrict__ w,
                                R scale) {
  const long total = nr * nq;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total;
       i += (long)gridDim.x * blockDim.x) {
    const R s = w[i % nr] * scale;
    typename Cx<R>::T v = P[i];
    P[i] = mk<R>(v.x * s, v.y * s);
  }
}

// real grids from packed grids (output type O: the grid type or FP64)
template <class R, class O>
__global__ void unpack_kernel(long nr, int nf, const typename Cx<R>::T *__restrict__ P, O *__restrict__ Rr) {
  const long total = nr * nf;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total;
       i += (long)gridDim.x * blockDim.x) {
    const int f = (int)(i / nr);
    const long r = i - (long)f * nr;
    const typename Cx<R>::T v = P[(long)(f >> 1) * nr + r];
    Rr[i] = (O)((f & 1) ? v.y : v.x);
  }
}

template <class R>
__global__ void pack_kernel(long nr, int nf, const R *__restrict__ Rr, typename Cx<R>::T *__restrict__ P) {
  const int nq = (nf + 1) / 2;
  const long total = nr * nq;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total;
       i += (long)gridDim.x * blockDim.x) {
    const int q = (int)(i / nr);
    const long r = i - (long)q * nr;
    const R a = Rr[(long)(2 * q) * nr + r];
    const R b = (2 * q + 1 < nf) ? Rr[(long)(2 * q + 1) * nr + r] : (R)0;
    P[i] = mk<R>(a, b);
  }
}

__global__ void fill_real_kernel(long nr, double2 *__restrict__ P, const double *__restrict__ R) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nr; i += (long)gridDim.x * blockDim.x)
    P[i] = make_double2(R[i], 0.0);
}

template <class R>
__global__ void pair_products_kernel(long nr, int np, const int2 *__restrict__ list,
                                     const R *__restrict__ A, const R *__restrict__ Bm,
                                     typename Cx<R>::T *__restrict__ P) {
  const int nq = (np + 1) / 2;
  const long total = nr * nq;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total;
       i += (long)gridDim.x * blockDim.x) {
    const int q = (int)(i / nr);
    const long r = i - (long)q * nr;
    const int2 p0 = list[2 * q];
    const R a = A[(long)p0.x * nr + r] * Bm[(long)p0.y * nr + r];
    R b = 0;
    if (2 * q + 1 < np) {
      const int2 p1 = list[2 * q + 1];
      b = A[(long)p1.x * nr + r] * Bm[(long)p1.y * nr + r];
    }
    P[i] = mk<R>(a, b);
  }
}

template <class T>
__global__ void scale_cols_kernel(int rows, int cols, T *__restrict__ Q, const T *__restrict__ s) {
  const long total = (long)rows * cols;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total;
       i += (long)gridDim.x * blockDim.x)
    Q[i] *= s[i % cols];
}

// Delta rho_b(r) = sum_v phi_v(r) a_{b,v}(r)  (Eq. 2b); a packed over f = b*nocc + v
template <class R>
__global__ void drho_kernel(long nr, int nocc, int nb, const R *__restrict__ phir,
                            const typename Cx<R>::T *__restrict__ Pa, typename Cx<R>::T *__restrict__ Pd) {
  const R *Pa_d = reinterpret_cast<const R *>(Pa);
  R *Pd_d = reinterpret_cast<R *>(Pd);
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < nr; r += (long)gridDim.x * blockDim.x) {
    for (int b = 0; b < nb; ++b) {
      R s = 0;
      for (int v = 0; v < nocc; ++v) {
        const long f = (long)b * nocc + v;
        s = fma(phir[(long)v * nr + r], Pa_d[2 * ((f >> 1) * nr + r) + (f & 1)], s);
      }
      Pd_d[2 * ((long)(b >> 1) * nr + r) + (b & 1)] = s;
    }
    if (nb & 1) Pd_d[2 * ((long)(nb >> 1) * nr + r) + 1] = 0;
  }
}

// Y_{b,v}(r) = V(r) a_{b,v} + 2 vH_b phi_v - sum_v' tau_{v'v} a_{b,v'}  (Eqs. 2a-2c on the grid)
template <class R, int NB, int TV>
__global__ void __launch_bounds__(128) combine_tau_kernel(
    long nr, int nocc, int nb_total, int b0, const R *__restrict__ phir,
    const R *__restrict__ vloc, const R *__restrict__ tau, const typename Cx<R>::T *__restrict__ Pa,
    const typename Cx<R>::T *__restrict__ Pvh, typename Cx<R>::T *__restrict__ Py, int use_vloc, int use_k1e,
    int use_k1d) {
  const long r = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (r >= nr) return;
  const int v0 = blockIdx.y * TV;
  const R *Pa_d = reinterpret_cast<const R *>(Pa);
  const R *Pv_d = reinterpret_cast<const R *>(Pvh);
  R *Py_d = reinterpret_cast<R *>(Py);
  R acc[NB][TV];
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int t = 0; t < TV; ++t) acc[b][t] = 0;
  if (use_k1d) {
    for (int vp = 0; vp < nocc; ++vp) {
      R a[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int bb = b0 + b;
        const long f = (long)bb * nocc + vp;
        a[b] = (bb < nb_total) ? Pa_d[2 * ((f >> 1) * nr + r) + (f & 1)] : (R)0;
      }
#pragma unroll
      for (int t = 0; t < TV; ++t) {
        const int v = v0 + t;
        if (v < nocc) {
          const int hi = v > vp ? v : vp, lo = v > vp ? vp : v;
          const R tv = __ldg(&tau[((long)hi * (hi + 1) / 2 + lo) * nr + r]);
#pragma unroll
          for (int b = 0; b < NB; ++b) acc[b][t] = fma(tv, a[b], acc[b][t]);
        }
      }
    }
  }
  const R V = use_vloc ? vloc[r] : (R)0;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int bb = b0 + b;
    if (bb >= nb_total) continue;
    const R vh = use_k1e ? (R)2 * Pv_d[2 * ((long)(bb >> 1) * nr + r) + (bb & 1)] : (R)0;
#pragma unroll
    for (int t = 0; t < TV; ++t) {
      const int v = v0 + t;
      if (v >= nocc) continue;
      const long f = (long)bb * nocc + v;
      const long o = 2 * ((f >> 1) * nr + r) + (f & 1);
      R y = -acc[b][t];
      if (use_vloc) y = fma(V, Pa_d[o], y);
      if (use_k1e) y = fma(vh, phir[(long)v * nr + r], y);
      Py_d[o] = y;
      if ((f & 1) == 0 && f == (long)nb_total * nocc - 1) Py_d[o + 1] = 0;  // unused partner
    }
  }
}

// The K1d term restricted to kept pairs (Wannier pair pruning): Y_{b,i} = V a_{b,i} + 2 vH_b w_i
// - sum_{(j, p) in nbr[off[i] .. off[i+1])} tau_p a_{b,j}, tau_p = W * (w_j w_i) on the grid.
template <class R, int NB, int TV>
__global__ void __launch_bounds__(128) combine_pruned_kernel(
    long nr, int nocc, int nb_total, int b0, const R *__restrict__ phir, const R *__restrict__ vloc,
    const R *__restrict__ tau, const int *__restrict__ off, const int2 *__restrict__ nbr,
    const typename Cx<R>::T *__restrict__ Pa, const typename Cx<R>::T *__restrict__ Pvh,
    typename Cx<R>::T *__restrict__ Py, int use_k1e, int use_k1d) {
  const long r = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (r >= nr) return;
  const int v0 = blockIdx.y * TV;
  const R *Pa_d = reinterpret_cast<const R *>(Pa);
  const R *Pv_d = reinterpret_cast<const R *>(Pvh);
  R *Py_d = reinterpret_cast<R *>(Py);
  const R V = vloc[r];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int bb = b0 + b;
    if (bb >= nb_total) continue;
    const R vh = use_k1e ? (R)2 * Pv_d[2 * ((long)(bb >> 1) * nr + r) + (bb & 1)] : (R)0;
    for (int t = 0; t < TV; ++t) {
      const int i = v0 + t;
      if (i >= nocc) break;
      R acc = 0;
      if (use_k1d) {
        for (int e = off[i]; e < off[i + 1]; ++e) {
          const int2 jp = nbr[e];
          const long fj = (long)bb * nocc + jp.x;
          acc = fma(__ldg(&tau[(long)jp.y * nr + r]), Pa_d[2 * ((fj >> 1) * nr + r) + (fj & 1)], acc);
        }
      }
      const long f = (long)bb * nocc + i;
      const long o = 2 * ((f >> 1) * nr + r) + (f & 1);
      R y = fma(V, Pa_d[o], -acc);
      if (use_k1e) y = fma(vh, phir[(long)i * nr + r], y);
      Py_d[o] = y;
      if ((f & 1) == 0 && f == (long)nb_total * nocc - 1) Py_d[o + 1] = 0;  // unused partner
    }
  }
}

// out_c[v][r] = phi_v(r) cos(2 pi j_k / N_k), out_s[v][r] = phi_v(r) sin(2 pi j_k / N_k) for the
// grid index j_k of point r along lattice vector k (r = j1 + N1 (j2 + N2 j3))
__global__ void phase_rows_kernel(long nr, int nocc, int n1, int n2, int n3, int k, const double *__restrict__ phir,
                                  double *__restrict__ oc, double *__restrict__ os) {
  const long total = (long)nocc * nr;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const long r = i % nr;
    const int j1 = (int)(r % n1), j2 = (int)((r / n1) % n2), j3 = (int)(r / ((long)n1 * n2));
    const int jk = k == 0 ? j1 : (k == 1 ? j2 : j3);
    const int nk = k == 0 ? n1 : (k == 1 ? n2 : n3);
    double sn, cs;
    sincospi(2.0 * jk / nk, &sn, &cs);
    oc[i] = phir[i] * cs;
    os[i] = phir[i] * sn;
  }
}

// P[q][r] += (T[2q][r], T[2q+1][r]) for nf real grids T packed in pairs
template <class R>
__global__ void add_packed_kernel(long nr, int nf, const R *__restrict__ T, typename Cx<R>::T *__restrict__ P) {
  const int nq = (nf + 1) / 2;
  const long total = nr * nq;
  R *Pd = reinterpret_cast<R *>(P);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int q = (int)(i / nr);
    const long r = i - (long)q * nr;
    Pd[2 * i] += T[(long)(2 * q) * nr + r];
    if (2 * q + 1 < nf) Pd[2 * i + 1] += T[(long)(2 * q + 1) * nr + r];
  }
}

// T_w(r) += coef sigma_{vw}(r) phi_v(r) and, when sym and v != w, T_v(r) += coef sigma_{vw}(r) phi_w(r)
template <class R>
__global__ void sigma_contract_kernel(long nr, int np, const int2 *__restrict__ list,
                                      const typename Cx<R>::T *__restrict__ Ps, const R *__restrict__ phir,
                                      R *__restrict__ T, R coef, int sym) {
  const R *Ps_d = reinterpret_cast<const R *>(Ps);
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < nr; r += (long)gridDim.x * blockDim.x) {
    for (int p = 0; p < np; ++p) {
      const int2 vw = list[p];
      const R s = coef * Ps_d[2 * ((long)(p >> 1) * nr + r) + (p & 1)];
      T[(long)vw.y * nr + r] = fma(s, phir[(long)vw.x * nr + r], T[(long)vw.y * nr + r]);
      if (sym && vw.x != vw.y)
        T[(long)vw.x * nr + r] = fma(s, phir[(long)vw.y * nr + r], T[(long)vw.x * nr + r]);
    }
  }
}

// Delta rho^(x) = sum_v a_v^2 - phi_v Psi_v  (Eq. 5 with Psi = O phi);  Delta rho^(z) = 2 sum_v Z_v phi_v  (Eq. 6)
template <class R>
__global__ void rel_density_kernel(long nr, int nocc, const R *__restrict__ phir,
                                   const double *__restrict__ ar, const double *__restrict__ psi,
                                   const double *__restrict__ zr, double *__restrict__ rx,
                                   double *__restrict__ rz) {
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < nr; r += (long)gridDim.x * blockDim.x) {
    double sx = 0.0, sz = 0.0;
    for (int v = 0; v < nocc; ++v) {
      const double p = (double)phir[(long)v * nr + r];
      const double a = ar[(long)v * nr + r];
      sx = fma(a, a, sx);
      sx = fma(-p, psi[(long)v * nr + r], sx);
      sz = fma(2.0 * zr[(long)v * nr + r], p, sz);
    }
    rx[r] = sx;
    rz[r] = sz;
  }
}

// out[r] = scale sum_v phi_v(r)^2 (the closed-shell ground-state density for scale 2)
__global__ void density_sum_kernel(long nr, int nocc, const double *__restrict__ phir, double scale,
                                   double *__restrict__ out) {
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < nr; r += (long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int v = 0; v < nocc; ++v) {
      const double p = phir[(long)v * nr + r];
      s = fma(p, p, s);
    }
    out[r] = scale * s;
  }
}

// Delta rho^(x)(r) = sum_v a_v(r)^2 - phi_v(r) Psi_v(r) in the grid precision (Eq. 5, Psi = O phi)
template <class R>
__global__ void xdensity_kernel(long nr, int nocc, const R *__restrict__ phir, const R *__restrict__ ar,
                                const R *__restrict__ psi, R *__restrict__ out) {
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < nr; r += (long)gridDim.x * blockDim.x) {
    R s = 0;
    for (int v = 0; v < nocc; ++v) {
      const R a = ar[(long)v * nr + r];
      s = fma(a, a, s);
      s = fma(-phir[(long)v * nr + r], psi[(long)v * nr + r], s);
    }
    out[r] = s;
  }
}

// out[r] = sum_v X_v(r) Y_v(r)
template <class R>
__global__ void pair_sum_kernel(long nr, int nocc, const R *__restrict__ X, const R *__restrict__ Y,
                                R *__restrict__ out) {
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < nr; r += (long)gridDim.x * blockDim.x) {
    R s = 0;
    for (int v = 0; v < nocc; ++v) s = fma(X[(long)v * nr + r], Y[(long)v * nr + r], s);
    out[r] = s;
  }
}

// T_w(r) += scale v(r) phi_w(r) for w < nocc
template <class R>
__global__ void add_product_kernel(long nr, int nocc, const R *__restrict__ v, const R *__restrict__ phir,
                                   R scale, R *__restrict__ T) {
  const long total = (long)nocc * nr;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x)
    T[i] = fma(scale * v[i % nr], phir[i], T[i]);
}

struct CellArgs {
  double B[9];       // rows b_i
  int n[3];
  double gmax2;      // density-sphere radius^2
  double omega;
  int natoms;
};

__device__ __forceinline__ bool grid_g(const CellArgs &c, long idx, double G[3], double &g2) {
  const int j1 = (int)(idx % c.n[0]);
  const int j2 = (int)((idx / c.n[0]) % c.n[1]);
  const int j3 = (int)(idx / ((long)c.n[0] * c.n[1]));
  const int m1 = j1 <= c.n[0] / 2 ? j1 : j1 - c.n[0];
  const int m2 = j2 <= c.n[1] / 2 ? j2 : j2 - c.n[1];
  const int m3 = j3 <= c.n[2] / 2 ? j3 : j3 - c.n[2];
#pragma unroll
  for (int a = 0; a < 3; ++a) G[a] = m1 * c.B[0 + a] + m2 * c.B[3 + a] + m3 * c.B[6 + a];
  g2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
  return g2 <= c.gmax2;
}

// Amplitude of atom a's external potential at |G|^2 = g2 (before the phase e^{-iG.R_a}): the
// Gaussian well -Z (2 pi s^2)^{3/2}/Omega e^{-s^2 G^2/2} plus, with ionic charges, the Coulomb
// potential of the Gaussian charge q: -4 pi q/(Omega G^2) e^{-s^2 G^2/2} (G = 0 dropped)
__device__ __forceinline__ double vext_amp(const CellArgs &c, const double *Z, const double *sig,
                                           const double *q, int a, double g2) {
  const double s2 = sig[a] * sig[a];
  double w = Z[a] * pow(2.0 * M_PI * s2, 1.5);
  if (q && g2 > 0.0) w += 4.0 * M_PI * q[a] / g2;
  return -w / c.omega * exp(-0.5 * s2 * g2);
}

// V(G) = sum_a vext_amp_a(G) exp(-i G.R_a) on the density sphere
__global__ void vloc_G_kernel(CellArgs c, long nr, const double *__restrict__ pos,
                              const double *__restrict__ Z, const double *__restrict__ sig,
                              const double *__restrict__ q, double2 *__restrict__ P) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nr; i += (long)gridDim.x * blockDim.x) {
    double G[3], g2;
    double2 v = make_double2(0.0, 0.0);
    if (grid_g(c, i, G, g2)) {
      for (int a = 0; a < c.natoms; ++a) {
        const double amp = vext_amp(c, Z, sig, q, a, g2);
        const double th = G[0] * pos[3 * a] + G[1] * pos[3 * a + 1] + G[2] * pos[3 * a + 2];
        double sn, cs;
        sincos(th, &sn, &cs);
        v.x += amp * cs;
        v.y -= amp * sn;
      }
    }
    P[i] = v;
  }
}

// partial[a][chunk][alpha] = sum_G -G_alpha v_a(G) (sin th rho_r + cos th rho_i), th = G.R_a,
// rho = P / nr (forward FFT of the real density).  d omega/dR = Omega * sum (Eq. 4).
__global__ void force_partial_kernel(CellArgs c, long nr, const double2 *__restrict__ P,
                                     const double *__restrict__ pos, const double *__restrict__ Z,
                                     const double *__restrict__ sig, const double *__restrict__ q, int nchunk,
                                     double *__restrict__ part) {
  const int a = blockIdx.y;
  const int ch = blockIdx.x;
  const long per = (nr + nchunk - 1) / nchunk;
  const long i0 = (long)ch * per, i1 = min(nr, i0 + per);
  const double R0 = pos[3 * a], R1 = pos[3 * a + 1], R2 = pos[3 * a + 2];
  double acc[3] = {0.0, 0.0, 0.0};
  for (long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    double G[3], g2;
    if (!grid_g(c, i, G, g2)) continue;
    const double2 rho = P[i];
    const double va = vext_amp(c, Z, sig, q, a, g2);
    double sn, cs;
    sincos(G[0] * R0 + G[1] * R1 + G[2] * R2, &sn, &cs);
    const double t = -va * (sn * rho.x + cs * rho.y) / (double)nr;
    acc[0] = fma(G[0], t, acc[0]);
    acc[1] = fma(G[1], t, acc[1]);
    acc[2] = fma(G[2], t, acc[2]);
  }
  __shared__ double red[3][256];
  for (int x = 0; x < 3; ++x) red[x][threadIdx.x] = acc[x];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int x = 0; x < 3; ++x) red[x][threadIdx.x] += red[x][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int x = 0; x < 3; ++x) part[((long)a * nchunk + ch) * 3 + x] = red[x][0];
}

__global__ void force_final_kernel(int natoms, int nchunk, const double *__restrict__ part, double omega,
                                   double *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= natoms * 3) return;
  const int a = i / 3, x = i % 3;
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += part[((long)a * nchunk + c) * 3 + x];
  out[i] = omega * s;
}

__global__ void residual_kernel(int k, long n, const double *__restrict__ AX, const double *__restrict__ X,
                                const double *__restrict__ th, double *__restrict__ R) {
  const long total = (long)k * n;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x)
    R[i] = AX[i] - th[i / n] * X[i];
}

__global__ void precond_kernel(int k, long n, const double *__restrict__ R, const double *__restrict__ kin,
                               int npw, const double *__restrict__ vshift, double tscale,
                               const double *__restrict__ th, double floor_, double *__restrict__ T) {
  const long total = (long)k * n;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const long row = i / n;
    const long j = i - row * n;
    const int v = (int)(j / npw);
    const int g = (int)(j - (long)v * npw);
    double d = kin[g] + (vshift ? vshift[v] : 0.0) - (th ? tscale * th[row] : 0.0);
    if (fabs(d) < floor_) d = d < 0 ? -floor_ : floor_;
    T[i] = R[i] / d;
  }
}

// C'[f][c] = C[f][c] / (eps_c - eps_v + shift - theta_i) - Ck[f][c],  f = i * nocc + v
__global__ void subspace_den_kernel(int rows, int ne, int nocc, const double *__restrict__ C,
                                    const double *__restrict__ Ck, const double *__restrict__ eps_e,
                                    const double *__restrict__ eps_o, double shift,
                                    const double *__restrict__ th, double floor_, double *__restrict__ out) {
  const long total = (long)rows * ne;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int f = (int)(i / ne), e = (int)(i % ne);
    double d = eps_e[e] - eps_o[f % nocc] + shift - th[f / nocc];
    if (fabs(d) < floor_) d = d < 0 ? -floor_ : floor_;
    out[i] = C[i] / d - Ck[i];
  }
}

__global__ void convert_kernel(long n, const double *__restrict__ src, float *__restrict__ dst) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

__global__ void axpby_f32_kernel(int M, int N, double alpha, const float *__restrict__ T, double beta,
                                 double *__restrict__ C, int ldc) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < (long)M * N; i += (long)gridDim.x * blockDim.x) {
    double *c = C + (i / N) * ldc + (i % N);
    const double t = alpha * (double)T[i];
    *c = beta == 0.0 ? t : t + beta * (*c);
  }
}

__global__ void sub_f32_kernel(long n, double *__restrict__ X, const float *__restrict__ T) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    X[i] -= (double)T[i];
}

CellArgs cell_args(const Ctx &c) {
  CellArgs a;
  for (int i = 0; i < 9; ++i) a.B[i] = c.B[i];
  for (int i = 0; i < 3; ++i) a.n[i] = c.N[i];
  a.gmax2 = 4.0 * c.desc.ecut;
  a.omega = c.omega;
  a.natoms = c.natoms;
  return a;
}

}  // namespace

template <class R, class I>
void scatter_pairs(const Ctx &c, int nf, const I *X, CT<R> *P, double scale, bool accumulate) {
  const long total = (long)((nf + 1) / 2) * (c.nhalf + 1);
  scatter_pairs_kernel<R, I><<<nblocks(total, 256), 256, 0, c.stream>>>(nf, c.npw, c.nhalf, c.nr, c.gp.get(),
                                                                         c.gm.get(), X, P, scale, accumulate);
  BSE_CHECK_LAUNCH();
}

template <class R, class O>
void gather_pairs(const Ctx &c, int nf, const CT<R> *P, O *Y, double scale, const double *Xd,
                  const double *shift, int period, double shift_const) {
  const long total = (long)((nf + 1) / 2) * (c.nhalf + 1);
  gather_pairs_kernel<R, O><<<nblocks(total, 256), 256, 0, c.stream>>>(
      nf, c.npw, c.nhalf, c.nr, c.gp.get(), c.gm.get(), P, Y, scale, Xd, c.kin.get(), shift,
      period > 0 ? period : 1, shift_const);
  BSE_CHECK_LAUNCH();
}

template <class R>
void mul_grid(long nr, int nq, CT<R> *P, const R *w, R scale, cudaStream_t s) {
  mul_grid_kernel<R><<<nblocks(nr * nq, 256), 256, 0, s>>>(nr, nq, P, w, scale);
  BSE_CHECK_LAUNCH();
}

template <class R, class O>
void unpack_real(long nr, int nf, const CT<R> *P, O *Rr, cudaStream_t s) {
  unpack_kernel<R, O><<<nblocks(nr * nf, 256), 256, 0, s>>>(nr, nf, P, Rr);
  BSE_CHECK_LAUNCH();
}

template <class R>
void pack_real(long nr, int nf, const R *Rr, CT<R> *P, cudaStream_t s) {
  pack_kernel<R><<<nblocks(nr * ((nf + 1) / 2), 256), 256, 0, s>>>(nr, nf, Rr, P);
  BSE_CHECK_LAUNCH();
}

template <class R>
void pair_products(long nr, int np, const int2 *list, const R *A, const R *Bm, CT<R> *P, cudaStream_t s) {
  pair_products_kernel<R><<<nblocks(nr * ((np + 1) / 2), 256), 256, 0, s>>>(nr, np, list, A, Bm, P);
  BSE_CHECK_LAUNCH();
}

template <class T>
void scale_cols(int rows, int cols, T *Q, const T *s, cudaStream_t st) {
  scale_cols_kernel<T><<<nblocks((long)rows * cols, 256), 256, 0, st>>>(rows, cols, Q, s);
  BSE_CHECK_LAUNCH();
}

template <class R>
void drho(const Ctx &c, int nb, const R *phir, const CT<R> *Pa, CT<R> *Pd) {
  drho_kernel<R><<<nblocks(c.nr, 256), 256, 0, c.stream>>>(c.nr, c.nocc, nb, phir, Pa, Pd);
  BSE_CHECK_LAUNCH();
}

template <class R>
void combine_tau(const Ctx &c, int nb, const R *phir, const R *vloc, const R *tau, const CT<R> *Pa,
                 const CT<R> *Pvh, CT<R> *Py, bool use_vloc, bool use_k1e, bool use_k1d) {
  constexpr int TV = 16;
  dim3 grid((unsigned)((c.nr + 127) / 128), (unsigned)((c.nocc + TV - 1) / TV));
  int b0 = 0;
  while (b0 < nb) {
    const int left = nb - b0;
    int step;
    // FP64: 4-vector passes run out of registers (lower occupancy, a third less FP64 rate), so
    // FP64 blocks go two vectors at a time
    if (left >= 4 && sizeof(R) == sizeof(float)) {
      step = 4;
      combine_tau_kernel<R, 4, TV><<<grid, 128, 0, c.stream>>>(c.nr, c.nocc, nb, b0, phir, vloc, tau, Pa, Pvh, Py,
                                                               use_vloc, use_k1e, use_k1d);
    } else if (left >= 2) {
      step = 2;
      combine_tau_kernel<R, 2, TV><<<grid, 128, 0, c.stream>>>(c.nr, c.nocc, nb, b0, phir, vloc, tau, Pa, Pvh, Py,
                                                               use_vloc, use_k1e, use_k1d);
    } else {
      step = 1;
      combine_tau_kernel<R, 1, TV><<<grid, 128, 0, c.stream>>>(c.nr, c.nocc, nb, b0, phir, vloc, tau, Pa, Pvh, Py,
                                                               use_vloc, use_k1e, use_k1d);
    }
    BSE_CHECK_LAUNCH();
    b0 += step;
  }
}

template <class R>
void sigma_contract(const Ctx &c, int np, const int2 *list, const CT<R> *Psig, const R *phir, R *T, bool sym) {
  sigma_contract_kernel<R><<<nblocks(c.nr, 256), 256, 0, c.stream>>>(c.nr, np, list, Psig, phir, T, (R)-1,
                                                                     sym ? 1 : 0);
  BSE_CHECK_LAUNCH();
}

void rel_density(const Ctx &c, const double *phir, const double *ar, const double *psi, const double *zr,
                 double *rx, double *rz) {
  rel_density_kernel<double><<<nblocks(c.nr, 256), 256, 0, c.stream>>>(c.nr, c.nocc, phir, ar, psi, zr, rx, rz);
  BSE_CHECK_LAUNCH();
}

void density_sum(long nr, int nocc, const double *phir, double scale, double *out, cudaStream_t s) {
  density_sum_kernel<<<nblocks(nr, 256), 256, 0, s>>>(nr, nocc, phir, scale, out);
  BSE_CHECK_LAUNCH();
}

template <class R>
void xdensity(long nr, int nocc, const R *phir, const R *ar, const R *psi, R *out, cudaStream_t s) {
  xdensity_kernel<R><<<nblocks(nr, 256), 256, 0, s>>>(nr, nocc, phir, ar, psi, out);
  BSE_CHECK_LAUNCH();
}

template <class R>
void combine_pruned(const Ctx &c, int nb, const R *phir, const R *vloc, const R *tau, const int *off, const int2 *nbr,
                    const CT<R> *Pa, const CT<R> *Pvh, CT<R> *Py, bool use_k1e, bool use_k1d) {
  constexpr int TV = 8;
  dim3 grid((unsigned)((c.nr + 127) / 128), (unsigned)((c.nocc + TV - 1) / TV));
  for (int b0 = 0; b0 < nb; b0 += 2) {
    if (nb - b0 >= 2)
      combine_pruned_kernel<R, 2, TV><<<grid, 128, 0, c.stream>>>(c.nr, c.nocc, nb, b0, phir, vloc, tau, off, nbr, Pa,
                                                                  Pvh, Py, use_k1e, use_k1d);
    else
      combine_pruned_kernel<R, 1, TV><<<grid, 128, 0, c.stream>>>(c.nr, c.nocc, nb, b0, phir, vloc, tau, off, nbr, Pa,
                                                                  Pvh, Py, use_k1e, use_k1d);
    BSE_CHECK_LAUNCH();
  }
}

void phase_rows(const Ctx &c, int k, const double *phir, double *oc, double *os) {
  phase_rows_kernel<<<nblocks((long)c.nocc * c.nr, 256), 256, 0, c.stream>>>(c.nr, c.nocc, c.N[0], c.N[1], c.N[2], k,
                                                                             phir, oc, os);
  BSE_CHECK_LAUNCH();
}

template <class R>
void add_packed(long nr, int nf, const R *T, CT<R> *P, cudaStream_t s) {
  add_packed_kernel<R><<<nblocks(nr * ((nf + 1) / 2), 256), 256, 0, s>>>(nr, nf, T, P);
  BSE_CHECK_LAUNCH();
}

template <class R>
void pair_sum(long nr, int nocc, const R *X, const R *Y, R *out, cudaStream_t s) {
  pair_sum_kernel<R><<<nblocks(nr, 256), 256, 0, s>>>(nr, nocc, X, Y, out);
  BSE_CHECK_LAUNCH();
}

template <class R>
void add_product(long nr, int nocc, const R *v, const R *phir, R scale, R *T, cudaStream_t s) {
  add_product_kernel<R><<<nblocks((long)nocc * nr, 256), 256, 0, s>>>(nr, nocc, v, phir, scale, T);
  BSE_CHECK_LAUNCH();
}

void vloc_G(const Ctx &c, const double *pos_d, const double *Z_d, const double *sig_d, const double *q_d,
            double2 *P) {
  vloc_G_kernel<<<nblocks(c.nr, 256), 256, 0, c.stream>>>(cell_args(c), c.nr, pos_d, Z_d, sig_d, q_d, P);
  BSE_CHECK_LAUNCH();
}

void force_reduce(const Ctx &c, const double2 *rhoG, const double *pos_d, const double *Z_d,
                  const double *sig_d, const double *q_d, double *partial, int nchunk, double *out) {
  force_partial_kernel<<<dim3(nchunk, c.natoms), 256, 0, c.stream>>>(cell_args(c), c.nr, rhoG, pos_d, Z_d,
                                                                      sig_d, q_d, nchunk, partial);
  BSE_CHECK_LAUNCH();
  force_final_kernel<<<(c.natoms * 3 + 127) / 128, 128, 0, c.stream>>>(c.natoms, nchunk, partial, c.omega, out);
  BSE_CHECK_LAUNCH();
}

void residual(int kk, long n, const double *AX, const double *X, const double *theta, double *R,
              cudaStream_t s) {
  residual_kernel<<<nblocks((long)kk * n, 256), 256, 0, s>>>(kk, n, AX, X, theta, R);
  BSE_CHECK_LAUNCH();
}

void precond_diag(int kk, long n, const double *R, const double *kin, int npw, const double *vshift,
                  double theta_scale, const double *theta, double floor, double *T, cudaStream_t s) {
  precond_kernel<<<nblocks((long)kk * n, 256), 256, 0, s>>>(kk, n, R, kin, npw, vshift, theta_scale, theta,
                                                            floor, T);
  BSE_CHECK_LAUNCH();
}

void subspace_den(int rows, int ne, int nocc, const double *C, const double *Ck, const double *eps_e,
                  const double *eps_o, double shift, const double *th, double floor, double *out, cudaStream_t s) {
  subspace_den_kernel<<<nblocks((long)rows * ne, 256), 256, 0, s>>>(rows, ne, nocc, C, Ck, eps_e, eps_o, shift, th,
                                                                     floor, out);
  BSE_CHECK_LAUNCH();
}

void fill_real_grid(long nr, double2 *P, const double *R, cudaStream_t s) {
  fill_real_kernel<<<nblocks(nr, 256), 256, 0, s>>>(nr, P, R);
  BSE_CHECK_LAUNCH();
}


void convert(long n, const double *src, float *dst, cudaStream_t s) {
  convert_kernel<<<nblocks(n, 256), 256, 0, s>>>(n, src, dst);
  BSE_CHECK_LAUNCH();
}

void axpby_f32(int M, int N, double alpha, const float *T, double beta, double *C, int ldc, cudaStream_t s) {
  axpby_f32_kernel<<<nblocks((long)M * N, 256), 256, 0, s>>>(M, N, alpha, T, beta, C, ldc);
  BSE_CHECK_LAUNCH();
}

void sub_f32(long n, double *X, const float *T, cudaStream_t s) {
  sub_f32_kernel<<<nblocks(n, 256), 256, 0, s>>>(n, X, T);
  BSE_CHECK_LAUNCH();
}

// explicit instantiations
template void scatter_pairs<double, double>(const Ctx &, int, const double *, double2 *, double, bool);
template void scatter_pairs<float, double>(const Ctx &, int, const double *, float2 *, double, bool);
template void scatter_pairs<float, float>(const Ctx &, int, const float *, float2 *, double, bool);
template void gather_pairs<double, double>(const Ctx &, int, const double2 *, double *, double, const double *,
                                           const double *, int, double);
template void gather_pairs<float, double>(const Ctx &, int, const float2 *, double *, double, const double *,
                                          const double *, int, double);
template void gather_pairs<float, float>(const Ctx &, int, const float2 *, float *, double, const double *,
                                         const double *, int, double);
template void mul_grid<double>(long, int, double2 *, const double *, double, cudaStream_t);
template void mul_grid<float>(long, int, float2 *, const float *, float, cudaStream_t);
template void unpack_real<double, double>(long, int, const double2 *, double *, cudaStream_t);
template void unpack_real<float, float>(long, int, const float2 *, float *, cudaStream_t);
template void unpack_real<double, float>(long, int, const double2 *, float *, cudaStream_t);
template void pack_real<double>(long, int, const double *, double2 *, cudaStream_t);
template void pack_real<float>(long, int, const float *, float2 *, cudaStream_t);
template void pair_products<double>(long, int, const int2 *, const double *, const double *, double2 *,
                                    cudaStream_t);
template void pair_products<float>(long, int, const int2 *, const float *, const float *, float2 *, cudaStream_t);
template void scale_cols<double>(int, int, double *, const double *, cudaStream_t);
template void scale_cols<float>(int, int, float *, const float *, cudaStream_t);
template void drho<double>(const Ctx &, int, const double *, const double2 *, double2 *);
template void drho<float>(const Ctx &, int, const float *, const float2 *, float2 *);
template void combine_tau<double>(const Ctx &, int, const double *, const double *, const double *,
                                  const double2 *, const double2 *, double2 *, bool, bool, bool);
template void combine_tau<float>(const Ctx &, int, const float *, const float *, const float *, const float2 *,
                                 const float2 *, float2 *, bool, bool, bool);
template void xdensity<double>(long, int, const double *, const double *, const double *, double *, cudaStream_t);
template void xdensity<float>(long, int, const float *, const float *, const float *, float *, cudaStream_t);
template void combine_pruned<double>(const Ctx &, int, const double *, const double *, const double *, const int *,
                                     const int2 *, const double2 *, const double2 *, double2 *, bool, bool);
template void combine_pruned<float>(const Ctx &, int, const float *, const float *, const float *, const int *,
                                    const int2 *, const float2 *, const float2 *, float2 *, bool, bool);
template void add_packed<double>(long, int, const double *, double2 *, cudaStream_t);
template void add_packed<float>(long, int, const float *, float2 *, cudaStream_t);
template void pair_sum<double>(long, int, const double *, const double *, double *, cudaStream_t);
template void pair_sum<float>(long, int, const float *, const float *, float *, cudaStream_t);
template void add_product<double>(long, int, const double *, const double *, double, double *, cudaStream_t);
template void add_product<float>(long, int, const float *, const float *, float, float *, cudaStream_t);
template void sigma_contract<double>(const Ctx &, int, const int2 *, const double2 *, const double *, double *,
                                     bool);
template void sigma_contract<float>(const Ctx &, int, const int2 *, const float2 *, const float *, float *, bool);

}  // namespace k
}  // namespace bse
