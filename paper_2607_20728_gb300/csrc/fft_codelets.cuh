// Radix-2/3/4/5/8/9 codelets and the Stockham butterfly shared by the batched 3D FFT (fft.cu)
// and the sphere-pruned transforms (sphere_fft.cu).
#pragma once
#include <cuda_runtime.h>

namespace bse {
namespace fftc {

template <class C>
struct AxisArgs {
  int n;
  int nstage;
  int radix[12];
  const C *tw;
};

template <class C> struct RealOf;
template <> struct RealOf<double2> { using T = double; };
template <> struct RealOf<float2> { using T = float; };

template <class C>
__device__ __forceinline__ C mkc(typename RealOf<C>::T x, typename RealOf<C>::T y) {
  C v;
  v.x = x;
  v.y = y;
  return v;
}
template <class C>
__device__ __forceinline__ C cmul(C a, C b) {
  return mkc<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <class C> __device__ __forceinline__ C cadd(C a, C b) { return mkc<C>(a.x + b.x, a.y + b.y); }
template <class C> __device__ __forceinline__ C csub(C a, C b) { return mkc<C>(a.x - b.x, a.y - b.y); }
template <class C>
__device__ __forceinline__ C cscale(C a, typename RealOf<C>::T s) { return mkc<C>(a.x * s, a.y * s); }
// a + sg * i * b
template <class C>
__device__ __forceinline__ C c_add_i(C a, C b, typename RealOf<C>::T sg) {
  return mkc<C>(a.x - sg * b.y, a.y + sg * b.x);
}

// small DFTs; sg = -1 forward (exp(-2 pi i jk/R)), +1 inverse
template <int R, class C>
__device__ __forceinline__ void dft(C *v, typename RealOf<C>::T sg);

template <>
__device__ __forceinline__ void dft<2, double2>(double2 *v, double) {
  double2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}
template <>
__device__ __forceinline__ void dft<2, float2>(float2 *v, float) {
  float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <int R, class C>
__device__ __forceinline__ void dft3(C *v, typename RealOf<C>::T sg) {
  using T = typename RealOf<C>::T;
  const T h = (T)0.86602540378443864676;  // sqrt(3)/2
  C t1 = cadd(v[1], v[2]);
  C t2 = csub(v[0], cscale(t1, (T)0.5));
  C t3 = cscale(csub(v[1], v[2]), h);
  v[0] = cadd(v[0], t1);
  v[1] = c_add_i(t2, t3, sg);
  v[2] = c_add_i(t2, t3, -sg);
}
template <> __device__ __forceinline__ void dft<3, double2>(double2 *v, double sg) { dft3<3, double2>(v, sg); }
template <> __device__ __forceinline__ void dft<3, float2>(float2 *v, float sg) { dft3<3, float2>(v, sg); }

template <class C>
__device__ __forceinline__ void dft4(C *v, typename RealOf<C>::T sg) {
  C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
  C t2 = cadd(v[1], v[3]), t3 = csub(v[1], v[3]);
  v[0] = cadd(t0, t2);
  v[2] = csub(t0, t2);
  v[1] = c_add_i(t1, t3, sg);
  v[3] = c_add_i(t1, t3, -sg);
}
template <> __device__ __forceinline__ void dft<4, double2>(double2 *v, double sg) { dft4(v, sg); }
template <> __device__ __forceinline__ void dft<4, float2>(float2 *v, float sg) { dft4(v, sg); }

template <class C>
__device__ __forceinline__ void dft5(C *v, typename RealOf<C>::T sg) {
  using T = typename RealOf<C>::T;
  // cos and sin of 2 pi/5 and 4 pi/5: (sqrt5 - 1)/4, -(sqrt5 + 1)/4,
  // sqrt((5 + sqrt5)/8), sqrt((5 - sqrt5)/8)
  const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;
  const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;
  C t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
  C t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
  C a = v[0];
  C m1 = cadd(a, cadd(cscale(t1, c1), cscale(t2, c2)));
  C m2 = cadd(a, cadd(cscale(t1, c2), cscale(t2, c1)));
  C n1 = cadd(cscale(t3, s1), cscale(t4, s2));
  C n2 = csub(cscale(t3, s2), cscale(t4, s1));
  v[0] = cadd(a, cadd(t1, t2));
  v[1] = c_add_i(m1, n1, sg);
  v[4] = c_add_i(m1, n1, -sg);
  v[2] = c_add_i(m2, n2, sg);
  v[3] = c_add_i(m2, n2, -sg);
}
template <> __device__ __forceinline__ void dft<5, double2>(double2 *v, double sg) { dft5(v, sg); }
template <> __device__ __forceinline__ void dft<5, float2>(float2 *v, float sg) { dft5(v, sg); }

// 8 points as 2 x 4: with w = exp(sg 2 pi i/8), X[2p] is the 4-point transform of
// a_n = x_n + x_{n+4} and X[2p+1] that of b_n w^n, b_n = x_n - x_{n+4} (n = 0..3).
template <class C>
__device__ __forceinline__ void dft8(C *v, typename RealOf<C>::T sg) {
  using T = typename RealOf<C>::T;
  const T h = (T)0.70710678118654752440;  // 1/sqrt(2)
  C a[4], b[4];
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    a[n] = cadd(v[n], v[n + 4]);
    b[n] = csub(v[n], v[n + 4]);
  }
  // b_1 w, b_2 w^2, b_3 w^3 with w = (1 + sg i)/sqrt2, w^2 = sg i, w^3 = (-1 + sg i)/sqrt2
  b[1] = mkc<C>((b[1].x - sg * b[1].y) * h, (b[1].y + sg * b[1].x) * h);
  b[2] = mkc<C>(-sg * b[2].y, sg * b[2].x);
  b[3] = mkc<C>((-b[3].x - sg * b[3].y) * h, (-b[3].y + sg * b[3].x) * h);
  dft4(a, sg);
  dft4(b, sg);
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    v[2 * p] = a[p];
    v[2 * p + 1] = b[p];
  }
}
template <> __device__ __forceinline__ void dft<8, double2>(double2 *v, double sg) { dft8(v, sg); }
template <> __device__ __forceinline__ void dft<8, float2>(float2 *v, float sg) { dft8(v, sg); }

// 9 points as 3 x 3: n = 3a + b, m = c + 3d; 3-point transforms over a, twiddles w^(b c) with
// w = exp(sg 2 pi i/9), 3-point transforms over b.
template <class C>
__device__ __forceinline__ void dft9(C *v, typename RealOf<C>::T sg) {
  using T = typename RealOf<C>::T;
  // cos and sin of 2 pi k/9 for k = 1, 2, 4
  const T c1 = (T)0.76604444311897803520, s1 = (T)0.64278760968653932632;
  const T c2 = (T)0.17364817766693034885, s2 = (T)0.98480775301220805936;
  const T c4 = (T)-0.93969262078590838405, s4 = (T)0.34202014332566873304;
  C y[3][3];  // y[b][c]
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    C t[3] = {v[b], v[3 + b], v[6 + b]};
    dft3<3, C>(t, sg);
#pragma unroll
    for (int c = 0; c < 3; ++c) y[b][c] = t[c];
  }
  // twiddles w^(b c): (b, c) = (1, 1) w, (1, 2) w^2, (2, 1) w^2, (2, 2) w^4
  y[1][1] = cmul(y[1][1], mkc<C>(c1, sg * s1));
  y[1][2] = cmul(y[1][2], mkc<C>(c2, sg * s2));
  y[2][1] = cmul(y[2][1], mkc<C>(c2, sg * s2));
  y[2][2] = cmul(y[2][2], mkc<C>(c4, sg * s4));
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    C t[3] = {y[0][c], y[1][c], y[2][c]};
    dft3<3, C>(t, sg);
#pragma unroll
    for (int d = 0; d < 3; ++d) v[c + 3 * d] = t[d];
  }
}
template <> __device__ __forceinline__ void dft<9, double2>(double2 *v, double sg) { dft9(v, sg); }
template <> __device__ __forceinline__ void dft<9, float2>(float2 *v, float sg) { dft9(v, sg); }

// One radix-R Stockham butterfly on a line with element stride es: inputs j + r N/R, outputs
// (j/Ns) Ns R + j%Ns + r Ns.
template <int R, class C>
__device__ __forceinline__ void stage_bfly(const C *__restrict__ src, C *__restrict__ dst, int j, int N, int Ns,
                                           const C *__restrict__ tw, typename RealOf<C>::T sg, int es = 1) {
  const int nb = N / R;
  C v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = src[(j + r * nb) * es];
  const int kk = j % Ns;
  if (Ns > 1) {
    const int step = kk * (N / (Ns * R));  // r * step < N for r < R
#pragma unroll
    for (int r = 1; r < R; ++r) {
      C w = __ldg(&tw[r * step]);
      w.y *= -sg;  // table holds exp(-2 pi i k/N); inverse uses the conjugate
      v[r] = cmul(v[r], w);
    }
  }
  dft<R, C>(v, sg);
  const int d0 = (j / Ns) * Ns * R + kk;
#pragma unroll
  for (int r = 0; r < R; ++r) dst[(d0 + r * Ns) * es] = v[r];
}

// one butterfly of the stage with radix R (run-time value)
template <class C>
__device__ __forceinline__ void stage_bfly_any(int R, const C *__restrict__ src, C *__restrict__ dst, int j, int N,
                                               int Ns, const C *__restrict__ tw, typename RealOf<C>::T sg,
                                               int es = 1) {
  switch (R) {
    case 8: stage_bfly<8, C>(src, dst, j, N, Ns, tw, sg, es); break;
    case 9: stage_bfly<9, C>(src, dst, j, N, Ns, tw, sg, es); break;
    case 4: stage_bfly<4, C>(src, dst, j, N, Ns, tw, sg, es); break;
    case 2: stage_bfly<2, C>(src, dst, j, N, Ns, tw, sg, es); break;
    case 3: stage_bfly<3, C>(src, dst, j, N, Ns, tw, sg, es); break;
    default: stage_bfly<5, C>(src, dst, j, N, Ns, tw, sg, es); break;
  }
}

}  // namespace fftc
}  // namespace bse
