// Radix-2/3/4/5 codelets and the Stockham butterfly shared by the batched 3D FFT (fft.cu)
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
    case 4: stage_bfly<4, C>(src, dst, j, N, Ns, tw, sg, es); break;
    case 2: stage_bfly<2, C>(src, dst, j, N, Ns, tw, sg, es); break;
    case 3: stage_bfly<3, C>(src, dst, j, N, Ns, tw, sg, es); break;
    default: stage_bfly<5, C>(src, dst, j, N, Ns, tw, sg, es); break;
  }
}

}  // namespace fftc
}  // namespace bse
