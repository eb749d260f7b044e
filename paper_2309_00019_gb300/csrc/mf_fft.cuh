// Register-resident small DFTs and Stockham pass helpers for the matched-filter
// kernels (sm_103a).  Everything here computes inverse-sign transforms,
// X[q] = sum_r v[r] exp(+2 pi i r q / R), unnormalised, which is the sign of the
// correlation over coalescence time in Eq. (1)-(2) (Sec. V.C: one inverse FFT
// per template and segment).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace mf {

// ---------------------------------------------------------------------------
// compile-time loops and constants
// ---------------------------------------------------------------------------

template <int... Is, class F>
__device__ __forceinline__ void sfor_impl(std::integer_sequence<int, Is...>, F&& f) {
  (f(std::integral_constant<int, Is>{}), ...);
}
// Calls f(std::integral_constant<int, i>) for i = 0..N-1 with compile-time i.
template <int N, class F>
__device__ __forceinline__ void sfor(F&& f) {
  sfor_impl(std::make_integer_sequence<int, N>{}, f);
}

// cos / sin of 2 pi e / R evaluated at compile time: argument reduced to
// [-pi/4, pi/4] by octant symmetry, then Taylor series to 1e-19.
__host__ __device__ constexpr double kpow_term(double x, int n) {
  double t = 1.0;
  for (int i = 1; i <= n; ++i) t *= x / i;
  return t;
}
__host__ __device__ constexpr double ksin_small(double x) {
  double s = 0.0;
  for (int n = 1, sg = 1; n < 30; n += 2, sg = -sg) s += sg * kpow_term(x, n);
  return s;
}
__host__ __device__ constexpr double kcos_small(double x) {
  double s = 0.0;
  for (int n = 0, sg = 1; n < 30; n += 2, sg = -sg) s += sg * kpow_term(x, n);
  return s;
}
// returns cos(2 pi e / R) (which = 0) or sin (which = 1)
__host__ __device__ constexpr double kcossin(long e, long R, int which) {
  const double kPi = 3.14159265358979323846264338327950288;
  e %= R;
  if (e < 0) e += R;
  // angle = 2 pi e / R = (pi/4) * (8e/R); octant o = floor(8e/R), remainder in [0, pi/4)
  long num = 8 * e;
  long o = num / R;
  double rem = (double)(num - o * R) / (double)R * (kPi / 4.0);  // [0, pi/4)
  double c = 0, s = 0;
  switch (o & 7) {
    case 0: c = kcos_small(rem); s = ksin_small(rem); break;
    case 1: c = ksin_small(kPi / 4 - rem); s = kcos_small(kPi / 4 - rem); break;
    case 2: c = -ksin_small(rem); s = kcos_small(rem); break;
    case 3: c = -kcos_small(kPi / 4 - rem); s = ksin_small(kPi / 4 - rem); break;
    case 4: c = -kcos_small(rem); s = -ksin_small(rem); break;
    case 5: c = -ksin_small(kPi / 4 - rem); s = -kcos_small(kPi / 4 - rem); break;
    case 6: c = ksin_small(rem); s = -kcos_small(rem); break;
    default: c = kcos_small(kPi / 4 - rem); s = -ksin_small(kPi / 4 - rem); break;
  }
  return which == 0 ? c : s;
}

// ---------------------------------------------------------------------------
// complex helpers (float2 = re, im)
// ---------------------------------------------------------------------------

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 mul_i(float2 a) { return make_float2(-a.y, a.x); }
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }

// a * exp(+2 pi i E / R) with E, R compile-time; trivial factors cost nothing.
template <long E, long R>
__device__ __forceinline__ float2 twiddle(float2 a) {
  constexpr long e = ((E % R) + R) % R;
  if constexpr (e == 0) {
    return a;
  } else if constexpr (4 * e == R) {
    return mul_i(a);
  } else if constexpr (2 * e == R) {
    return make_float2(-a.x, -a.y);
  } else if constexpr (4 * e == 3 * R) {
    return mul_mi(a);
  } else if constexpr (8 * e == R) {
    constexpr float h = 0.707106781186547524f;
    return make_float2(h * (a.x - a.y), h * (a.x + a.y));
  } else if constexpr (8 * e == 3 * R) {
    constexpr float h = 0.707106781186547524f;
    return make_float2(-h * (a.x + a.y), h * (a.x - a.y));
  } else if constexpr (8 * e == 5 * R) {
    constexpr float h = 0.707106781186547524f;
    return make_float2(h * (a.y - a.x), -h * (a.x + a.y));
  } else if constexpr (8 * e == 7 * R) {
    constexpr float h = 0.707106781186547524f;
    return make_float2(h * (a.x + a.y), h * (a.y - a.x));
  } else {
    constexpr float c = (float)kcossin(e, R, 0);
    constexpr float s = (float)kcossin(e, R, 1);
    return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
  }
}

// ---------------------------------------------------------------------------
// in-register DFT of size R (inverse sign, natural order in and out).
// ZH: the upper half of the inputs (v[R/2..R-1]) is known to be zero.
// ---------------------------------------------------------------------------

template <int R, bool ZH = false>
struct Dft;

template <bool ZH>
struct Dft<1, ZH> {
  template <class V>
  __device__ __forceinline__ static void run(V& v, int o, int s) {}
};

template <bool ZH>
struct Dft<2, ZH> {
  // v[o], v[o+s]
  template <class V>
  __device__ __forceinline__ static void run(V& v, int o, int s) {
    if constexpr (ZH) {
      v[o + s] = v[o];
    } else {
      float2 a = v[o], b = v[o + s];
      v[o] = cadd(a, b);
      v[o + s] = csub(a, b);
    }
  }
};

template <bool ZH>
struct Dft<4, ZH> {
  template <class V>
  __device__ __forceinline__ static void run(V& v, int o, int s) {
    float2 x0 = v[o], x1 = v[o + s];
    if constexpr (ZH) {
      float2 ix1 = mul_i(x1);
      v[o] = cadd(x0, x1);
      v[o + s] = cadd(x0, ix1);
      v[o + 2 * s] = csub(x0, x1);
      v[o + 3 * s] = csub(x0, ix1);
    } else {
      float2 x2 = v[o + 2 * s], x3 = v[o + 3 * s];
      float2 t0 = cadd(x0, x2), t1 = csub(x0, x2);
      float2 t2 = cadd(x1, x3), t3 = mul_i(csub(x1, x3));
      v[o] = cadd(t0, t2);
      v[o + 2 * s] = csub(t0, t2);
      v[o + s] = cadd(t1, t3);
      v[o + 3 * s] = csub(t1, t3);
    }
  }
};

// Generic R = A * B in registers:
//   r = B r1 + r2, q = q1 + A q2:
//   X[q1 + A q2] = sum_r2 w_B^{r2 q2} w_R^{r2 q1} sum_r1 v[B r1 + r2] w_A^{r1 q1}
template <int R>
struct Split {
  static constexpr int A = (R >= 16) ? 4 : 2;
  static constexpr int B = R / A;
};

template <int R, bool ZH>
struct Dft {
  static constexpr int A = Split<R>::A;
  static constexpr int B = Split<R>::B;
  // operates on v[o + s*i], i = 0..R-1, with a local copy (registers)
  template <class V>
  __device__ __forceinline__ static void run(V& v, int o, int s) {
    float2 u[R];
#pragma unroll
    for (int i = 0; i < R; ++i) u[i] = v[o + s * i];
    // step 1: A-point DFTs over r1 for each r2 (stride B); upper half of r1 zero if ZH
    sfor<B>([&](auto r2c) {
      constexpr int r2 = decltype(r2c)::value;
      Dft<A, ZH>::run(u, r2, B);
    });
    // after step 1: u[r2 + B q1] holds U[r2][q1]; twiddle by w_R^{r2 q1}
    sfor<B>([&](auto r2c) {
      constexpr int r2 = decltype(r2c)::value;
      sfor<A>([&](auto q1c) {
        constexpr int q1 = decltype(q1c)::value;
        u[r2 + B * q1] = twiddle<(long)r2 * q1, R>(u[r2 + B * q1]);
      });
    });
    // step 2: B-point DFT over r2 for each q1: elements u[B q1 + r2], stride 1
    sfor<A>([&](auto q1c) {
      constexpr int q1 = decltype(q1c)::value;
      Dft<B, false>::run(u, B * q1, 1);
    });
    // u[B q1 + q2] = X[q1 + A q2]
#pragma unroll
    for (int q1 = 0; q1 < A; ++q1)
#pragma unroll
      for (int q2 = 0; q2 < B; ++q2) v[o + s * (q1 + A * q2)] = u[B * q1 + q2];
  }
};

template <int R, bool ZH = false>
__device__ __forceinline__ void dft(float2 (&v)[R]) {
  Dft<R, ZH>::run(v, 0, 1);
}

// exp(+2 pi i p / q) for integers 0 <= p < q <= 2^24, q a power of two.
__device__ __forceinline__ float2 unit_root(uint32_t p, uint32_t q) {
  float s, c;
  sincospif(2.0f * (float)p / (float)q, &s, &c);
  return make_float2(c, s);
}

// ---------------------------------------------------------------------------
// two-pass Stockham geometry of an M-point sub-FFT: radices (RA, RB), M = RA*RB,
// RA >= RB, T = RB threads.  Pass a: thread t reads x[t + r RB] (r < RA),
// writes shared[t RA + a].  Pass b: thread t does RA/RB butterflies
// j = t + T i; reads shared[j + r RA] (r < RB), twiddles by w_M^{r j}, and
// produces X[j + a RA] (a < RB).
// ---------------------------------------------------------------------------

template <int M>
struct Geo;
template <>
struct Geo<64> { static constexpr int RA = 8, RB = 8; };
template <>
struct Geo<128> { static constexpr int RA = 16, RB = 8; };
template <>
struct Geo<256> { static constexpr int RA = 16, RB = 16; };
template <>
struct Geo<512> { static constexpr int RA = 32, RB = 16; };
template <>
struct Geo<1024> { static constexpr int RA = 32, RB = 32; };

template <int M>
struct SubFft {
  static constexpr int RA = Geo<M>::RA;
  static constexpr int RB = Geo<M>::RB;
  static constexpr int T = RB;           // threads per sub-FFT
  static constexpr int NB = RA / RB;     // pass-b butterflies per thread
  static constexpr int PAD = M + M / RA; // padded shared length (one pad per RA entries)
  // padded shared index of logical index i
  __device__ __forceinline__ static int pidx(int i) { return i + i / RA; }
};

}  // namespace mf
