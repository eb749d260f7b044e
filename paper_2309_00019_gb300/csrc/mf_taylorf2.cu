// On-GPU TaylorF2 templates (the bank waveforms the search filters, Sec. II;
// non-spinning stationary-phase approximant with the 3.5PN phase of Buonanno,
// Iyer, Ochsner, Pan & Sathyaprakash 2009, Eq. 3.18, and Newtonian amplitude):
//   h~(f) = f^{-7/6} exp(-i Psi(f)),  f_low <= f <= min(f_ISCO, Nyquist), k < N/2,
//   Psi(f) = -pi/4 + 3 / (128 eta v^5) [1 + sum_k psi_k v^k (+ log terms)],  v = (pi M f)^{1/3},
// zero elsewhere.  Psi reaches ~1e5 rad at the lower frequencies, so it is
// evaluated in FP64 only at anchors K bins apart (K = 2^j with K df <= 0.25 Hz
// and K <= k_low / 4); each anchor keeps Psi mod 2 pi and the FP64 difference
// to the next anchor, both as FP32.  Between anchors the phase is the cubic
// Lagrange interpolant through the four nearest anchors, evaluated in FP32
// (differences of at most 3 K bins' worth of phase, so FP32 rounding stays
// near 1e-5 rad; the interpolation error is below 2e-4 rad, at the
// lightest templates' lowest frequencies), reduced to [-pi, pi] and turned into
// cos / sin.  The amplitude is exp2(-7/6 log2 f) (fast base-2 logarithm, ~1e-6 relative).
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "../../include/mf.h"
#include "mf_internal.h"

namespace mf {

namespace {

constexpr int kGenThreads = 256;
constexpr int kGenChunk = 2048;  // bins per CTA
constexpr double kMtsun = 4.925491025543576e-06;  // G M_sun / c^3, seconds
constexpr double kEulerGamma = 0.5772156649015329;
constexpr double kPi = 3.141592653589793;

struct TF2 {
  double p[8];        // psi_0 .. psi_7
  double log5, log6;  // coefficients of ln(v / v_lso) at v^5 and of ln v at v^6
  double piM;         // pi M (seconds)
  double pre;         // 3 / (128 eta)
  int64_t k_lo, k_hi; // band, inclusive
  int K_log2;         // anchors every 2^K_log2 bins
};

__device__ __forceinline__ double tf2_phase(const TF2& t, double f) {
  const double v = cbrt(t.piM * f);
  const double lv = log(v);
  const double v2 = v * v;
  const double s = t.p[0] + v2 * (t.p[2] + v * (t.p[3] + v * (t.p[4] + v * (t.p[5] + t.log5 * (lv + 0.8958797346140275) +
                                                                               v * (t.p[6] + t.log6 * lv + v * t.p[7])))));
  // 0.8958797346140275 = -ln(v_lso), v_lso = 6^{-1/2}
  const double v5 = v2 * v2 * v;
  return -0.25 * kPi + t.pre / v5 * s;
}

__global__ void __launch_bounds__(kGenThreads) k_taylorf2(const TF2* __restrict__ tmpl, double df, float2* __restrict__ out,
                                                          int64_t ld, int64_t nb) {
  __shared__ double psi[kGenChunk + 4];    // anchor phases (FP64), then
  __shared__ float mod2pi[kGenChunk + 4];  // anchor phase mod 2 pi
  __shared__ float dnext[kGenChunk + 4];   // Psi(anchor + 1) - Psi(anchor)
  const TF2 t = tmpl[blockIdx.y];
  float2* row = out + (int64_t)blockIdx.y * ld;
  const int64_t k0 = (int64_t)blockIdx.x * kGenChunk;
  const int64_t k1 = k0 + kGenChunk < nb ? k0 + kGenChunk : nb;
  if (k1 <= t.k_lo || k0 > t.k_hi) {  // chunk outside the band
    for (int64_t k = k0 + threadIdx.x; k < k1; k += kGenThreads) row[k] = make_float2(0.f, 0.f);
    return;
  }
  const int K = 1 << t.K_log2;
  // anchors a = -1 .. n_in + 1 at bins k0 + a K (bins of the chunk lie in intervals 0 .. n_in - 1)
  const int n_in = (int)((k1 - k0 + K - 1) >> t.K_log2);
  for (int a = threadIdx.x; a < n_in + 4; a += kGenThreads) {  // one FP64 phase per anchor
    const int64_t ka = k0 + (int64_t)(a - 1) * K;
    // anchors below half the lower band edge only serve bins that are zeroed; keep them finite
    psi[a] = tf2_phase(t, (double)(ka > t.k_lo / 2 ? ka : t.k_lo / 2) * df);
  }
  __syncthreads();
  for (int a = threadIdx.x; a < n_in + 3; a += kGenThreads) {
    const double pa = psi[a];
    const double two_pi = 2.0 * kPi;
    mod2pi[a] = (float)(pa - two_pi * floor(pa / two_pi));
    dnext[a] = (float)(psi[a + 1] - pa);
  }
  __syncthreads();
  const float two_pi_f = 6.283185307179586f, inv_two_pi = 0.15915494309189535f;
  for (int64_t k = k0 + threadIdx.x; k < k1; k += kGenThreads) {
    if (k < t.k_lo || k > t.k_hi) {
      row[k] = make_float2(0.f, 0.f);
      continue;
    }
    const int64_t off = k - k0;
    const int i = (int)(off >> t.K_log2) + 1;  // anchor index of the interval's left end
    const float x = (float)(off & (K - 1)) * (1.0f / (float)K);
    // cubic Lagrange weights at nodes -1, 0, 1, 2 (node 0 contributes its own value, i.e. 0 here)
    const float wm = -x * (x - 1.f) * (x - 2.f) * (1.f / 6.f);
    const float w1 = -(x + 1.f) * x * (x - 2.f) * 0.5f;
    const float w2 = (x + 1.f) * x * (x - 1.f) * (1.f / 6.f);
    const float d0 = dnext[i], d1 = dnext[i + 1];
    float ph = mod2pi[i] - wm * dnext[i - 1] + w1 * d0 + w2 * (d0 + d1);
    ph -= two_pi_f * rintf(ph * inv_two_pi);
    float s, c;
    __sincosf(ph, &s, &c);
    const float f = (float)((double)k * df);
    const float amp = exp2f(-1.1666666666666667f * __log2f(f));
    row[k] = make_float2(amp * c, -amp * s);
  }
}

}  // namespace

// host: per-template coefficients; the band uses the same float64 arithmetic as the host-side generators
static TF2 make_tf2(double m1, double m2, double fs, int64_t n, double f_low) {
  TF2 t{};
  const double M = (m1 + m2) * kMtsun;
  const double eta = m1 * m2 / ((m1 + m2) * (m1 + m2));
  const double pi = kPi;
  t.p[0] = 1.0;
  t.p[1] = 0.0;
  t.p[2] = 20.0 / 9.0 * (743.0 / 336.0 + 11.0 / 4.0 * eta);
  t.p[3] = -16.0 * pi;
  t.p[4] = 10.0 * (3058673.0 / 1016064.0 + 5429.0 / 1008.0 * eta + 617.0 / 144.0 * eta * eta);
  t.p[5] = pi * (38645.0 / 756.0 - 65.0 / 9.0 * eta);
  t.p[6] = 11583231236531.0 / 4694215680.0 - 640.0 / 3.0 * pi * pi - 6848.0 / 21.0 * kEulerGamma +
           eta * (-15737765635.0 / 3048192.0 + 2255.0 / 12.0 * pi * pi) + 76055.0 / 1728.0 * eta * eta -
           127825.0 / 1296.0 * eta * eta * eta - 6848.0 / 21.0 * std::log(4.0);
  t.p[7] = pi * (77096675.0 / 254016.0 + 378515.0 / 1512.0 * eta - 74045.0 / 756.0 * eta * eta);
  t.log5 = 3.0 * t.p[5];
  t.log6 = -6848.0 / 21.0;
  t.piM = pi * M;
  t.pre = 3.0 / (128.0 * eta);
  const double df = fs / (double)n;
  const double f_isco = 1.0 / (std::pow(6.0, 1.5) * pi * M);
  const double fhi = std::min(f_isco, fs / 2.0);
  int64_t lo = (int64_t)std::ceil(f_low / df);
  while (lo > 0 && (double)(lo - 1) * df >= f_low) --lo;
  while ((double)lo * df < f_low) ++lo;
  int64_t hi = (int64_t)std::floor(fhi / df);
  while ((double)(hi + 1) * df <= fhi) ++hi;
  while (hi >= 0 && (double)hi * df > fhi) --hi;
  hi = std::min<int64_t>(hi, n / 2 - 1);
  t.k_lo = lo;
  t.k_hi = hi;
  int K = 1;
  while (2.0 * K * df <= 0.25 && 2 * K <= std::max<int64_t>(lo / 4, 1) && K < 1024) K *= 2;
  int lg = 0;
  while ((1 << lg) < K) ++lg;
  t.K_log2 = lg;
  return t;
}

cudaError_t launch_taylorf2(const double* m1, const double* m2, int64_t n_tmpl, double fs, int64_t n, double f_low,
                            float2* out, int64_t ld, cudaStream_t st) {
  if (n_tmpl < 1 || n < 16 || !(fs > 0) || !(f_low > 0) || ld < n / 2 + 1) return cudaErrorInvalidValue;
  std::vector<TF2> h((size_t)n_tmpl);
  for (int64_t i = 0; i < n_tmpl; ++i) {
    if (!(m1[i] > 0) || !(m2[i] > 0)) return cudaErrorInvalidValue;
    h[(size_t)i] = make_tf2(m1[i], m2[i], fs, n, f_low);
  }
  TF2* d = nullptr;
  cudaError_t e = cudaMallocAsync(&d, (size_t)n_tmpl * sizeof(TF2), st);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(d, h.data(), (size_t)n_tmpl * sizeof(TF2), cudaMemcpyHostToDevice, st);
  const int64_t nb = n / 2 + 1;
  for (int64_t t0 = 0; e == cudaSuccess && t0 < n_tmpl; t0 += 65535) {
    const dim3 grid((unsigned)((nb + kGenChunk - 1) / kGenChunk), (unsigned)std::min<int64_t>(65535, n_tmpl - t0));
    k_taylorf2<<<grid, kGenThreads, 0, st>>>(d + t0, fs / (double)n, out + t0 * ld, ld, nb);
    add_launches(1);
    e = cudaGetLastError();
  }
  // the host table must outlive the copy: wait for it before the vector goes away
  cudaError_t e2 = cudaStreamSynchronize(st);
  cudaFreeAsync(d, st);
  return e != cudaSuccess ? e : e2;
}

}  // namespace mf

extern "C" mf_status mf_taylorf2(const double* m1, const double* m2, int64_t n_tmpl, double fs, int64_t n,
                                 double f_low, void* out, int64_t ld, void* cuda_stream) {
  if (!m1 || !m2 || !out) {
    mf::set_global_error("mf_taylorf2: null argument");
    return MF_EINVAL;
  }
  cudaError_t e = mf::launch_taylorf2(m1, m2, n_tmpl, fs, n, f_low, static_cast<float2*>(out), ld,
                                      static_cast<cudaStream_t>(cuda_stream));
  if (e == cudaErrorInvalidValue) {
    mf::set_global_error("mf_taylorf2: bad sizes, masses or band");
    return MF_EINVAL;
  }
  if (e != cudaSuccess) {
    mf::set_global_error(std::string("mf_taylorf2: ") + cudaGetErrorString(e));
    return MF_ECUDA;
  }
  return MF_OK;
}
