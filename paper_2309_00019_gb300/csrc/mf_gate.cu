// Gating of loud short transients before the filter (Sec. VI: short-duration
// artifacts are removed from the data by gating before matched filtering; the
// paper cites the method without its statistic or parameters, so the ones here
// are readings).
//   k_gate_row    h[k] = sqrt(4 df / w[k]) = sqrt(S_n[k]) on the band of Eq. (2)
//                 (w > 0), 0 elsewhere: with this one-row bank mf_filter computes
//                 the gate statistic, the envelope of the band-limited whitened
//                 strain in matched-filter SNR units, and its per-window peaks
//                 over the plan's threshold are the gates.
//   k_gate_apply  out[d][j] = x[d][j] prod over row d's gates c of W(|j - c| / fs),
//                 W the inverse Tukey window (0 within t_zero, cosine taper over
//                 t_taper, 1 beyond), in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "../../include/mf.h"
#include "mf_common.cuh"

namespace mf {
namespace {

__global__ void k_gate_row(const double* __restrict__ w, int64_t nb, double df, float2* __restrict__ row) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nb; k += (int64_t)gridDim.x * blockDim.x)
    row[k] = w[k] > 0.0 ? make_float2((float)sqrt(4.0 * df / w[k]), 0.f) : make_float2(0.f, 0.f);
}

// gates: sorted by (det, sample) (one-template trigger list); the first min(*count, max_g) are used
__global__ void k_gate_apply(const float* __restrict__ x, int64_t ld, int n_det, int64_t n, double inv_fs,
                             const mf_trigger* __restrict__ g, const int64_t* __restrict__ count, int64_t max_g,
                             double t_zero, double t_taper, int64_t reach, float* out, int64_t ld_out) {
  const int64_t cnt = min(*count, max_g);
  const int64_t total = (int64_t)n_det * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int d = (int)(i / n);
    const int64_t j = i - (int64_t)d * n;
    // first gate with (det, sample) >= (d, j - reach)
    int64_t lo = 0, hi = cnt;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      const bool before = g[mid].det < d || (g[mid].det == d && g[mid].sample < j - reach);
      if (before) lo = mid + 1; else hi = mid;
    }
    double gw = 1.0;
    for (int64_t m = lo; m < cnt && g[m].det == d && g[m].sample <= j + reach; ++m) {
      const double t = fabs((double)(j - g[m].sample)) * inv_fs;
      if (t <= t_zero) {
        gw = 0.0;
        break;
      }
      if (t < t_zero + t_taper) gw *= 0.5 * (1.0 - cospi((t - t_zero) / t_taper));
    }
    out[(int64_t)d * ld_out + j] = (float)((double)x[(int64_t)d * ld + j] * gw);
  }
}

int gate_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

}  // namespace

cudaError_t launch_gate_row(const double* w, int64_t nb, double df, float2* row, cudaStream_t st) {
  k_gate_row<<<(int)std::min<int64_t>((nb + 255) / 256, 1024), 256, 0, st>>>(w, nb, df, row);
  add_launches(1);
  return cudaGetLastError();
}

}  // namespace mf

extern "C" mf_status mf_gate_apply(const float* strain, int64_t ld, int32_t n_det, int64_t n, double fs,
                                   const mf_trigger* gates, const int64_t* count, int64_t max_gates, double t_zero,
                                   double t_taper, float* out, int64_t ld_out, void* cuda_stream) {
  auto bad = [](const char* m) {
    mf::set_global_error(std::string("mf_gate_apply: ") + m);
    return MF_EINVAL;
  };
  if (!strain || !out || !count || (max_gates > 0 && !gates)) return bad("null argument");
  if (!(fs > 0) || n_det < 1 || n < 1 || ld < n || ld_out < n || max_gates < 0) return bad("fs, n_det, n, ld or max_gates");
  if (!(t_zero >= 0) || !(t_taper >= 0)) return bad("t_zero and t_taper must be >= 0");
  const int64_t reach = (int64_t)std::ceil((t_zero + t_taper) * fs) + 1;
  const int64_t total = (int64_t)n_det * n;
  const int grid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)mf::gate_sms() * 8);
  mf::k_gate_apply<<<grid, 256, 0, (cudaStream_t)cuda_stream>>>(strain, ld, n_det, n, 1.0 / fs, gates, count,
                                                                   max_gates, t_zero, t_taper, reach, out, ld_out);
  mf::add_launches(1);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    mf::set_global_error(std::string("mf_gate_apply: ") + cudaGetErrorString(e));
    return MF_ECUDA;
  }
  return MF_OK;
}
