// Device helpers shared by the filter kernels (mf_kernels.cu, mf_filter.cu):
// shared-memory strides, bank element loads and the SNR / threshold /
// window-maximum epilogue of Eq. (1) with the Sec. II threshold.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "mf_fft.cuh"
#include "mf_internal.h"

namespace mf {

// Shared-memory stride of one column/row: >= pad and congruent to L (mod 16),
// where L = consecutive-thread lanes a group contributes to a half-warp, so
// 64-bit shared accesses of a half-warp hit 16 distinct bank pairs.
constexpr int stride_for(int pad, int lanes) {
  int L = lanes >= 16 ? 0 : lanes;
  int s = pad;
  if (L == 0) return s;
  while (s % 16 != L) ++s;
  return s;
}

template <int BT>
struct BankElem;
template <>
struct BankElem<kBankF32> {
  __device__ __forceinline__ static float2 get(const void* p, int64_t i) {
    return __ldg(reinterpret_cast<const float2*>(p) + i);
  }
};
template <>
struct BankElem<kBankF16> {
  __device__ __forceinline__ static float2 get(const void* p, int64_t i) {
    __half2 h = __ldg(reinterpret_cast<const __half2*>(p) + i);
    return __half22float2(h);
  }
};
template <>
struct BankElem<kBankBF16> {
  __device__ __forceinline__ static float2 get(const void* p, int64_t i) {
    __nv_bfloat162 h = __ldg(reinterpret_cast<const __nv_bfloat162*>(p) + i);
    return __bfloat1622float2(h);
  }
};

// Power-of-two scale of one series of the FP16 intermediate: 2^(e-1) with ratio = m 2^e, m in [0.5, 1),
// so that ratio / scale is in [1, 2).  ratio = sigma_ref / sigma of the template; the pre-scaled data give
// pass-1 outputs of RMS ~ sqrt(2 / N2) / ratio in Gaussian noise, so the scaled ones sit near sqrt(2 / N2)
// whatever the template (far inside FP16's normal range).  The row pass divides it out of rho exactly.
__device__ __forceinline__ float series_scale16(float ratio) {
  if (!(ratio > 0.f) || !isfinite(ratio)) return 1.f;
  int e = 0;
  frexpf(ratio, &e);
  e = max(-24, min(24, e - 1));
  return ldexpf(1.f, e);
}

// Record a sample that passed the threshold: packed (rho^2, sample, phase)
// atomic maximum into its window slot.  Out of line: it runs for a small
// fraction of samples and keeping it out of the unrolled hot loop keeps that
// loop's code small.
static __device__ __noinline__ void record_peak(unsigned long long* slot_row, int64_t n, int64_t window, float a, float b,
                                        float r2) {
  const float ph = atan2f(b, a);
  const uint32_t code = (uint32_t)__float2int_rn(fmaf(ph, 0.15915494309189535f, 0.5f) * 2048.0f) & 2047u;
  const unsigned long long key = ((unsigned long long)__float_as_uint(r2) << 32) |
                                 ((unsigned long long)(((1u << kSampleBits) - 1u) - (uint32_t)n) << kPhaseBits) |
                                 code;
  atomicMax(slot_row + n / window, key);
}

struct FilterEpi {
  const int32_t* sel;
  const float* inv_sigma;
  int64_t pos0;
  int n_det;
  float thr2;
  int64_t window, vb, ve, n_win, n_sel_total;
  unsigned long long* slots;
  struct Ser {
    float is;
    unsigned long long* slot;
  };
  __device__ __forceinline__ Ser series(int s) const {
    const int d = s % n_det;
    const int64_t pos = pos0 + s / n_det;
    return Ser{__ldg(inv_sigma + sel[pos]), slots + ((int64_t)d * n_sel_total + pos) * n_win};
  }
  __device__ __forceinline__ void operator()(const Ser& se, int64_t n, float2 z) const {
    const float a = z.x * se.is, b = z.y * se.is;
    const float r2 = fmaf(a, a, b * b);
    if (r2 >= thr2) {
      if (n >= vb && n < ve) record_peak(se.slot, n, window, a, b, r2);
    }
  }
};

// Epilogue on raw |z|^2: the data are pre-scaled by 1/sigma_ref, so |z'|^2 is in
// range, and each template carries thr_raw = rho_thr^2 / ratio^2 and ratio =
// scale * sigma_ref / sigma (rho = |z'| ratio).  Two instructions and a
// compare per sample; rho^2 and the phase only for samples over threshold.
struct RawEpi {
  const int32_t* sel;
  const float* ratio;
  const float* thr_raw;
  const float* dscale;  // per detector: power-of-two scale of 16-bit data (z' carries it), or null
  int64_t pos0;
  int n_det;
  int64_t window, vb, ve, n_win, n_sel_total;
  unsigned long long* slots;
  const int2* row_valid;  // per data row [begin, end), or null: [vb, ve) for every row
  struct Ser {
    float ratio, thr;
    int vb, ve;
    unsigned long long* slot;
  };
  __device__ __forceinline__ Ser series(int s) const {
    const int d = s % n_det;
    const int64_t pos = pos0 + s / n_det;
    const int t = sel[pos];
    float r = __ldg(ratio + t), th = __ldg(thr_raw + t);
    if (dscale) {  // exact: c is a power of two
      const float c = __ldg(dscale + d);
      r /= c;
      th *= c * c;
    }
    int b = (int)vb, e = (int)ve;
    if (row_valid) {
      const int2 rv = __ldg(row_valid + d);
      b = rv.x;
      e = rv.y;
    }
    return Ser{r, th, b, e, slots + ((int64_t)d * n_sel_total + pos) * n_win};
  }
  __device__ __forceinline__ void operator()(const Ser& se, int64_t n, float2 z) const {
    const float m2 = fmaf(z.x, z.x, z.y * z.y);
    if (m2 >= se.thr) {
      if (n >= se.vb && n < se.ve) {
        const float a = z.x * se.ratio, b = z.y * se.ratio;
        record_peak(se.slot, n, window, a, b, fmaf(a, a, b * b));
      }
    }
  }
};

}  // namespace mf
