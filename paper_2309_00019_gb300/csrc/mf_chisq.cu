// Signal-based veto at trigger times: Allen's chi^2 over p bands of equal
// template power and the re-weighted SNR of Eq. (4).
//
// The filter output of a trigger, z = sum_k w s~ h~* e^{+2 pi i k j / N},
// is split by frequency band, z_l = the same sum over band l, and
//   chi^2 = p sum_l |z_l - z / p|^2 / sigma^2   (2p - 2 degrees of freedom),
//   rho~ = rho / [(1 + chi2_r^3) / 2]^{1/6} if chi2_r = chi^2 / (2p - 2) >= 1.
// Band l holds the bins k whose template power below k, C(k), satisfies
// floor(p C(k) / sigma^2) = l (clamped to p - 1): k_block_power and
// k_chisq_edges find the first bin of every band with FP64 block sums, once
// per bank and p; k_chisq then
// sums each trigger's terms in the bank's column layout (contiguous reads of
// the template and the weighted data), one CTA per trigger.
#include <algorithm>

#include "mf_common.cuh"

namespace mf {

namespace {

constexpr int kCT = 128;  // threads per CTA

template <int BT>
__device__ __forceinline__ float2 elem(const void* p, int64_t i) {
  return BankElem<BT>::get(p, i);
}

// Template power per block of PB = min(256, N2) consecutive bins in frequency
// order (block b = bins [b PB, (b + 1) PB), all in one row k1 of the column
// layout), FP64, from the column-layout bank: bpow[t][b] = sum w |h|^2.
// grid (N2 / PB, n_tmpl); each thread owns rows k1 and walks the PB columns of
// its block, so the reads of every column are contiguous and the sums have a
// fixed order.
template <int BT>
__global__ void __launch_bounds__(kCT) k_block_power(const void* __restrict__ bank, int64_t ld_bank, int n1, int n2,
                                                     int pb, const double* __restrict__ w, double* __restrict__ bpow) {
  const int64_t t = blockIdx.y;
  const int cb = blockIdx.x;
  const int R = n1 / 2;
  const int nbl_row = n2 / pb;
  const void* row = static_cast<const unsigned char*>(bank) + t * ld_bank * (BT == kBankF32 ? 8 : 4);
  for (int k1 = threadIdx.x; k1 < R; k1 += blockDim.x) {
    double acc = 0.0;
    for (int c = 0; c < pb; ++c) {
      const int k2 = cb * pb + c;
      const int64_t k = (int64_t)k1 * n2 + k2;
      const double wk = w[k];
      if (wk != 0.0) {
        const float2 h = BankElem<BT>::get(row, (int64_t)k2 * R + k1);
        acc += wk * ((double)h.x * h.x + (double)h.y * h.y);
      }
    }
    bpow[t * ((int64_t)R * nbl_row) + (int64_t)k1 * nbl_row + cb] = acc;
  }
}

// edges[t][l] = first bin k of band l, i.e. the first k with w[k] != 0 and
// floor(p C(k) / sigma^2) >= l, with C(k) the template power below k (l < p);
// edges[t][p] = nb.  One warp per template: lane l < p finds edge l from the
// block sums, then within its block from the column-layout bank.
template <int BT>
__global__ void k_chisq_edges(const void* __restrict__ bank, int64_t ld_bank, int n1, int n2, int pb,
                              const double* __restrict__ w, int64_t nb, const double* __restrict__ bpow,
                              int64_t n_blocks, int64_t n_tmpl, int p, int32_t* __restrict__ edges) {
  const int64_t t = blockIdx.x * (int64_t)(blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (t >= n_tmpl) return;
  const double* bp = bpow + t * n_blocks;
  double total = 0.0;
  for (int64_t b = 0; b < n_blocks; ++b) total += bp[b];
  const int R = n1 / 2;
  const void* row = static_cast<const unsigned char*>(bank) + t * ld_bank * (BT == kBankF32 ? 8 : 4);
  for (int l = lane; l <= p; l += 32) {
    int64_t e = nb;
    if (l < p && total > 0.0) {
      double below = 0.0;
      int64_t b = 0;
      // the first block whose end reaches band l (band(k) >= l needs p C(k) / total >= l)
      while (b < n_blocks - 1 && floor((double)p * (below + bp[b]) / total) < (double)l) below += bp[b++];
      for (int64_t k = b * pb; k < nb && e == nb; ++k) {
        const double wk = w[k];
        if (wk != 0.0 && floor((double)p * below / total) >= (double)l) {
          e = k;
          break;
        }
        if (wk != 0.0 && k < (int64_t)R * n2) {
          const float2 h = BankElem<BT>::get(row, (k % n2) * R + k / n2);
          below += wk * ((double)h.x * h.x + (double)h.y * h.y);
        }
      }
    }
    edges[t * (p + 1) + l] = (int32_t)e;
  }
}

struct TrigRecC {
  int32_t det, tmpl;
  int64_t sample;
  float snr, phase;
};

// One CTA per trigger: thread-owned band partials in shared memory, then a
// fixed-order reduction, so the result is bitwise reproducible.
template <int BT, int QT>
__global__ void __launch_bounds__(kCT) k_chisq(const TrigRecC* __restrict__ trig, const int64_t* __restrict__ count,
                                               int64_t cap, const void* __restrict__ bank, int64_t ld_bank,
                                               const void* __restrict__ q, int64_t ld_q, int n1, int n2,
                                               const int32_t* __restrict__ edges, int p, const float* __restrict__ ratio,
                                               const float* __restrict__ dscale, float* __restrict__ chi2,
                                               float* __restrict__ newsnr) {
  extern __shared__ float2 zs[];  // [kCT][p]
  const int64_t n_trig = *count < cap ? *count : cap;
  const int R = n1 / 2;
  const int64_t half = (int64_t)R * n2;
  const uint32_t N = (uint32_t)n1 * (uint32_t)n2;
  for (int64_t it = blockIdx.x; it < n_trig; it += gridDim.x) {
    const TrigRecC tr = trig[it];
    const int32_t* e = edges + (int64_t)tr.tmpl * (p + 1);
    const void* hrow = static_cast<const unsigned char*>(bank) + (int64_t)tr.tmpl * ld_bank * (BT == kBankF32 ? 8 : 4);
    const void* qrow = static_cast<const unsigned char*>(q) + (int64_t)tr.det * ld_q * (QT == kBankF32 ? 8 : 4);
    float2* my = zs + threadIdx.x * p;
    for (int l = 0; l < p; ++l) my[l] = make_float2(0.f, 0.f);
    const uint32_t j = (uint32_t)tr.sample;
    // step of the phase along a column (k += N2): exp(+2 pi i j / N1)
    float ss, cs;
    sincospif(2.0f * (float)(j % (uint32_t)n1) / (float)n1, &ss, &cs);
    const float2 step = make_float2(cs, ss);
    const int64_t L = (half + kCT - 1) / kCT;
    const int64_t i0 = threadIdx.x * L, i1 = i0 + L < half ? i0 + L : half;
    float2 acc = make_float2(0.f, 0.f), ph = make_float2(1.f, 0.f);
    int band = -1;
    int64_t next = 0;  // first bin of the next band
    for (int64_t i = i0; i < i1; ++i) {
      const int k1 = (int)(i % R);
      const int64_t k = (int64_t)k1 * n2 + i / R;
      if (i == i0 || k1 == 0 || (k1 & 31) == 0) {
        if (i == i0 || k1 == 0) {  // new column: find the band by bisection over the edges
          if (band >= 0) {
            my[band].x += acc.x;
            my[band].y += acc.y;
            acc = make_float2(0.f, 0.f);
          }
          int lo = -1, hi = p;  // largest l with e[l] <= k (-1: below the band)
          while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (e[mid] <= k) lo = mid; else hi = mid;
          }
          band = lo;
          next = band + 1 <= p ? e[band + 1] : (int64_t)1 << 62;
        }
        // exact phase exp(+2 pi i k j / N) every 32 bins of a column
        const uint32_t m = (uint32_t)(((uint64_t)k * j) % N);
        sincospif(2.0f * (float)m / (float)N, &ss, &cs);
        ph = make_float2(cs, ss);
      }
      while (k >= next && band < p) {  // bands advance with k inside a column
        if (band >= 0) {
          my[band].x += acc.x;
          my[band].y += acc.y;
        }
        acc = make_float2(0.f, 0.f);
        ++band;
        next = band + 1 <= p ? e[band + 1] : (int64_t)1 << 62;
      }
      if (band >= 0 && band < p) {
        const float2 x = cmulc(elem<QT>(qrow, i), elem<BT>(hrow, i));
        const float2 y = cmul(x, ph);
        acc.x += y.x;
        acc.y += y.y;
      }
      ph = cmul(ph, step);
    }
    if (band >= 0 && band < p) {
      my[band].x += acc.x;
      my[band].y += acc.y;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      // z_l in stored units (data / sigma_ref, template / scale): |z_true| = |z| ratio / c_d
      float r = ratio[tr.tmpl];
      if (dscale) r /= dscale[tr.det];
      double zl_re[64], zl_im[64], z_re = 0.0, z_im = 0.0;
      for (int l = 0; l < p; ++l) {
        double a = 0.0, b = 0.0;
        for (int th = 0; th < kCT; ++th) {
          a += zs[th * p + l].x;
          b += zs[th * p + l].y;
        }
        zl_re[l] = a;
        zl_im[l] = b;
        z_re += a;
        z_im += b;
      }
      double c2 = 0.0;
      for (int l = 0; l < p; ++l) {
        const double dr = zl_re[l] - z_re / p, di = zl_im[l] - z_im / p;
        c2 += dr * dr + di * di;
      }
      c2 *= (double)p * (double)r * (double)r;
      chi2[it] = (float)c2;
      const double cr = c2 / (2.0 * p - 2.0);
      newsnr[it] = cr >= 1.0 ? (float)((double)tr.snr / pow((1.0 + cr * cr * cr) / 2.0, 1.0 / 6.0)) : tr.snr;
    }
    __syncthreads();
  }
}

int sms_c() {
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

// blocks of the template-power prefix: PB = min(256, N2) bins, N/2 / PB blocks
int chisq_pb(int n2) { return n2 < 256 ? n2 : 256; }
int64_t chisq_blocks(int n1, int n2) { return (int64_t)n1 / 2 * n2 / chisq_pb(n2); }

cudaError_t launch_chisq_edges(const void* bank, int bank_type, int64_t ld_bank, int64_t n_tmpl, int n1, int n2,
                               const double* w, int64_t nb, double* bpow, int p, int32_t* edges, cudaStream_t st) {
  if (p < 2 || p > 64 || n_tmpl <= 0) return cudaErrorInvalidValue;
  const int pb = chisq_pb(n2);
  const int64_t nbl = chisq_blocks(n1, n2);
  const unsigned g = (unsigned)((n_tmpl + 3) / 4);
  for (int64_t t0 = 0; t0 < n_tmpl; t0 += 65535) {
    const dim3 gp((unsigned)(n2 / pb), (unsigned)std::min<int64_t>(65535, n_tmpl - t0));
    const int64_t eb = bank_type == kBankF32 ? 8 : 4;
    const void* b0 = static_cast<const unsigned char*>(bank) + t0 * ld_bank * eb;
    double* o = bpow + t0 * nbl;
    switch (bank_type) {
      case kBankF32: k_block_power<kBankF32><<<gp, kCT, 0, st>>>(b0, ld_bank, n1, n2, pb, w, o); break;
      case kBankF16: k_block_power<kBankF16><<<gp, kCT, 0, st>>>(b0, ld_bank, n1, n2, pb, w, o); break;
      case kBankBF16: k_block_power<kBankBF16><<<gp, kCT, 0, st>>>(b0, ld_bank, n1, n2, pb, w, o); break;
      default: return cudaErrorInvalidValue;
    }
    add_launches(1);
  }
  switch (bank_type) {
    case kBankF32: k_chisq_edges<kBankF32><<<g, 128, 0, st>>>(bank, ld_bank, n1, n2, pb, w, nb, bpow, nbl, n_tmpl, p, edges); break;
    case kBankF16: k_chisq_edges<kBankF16><<<g, 128, 0, st>>>(bank, ld_bank, n1, n2, pb, w, nb, bpow, nbl, n_tmpl, p, edges); break;
    case kBankBF16: k_chisq_edges<kBankBF16><<<g, 128, 0, st>>>(bank, ld_bank, n1, n2, pb, w, nb, bpow, nbl, n_tmpl, p, edges); break;
    default: return cudaErrorInvalidValue;
  }
  add_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_chisq(const void* trig, const int64_t* count, int64_t cap, const void* bank, int bank_type,
                         int64_t ld_bank, const void* q, int q_type, int64_t ld_q, int n1, int n2, const int32_t* edges,
                         int p, const float* ratio, const float* dscale, float* chi2, float* newsnr, cudaStream_t st) {
  if (p < 2 || p > 64) return cudaErrorInvalidValue;
  const int grid = sms_c() * 4;
  const size_t smem = (size_t)kCT * p * sizeof(float2);
  const TrigRecC* t = static_cast<const TrigRecC*>(trig);
#define MF_CHISQ(BT, QT)                                                                                             \
  k_chisq<BT, QT><<<grid, kCT, smem, st>>>(t, count, cap, bank, ld_bank, q, ld_q, n1, n2, edges, p, ratio, dscale, \
                                           chi2, newsnr)
  if (q_type == kBankF32) {
    switch (bank_type) {
      case kBankF32: MF_CHISQ(kBankF32, kBankF32); break;
      case kBankF16: MF_CHISQ(kBankF16, kBankF32); break;
      case kBankBF16: MF_CHISQ(kBankBF16, kBankF32); break;
      default: return cudaErrorInvalidValue;
    }
  } else if (q_type == bank_type && q_type == kBankF16) {
    MF_CHISQ(kBankF16, kBankF16);
  } else if (q_type == bank_type && q_type == kBankBF16) {
    MF_CHISQ(kBankBF16, kBankBF16);
  } else {
    return cudaErrorInvalidValue;
  }
#undef MF_CHISQ
  add_launches(1);
  return cudaGetLastError();
}

namespace {

// One CTA per trigger: for a trigger of a template heavier than m_min and with rho~ >= snr_min, the SNR of
// every sine-Gaussian tile at the trigger sample.  Tile l of template t: f_l = f_final[t] + offsets[l]
// (skipped at or above f_high), g~[k] = exp(-(pi tau (f_k - f_l))^2), tau = qf / (sqrt(2) pi f_l); only the
// bins within 6 / (pi tau) of f_l enter (beyond, g~ < 3e-16).  rho_l^2 = |sum_k w s~ g~ e^{+2 pi i k j / N}|^2
// / sum_k w g~^2 with the weighted data read in the column layout and rescaled from its stored units.
template <int QT>
__global__ void __launch_bounds__(kCT) k_sgchisq(const TrigRecC* __restrict__ trig, const int64_t* __restrict__ count,
                                                 int64_t cap, const void* __restrict__ q, int64_t ld_q, int n1, int n2,
                                                 const double* __restrict__ w, double df, double f_high,
                                                 const float* __restrict__ f_final, const float* __restrict__ mtotal,
                                                 float m_min, float snr_min, SgTiles tiles, double q_to_true,
                                                 const float* __restrict__ dscale, const float* __restrict__ snr_in,
                                                 float* __restrict__ chi2_r, float* __restrict__ snr_hat) {
  __shared__ double red[3][kCT];
  const int64_t n_trig = *count < cap ? *count : cap;
  const int R = n1 / 2;
  const int64_t nb = (int64_t)R * n2 + 1;  // bins 0 .. N/2
  const uint64_t N = (uint64_t)n1 * (uint64_t)n2;
  for (int64_t it = blockIdx.x; it < n_trig; it += gridDim.x) {
    const TrigRecC tr = trig[it];
    const float rho = snr_in[it];
    if (!(mtotal[tr.tmpl] > m_min) || !(rho >= snr_min)) {
      if (threadIdx.x == 0) {
        chi2_r[it] = 0.f;
        snr_hat[it] = rho;
      }
      continue;
    }
    const void* qrow = static_cast<const unsigned char*>(q) + (int64_t)tr.det * ld_q * (QT == kBankF32 ? 8 : 4);
    const double scale = dscale ? q_to_true / (double)dscale[tr.det] : q_to_true;
    const uint64_t j = (uint64_t)tr.sample;
    double total = 0.0;
    int used = 0;
    for (int l = 0; l < tiles.n; ++l) {
      const double f0 = (double)f_final[tr.tmpl] + tiles.offset[l];
      if (!(f0 < f_high)) continue;
      const double tau = tiles.q / (1.4142135623730951 * 3.141592653589793 * f0);
      const double half = 6.0 / (3.141592653589793 * tau);
      const int64_t klo = max((int64_t)1, (int64_t)ceil((f0 - half) / df));
      const int64_t khi = min(nb - 2, (int64_t)floor((f0 + half) / df));
      float ar = 0.f, ai = 0.f;
      double s2 = 0.0;
      for (int64_t k = klo + threadIdx.x; k <= khi; k += kCT) {
        const double wk = w[k];
        if (wk == 0.0) continue;
        const float x = (float)(3.141592653589793 * tau * ((double)k * df - f0));
        const float g = expf(-x * x);
        const float2 qk = BankElem<QT>::get(qrow, (int64_t)(k % n2) * R + k / n2);  // column layout
        float sn, cs;
        sincospif(2.0f * (float)((k * j) % N) / (float)N, &sn, &cs);
        ar += g * (qk.x * cs - qk.y * sn);
        ai += g * (qk.x * sn + qk.y * cs);
        s2 += wk * (double)g * (double)g;
      }
      red[0][threadIdx.x] = ar;
      red[1][threadIdx.x] = ai;
      red[2][threadIdx.x] = s2;
      __syncthreads();
      if (threadIdx.x == 0) {  // fixed-order sums
        double zr = 0.0, zi = 0.0, ss = 0.0;
        for (int i = 0; i < kCT; ++i) {
          zr += red[0][i];
          zi += red[1][i];
          ss += red[2][i];
        }
        if (ss > 0.0) {
          total += (zr * zr + zi * zi) * scale * scale / ss;
          ++used;
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const float c = used ? (float)(total / (2.0 * used)) : 0.f;
      chi2_r[it] = c;
      // Eq. 3, inclusive at 6; decided on the stored single-precision value
      snr_hat[it] = c >= 6.f ? (float)((double)rho / sqrt((double)c)) : rho;
    }
  }
}

}  // namespace

cudaError_t launch_sgchisq(const void* trig, const int64_t* count, int64_t cap, const void* q, int q_type, int64_t ld_q,
                           int n1, int n2, const double* w, double df, double f_high, const float* f_final,
                           const float* mtotal, float m_min, float snr_min, const SgTiles& tiles, double q_to_true,
                           const float* dscale, const float* snr_in, float* chi2_r, float* snr_hat, cudaStream_t st) {
  if (tiles.n < 1 || tiles.n > kMaxSgTiles || !(tiles.q > 0)) return cudaErrorInvalidValue;
  const int grid = sms_c() * 4;
  const TrigRecC* t = static_cast<const TrigRecC*>(trig);
#define MF_SG(QT)                                                                                                  \
  k_sgchisq<QT><<<grid, kCT, 0, st>>>(t, count, cap, q, ld_q, n1, n2, w, df, f_high, f_final, mtotal, m_min, snr_min, \
                                      tiles, q_to_true, dscale, snr_in, chi2_r, snr_hat)
  switch (q_type) {
    case kBankF32: MF_SG(kBankF32); break;
    case kBankF16: MF_SG(kBankF16); break;
    case kBankBF16: MF_SG(kBankBF16); break;
    default: return cudaErrorInvalidValue;
  }
#undef MF_SG
  add_launches(1);
  return cudaGetLastError();
}

}  // namespace mf
