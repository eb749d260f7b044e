// mf_filter_noalloc: the matched filter for callers that cannot allocate GPU
// memory (for example code running where cudaMalloc is forbidden or
// unavailable: inside another framework's memory pool, a real-time loop that
// must not allocate, or a plug-in that only receives buffers).  It keeps all
// of its working memory in one file-scope __device__ array and allocates
// nothing on the device or the host.
//
// In host code the array (kNoAllocBytes) is only a host-side stand-in, not a
// device address.  Every call therefore asks the runtime for the array's
// address on the current device (cudaGetSymbolAddress, a host-side query
// that enqueues no work) and hands that pointer to the kernels.  Looking it
// up on every call, instead of caching it, keeps it right after the device's
// context is torn down and created again (cudaDeviceReset), when the module
// is reloaded and the array can move, and needs no shared host state between
// caller threads.  Every call shares the array, so calls that overlap on the
// GPU (different streams or threads) race; serialise them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "../../include/mf.h"
#include "mf_internal.h"

namespace {

constexpr size_t kNoAllocBytes = size_t(32) << 20;  // 32 MiB on every device that loads the library

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// analysis-band weights w[k] = 4 df / S_n[k] on f_low <= k df < f_high, 0 < k < N/2
__global__ void k_weights(const double* __restrict__ psd, int64_t nb, int64_t k_lo, int64_t k_hi, double four_df,
                          double* __restrict__ w) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nb; k += (int64_t)gridDim.x * blockDim.x) {
    const double s = psd[k];
    w[k] = (k >= k_lo && k <= k_hi && isfinite(s) && s > 0.0) ? four_df / s : 0.0;
  }
}

__global__ void k_iota_zero(int32_t* sel, int64_t n, int* status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    sel[i] = (int32_t)i;
  if (blockIdx.x == 0 && threadIdx.x == 0) *status = 0;
}

mf_status fail(mf_status s, const std::string& m) {
  mf::set_global_error(m);
  return s;
}

}  // namespace

extern "C" mf_status mf_filter_noalloc(double fs, int64_t n, int32_t n_det, double f_low, double f_high,
                                       double snr_thr, int64_t window, const double* psd, const void* htilde,
                                       int64_t n_tmpl, int64_t ld_h, const void* dtilde, int64_t ld_d,
                                       mf_trigger* trig, int64_t trig_cap, int64_t* count, void* cuda_stream) {
  // ---- arguments and limits ----
  if (!psd || !htilde || !dtilde || !trig || !count) return fail(MF_EINVAL, "mf_filter_noalloc: null pointer");
  if (n < (1 << 12) || n > (1 << 16) || (n & (n - 1)) != 0)
    return fail(MF_EINVAL, "mf_filter_noalloc: n must be a power of two in [2^12, 2^16]");
  if (n_det < 1 || n_det > 2) return fail(MF_EINVAL, "mf_filter_noalloc: n_det must be 1 or 2");
  if (n_tmpl < 1 || n_tmpl > 1024) return fail(MF_EINVAL, "mf_filter_noalloc: n_tmpl must be in [1, 1024]");
  if (!(fs > 0) || !(f_low >= 0) || !(f_high > f_low) || !(snr_thr > 0) || window < 1 || window > n)
    return fail(MF_EINVAL, "mf_filter_noalloc: bad fs / band / threshold / window");
  const int64_t nb = n / 2 + 1;
  const int64_t n_win = (n + window - 1) / window;
  if (n_win > 256) return fail(MF_EINVAL, "mf_filter_noalloc: more than 256 windows per segment");
  if (ld_h < nb || ld_d < nb || trig_cap < 1) return fail(MF_EINVAL, "mf_filter_noalloc: leading dimension / capacity");

  // ---- the static array's address on the current device (looked up on every call) ----
  void* addr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
  if (e != cudaSuccess || !addr)
    return fail(MF_ECUDA, std::string("mf_filter_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  unsigned char* base = static_cast<unsigned char*>(addr);

  // ---- carve the array ----
  const int64_t ld_q = (nb + 63) / 64 * 64;
  const int64_t n_slots = (int64_t)n_det * n_tmpl * n_win;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* p = base + off;
    off += align256(bytes);
    return p;
  };
  double* w = reinterpret_cast<double*>(take(nb * sizeof(double)));
  float2* q = reinterpret_cast<float2*>(take((size_t)n_det * ld_q * sizeof(float2)));
  double* sigmasq = reinterpret_cast<double*>(take(n_tmpl * sizeof(double)));
  float* inv_sigma = reinterpret_cast<float*>(take(n_tmpl * sizeof(float)));
  int32_t* sel = reinterpret_cast<int32_t*>(take(n_tmpl * sizeof(int32_t)));
  int* status = reinterpret_cast<int*>(take(sizeof(int)));
  unsigned long long* slots = reinterpret_cast<unsigned long long*>(take(n_slots * sizeof(unsigned long long)));
  const int64_t n_blk = mf::compact_blocks(n_slots);
  int64_t* bc = reinterpret_cast<int64_t*>(take(n_blk * sizeof(int64_t)));
  const size_t per = (size_t)n_det * n * sizeof(float2);
  if (off + per > kNoAllocBytes) return fail(MF_EINVAL, "mf_filter_noalloc: problem exceeds the static scratch");
  const int batch = (int)std::min<int64_t>((int64_t)((kNoAllocBytes - off) / per), n_tmpl);
  float2* fft_scratch = reinterpret_cast<float2*>(take((size_t)batch * per));

  // ---- enqueue ----
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const double df = fs / (double)n;
  int64_t k_lo = (int64_t)std::ceil(f_low / df - 1e-9);
  int64_t k_hi = (int64_t)std::ceil(f_high / df - 1e-9) - 1;
  if (k_lo < 1) k_lo = 1;
  if (k_hi > n / 2 - 1) k_hi = n / 2 - 1;
  k_weights<<<64, 256, 0, st>>>(psd, nb, k_lo, k_hi, 4.0 * df, w);
  k_iota_zero<<<8, 256, 0, st>>>(sel, n_tmpl, status);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = mf::launch_sigmasq(htilde, mf::kBankF32, ld_h, nullptr, 0, n_tmpl, w, nb, sigmasq, inv_sigma, st);
  if (e == cudaSuccess)
    e = mf::launch_prep(static_cast<const float2*>(dtilde), ld_d, w, nb, n_det, q, ld_q, slots, n_slots, st);
  mf::FilterArgs a{};
  a.n = n;
  int lg = 0;
  while ((int64_t(1) << lg) < n) ++lg;
  a.n1 = 1 << ((lg + 1) / 2);
  a.n2 = 1 << (lg / 2);
  a.n_det = n_det;
  a.nb = nb;
  a.bank = htilde;
  a.bank_type = mf::kBankF32;
  a.ld_bank = ld_h;
  a.q = q;
  a.ld_q = ld_q;
  a.sel = sel;
  a.inv_sigma = inv_sigma;
  a.scratch = fft_scratch;
  a.thr2 = (float)(snr_thr * snr_thr);
  a.window = window;
  a.valid_begin = 0;
  a.valid_end = n;
  a.n_win = n_win;
  a.n_sel_total = n_tmpl;
  a.slots = slots;
  a.status = status;
  for (int64_t pos0 = 0; e == cudaSuccess && pos0 < n_tmpl; pos0 += batch) {
    a.pos0 = pos0;
    a.count = (int)std::min<int64_t>(batch, n_tmpl - pos0);
    e = mf::launch_filter_batch(a, st);
  }
  if (e == cudaSuccess)
    e = mf::launch_compact(slots, n_det, n_tmpl, n_win, window, sel, trig, trig_cap, count, bc, n_blk, st);
  if (e != cudaSuccess) return fail(MF_ECUDA, std::string("mf_filter_noalloc: ") + cudaGetErrorString(e));
  return MF_OK;
}
