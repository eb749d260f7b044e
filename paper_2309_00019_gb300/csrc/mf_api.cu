// C ABI of libmf (declared in include/mf.h): plan management, argument checks,
// device memory ownership and the enqueueing of the kernels in
// mf_kernels.cu / mf_glue.cu on the plan's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "../../include/mf.h"
#include "mf_internal.h"

struct mf_plan_s {
  mf_plan_desc d{};
  cudaStream_t st = nullptr;
  int n1 = 0, n2 = 0;
  int64_t nb = 0, n_win = 0;
  std::string err;
  // PSD weights
  std::vector<double> w_host;
  double* w_dev = nullptr;
  bool psd_set = false;
  // bank
  void* bank = nullptr;
  mf_dtype bank_dtype = MF_F32;
  int64_t n_tmpl = 0, ld_bank = 0;
  float* scales_dev = nullptr;
  double* sigmasq_dev = nullptr;
  float* inv_sigma_dev = nullptr;
  int32_t* sel_all = nullptr;
  // data pre-scaling for the raw-|z|^2 epilogue: q' = w s~ / sigma_ref,
  // ratio[t] = scale_t sigma_ref / sigma_t, thr_raw[t] = rho_thr^2 / ratio[t]^2
  double sigma_ref = 1.0;
  float* ratio_dev = nullptr;
  float* thr_raw_dev = nullptr;
  bool scale_valid = false;
  // filter work space
  float2* q = nullptr;
  int64_t ld_q = 0;
  mf_dtype data_dtype = MF_F32;   // storage of the weighted data the filter reads
  int inter = 0;                  // pass-1 -> pass-2 intermediate: 0 complex64, 1 FP16, 2 FP16 pairs (FilterArgs)
  void* q_lp = nullptr;           // 16-bit weighted data [n_det][ld_q]
  unsigned* dmax = nullptr;       // per-detector max |q| (float bits)
  float* dscale = nullptr;        // per-detector power-of-two data scale
  int2* row_valid = nullptr;      // per-row analysed range (overlapping segments), or null
  // chi^2 veto: band edges for chisq_p bands (valid until the bank or the PSD changes)
  double* bpow = nullptr;
  int32_t* edges = nullptr;
  int chisq_p = 0;
  float2* scratch = nullptr;
  int batch = 1;
  CUtensorMap scratch_map{};  // pass-2 view of the scratch (mf::encode_scratch_map)
  unsigned long long* slots = nullptr;
  int64_t slots_cap = 0;        // in slots
  int32_t* sel_copy = nullptr;  // the selection of the last filter (device copy)
  int64_t sel_cap = 0;
  int64_t n_sel = 0;
  bool filtered = false;
  void* trig = nullptr;         // mf_trigger [max_triggers]
  int64_t* count = nullptr;     // device int64
  int64_t* bc = nullptr;        // compaction block offsets
  int64_t bc_cap = 0;
  // coincidence
  void* coincs = nullptr;
  int64_t coinc_cap = 0;
  unsigned long long* n_coinc = nullptr;
  float* maxrho = nullptr;
  int64_t maxrho_cap = 0;
  bool coinc_done = false;
  // neighbourhood map
  int64_t* nb_ptr = nullptr;
  int32_t* nb_idx = nullptr;
  int64_t n_coarse = 0;
  int32_t* flags = nullptr;
  int64_t flags_cap = 0;
  int64_t* ubc = nullptr;
  int64_t* ucount = nullptr;
  // TMA-staged filter
  int* status = nullptr;    // device status word
  float2* tw = nullptr;     // sub-FFT twiddle tables [2][1024]
  float2* tw4 = nullptr;    // four-step twiddles by column (launch_fill_tw4)
  // instrumentation
  mf_plan_stats stats{};
  bool prof = false;
  int prof_stride = 1;              // time every prof_stride-th launch pair
  int64_t prof_count = 0;           // launch pairs since profiling was turned on
  std::vector<cudaEvent_t> ev;      // pool, 3 per sampled batch
  struct Sample {
    int e0;
    int64_t series;
  };
  std::vector<Sample> samples;      // batch samples awaiting read
};

namespace mf {
int64_t plan_templates(const mf_plan_s* p) { return p ? p->n_tmpl : 0; }

uint64_t plan_fingerprint(const mf_plan_s* p) {
  uint64_t h = 1469598103934665603ull;  // FNV-1a over the values a captured filter depends on
  auto mix = [&](uint64_t v) {
    for (int i = 0; i < 8; ++i) {
      h ^= (v >> (8 * i)) & 0xffu;
      h *= 1099511628211ull;
    }
  };
  mix((uint64_t)(uintptr_t)p->bank);
  mix((uint64_t)p->n_tmpl);
  mix((uint64_t)p->batch);
  mix((uint64_t)p->data_dtype);
  mix((uint64_t)p->inter);
  mix((uint64_t)(uintptr_t)p->row_valid);
  mix((uint64_t)(uintptr_t)p->scratch);
  mix((uint64_t)(uintptr_t)p->slots);
  return h;
}

bool plan_capturable(const mf_plan_s* p) {
  if (!p || !p->scale_valid || p->prof) return false;
  const int64_t need = (int64_t)p->d.n_det * p->n_tmpl * p->n_win;
  return p->slots_cap >= need && p->sel_cap >= p->n_tmpl && p->bc_cap >= mf::compact_blocks(need);
}
}  // namespace mf

namespace {
constexpr int kProfBatches = 4096;  // launch pairs timed between two reads of the counters

// counts the kernels a block of code launches into p->stats.launches
struct LaunchScope {
  mf_plan_t p;
  int64_t before;
  explicit LaunchScope(mf_plan_t pp) : p(pp), before(mf::launch_count()) {}
  ~LaunchScope() { p->stats.launches += mf::launch_count() - before; }
};
}  // namespace

namespace {

thread_local std::string g_err;

mf_status fail(mf_plan_t p, mf_status s, const std::string& msg) {
  if (p) p->err = msg; else g_err = msg;
  return s;
}

mf_status cuda_fail(mf_plan_t p, cudaError_t e, const char* what) {
  return fail(p, MF_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <class T>
mf_status dalloc(mf_plan_t p, T** ptr, size_t bytes, const char* what) {
  if (*ptr) {
    cudaFree(*ptr);
    *ptr = nullptr;
  }
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc((void**)ptr, bytes);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
    return fail(p, MF_ENOMEM, std::string("cudaMalloc ") + what + " (" + std::to_string(bytes) + " bytes): " +
                                  cudaGetErrorString(e));
  }
  return MF_OK;
}

template <class T>
void dfree(T*& ptr) {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
}

bool is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }

// Device rows handed to a bank call are read on the plan's stream.  Order it after the work already
// submitted to the legacy default stream, which every blocking stream's earlier work precedes: rows written
// there (or on a blocking stream) before the call are complete when the plan reads them.
cudaError_t after_default_stream(mf_plan_t p) {
  cudaEvent_t ev = nullptr;
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev, cudaStreamLegacy);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->st, ev, 0);
  if (ev) cudaEventDestroy(ev);
  return e;
}

size_t elem_bytes(mf_dtype t) { return t == MF_F32 ? 8 : 4; }

int bank_type(mf_dtype t) { return t == MF_F32 ? mf::kBankF32 : (t == MF_F16 ? mf::kBankF16 : mf::kBankBF16); }

// Analysis-band weights w[k] = 4 df / S_n[k] (Eq. 2): f_low <= k df < f_high,
// 1 <= k <= N/2 - 1, S_n[k] positive and finite.
void make_weights(const mf_plan_desc& d, const double* psd, std::vector<double>& w) {
  const int64_t nb = d.n / 2 + 1;
  const double df = d.fs / (double)d.n;
  w.assign(nb, 0.0);
  int64_t k_lo = (int64_t)std::ceil(d.f_low / df - 1e-9);
  int64_t k_hi = (int64_t)std::ceil(d.f_high / df - 1e-9) - 1;
  k_lo = std::max<int64_t>(k_lo, 1);
  k_hi = std::min<int64_t>(k_hi, d.n / 2 - 1);
  for (int64_t k = k_lo; k <= k_hi; ++k) {
    const double s = psd[k];
    if (std::isfinite(s) && s > 0.0) w[k] = 4.0 * df / s;
  }
}

mf_status recompute_sigmasq(mf_plan_t p, int64_t row0, int64_t n_rows) {
  p->scale_valid = false;
  p->chisq_p = 0;  // band edges follow the bank and the PSD
  if (!p->psd_set || !p->bank || n_rows <= 0) return MF_OK;
  cudaError_t e = mf::launch_sigmasq(p->bank, bank_type(p->bank_dtype), p->ld_bank, p->scales_dev, row0, n_rows,
                                     p->w_dev, p->nb, p->sigmasq_dev, p->inv_sigma_dev, p->st, p->n1, p->n2);
  if (e != cudaSuccess) return cuda_fail(p, e, "sigma^2 kernel");
  return MF_OK;
}

// sigma_ref = max_t sigma_t (host copy of the FP64 norms), then ratio / thr_raw on the device
mf_status refresh_scale(mf_plan_t p) {
  if (p->scale_valid) return MF_OK;
  std::vector<double> s2(p->n_tmpl);
  cudaError_t e = cudaMemcpyAsync(s2.data(), p->sigmasq_dev, p->n_tmpl * sizeof(double), cudaMemcpyDeviceToHost, p->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_filter sigma^2 readback");
  double mx = 0.0;
  for (double v : s2)
    if (std::isfinite(v) && v > mx) mx = v;
  p->sigma_ref = mx > 0.0 ? std::sqrt(mx) : 1.0;
  e = mf::launch_tmpl_scale(p->inv_sigma_dev, p->n_tmpl, p->sigma_ref, p->d.snr_thr * p->d.snr_thr, p->ratio_dev,
                            p->thr_raw_dev, p->st);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_filter template scales");
  p->scale_valid = true;
  return MF_OK;
}

mf_status ensure_slots(mf_plan_t p, int64_t n_sel) {
  const int64_t need = (int64_t)p->d.n_det * n_sel * p->n_win;
  if (need > p->slots_cap) {
    mf_status s = dalloc(p, &p->slots, (size_t)need * sizeof(unsigned long long), "window slots");
    if (s != MF_OK) {
      p->slots_cap = 0;
      return s;
    }
    p->slots_cap = need;
  }
  const int64_t nblk = mf::compact_blocks(need);
  if (nblk > p->bc_cap) {
    mf_status s = dalloc(p, &p->bc, (size_t)std::max<int64_t>(nblk, 1) * sizeof(int64_t), "block offsets");
    if (s != MF_OK) {
      p->bc_cap = 0;
      return s;
    }
    p->bc_cap = nblk;
  }
  if (n_sel > p->sel_cap) {
    mf_status s = dalloc(p, &p->sel_copy, (size_t)std::max<int64_t>(n_sel, 1) * sizeof(int32_t), "selection");
    if (s != MF_OK) {
      p->sel_cap = 0;
      return s;
    }
    p->sel_cap = n_sel;
  }
  return MF_OK;
}

}  // namespace

namespace mf {
void set_global_error(const char* msg) { g_err = msg ? msg : ""; }
}  // namespace mf

extern "C" {

const char* mf_last_error(mf_plan_t plan) { return plan ? plan->err.c_str() : g_err.c_str(); }

mf_status mf_plan(mf_plan_t* out, const mf_plan_desc* desc) {
  if (!out || !desc) return fail(nullptr, MF_EINVAL, "mf_plan: null argument");
  const mf_plan_desc& d = *desc;
  if (!is_pow2(d.n) || d.n < (1 << 12) || d.n > mf::kMaxN)
    return fail(nullptr, MF_EINVAL, "mf_plan: n must be a power of two in [2^12, 2^20]");
  if (!(d.fs > 0) || !std::isfinite(d.fs)) return fail(nullptr, MF_EINVAL, "mf_plan: fs must be positive");
  if (d.n_det < 1 || d.n_det > 65536) return fail(nullptr, MF_EINVAL, "mf_plan: n_det must be in 1..65536");
  if (!(d.f_low >= 0) || !(d.f_high > d.f_low)) return fail(nullptr, MF_EINVAL, "mf_plan: need 0 <= f_low < f_high");
  if (d.dtype != MF_F32 && d.dtype != MF_F16 && d.dtype != MF_BF16) return fail(nullptr, MF_EINVAL, "mf_plan: dtype");
  if (!(d.snr_thr > 0) || !std::isfinite(d.snr_thr)) return fail(nullptr, MF_EINVAL, "mf_plan: snr_thr must be > 0");
  if (d.window < 1 || d.window > d.n) return fail(nullptr, MF_EINVAL, "mf_plan: window must be in [1, N]");
  if (d.valid_begin < 0 || d.valid_end > d.n || d.valid_begin >= d.valid_end)
    return fail(nullptr, MF_EINVAL, "mf_plan: need 0 <= valid_begin < valid_end <= N");
  if (d.max_triggers < 1) return fail(nullptr, MF_EINVAL, "mf_plan: max_triggers must be >= 1");

  mf_plan_t p = new (std::nothrow) mf_plan_s();
  if (!p) return fail(nullptr, MF_ENOMEM, "mf_plan: host allocation");
  p->d = d;
  p->st = (cudaStream_t)d.cuda_stream;
  int lg = 0;
  while ((int64_t(1) << lg) < d.n) ++lg;
  p->n1 = 1 << ((lg + 1) / 2);
  p->n2 = 1 << (lg / 2);
  p->nb = d.n / 2 + 1;
  p->n_win = (d.n + d.window - 1) / d.window;
  p->ld_q = (p->nb + 63) / 64 * 64;
  // templates per pass pair: as many as fit a 1 GB pass-1 -> pass-2 intermediate (fewer, longer
  // launches; the intermediate does not stay in L2 at any size that keeps launches efficient)
  const int64_t per = (int64_t)d.n_det * d.n * (int64_t)sizeof(float2);
  int64_t budget = int64_t(1024) << 20;
  if (const char* b = std::getenv("MF_SCRATCH_MB")) budget = std::max<int64_t>(1, std::atoll(b)) << 20;
  p->batch = (int)std::max<int64_t>(1, std::min<int64_t>(budget / per, 4096));
  const int64_t scratch_series = p->batch;
  mf_status s;
  if ((s = dalloc(p, &p->w_dev, p->nb * sizeof(double), "weights")) != MF_OK ||
      (s = dalloc(p, &p->q, (size_t)d.n_det * p->ld_q * sizeof(float2), "weighted data")) != MF_OK ||
      (s = dalloc(p, &p->scratch, (size_t)scratch_series * per, "scratch")) != MF_OK ||
      (s = dalloc(p, &p->trig, (size_t)d.max_triggers * sizeof(mf_trigger), "triggers")) != MF_OK ||
      (s = dalloc(p, &p->count, sizeof(int64_t), "count")) != MF_OK ||
      (s = dalloc(p, &p->status, sizeof(int), "status")) != MF_OK ||
      (s = dalloc(p, &p->tw, 2 * 1024 * sizeof(float2), "twiddles")) != MF_OK ||
      (s = dalloc(p, &p->tw4, (size_t)mf::tw4_count(d.n) * sizeof(float2), "four-step twiddles")) != MF_OK) {
    g_err = p->err;
    mf_destroy(p);
    return s;
  }
  if (mf::encode_scratch_map(d.n, p->scratch, scratch_series * d.n_det, &p->scratch_map) != cudaSuccess) {
    g_err = "mf_plan: tensor map of the scratch";
    mf_destroy(p);
    return MF_ECUDA;
  }
  cudaMemsetAsync(p->count, 0, sizeof(int64_t), p->st);
  cudaMemsetAsync(p->status, 0, sizeof(int), p->st);
  if (mf::launch_fill_twiddles(d.n, p->tw, p->tw + 1024, p->st) != cudaSuccess ||
      mf::launch_fill_tw4(d.n, p->tw4, p->st) != cudaSuccess) {
    g_err = "mf_plan: twiddle table kernel";
    mf_destroy(p);
    return MF_ECUDA;
  }
  *out = p;
  return MF_OK;
}

void mf_destroy(mf_plan_t p) {
  if (!p) return;
  if (p->st) cudaStreamSynchronize(p->st); else cudaDeviceSynchronize();
  dfree(p->w_dev); dfree(p->bank); dfree(p->scales_dev); dfree(p->sigmasq_dev); dfree(p->inv_sigma_dev); dfree(p->ratio_dev); dfree(p->thr_raw_dev);
  dfree(p->sel_all); dfree(p->q); dfree(p->scratch); dfree(p->slots); dfree(p->sel_copy); dfree(p->trig);
  dfree(p->count); dfree(p->bc); dfree(p->coincs); dfree(p->n_coinc); dfree(p->maxrho); dfree(p->nb_ptr);
  dfree(p->q_lp); dfree(p->dmax); dfree(p->dscale); dfree(p->row_valid); dfree(p->bpow); dfree(p->edges);
  dfree(p->nb_idx); dfree(p->flags); dfree(p->ubc); dfree(p->ucount); dfree(p->status); dfree(p->tw); dfree(p->tw4);
  for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
  delete p;
}

mf_status mf_set_psd(mf_plan_t p, const double* psd, int64_t nbins) {
  if (!p || !psd) return fail(p, MF_EINVAL, "mf_set_psd: null argument");
  if (nbins != p->nb) return fail(p, MF_EINVAL, "mf_set_psd: nbins must be N/2+1");
  make_weights(p->d, psd, p->w_host);
  cudaError_t e = cudaMemcpyAsync(p->w_dev, p->w_host.data(), p->nb * sizeof(double), cudaMemcpyHostToDevice, p->st);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_set_psd copy");
  e = cudaStreamSynchronize(p->st);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_set_psd sync");
  p->psd_set = true;
  return recompute_sigmasq(p, 0, p->n_tmpl);
}

mf_status mf_bank_reserve(mf_plan_t p, mf_dtype dtype, int64_t n_tmpl) {
  if (!p) return fail(p, MF_EINVAL, "mf_bank_reserve: null plan");
  if (dtype != MF_F32 && dtype != MF_F16 && dtype != MF_BF16) return fail(p, MF_EINVAL, "mf_bank_reserve: dtype");
  if (n_tmpl < 1 || n_tmpl > 0x7fffffff) return fail(p, MF_EINVAL, "mf_bank_reserve: n_tmpl must be in [1, 2^31)");
  cudaStreamSynchronize(p->st);
  p->n_tmpl = 0;
  p->scale_valid = false;
  p->chisq_p = 0;
  p->bank_dtype = dtype;
  p->ld_bank = p->d.n / 2;  // column layout of the N/2 bins below Nyquist (launch_to_cols)
  const size_t bytes = (size_t)n_tmpl * p->ld_bank * elem_bytes(dtype);
  mf_status s;
  if ((s = dalloc(p, &p->bank, bytes, "bank")) != MF_OK ||
      (s = dalloc(p, &p->sigmasq_dev, n_tmpl * sizeof(double), "sigma^2")) != MF_OK ||
      (s = dalloc(p, &p->inv_sigma_dev, n_tmpl * sizeof(float), "1/sigma")) != MF_OK ||
      (s = dalloc(p, &p->ratio_dev, n_tmpl * sizeof(float), "sigma ratio")) != MF_OK ||
      (s = dalloc(p, &p->thr_raw_dev, n_tmpl * sizeof(float), "raw thresholds")) != MF_OK ||
      (s = dalloc(p, &p->sel_all, n_tmpl * sizeof(int32_t), "all-template selection")) != MF_OK)
    return s;
  if (dtype != MF_F32) {
    if ((s = dalloc(p, &p->scales_dev, n_tmpl * sizeof(float), "scales")) != MF_OK) return s;
  } else {
    dfree(p->scales_dev);
  }
  cudaError_t e = cudaMemsetAsync(p->bank, 0, bytes, p->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->sigmasq_dev, 0, n_tmpl * sizeof(double), p->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->inv_sigma_dev, 0, n_tmpl * sizeof(float), p->st);
  std::vector<int32_t> ids(n_tmpl);
  for (int64_t i = 0; i < n_tmpl; ++i) ids[i] = (int32_t)i;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->sel_all, ids.data(), n_tmpl * sizeof(int32_t), cudaMemcpyHostToDevice, p->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_bank_reserve");
  p->n_tmpl = n_tmpl;
  return MF_OK;
}

mf_status mf_bank_set_rows(mf_plan_t p, int64_t row0, int64_t n_rows, const void* htilde, int64_t ld,
                           const float* scales, int on_device) {
  if (!p || !htilde) return fail(p, MF_EINVAL, "mf_bank_set_rows: null argument");
  if (!p->bank) return fail(p, MF_ESTATE, "mf_bank_set_rows: no bank reserved");
  if (row0 < 0 || n_rows < 0 || row0 + n_rows > p->n_tmpl)
    return fail(p, MF_EINVAL, "mf_bank_set_rows: rows out of range");
  if (ld < p->nb) return fail(p, MF_EINVAL, "mf_bank_set_rows: ld must be >= N/2+1");
  if ((p->bank_dtype == MF_F32) != (scales == nullptr))
    return fail(p, MF_EINVAL, "mf_bank_set_rows: scales required for 16-bit banks and forbidden for MF_F32");
  if (n_rows == 0) return MF_OK;
  const size_t eb = elem_bytes(p->bank_dtype);
  char* dst = (char*)p->bank + (size_t)row0 * p->ld_bank * eb;
  const void* src = htilde;
  void* tmp = nullptr;
  cudaError_t e = on_device ? after_default_stream(p) : cudaSuccess;
  if (!on_device) {  // stage host rows through a temporary device buffer
    mf_status s = dalloc(p, &tmp, (size_t)n_rows * ld * eb, "bank staging");
    if (s != MF_OK) return s;
    e = cudaMemcpyAsync(tmp, htilde, (size_t)n_rows * ld * eb, cudaMemcpyHostToDevice, p->st);
    src = tmp;
  }
  if (e == cudaSuccess) e = mf::launch_to_cols(src, ld, dst, p->ld_bank, n_rows, p->n1, p->n2, (int)eb, p->st);
  if (e == cudaSuccess && scales)
    e = cudaMemcpyAsync(p->scales_dev + row0, scales, n_rows * sizeof(float), cudaMemcpyHostToDevice, p->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_bank_set_rows copy");
  mf_status s = recompute_sigmasq(p, row0, n_rows);
  if (s != MF_OK) return s;
  e = cudaStreamSynchronize(p->st);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_bank_set_rows sigma^2");
  return MF_OK;
}

mf_status mf_bank_quantize_rows(mf_plan_t p, int64_t row0, int64_t n_rows, const void* htilde, int64_t ld,
                                int on_device) {
  if (!p || !htilde) return fail(p, MF_EINVAL, "mf_bank_quantize_rows: null argument");
  if (!p->bank) return fail(p, MF_ESTATE, "mf_bank_quantize_rows: no bank reserved");
  if (p->bank_dtype == MF_F32) return fail(p, MF_ESTATE, "mf_bank_quantize_rows: the bank is MF_F32");
  if (row0 < 0 || n_rows < 0 || row0 + n_rows > p->n_tmpl)
    return fail(p, MF_EINVAL, "mf_bank_quantize_rows: rows out of range");
  if (ld < p->nb) return fail(p, MF_EINVAL, "mf_bank_quantize_rows: ld must be >= N/2+1");
  if (n_rows == 0) return MF_OK;
  const float2* src = (const float2*)htilde;
  float2* tmp = nullptr;
  cudaError_t e = on_device ? after_default_stream(p) : cudaSuccess;
  if (!on_device) {  // stage host rows through a temporary device buffer
    mf_status s = dalloc(p, &tmp, (size_t)n_rows * ld * sizeof(float2), "quantisation staging");
    if (s != MF_OK) return s;
    e = cudaMemcpyAsync(tmp, htilde, (size_t)n_rows * ld * sizeof(float2), cudaMemcpyHostToDevice, p->st);
    src = tmp;
  }
  const size_t eb = elem_bytes(p->bank_dtype);
  void* q16 = nullptr;  // quantised rows in natural layout, then into the bank's column layout
  if (e == cudaSuccess) {
    mf_status s = dalloc(p, &q16, (size_t)n_rows * p->nb * eb, "quantised rows");
    if (s != MF_OK) {
      dfree(tmp);
      return s;
    }
    e = mf::launch_quant_bank(src, ld, n_rows, p->nb, bank_type(p->bank_dtype), q16, p->nb, p->scales_dev + row0, p->st);
  }
  if (e == cudaSuccess)
    e = mf::launch_to_cols(q16, p->nb, (char*)p->bank + (size_t)row0 * p->ld_bank * eb, p->ld_bank, n_rows, p->n1, p->n2,
                           (int)eb, p->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
  dfree(tmp);
  if (q16) cudaFree(q16);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_bank_quantize_rows");
  mf_status s = recompute_sigmasq(p, row0, n_rows);
  if (s != MF_OK) return s;
  e = cudaStreamSynchronize(p->st);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_bank_quantize_rows sigma^2");
  return MF_OK;
}

mf_status mf_set_data_dtype(mf_plan_t p, mf_dtype dtype) {
  if (!p) return fail(p, MF_EINVAL, "mf_set_data_dtype: null plan");
  if (dtype != MF_F32 && dtype != MF_F16 && dtype != MF_BF16) return fail(p, MF_EINVAL, "mf_set_data_dtype: dtype");
  cudaStreamSynchronize(p->st);
  if (dtype != MF_F32) {
    mf_status s;
    if (!p->q_lp && (s = dalloc(p, &p->q_lp, (size_t)p->d.n_det * p->ld_q * 4, "16-bit weighted data")) != MF_OK) return s;
    if (!p->dmax && (s = dalloc(p, &p->dmax, (size_t)p->d.n_det * sizeof(unsigned), "data maxima")) != MF_OK) return s;
    if (!p->dscale && (s = dalloc(p, &p->dscale, (size_t)p->d.n_det * sizeof(float), "data scales")) != MF_OK) return s;
    cudaError_t e = cudaMemsetAsync(p->q_lp, 0, (size_t)p->d.n_det * p->ld_q * 4, p->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
    if (e != cudaSuccess) return cuda_fail(p, e, "mf_set_data_dtype");
  }
  p->data_dtype = dtype;
  return MF_OK;
}

mf_status mf_bank_generate_taylorf2(mf_plan_t p, int64_t row0, int64_t n_rows, const double* m1, const double* m2,
                                    double f_low) {
  if (!p || !m1 || !m2) return fail(p, MF_EINVAL, "mf_bank_generate_taylorf2: null argument");
  if (!p->bank) return fail(p, MF_ESTATE, "mf_bank_generate_taylorf2: no bank reserved");
  if (row0 < 0 || n_rows < 0 || row0 + n_rows > p->n_tmpl)
    return fail(p, MF_EINVAL, "mf_bank_generate_taylorf2: rows out of range");
  if (!(f_low > 0)) return fail(p, MF_EINVAL, "mf_bank_generate_taylorf2: f_low must be > 0");
  if (n_rows == 0) return MF_OK;
  const int64_t ld = (p->nb + 63) / 64 * 64;
  const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(n_rows, (int64_t(256) << 20) / (ld * 8)));
  float2* tmp = nullptr;
  mf_status s = dalloc(p, &tmp, (size_t)chunk * ld * sizeof(float2), "generated rows");
  if (s != MF_OK) return s;
  for (int64_t r = 0; r < n_rows && s == MF_OK; r += chunk) {
    const int64_t cnt = std::min<int64_t>(chunk, n_rows - r);
    cudaError_t e = mf::launch_taylorf2(m1 + r, m2 + r, cnt, p->d.fs, p->d.n, f_low, tmp, ld, p->st);
    if (e == cudaErrorInvalidValue) {
      s = fail(p, MF_EINVAL, "mf_bank_generate_taylorf2: bad masses or band");
    } else if (e != cudaSuccess) {
      s = cuda_fail(p, e, "mf_bank_generate_taylorf2");
    } else {
      s = p->bank_dtype == MF_F32 ? mf_bank_set_rows(p, row0 + r, cnt, tmp, ld, nullptr, 1)
                                  : mf_bank_quantize_rows(p, row0 + r, cnt, tmp, ld, 1);
    }
  }
  cudaStreamSynchronize(p->st);
  cudaFree(tmp);
  return s;
}

mf_status mf_set_intermediate(mf_plan_t p, mf_dtype dtype) {
  if (!p) return fail(p, MF_EINVAL, "mf_set_intermediate: null plan");
  if (dtype != MF_F32 && dtype != MF_F16 && dtype != MF_F16X2)
    return fail(p, MF_EINVAL, "mf_set_intermediate: dtype must be F32, F16 or F16X2");
  if (dtype != MF_F32 && p->d.n != (int64_t(1) << 20))
    return fail(p, MF_EINVAL, "mf_set_intermediate: the FP16 intermediates need N = 2^20");
  cudaStreamSynchronize(p->st);
  p->inter = dtype == MF_F32 ? 0 : (dtype == MF_F16 ? 1 : 2);
  return MF_OK;
}

mf_status mf_set_row_valid(mf_plan_t p, const int64_t* range) {
  if (!p) return fail(p, MF_EINVAL, "mf_set_row_valid: null plan");
  cudaStreamSynchronize(p->st);
  if (!range) {
    dfree(p->row_valid);
    return MF_OK;
  }
  std::vector<int2> r(p->d.n_det);
  for (int i = 0; i < p->d.n_det; ++i) {
    const int64_t b = range[2 * i], e = range[2 * i + 1];
    if (b < 0 || e < b || e > p->d.n) return fail(p, MF_EINVAL, "mf_set_row_valid: need 0 <= begin <= end <= N");
    r[i] = make_int2((int)b, (int)e);
  }
  mf_status s;
  if (!p->row_valid && (s = dalloc(p, &p->row_valid, r.size() * sizeof(int2), "row ranges")) != MF_OK) return s;
  cudaError_t e = cudaMemcpyAsync(p->row_valid, r.data(), r.size() * sizeof(int2), cudaMemcpyHostToDevice, p->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_set_row_valid");
  return MF_OK;
}

mf_status mf_set_batch(mf_plan_t p, int32_t batch) {
  if (!p) return fail(p, MF_EINVAL, "mf_set_batch: null plan");
  if (batch < 1) return fail(p, MF_EINVAL, "mf_set_batch: batch must be >= 1");
  cudaStreamSynchronize(p->st);
  const int64_t per = (int64_t)p->d.n_det * p->d.n * (int64_t)sizeof(float2);
  const int64_t series = batch;
  mf_status s = dalloc(p, &p->scratch, (size_t)series * per, "scratch");
  if (s != MF_OK) return s;
  p->batch = batch;
  if (mf::encode_scratch_map(p->d.n, p->scratch, series * p->d.n_det, &p->scratch_map) != cudaSuccess)
    return fail(p, MF_ECUDA, "mf_set_batch: tensor map of the scratch");
  return MF_OK;
}

mf_status mf_load_gate_template(mf_plan_t p) {
  if (!p) return fail(p, MF_EINVAL, "mf_load_gate_template: null plan");
  if (!p->psd_set) return fail(p, MF_ESTATE, "mf_load_gate_template: PSD not set");
  mf_status s = mf_bank_reserve(p, MF_F32, 1);
  if (s != MF_OK) return s;
  float2* row = nullptr;
  s = dalloc(p, &row, (size_t)p->nb * sizeof(float2), "gate row");
  if (s != MF_OK) return s;
  cudaError_t e = mf::launch_gate_row(p->w_dev, p->nb, p->d.fs / (double)p->d.n, row, p->st);
  if (e != cudaSuccess) {
    cudaFree(row);
    return cuda_fail(p, e, "mf_load_gate_template");
  }
  s = mf_bank_set_rows(p, 0, 1, row, p->nb, nullptr, 1);  // synchronises before returning
  cudaFree(row);
  return s;
}

mf_status mf_load_bank(mf_plan_t p, const void* htilde, mf_dtype dtype, int64_t n_tmpl, int64_t ld, const float* scales,
                       int on_device) {
  if (!p || !htilde) return fail(p, MF_EINVAL, "mf_load_bank: null argument");
  mf_status s = mf_bank_reserve(p, dtype, n_tmpl);
  if (s != MF_OK) return s;
  return mf_bank_set_rows(p, 0, n_tmpl, htilde, ld, scales, on_device);
}

mf_status mf_get_sigmasq(mf_plan_t p, double* out, int64_t n) {
  if (!p || !out) return fail(p, MF_EINVAL, "mf_get_sigmasq: null argument");
  if (n < 0 || n > p->n_tmpl) return fail(p, MF_EINVAL, "mf_get_sigmasq: n out of range");
  if (!p->psd_set) return fail(p, MF_ESTATE, "mf_get_sigmasq: PSD not set");
  cudaError_t e = cudaMemcpyAsync(out, p->sigmasq_dev, n * sizeof(double), cudaMemcpyDeviceToHost, p->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_get_sigmasq");
  return MF_OK;
}

mf_status mf_strain_to_fd(mf_plan_t p, const float* strain, int64_t ld_strain, void* dtilde, int64_t ld_dtilde) {
  if (!p || !strain || !dtilde) return fail(p, MF_EINVAL, "mf_strain_to_fd: null argument");
  if (ld_strain < p->d.n || ld_dtilde < p->nb) return fail(p, MF_EINVAL, "mf_strain_to_fd: leading dimension");
  LaunchScope ls(p);
  cudaError_t e = mf::launch_rfft(strain, ld_strain, p->d.n_det, p->d.n, p->n1, p->n2, 1.0 / p->d.fs, p->scratch,
                                  (float2*)dtilde, ld_dtilde, p->st);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_strain_to_fd");
  return MF_OK;
}

mf_status mf_decimate(mf_plan_t p, const void* in, int64_t ld_in, void* out, int64_t ld_out) {
  if (!p || !in || !out) return fail(p, MF_EINVAL, "mf_decimate: null argument");
  if (ld_in < p->nb || ld_out < p->nb) return fail(p, MF_EINVAL, "mf_decimate: leading dimension < N/2+1");
  LaunchScope ls(p);
  cudaError_t e = mf::launch_decimate((const float2*)in, ld_in, (float2*)out, ld_out, p->nb, p->d.n_det, p->st);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_decimate");
  return MF_OK;
}

mf_status mf_filter(mf_plan_t p, const void* dtilde, int64_t ld_dtilde, const int32_t* subset, int64_t n_subset) {
  if (!p || !dtilde) return fail(p, MF_EINVAL, "mf_filter: null argument");
  if (!p->psd_set) return fail(p, MF_ESTATE, "mf_filter: PSD not set");
  if (!p->bank || p->n_tmpl == 0) return fail(p, MF_ESTATE, "mf_filter: no bank loaded");
  if (ld_dtilde < p->nb) return fail(p, MF_EINVAL, "mf_filter: ld_dtilde < N/2+1");
  if (n_subset < 0 && subset) return fail(p, MF_EINVAL, "mf_filter: n_subset < 0 (all templates) needs subset NULL");
  if (n_subset > 0 && !subset) return fail(p, MF_EINVAL, "mf_filter: subset is NULL");
  if (p->data_dtype != MF_F32 && p->data_dtype != p->bank_dtype)
    return fail(p, MF_EINVAL, "mf_filter: 16-bit data need a bank of the same 16-bit type");
  if (p->inter && p->data_dtype != MF_F32)
    return fail(p, MF_EINVAL, "mf_filter: the FP16 intermediate needs FP32 weighted data");
  const int64_t n_sel = n_subset < 0 ? p->n_tmpl : n_subset;
  mf_status s = ensure_slots(p, std::max<int64_t>(n_sel, 1));
  if (s != MF_OK) return s;
  if ((s = refresh_scale(p)) != MF_OK) return s;
  cudaError_t e = cudaSuccess;
  if (n_sel > 0)
    e = cudaMemcpyAsync(p->sel_copy, n_subset < 0 ? p->sel_all : subset, n_sel * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                        p->st);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_filter selection copy");
  const int64_t n_slots = (int64_t)p->d.n_det * n_sel * p->n_win;
  const int64_t launches_before = mf::launch_count();
  e = mf::launch_prep_cols((const float2*)dtilde, ld_dtilde, p->w_dev, p->n1, p->n2, p->d.n_det, p->q, p->ld_q,
                           p->slots, n_slots, p->st, 1.0 / p->sigma_ref);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_filter prep");
  if (p->data_dtype != MF_F32) {
    e = mf::launch_quant_q(p->q, p->ld_q, p->d.n / 2, p->d.n_det, bank_type(p->data_dtype), p->q_lp, p->dmax, p->dscale,
                           p->st);
    if (e != cudaSuccess) return cuda_fail(p, e, "mf_filter data quantisation");
  }
  mf::FilterArgs a{};
  a.n = p->d.n;
  a.n1 = p->n1;
  a.n2 = p->n2;
  a.n_det = p->d.n_det;
  a.nb = p->nb;
  a.bank = p->bank;
  a.bank_type = bank_type(p->bank_dtype);
  a.ld_bank = p->ld_bank;
  a.scales = p->scales_dev;
  a.q = p->q;
  a.ld_q = p->ld_q;
  a.sel = p->sel_copy;
  a.inv_sigma = p->ratio_dev;  // 1/sigma on the data scaled by 1/sigma_ref
  a.thr_raw = p->thr_raw_dev;
  a.scratch = p->scratch;
  const double thr = p->d.snr_thr;
  a.thr2 = (float)(thr * thr);
  a.window = p->d.window;
  a.valid_begin = p->d.valid_begin;
  a.valid_end = p->d.valid_end;
  a.n_win = p->n_win;
  a.n_sel_total = n_sel;
  a.slots = p->slots;
  a.status = p->status;
  a.tw1 = p->tw;
  a.tw2 = p->tw + 1024;
  a.tw4 = p->tw4;
  a.row_valid = p->row_valid;
  a.q_type = bank_type(p->data_dtype);
  a.q_lp = p->q_lp;
  a.dscale = p->dscale;
  a.inter = p->inter;
  LaunchScope ls(p);
  ls.before = launches_before;
  for (int64_t pos0 = 0; pos0 < n_sel; pos0 += p->batch) {
    a.pos0 = pos0;
    a.first_batch = pos0 == 0 ? 1 : 0;
    a.count = (int)std::min<int64_t>(p->batch, n_sel - pos0);
    const bool prof = p->prof && p->prof_count++ % p->prof_stride == 0 && (int)p->samples.size() < kProfBatches;
    const int e0 = prof ? (int)p->samples.size() * 3 : 0;
    if (prof) cudaEventRecord(p->ev[e0], p->st);
    e = mf::launch_filter2_pass1(a, p->st);
    if (e != cudaSuccess) return cuda_fail(p, e, "mf_filter pass 1");
    if (prof) cudaEventRecord(p->ev[e0 + 1], p->st);
    e = mf::launch_filter2_pass2(a, p->scratch_map, p->st);
    if (e != cudaSuccess) return cuda_fail(p, e, "mf_filter pass 2");
    if (prof) {
      cudaEventRecord(p->ev[e0 + 2], p->st);
      p->samples.push_back({e0, (int64_t)a.count * p->d.n_det});
    }
  }
  e = mf::launch_compact(p->slots, p->d.n_det, n_sel, p->n_win, p->d.window, p->sel_copy, p->trig, p->d.max_triggers,
                         p->count, p->bc, p->bc_cap, p->st);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_filter compaction");
  p->n_sel = n_sel;
  p->filtered = true;
  p->coinc_done = false;
  return MF_OK;
}

mf_status mf_profile(mf_plan_t p, int enable) {
  if (!p) return fail(p, MF_EINVAL, "mf_profile: null plan");
  if (enable < 0) return fail(p, MF_EINVAL, "mf_profile: enable must be >= 0");
  if (enable && p->ev.empty()) {
    p->ev.resize(3 * kProfBatches);
    for (auto& e : p->ev) {
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return cuda_fail(p, r, "mf_profile event");
    }
  }
  p->prof = enable != 0;
  p->prof_stride = enable > 1 ? enable : 1;
  p->prof_count = 0;
  return MF_OK;
}

mf_status mf_get_stats(mf_plan_t p, mf_plan_stats* out, int reset) {
  if (!p || !out) return fail(p, MF_EINVAL, "mf_get_stats: null argument");
  cudaError_t e = cudaStreamSynchronize(p->st);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_get_stats sync");
  for (const auto& sm : p->samples) {
    float t1 = 0, t2 = 0;
    e = cudaEventElapsedTime(&t1, p->ev[sm.e0], p->ev[sm.e0 + 1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t2, p->ev[sm.e0 + 1], p->ev[sm.e0 + 2]);
    if (e != cudaSuccess) return cuda_fail(p, e, "mf_get_stats elapsed");
    p->stats.pass1_launches += 1;
    p->stats.pass1_series += sm.series;
    p->stats.pass1_ms += t1;
    p->stats.pass2_launches += 1;
    p->stats.pass2_series += sm.series;
    p->stats.pass2_ms += t2;
  }
  p->samples.clear();
  p->stats.impl = 2 + p->inter;
  p->stats.batch = p->batch;
  *out = p->stats;
  if (reset) p->stats = mf_plan_stats{};
  return MF_OK;
}

mf_status mf_get_triggers(mf_plan_t p, mf_trigger* out, int64_t cap, int64_t* n_found) {
  if (!p || !n_found || (cap > 0 && !out)) return fail(p, MF_EINVAL, "mf_get_triggers: null argument");
  if (!p->filtered) return fail(p, MF_ESTATE, "mf_get_triggers: no filter run");
  int64_t n = 0;
  cudaError_t e = cudaMemcpyAsync(&n, p->count, sizeof(int64_t), cudaMemcpyDeviceToHost, p->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_get_triggers count");
  *n_found = n;
  int dst = 0;
  e = cudaMemcpy(&dst, p->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_get_triggers status");
  if (dst != 0) {
    cudaMemset(p->status, 0, sizeof(int));
    std::string m = "mf_get_triggers: a bounded device wait timed out; results are incomplete";
    if (dst >> 8)  // waits that record where they gave up: site and item
      m += " (wait site " + std::to_string((dst >> 8) & 0xff) + ", item " + std::to_string((unsigned)dst >> 16) + ")";
    return fail(p, MF_ETIMEOUT, m);
  }
  const int64_t m = std::min<int64_t>(std::min<int64_t>(n, cap), p->d.max_triggers);
  if (m > 0) {
    e = cudaMemcpyAsync(out, p->trig, m * sizeof(mf_trigger), cudaMemcpyDeviceToHost, p->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
    if (e != cudaSuccess) return cuda_fail(p, e, "mf_get_triggers copy");
  }
  if (n > cap || n > p->d.max_triggers)
    return fail(p, MF_EOVERFLOW, "mf_get_triggers: " + std::to_string(n) + " triggers exceed the buffer");
  return MF_OK;
}

mf_status mf_chisq(mf_plan_t p, int32_t n_bands, float* chi2, float* newsnr) {
  if (!p || !chi2 || !newsnr) return fail(p, MF_EINVAL, "mf_chisq: null argument");
  if (n_bands < 2 || n_bands > 64) return fail(p, MF_EINVAL, "mf_chisq: bands must be in [2, 64]");
  if (!p->filtered) return fail(p, MF_ESTATE, "mf_chisq: no filter run");
  if (p->chisq_p != n_bands) {
    mf_status s;
    if ((s = dalloc(p, &p->bpow, (size_t)p->n_tmpl * mf::chisq_blocks(p->n1, p->n2) * sizeof(double), "band power")) !=
            MF_OK ||
        (s = dalloc(p, &p->edges, (size_t)p->n_tmpl * (n_bands + 1) * sizeof(int32_t), "band edges")) != MF_OK)
      return s;
    cudaError_t e = mf::launch_chisq_edges(p->bank, bank_type(p->bank_dtype), p->ld_bank, p->n_tmpl, p->n1, p->n2,
                                           p->w_dev, p->nb, p->bpow, n_bands, p->edges, p->st);
    if (e != cudaSuccess) return cuda_fail(p, e, "mf_chisq band edges");
    p->chisq_p = n_bands;
  }
  const bool lp = p->data_dtype != MF_F32;
  cudaError_t e = mf::launch_chisq(p->trig, p->count, p->d.max_triggers, p->bank, bank_type(p->bank_dtype), p->ld_bank,
                                   lp ? p->q_lp : (const void*)p->q, bank_type(p->data_dtype), p->ld_q, p->n1, p->n2,
                                   p->edges, n_bands, p->ratio_dev, lp ? p->dscale : nullptr, chi2, newsnr, p->st);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_chisq");
  return MF_OK;
}

mf_status mf_sgchisq(mf_plan_t p, const float* f_final, const float* mtotal, float m_min, float snr_min,
                     int32_t n_tiles, const double* offsets, double q, const float* newsnr, float* chi2_r,
                     float* snr_hat) {
  if (!p || !f_final || !mtotal || !offsets || !newsnr || !chi2_r || !snr_hat)
    return fail(p, MF_EINVAL, "mf_sgchisq: null argument");
  if (n_tiles < 1 || n_tiles > mf::kMaxSgTiles || !(q > 0)) return fail(p, MF_EINVAL, "mf_sgchisq: tiles or q");
  if (!p->filtered) return fail(p, MF_ESTATE, "mf_sgchisq: no filter run");
  mf::SgTiles tiles{};
  tiles.n = n_tiles;
  tiles.q = q;
  for (int i = 0; i < n_tiles; ++i) tiles.offset[i] = offsets[i];
  const bool lp = p->data_dtype != MF_F32;
  // the band's upper edge: tiles at or above it are skipped
  const double f_high = std::min(p->d.f_high, p->d.fs / 2.0);
  cudaError_t e = mf::launch_sgchisq(p->trig, p->count, p->d.max_triggers, lp ? p->q_lp : (const void*)p->q,
                                     bank_type(p->data_dtype), p->ld_q, p->n1, p->n2, p->w_dev, p->d.fs / (double)p->d.n,
                                     f_high, f_final, mtotal, m_min, snr_min, tiles, p->sigma_ref,
                                     lp ? p->dscale : nullptr, newsnr, chi2_r, snr_hat, p->st);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_sgchisq");
  return MF_OK;
}

mf_status mf_far(const float* stat_fg, int64_t n_fg, const float* stat_bg, int64_t n_bg, double t_bg, double scale,
                 double fit_min, double* far_count, double* far_fit, double* alpha, double* beta) {
  if (n_fg < 0 || n_bg < 0 || (n_fg > 0 && (!stat_fg || !far_count)) || (n_bg > 0 && !stat_bg))
    return fail(nullptr, MF_EINVAL, "mf_far: null argument or negative size");
  if (!(t_bg > 0) || !(scale > 0)) return fail(nullptr, MF_EINVAL, "mf_far: t_bg and scale must be positive");
  std::vector<double> bg(stat_bg, stat_bg + n_bg);
  std::sort(bg.begin(), bg.end());
  auto count_ge = [&](double x) {
    return scale * (double)(bg.end() - std::lower_bound(bg.begin(), bg.end(), x));
  };
  for (int64_t i = 0; i < n_fg; ++i) far_count[i] = (1.0 + count_ge((double)stat_fg[i])) / t_bg;
  // least-squares line through (x, log n_b(x)) at every background value x >= fit_min
  double sx = 0, sy = 0, sxx = 0, sxy = 0;
  int64_t m = 0;
  for (size_t i = std::lower_bound(bg.begin(), bg.end(), fit_min) - bg.begin(); i < bg.size(); ++i) {
    const double x = bg[i], y = std::log(scale * (double)(bg.size() - (std::lower_bound(bg.begin(), bg.end(), x) - bg.begin())));
    sx += x;
    sy += y;
    sxx += x * x;
    sxy += x * y;
    ++m;
  }
  const double det = (double)m * sxx - sx * sx;
  const bool ok = m >= 2 && det > 0;
  const double b = ok ? ((double)m * sxy - sx * sy) / det : std::nan("");
  const double a = ok ? (sy - b * sx) / (double)m : std::nan("");
  if (alpha) *alpha = a;
  if (beta) *beta = b;
  if (far_fit)
    for (int64_t i = 0; i < n_fg; ++i) far_fit[i] = ok ? (1.0 + std::exp(a + b * (double)stat_fg[i])) / t_bg : std::nan("");
  return MF_OK;
}

mf_status mf_fma_probe(double* tflops, void* cuda_stream) {
  if (!tflops) return fail(nullptr, MF_EINVAL, "mf_fma_probe: null argument");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = std::max(1, sms) * 8, iters = 4096;
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc((void**)&out, (size_t)blocks * 256 * sizeof(float));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = mf::launch_fma_probe(out, blocks, iters / 8, st);  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) e = mf::launch_fma_probe(out, blocks, iters, st);
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (out) cudaFree(out);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail(nullptr, MF_ECUDA, std::string("mf_fma_probe: ") + cudaGetErrorString(e));
  const double flops = 2.0 * (double)blocks * 256.0 * 8.0 * 16.0 * (double)iters;
  *tflops = flops / ((double)ms * 1e-3) / 1e12;
  return MF_OK;
}

mf_status mf_selftest_wait(mf_plan_t p, int32_t* returned) {
  if (!p || !returned) return fail(p, MF_EINVAL, "mf_selftest_wait: null argument");
  int* cnt = nullptr;
  mf_status s = dalloc(p, &cnt, sizeof(int), "self-test counter");
  if (s != MF_OK) return s;
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int), p->st);
  if (e == cudaSuccess) e = mf::launch_wait_selftest(p->status, cnt, p->st);
  int r = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&r, cnt, sizeof(int), cudaMemcpyDeviceToHost, p->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
  cudaFree(cnt);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_selftest_wait");
  *returned = r;
  return MF_OK;
}

mf_status mf_device_triggers(mf_plan_t p, const mf_trigger** trig, const int64_t** count) {
  if (!p || !trig || !count) return fail(p, MF_EINVAL, "mf_device_triggers: null argument");
  if (!p->filtered) return fail(p, MF_ESTATE, "mf_device_triggers: no filter run");
  *trig = (const mf_trigger*)p->trig;
  *count = p->count;
  return MF_OK;
}

mf_status mf_coincide(mf_plan_t p, const mf_coinc_desc* c, int32_t* followed) {
  if (!p || !c || !followed) return fail(p, MF_EINVAL, "mf_coincide: null argument");
  if (p->d.n_det != 2) return fail(p, MF_EINVAL, "mf_coincide: needs a 2-detector plan");
  if (!p->filtered) return fail(p, MF_ESTATE, "mf_coincide: no filter run");
  const int64_t R = p->d.valid_end - p->d.valid_begin;
  if (c->shift_samples <= 0 || c->n_shifts < 0 || c->window_samples < 0 || 2 * c->window_samples >= R ||
      c->max_coincs < 1 || !(c->rho_c_thr > 0) || !(c->rho_c_store > 0))
    return fail(p, MF_EINVAL, "mf_coincide: bad coincidence description");
  mf_status s;
  if (c->max_coincs > p->coinc_cap) {
    if ((s = dalloc(p, &p->coincs, (size_t)c->max_coincs * sizeof(mf_coinc), "coincidences")) != MF_OK) {
      p->coinc_cap = 0;
      return s;
    }
    p->coinc_cap = c->max_coincs;
  }
  if (!p->n_coinc && (s = dalloc(p, &p->n_coinc, sizeof(unsigned long long), "coincidence count")) != MF_OK) return s;
  if (p->n_sel > p->maxrho_cap) {
    if ((s = dalloc(p, &p->maxrho, (size_t)p->n_sel * sizeof(float), "max rho^2")) != MF_OK) {
      p->maxrho_cap = 0;
      return s;
    }
    p->maxrho_cap = p->n_sel;
  }
  cudaError_t e = cudaMemsetAsync(followed, 0, p->n_tmpl * sizeof(int32_t), p->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->n_coinc, 0, sizeof(unsigned long long), p->st);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_coincide reset");
  mf::CoincArgs a{};
  a.slots = p->slots;
  a.sel = p->sel_copy;
  a.n_sel = p->n_sel;
  a.n_win = p->n_win;
  a.window = p->d.window;
  a.ring_begin = p->d.valid_begin;
  a.ring_end = p->d.valid_end;
  a.shift = c->shift_samples;
  a.n_shifts = c->n_shifts;
  a.coinc_window = c->window_samples;
  a.rho_c_thr2 = (float)(c->rho_c_thr * c->rho_c_thr);
  a.rho_c_store2 = (float)(c->rho_c_store * c->rho_c_store);
  a.followed = followed;
  a.coincs = p->coincs;
  a.coinc_cap = p->coinc_cap;
  a.n_coinc = p->n_coinc;
  LaunchScope ls(p);
  e = mf::launch_coinc(a, p->maxrho, p->st);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_coincide kernels");
  p->coinc_done = true;
  return MF_OK;
}

mf_status mf_get_coincs(mf_plan_t p, mf_coinc* out, int64_t cap, int64_t* n_found) {
  if (!p || !n_found || (cap > 0 && !out)) return fail(p, MF_EINVAL, "mf_get_coincs: null argument");
  if (!p->coinc_done) return fail(p, MF_ESTATE, "mf_get_coincs: no coincidence run");
  unsigned long long n = 0;
  cudaError_t e = cudaMemcpyAsync(&n, p->n_coinc, sizeof(n), cudaMemcpyDeviceToHost, p->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_get_coincs count");
  *n_found = (int64_t)n;
  const int64_t have = std::min<int64_t>((int64_t)n, p->coinc_cap);
  const int64_t m = std::min<int64_t>(have, cap);
  if (m > 0) try {  // a count-only call (cap 0) copies nothing; no allocation failure crosses the ABI
    std::unique_ptr<mf_coinc[]> rec(new mf_coinc[have]);
    e = cudaMemcpyAsync(rec.get(), p->coincs, have * sizeof(mf_coinc), cudaMemcpyDeviceToHost, p->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
    if (e != cudaSuccess) return cuda_fail(p, e, "mf_get_coincs copy");
    // order by (tmpl, shift, sample0, sample1) through packed keys: tmpl and shift are non-negative int32;
    // the samples are compared as int64 (sign bit flipped, so that unsigned order is signed order)
    struct Key {
      uint64_t ts, s0, s1;
      int64_t i;
    };
    std::vector<Key> key((size_t)have);
    for (int64_t i = 0; i < have; ++i) {
      const mf_coinc& c = rec[i];
      key[(size_t)i] = Key{((uint64_t)(uint32_t)c.tmpl << 32) | (uint32_t)c.shift,
                           (uint64_t)c.sample0 ^ (uint64_t(1) << 63), (uint64_t)c.sample1 ^ (uint64_t(1) << 63), i};
    }
    auto less = [](const Key& a, const Key& b) {
      if (a.ts != b.ts) return a.ts < b.ts;
      if (a.s0 != b.s0) return a.s0 < b.s0;
      return a.s1 < b.s1;
    };
    // counting sort by template id (ids are < n_tmpl), then each template's few records by the rest of the key
    std::vector<int64_t> start((size_t)p->n_tmpl + 1, 0);
    bool ids_ok = true;
    for (int64_t i = 0; i < have && ids_ok; ++i) {
      const int32_t t = rec[i].tmpl;
      if (t < 0 || t >= p->n_tmpl) ids_ok = false;
      else ++start[(size_t)t + 1];
    }
    if (ids_ok) {
      for (int64_t t = 0; t < p->n_tmpl; ++t) start[(size_t)t + 1] += start[(size_t)t];
      std::vector<Key> by((size_t)have);
      std::vector<int64_t> pos(start.begin(), start.end() - 1);
      for (int64_t i = 0; i < have; ++i) by[(size_t)pos[(size_t)rec[i].tmpl]++] = key[(size_t)i];
      for (int64_t t = 0; t < p->n_tmpl; ++t)
        if (start[(size_t)t + 1] - start[(size_t)t] > 1)
          std::sort(by.begin() + start[(size_t)t], by.begin() + start[(size_t)t + 1], less);
      key.swap(by);
    } else {
      std::sort(key.begin(), key.end(), less);
    }
    for (int64_t j = 0; j < m; ++j) out[j] = rec[key[(size_t)j].i];
  } catch (const std::bad_alloc&) {
    return fail(p, MF_ENOMEM, "mf_get_coincs: host memory for " + std::to_string(have) + " records");
  }
  if ((int64_t)n > cap || (int64_t)n > p->coinc_cap)
    return fail(p, MF_EOVERFLOW, "mf_get_coincs: " + std::to_string(n) + " coincidences exceed the buffer");
  return MF_OK;
}

mf_status mf_set_nbhd(mf_plan_t p, const int64_t* ptr, const int32_t* idx, int64_t n_coarse, int on_device) {
  if (!p || !ptr || (n_coarse > 0 && !idx)) return fail(p, MF_EINVAL, "mf_set_nbhd: null argument");
  if (n_coarse < 0) return fail(p, MF_EINVAL, "mf_set_nbhd: negative n_coarse");
  int64_t nnz = 0;
  cudaError_t e = cudaSuccess;
  if (on_device) {
    e = cudaMemcpy(&nnz, ptr + n_coarse, sizeof(int64_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(p, e, "mf_set_nbhd read nnz");
  } else {
    nnz = ptr[n_coarse];
    if (ptr[0] != 0) return fail(p, MF_EINVAL, "mf_set_nbhd: ptr[0] must be 0");
    for (int64_t c = 0; c < n_coarse; ++c)
      if (ptr[c + 1] < ptr[c]) return fail(p, MF_EINVAL, "mf_set_nbhd: ptr must be non-decreasing");
    for (int64_t i = 0; i < nnz; ++i)
      if (idx[i] < 0 || idx[i] >= p->n_tmpl) return fail(p, MF_EINVAL, "mf_set_nbhd: fine id out of range");
  }
  if (nnz < 0) return fail(p, MF_EINVAL, "mf_set_nbhd: negative nnz");
  mf_status s;
  if ((s = dalloc(p, &p->nb_ptr, (n_coarse + 1) * sizeof(int64_t), "nbhd ptr")) != MF_OK ||
      (s = dalloc(p, &p->nb_idx, std::max<int64_t>(nnz, 1) * sizeof(int32_t), "nbhd idx")) != MF_OK)
    return s;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  e = cudaMemcpy(p->nb_ptr, ptr, (n_coarse + 1) * sizeof(int64_t), kind);
  if (e == cudaSuccess && nnz > 0) e = cudaMemcpy(p->nb_idx, idx, nnz * sizeof(int32_t), kind);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_set_nbhd copy");
  p->n_coarse = n_coarse;
  return MF_OK;
}

mf_status mf_nbhd_union(mf_plan_t p, const int32_t* followed, int32_t* subset, int64_t* n_subset) {
  if (!p || !followed || !subset || !n_subset) return fail(p, MF_EINVAL, "mf_nbhd_union: null argument");
  if (!p->nb_ptr) return fail(p, MF_ESTATE, "mf_nbhd_union: no neighbourhood map");
  if (p->n_tmpl < 1) return fail(p, MF_ESTATE, "mf_nbhd_union: no bank");
  mf_status s;
  if (p->flags_cap < p->n_tmpl) {
    p->flags_cap = 0;
    if ((s = dalloc(p, &p->flags, p->n_tmpl * sizeof(int32_t), "union flags")) != MF_OK ||
        (s = dalloc(p, &p->ubc, ((p->n_tmpl + 1023) / 1024 + 1) * sizeof(int64_t), "union blocks")) != MF_OK ||
        (s = dalloc(p, &p->ucount, sizeof(int64_t), "union count")) != MF_OK)
      return s;
    p->flags_cap = p->n_tmpl;
  }
  LaunchScope ls(p);
  cudaError_t e = mf::launch_union(p->nb_ptr, p->nb_idx, p->n_coarse, followed, p->flags, p->n_tmpl, subset,
                                   p->ucount, p->ubc, p->st);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_nbhd_union kernels");
  int64_t n = 0;
  e = cudaMemcpyAsync(&n, p->ucount, sizeof(int64_t), cudaMemcpyDeviceToHost, p->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
  if (e != cudaSuccess) return cuda_fail(p, e, "mf_nbhd_union count");
  *n_subset = n;
  return MF_OK;
}

}  // extern "C"

namespace mf {

int plan_batch(const mf_plan_s* p) { return p ? p->batch : 0; }

int filter_fused(mf_plan_s* const* plans, const void* const* dtilde, const int64_t* ld, int n_plans, void* scratch,
                 int64_t scratch_series, const CUtensorMap& scratch_map, cudaStream_t st, std::string* err) {
  auto bad = [&](mf_status s, const std::string& m) {
    if (err) *err = m;
    return s;
  };
  auto from_plan = [&](mf_plan_s* p, mf_status s) {
    if (err) *err = p->err;
    return s;
  };
  if (n_plans < 1 || n_plans > kMaxParts || !plans || !dtilde || !ld || !scratch)
    return bad(MF_EINVAL, "fused filter: bad arguments");
  mf_plan_s* p0 = plans[0];
  for (int i = 0; i < n_plans; ++i) {
    mf_plan_s* p = plans[i];
    if (!p || !dtilde[i]) return bad(MF_EINVAL, "fused filter: null plan or data");
    if (!p->psd_set || !p->bank || p->n_tmpl == 0) return bad(MF_ESTATE, "fused filter: a plan has no PSD or bank");
    if (ld[i] < p->nb) return bad(MF_EINVAL, "fused filter: ld_dtilde < N/2+1");
    if (p->d.n != p0->d.n || p->bank_dtype != MF_F32 || p->data_dtype != MF_F32 || p->inter != p0->inter ||
        p->d.window != p0->d.window || p->n_win != p0->n_win)
      return bad(MF_EINVAL, "fused filter: the plans differ in N, window or intermediate, or store 16-bit data");
    if (p->d.n_det > scratch_series) return bad(MF_EINVAL, "fused filter: scratch smaller than a plan's rows");
  }
  const int64_t launches_before = launch_count();
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < n_plans; ++i) {
    mf_plan_s* p = plans[i];
    mf_status s = ensure_slots(p, p->n_tmpl);
    if (s != MF_OK) return from_plan(p, s);
    if (!p->scale_valid) {  // first use: the template scales are written on the plan's own stream
      if ((s = refresh_scale(p)) != MF_OK) return from_plan(p, s);
      if ((e = cudaStreamSynchronize(p->st)) != cudaSuccess) return bad(MF_ECUDA, "fused filter: template scales");
    }
    e = cudaMemcpyAsync(p->sel_copy, p->sel_all, p->n_tmpl * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
      e = launch_prep_cols(static_cast<const float2*>(dtilde[i]), ld[i], p->w_dev, p->n1, p->n2, p->d.n_det, p->q,
                           p->ld_q, p->slots, (int64_t)p->d.n_det * p->n_tmpl * p->n_win, st, 1.0 / p->sigma_ref);
    if (e != cudaSuccess) return bad(MF_ECUDA, std::string("fused filter prep: ") + cudaGetErrorString(e));
  }
  FilterArgs a{};
  a.n = p0->d.n;
  a.n1 = p0->n1;
  a.n2 = p0->n2;
  a.n_det = p0->d.n_det;
  a.nb = p0->nb;
  a.bank_type = kBankF32;
  a.scratch = static_cast<float2*>(scratch);
  a.window = p0->d.window;
  a.n_win = p0->n_win;
  a.status = p0->status;
  a.tw1 = p0->tw;
  a.tw2 = p0->tw + 1024;
  a.tw4 = p0->tw4;
  a.q_type = kBankF32;
  a.inter = p0->inter;
  // the work queue: (plan, template, row) series in order, cut into launches of at most scratch_series
  int i = 0;
  int64_t t = 0;
  bool first = true;
  while (i < n_plans) {
    FilterParts ps{};
    int64_t ser = 0;
    while (i < n_plans && ps.n < kMaxParts) {
      mf_plan_s* p = plans[i];
      const int64_t rows = p->d.n_det;
      const int64_t cnt = std::min<int64_t>((scratch_series - ser) / rows, p->n_tmpl - t);
      if (cnt < 1) break;
      FilterPart& f = ps.p[ps.n++];
      f.bank = p->bank;
      f.ld_bank = p->ld_bank;
      f.q = p->q;
      f.ld_q = p->ld_q;
      f.sel = p->sel_copy;
      f.inv_sigma = p->ratio_dev;
      f.thr_raw = p->thr_raw_dev;
      f.pos0 = t;
      f.count = (int)cnt;
      f.n_det = (int)rows;
      f.valid_begin = p->d.valid_begin;
      f.valid_end = p->d.valid_end;
      f.n_sel_total = p->n_tmpl;
      f.slots = p->slots;
      f.row_valid = p->row_valid;
      f.series0 = (int)ser;
      ser += cnt * rows;
      t += cnt;
      if (t == p->n_tmpl) {
        ++i;
        t = 0;
      }
    }
    ps.n_series = (int)ser;
    a.first_batch = first ? 1 : 0;
    first = false;
    const bool prof =
        p0->prof && p0->prof_count++ % p0->prof_stride == 0 && (int)p0->samples.size() < kProfBatches;
    const int e0 = prof ? (int)p0->samples.size() * 3 : 0;
    if (prof) cudaEventRecord(p0->ev[e0], st);
    if ((e = launch_filter2_fused(a, ps, scratch_map, st, prof ? p0->ev[e0 + 1] : nullptr)) != cudaSuccess)
      return bad(MF_ECUDA, std::string("fused filter launch: ") + cudaGetErrorString(e));
    if (prof) {
      cudaEventRecord(p0->ev[e0 + 2], st);
      p0->samples.push_back({e0, ser});
    }
  }
  for (int j = 0; j < n_plans; ++j) {
    mf_plan_s* p = plans[j];
    e = launch_compact(p->slots, p->d.n_det, p->n_tmpl, p->n_win, p->d.window, p->sel_copy, p->trig,
                       p->d.max_triggers, p->count, p->bc, p->bc_cap, st);
    if (e != cudaSuccess) return bad(MF_ECUDA, std::string("fused filter compaction: ") + cudaGetErrorString(e));
    p->n_sel = p->n_tmpl;
    p->filtered = true;
    p->coinc_done = false;
  }
  p0->stats.launches += launch_count() - launches_before;
  return MF_OK;
}

}  // namespace mf
