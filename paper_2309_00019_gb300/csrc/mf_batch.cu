// Long data in overlapping segments, one plan per template-length class
// (include/mf.h, "long data in overlapping segments"; Sec. V.C analyses the
// data in overlapping segments).  This file is host runtime plus one gather
// kernel: it cuts the stream into each class's segment rows, runs the
// plan's own transform and filter kernels on them, and maps the triggers
// back to stream time.  Classes run one after another, on concurrent streams,
// or as one captured CUDA graph; an autotuner picks each class's segment
// length and launch batch from timed probe runs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "../../include/mf.h"
#include "mf_internal.h"

namespace {

// out[r][j] = x[d][s stride + j] for row r = s n_det + d, zero past the stream
__global__ void k_segments(const float* __restrict__ x, int64_t ld, int n_det, int64_t n_samples, int64_t stride,
                           int lg_n, int64_t rows, float* __restrict__ out) {
  const int64_t total = rows << lg_n;
  const int64_t mask = (int64_t(1) << lg_n) - 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i >> lg_n, j = i & mask;
    const int64_t s = r / n_det;
    const int d = (int)(r - s * n_det);
    const int64_t g = s * stride + j;
    out[i] = g < n_samples ? __ldg(x + d * ld + g) : 0.f;
  }
}

int sm_count_b() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

int ilog2(int64_t n) {
  int l = 0;
  while ((int64_t(1) << l) < n) ++l;
  return l;
}

bool pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }

}  // namespace

struct mf_batch_s {
  mf_batch_desc d{};
  std::vector<double> len;
  std::string err;
  cudaStream_t user = nullptr, main = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<double> psd;
  int64_t n_psd = 0;
  struct Cls {
    int64_t L = 0, n = 0, stride = 0, n_seg = 0, rows = 0, ld = 0;
    int32_t batch = 0;
    double est_ms = 0.0;
    mf_plan_t plan = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr, join = nullptr;
    bool timed = false;
    float* seg = nullptr;
    float2* fd = nullptr;
  };
  std::vector<Cls> cls;
  // fused runs: the scratch of one launch pair (fscratch_series series of N = fscratch_n) and its pass-2 map
  float2* fscratch = nullptr;
  int64_t fscratch_series = 0, fscratch_n = 0;
  CUtensorMap fmap{};
  // captured graph of one MF_RUN_STREAMS (or MF_RUN_FUSED) pass
  cudaGraphExec_t exec = nullptr;
  int32_t g_mode = -1;
  const float* g_strain = nullptr;
  int64_t g_ld = 0;
  std::vector<uint64_t> g_fp;
  bool ran = false;
};

namespace {

thread_local std::string g_berr;

mf_status bfail(mf_batch_t b, mf_status s, const std::string& m) {
  if (b) b->err = m; else g_berr = m;
  return s;
}

mf_status bcuda(mf_batch_t b, cudaError_t e, const char* what) {
  return bfail(b, MF_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

mf_status bplan(mf_batch_t b, mf_plan_t p, mf_status s, const char* what) {
  return bfail(b, s, std::string(what) + ": " + mf_last_error(p));
}

void free_class(mf_batch_s::Cls& c) {
  if (c.plan) mf_destroy(c.plan);
  c.plan = nullptr;
  if (c.seg) cudaFree(c.seg);
  if (c.fd) cudaFree(c.fd);
  c.seg = nullptr;
  c.fd = nullptr;
}

// geometry of a class at segment length n (false if inadmissible)
bool geometry(const mf_batch_s* b, int c, int64_t n, int64_t* L, int64_t* stride, int64_t* n_seg) {
  const int64_t W = b->d.window;
  const int64_t l = (int64_t)std::ceil(b->len[c] * b->d.fs - 1e-9);
  const int64_t Lw = (l + W - 1) / W * W;
  const int64_t s = (n - Lw) / W * W;
  if (s <= 0 || Lw >= b->d.n_samples) return false;
  *L = Lw;
  *stride = s;
  *n_seg = (b->d.n_samples - Lw + s - 1) / s;
  return *n_seg * b->d.n_det <= 65536;
}

std::vector<double> class_psd(const mf_batch_s* b, int64_t n) {
  const int64_t step = b->n_psd / n;
  std::vector<double> out(n / 2 + 1);
  for (int64_t k = 0; k <= n / 2; ++k) out[k] = b->psd[k * step];
  return out;
}

mf_status make_plan(mf_batch_s* b, int64_t n, int64_t rows, int64_t vb, int64_t max_trig, cudaStream_t st,
                    mf_plan_t* out) {
  mf_plan_desc pd{};
  pd.fs = b->d.fs;
  pd.n = n;
  pd.n_det = (int32_t)rows;
  pd.f_low = b->d.f_low;
  pd.f_high = b->d.f_high;
  pd.dtype = MF_F32;
  pd.snr_thr = b->d.snr_thr;
  pd.window = b->d.window;
  pd.valid_begin = vb;
  pd.valid_end = n;
  pd.max_triggers = max_trig;
  pd.cuda_stream = st;
  mf_plan_t p = nullptr;
  mf_status s = mf_plan(&p, &pd);
  if (s != MF_OK) return bfail(b, s, std::string("class plan: ") + mf_last_error(nullptr));
  std::vector<double> ps = class_psd(b, n);
  if ((s = mf_set_psd(p, ps.data(), (int64_t)ps.size())) != MF_OK) {
    mf_status r = bplan(b, p, s, "class PSD");
    mf_destroy(p);
    return r;
  }
  *out = p;
  return MF_OK;
}

mf_status enqueue_spectra(mf_batch_s* b, mf_batch_s::Cls& c, const float* strain, int64_t ld);

mf_status enqueue_class(mf_batch_s* b, mf_batch_s::Cls& c, const float* strain, int64_t ld) {
  mf_status s = enqueue_spectra(b, c, strain, ld);
  if (s != MF_OK) return s;
  s = mf_filter(c.plan, c.fd, c.ld, nullptr, -1);
  if (s != MF_OK) return bplan(b, c.plan, s, "class filter");
  return MF_OK;
}

bool has_bank(const mf_batch_s::Cls& c) { return c.plan && mf::plan_templates(c.plan) > 0; }

struct Probe {  // the autotuner's timing events
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  Probe() {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
  }
  ~Probe() {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
};

// Time class ci at segment length n: 2 filter calls of a zero probe bank on the class's real row
// count for each of 3 launch batches (the largest fitting 128 MB, 256 MB and 1 GB of
// intermediate).  *ms = the least n_tmpl x time per template (+inf if n is inadmissible), *batch its batch.
mf_status probe_class(mf_batch_t b, int ci, int64_t n, int64_t n_tmpl, Probe& pr, double* ms_out, int32_t* batch) {
  *ms_out = INFINITY;
  int64_t L, stride, n_seg;
  if (!geometry(b, ci, n, &L, &stride, &n_seg)) return MF_OK;
  const int64_t rows = n_seg * b->d.n_det;
  const int64_t per = rows * n * (int64_t)sizeof(float2);
  std::vector<int32_t> cands;
  for (int64_t budget : {int64_t(128) << 20, int64_t(256) << 20, int64_t(1) << 30}) {
    const int32_t bb = (int32_t)std::max<int64_t>(1, std::min<int64_t>({budget / per, n_tmpl, 256}));
    if (std::find(cands.begin(), cands.end(), bb) == cands.end()) cands.push_back(bb);
  }
  const int32_t probe = std::max<int32_t>(8, std::min<int32_t>(64, 2 * *std::max_element(cands.begin(), cands.end())));
  mf_plan_t p = nullptr;
  mf_status s = make_plan(b, n, rows, L, 1024, b->main, &p);
  if (s != MF_OK) return s;
  float2* fd = nullptr;
  const int64_t ld = (n / 2 + 1 + 63) / 64 * 64;
  cudaError_t ce = cudaMalloc((void**)&fd, (size_t)rows * ld * sizeof(float2));
  if (ce == cudaSuccess) ce = cudaMemsetAsync(fd, 0, (size_t)rows * ld * sizeof(float2), b->main);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    if (fd) cudaFree(fd);
    mf_destroy(p);
    return bfail(b, MF_ENOMEM, "mf_batch_autotune probe data");
  }
  s = mf_bank_reserve(p, MF_F32, probe);
  for (int32_t bb : cands) {
    if (s == MF_OK) s = mf_set_batch(p, bb);
    if (s == MF_OK) s = mf_filter(p, fd, ld, nullptr, -1);  // warm-up (tables, tensor maps)
    if (s != MF_OK) break;
    cudaEventRecord(pr.e0, b->main);
    for (int it = 0; it < 2 && s == MF_OK; ++it) s = mf_filter(p, fd, ld, nullptr, -1);
    cudaEventRecord(pr.e1, b->main);
    if (cudaEventSynchronize(pr.e1) != cudaSuccess || s != MF_OK) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, pr.e0, pr.e1);
    const double est = (double)ms / (2.0 * probe) * (double)n_tmpl;
    if (est < *ms_out) {
      *ms_out = est;
      *batch = bb;
    }
  }
  if (s != MF_OK) s = bplan(b, p, s, "mf_batch_autotune probe");
  cudaFree(fd);
  mf_destroy(p);
  return s;
}

// spectra of class c's segment rows: gather from the stream, then the plan's real-input transform
mf_status enqueue_spectra(mf_batch_s* b, mf_batch_s::Cls& c, const float* strain, int64_t ld) {
  const int64_t total = c.rows * c.n;
  const int grid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)sm_count_b() * 8);
  k_segments<<<grid, 256, 0, c.st>>>(strain, ld, b->d.n_det, b->d.n_samples, c.stride, ilog2(c.n), c.rows, c.seg);
  mf::add_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return bcuda(b, e, "segment gather");
  mf_status s = mf_strain_to_fd(c.plan, c.seg, c.n, c.fd, c.ld);
  if (s != MF_OK) return bplan(b, c.plan, s, "segment spectra");
  return MF_OK;
}

// series per fused launch: the largest launch pair a class makes on its own (its batch x rows)
int64_t fused_series(const mf_batch_s* b) {
  int64_t n = 0;
  for (const auto& c : b->cls)
    if (has_bank(c)) n = std::max<int64_t>(n, (int64_t)mf::plan_batch(c.plan) * c.rows);
  return n;
}

// the fused run's scratch (and its pass-2 map) for the classes' common segment length
mf_status ensure_fused(mf_batch_s* b) {
  int64_t n = 0;
  for (const auto& c : b->cls) {
    if (!has_bank(c)) continue;
    if (n != 0 && c.n != n)
      return bfail(b, MF_ESTATE, "mf_batch_run: a fused run needs one segment length for every class with a bank");
    n = c.n;
  }
  const int64_t series = fused_series(b);
  if (b->fscratch && b->fscratch_n == n && b->fscratch_series == series) return MF_OK;
  cudaStreamSynchronize(b->main);  // the old scratch may still be read
  if (b->fscratch) cudaFree(b->fscratch);
  b->fscratch = nullptr;
  b->fscratch_series = 0;
  cudaError_t e = cudaMalloc((void**)&b->fscratch, (size_t)series * n * sizeof(float2));
  if (e != cudaSuccess) {
    cudaGetLastError();
    b->fscratch = nullptr;
    return bfail(b, MF_ENOMEM, std::string("mf_batch_run fused scratch: ") + cudaGetErrorString(e));
  }
  e = mf::encode_scratch_map(n, b->fscratch, series, &b->fmap);
  if (e != cudaSuccess) return bcuda(b, e, "mf_batch_run fused scratch map");
  b->fscratch_n = n;
  b->fscratch_series = series;
  return MF_OK;
}

// one fused pass: every class's spectra on its own stream, then the classes' work queue on the main stream
mf_status enqueue_fused(mf_batch_s* b, const float* strain, int64_t ld) {
  cudaError_t e = cudaEventRecord(b->ev_in, b->main);
  std::vector<mf_plan_t> plans;
  std::vector<const void*> fd;
  std::vector<int64_t> lds;
  for (auto& c : b->cls) {
    if (!has_bank(c) || e != cudaSuccess) continue;
    e = cudaStreamWaitEvent(c.st, b->ev_in, 0);
    if (e != cudaSuccess) break;
    mf_status s = enqueue_spectra(b, c, strain, ld);
    if (s != MF_OK) return s;
    e = cudaEventRecord(c.join, c.st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->main, c.join, 0);
    plans.push_back(c.plan);
    fd.push_back(c.fd);
    lds.push_back(c.ld);
  }
  if (e != cudaSuccess) return bcuda(b, e, "mf_batch_run fused order");
  std::string m;
  const int s = mf::filter_fused(plans.data(), fd.data(), lds.data(), (int)plans.size(), b->fscratch,
                                 b->fscratch_series, b->fmap, b->main, &m);
  if (s != MF_OK) return bfail(b, (mf_status)s, m);
  return MF_OK;
}

}  // namespace

extern "C" {

const char* mf_batch_last_error(mf_batch_t b) { return b ? b->err.c_str() : g_berr.c_str(); }

mf_status mf_batch_create(mf_batch_t* out, const mf_batch_desc* desc) {
  if (!out || !desc) return bfail(nullptr, MF_EINVAL, "mf_batch_create: null argument");
  const mf_batch_desc& d = *desc;
  if (!(d.fs > 0) || d.n_det < 1 || d.n_det > 8 || d.n_samples < 1 || d.window < 1 || d.n_class < 1 ||
      d.n_class > 8 || !d.class_len || !(d.snr_thr > 0) || !(d.f_high > d.f_low) || d.max_triggers < 1)
    return bfail(nullptr, MF_EINVAL, "mf_batch_create: bad description");
  for (int c = 0; c < d.n_class; ++c)
    if (!(d.class_len[c] > 0) || (c > 0 && !(d.class_len[c] > d.class_len[c - 1])))
      return bfail(nullptr, MF_EINVAL, "mf_batch_create: class lengths must be positive and increasing");
  mf_batch_s* b = new (std::nothrow) mf_batch_s();
  if (!b) return bfail(nullptr, MF_ENOMEM, "mf_batch_create: host allocation");
  b->d = d;
  b->len.assign(d.class_len, d.class_len + d.n_class);
  b->d.class_len = b->len.data();
  b->user = (cudaStream_t)d.cuda_stream;
  b->cls.resize(d.n_class);
  cudaError_t e = cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
  for (auto& c : b->cls) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c.st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&c.t0);
    if (e == cudaSuccess) e = cudaEventCreate(&c.t1);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.join, cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    mf_status s = bcuda(nullptr, e, "mf_batch_create streams");
    mf_batch_destroy(b);
    return s;
  }
  *out = b;
  return MF_OK;
}

void mf_batch_destroy(mf_batch_t b) {
  if (!b) return;
  if (b->main) cudaStreamSynchronize(b->main);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (auto& c : b->cls) {
    free_class(c);
    if (c.st) cudaStreamDestroy(c.st);
    if (c.t0) cudaEventDestroy(c.t0);
    if (c.t1) cudaEventDestroy(c.t1);
    if (c.join) cudaEventDestroy(c.join);
  }
  if (b->fscratch) cudaFree(b->fscratch);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->main) cudaStreamDestroy(b->main);
  delete b;
}

mf_status mf_batch_set_psd(mf_batch_t b, const double* psd, int64_t n_psd) {
  if (!b || !psd) return bfail(b, MF_EINVAL, "mf_batch_set_psd: null argument");
  if (!pow2(n_psd) || n_psd < 4096) return bfail(b, MF_EINVAL, "mf_batch_set_psd: n_psd must be a power of two >= 2^12");
  for (auto& c : b->cls)
    if (c.plan && c.n > n_psd) return bfail(b, MF_EINVAL, "mf_batch_set_psd: grid coarser than a class's segments");
  b->psd.assign(psd, psd + n_psd / 2 + 1);
  b->n_psd = n_psd;
  for (auto& c : b->cls) {
    if (!c.plan) continue;
    std::vector<double> ps = class_psd(b, c.n);
    mf_status s = mf_set_psd(c.plan, ps.data(), (int64_t)ps.size());
    if (s != MF_OK) return bplan(b, c.plan, s, "mf_batch_set_psd");
  }
  return MF_OK;
}

mf_status mf_batch_set_segment(mf_batch_t b, int32_t ci, int64_t n, int32_t per_launch) {
  if (!b || ci < 0 || ci >= b->d.n_class) return bfail(b, MF_EINVAL, "mf_batch_set_segment: class");
  if (b->n_psd == 0) return bfail(b, MF_ESTATE, "mf_batch_set_segment: PSD not set");
  if (!pow2(n) || n < 4096 || n > mf::kMaxN || n > b->n_psd)
    return bfail(b, MF_EINVAL, "mf_batch_set_segment: n must be a power of two in [2^12, min(2^20, n_psd)]");
  if (per_launch < 0) return bfail(b, MF_EINVAL, "mf_batch_set_segment: templates per launch");
  mf_batch_s::Cls& c = b->cls[ci];
  int64_t L, stride, n_seg;
  if (!geometry(b, ci, n, &L, &stride, &n_seg))
    return bfail(b, MF_EINVAL, "mf_batch_set_segment: segment too short for the class (or too many rows)");
  cudaStreamSynchronize(c.st);
  free_class(c);
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  c.n = n;
  c.L = L;
  c.stride = stride;
  c.n_seg = n_seg;
  c.rows = n_seg * b->d.n_det;
  c.ld = (n / 2 + 1 + 63) / 64 * 64;
  c.batch = per_launch;
  c.timed = false;
  mf_status s = make_plan(b, n, c.rows, L, b->d.max_triggers, c.st, &c.plan);
  if (s != MF_OK) return s;
  std::vector<int64_t> rv(2 * c.rows);
  for (int64_t r = 0; r < c.rows; ++r) {
    const int64_t seg = r / b->d.n_det;
    rv[2 * r] = L;
    rv[2 * r + 1] = std::min<int64_t>(L + stride, b->d.n_samples - seg * stride);
  }
  if ((s = mf_set_row_valid(c.plan, rv.data())) != MF_OK) return bplan(b, c.plan, s, "class row ranges");
  if (per_launch > 0 && (s = mf_set_batch(c.plan, per_launch)) != MF_OK) return bplan(b, c.plan, s, "class batch");
  cudaError_t e = cudaMalloc((void**)&c.seg, (size_t)c.rows * n * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c.fd, (size_t)c.rows * c.ld * sizeof(float2));
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_class(c);
    return bfail(b, MF_ENOMEM, std::string("mf_batch_set_segment buffers: ") + cudaGetErrorString(e));
  }
  return MF_OK;
}

mf_status mf_batch_autotune(mf_batch_t b, const int64_t* n_tmpl) {
  if (!b || !n_tmpl) return bfail(b, MF_EINVAL, "mf_batch_autotune: null argument");
  if (b->n_psd == 0) return bfail(b, MF_ESTATE, "mf_batch_autotune: PSD not set");
  Probe pr;
  mf_status result = MF_OK;
  for (int ci = 0; ci < b->d.n_class && result == MF_OK; ++ci) {
    if (n_tmpl[ci] <= 0) continue;
    double best = INFINITY;
    int64_t best_n = 0;
    int32_t best_b = 0;
    for (int64_t n = 4096; n <= std::min<int64_t>(mf::kMaxN, b->n_psd) && result == MF_OK; n *= 2) {
      double ms = INFINITY;
      int32_t bb = 0;
      result = probe_class(b, ci, n, n_tmpl[ci], pr, &ms, &bb);
      if (ms < best) {
        best = ms;
        best_n = n;
        best_b = bb;
      }
    }
    if (result != MF_OK) break;
    if (best_n == 0) {
      result = bfail(b, MF_EINVAL, "mf_batch_autotune: no admissible segment length for class " + std::to_string(ci));
      break;
    }
    result = mf_batch_set_segment(b, ci, best_n, best_b);
    if (result == MF_OK) b->cls[ci].est_ms = best;
  }
  return result;
}

mf_status mf_batch_autotune_fused(mf_batch_t b, const int64_t* n_tmpl) {
  if (!b || !n_tmpl) return bfail(b, MF_EINVAL, "mf_batch_autotune_fused: null argument");
  if (b->n_psd == 0) return bfail(b, MF_ESTATE, "mf_batch_autotune_fused: PSD not set");
  Probe pr;
  const int nc = b->d.n_class;
  double best = INFINITY;
  int64_t best_n = 0;
  std::vector<double> best_ms(nc, 0.0), ms(nc, 0.0);
  std::vector<int32_t> best_b(nc, 0), bb(nc, 0);
  for (int64_t n = 4096; n <= std::min<int64_t>(mf::kMaxN, b->n_psd); n *= 2) {
    bool fits = true;  // probe only lengths that every class with templates admits
    for (int ci = 0; ci < nc; ++ci) {
      int64_t L, stride, n_seg;
      if (n_tmpl[ci] > 0 && !geometry(b, ci, n, &L, &stride, &n_seg)) fits = false;
    }
    if (!fits) continue;
    double total = 0.0;
    bool any = false;
    for (int ci = 0; ci < nc && std::isfinite(total); ++ci) {
      if (n_tmpl[ci] <= 0) continue;
      ms[ci] = INFINITY;
      mf_status s = probe_class(b, ci, n, n_tmpl[ci], pr, &ms[ci], &bb[ci]);
      if (s != MF_OK) return s;
      total += ms[ci];  // +inf when the class does not fit segments of n
      any = true;
    }
    if (any && total < best) {
      best = total;
      best_n = n;
      best_ms = ms;
      best_b = bb;
    }
  }
  if (best_n == 0) return bfail(b, MF_EINVAL, "mf_batch_autotune_fused: no segment length admissible for every class");
  for (int ci = 0; ci < nc; ++ci) {
    if (n_tmpl[ci] <= 0) continue;
    mf_status s = mf_batch_set_segment(b, ci, best_n, best_b[ci]);
    if (s != MF_OK) return s;
    b->cls[ci].est_ms = best_ms[ci];
  }
  return MF_OK;
}

mf_status mf_batch_segment(mf_batch_t b, int32_t ci, int64_t* n, int64_t* tmpl_len, int64_t* stride, int64_t* n_seg,
                           double* est_ms, double* run_ms) {
  if (!b || ci < 0 || ci >= b->d.n_class) return bfail(b, MF_EINVAL, "mf_batch_segment: class");
  const mf_batch_s::Cls& c = b->cls[ci];
  if (n) *n = c.n;
  if (tmpl_len) *tmpl_len = c.L;
  if (stride) *stride = c.stride;
  if (n_seg) *n_seg = c.n_seg;
  if (est_ms) *est_ms = c.est_ms;
  if (run_ms) {
    float ms = 0.f;
    if (c.timed && cudaEventSynchronize(c.t1) == cudaSuccess) cudaEventElapsedTime(&ms, c.t0, c.t1);
    *run_ms = ms;
  }
  return MF_OK;
}

mf_status mf_batch_plan(mf_batch_t b, int32_t ci, mf_plan_t* plan) {
  if (!b || !plan || ci < 0 || ci >= b->d.n_class) return bfail(b, MF_EINVAL, "mf_batch_plan: argument");
  if (!b->cls[ci].plan) return bfail(b, MF_ESTATE, "mf_batch_plan: segment length not set");
  *plan = b->cls[ci].plan;
  return MF_OK;
}

mf_status mf_batch_run(mf_batch_t b, const float* strain, int64_t ld, int32_t mode) {
  if (!b || !strain) return bfail(b, MF_EINVAL, "mf_batch_run: null argument");
  if (ld < b->d.n_samples) return bfail(b, MF_EINVAL, "mf_batch_run: ld < n_samples");
  if (mode < MF_RUN_SERIAL || mode > MF_RUN_FUSED_GRAPH) return bfail(b, MF_EINVAL, "mf_batch_run: mode");
  bool any = false;
  for (auto& c : b->cls) any |= has_bank(c);
  if (!any) return bfail(b, MF_ESTATE, "mf_batch_run: no class has a bank");
  const bool fused = mode == MF_RUN_FUSED || mode == MF_RUN_FUSED_GRAPH;
  mf_status s = MF_OK;
  if (fused && (s = ensure_fused(b)) != MF_OK) return s;
  cudaError_t e = cudaEventRecord(b->ev_in, b->user);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->main, b->ev_in, 0);
  if (e != cudaSuccess) return bcuda(b, e, "mf_batch_run order");
  if (mode == MF_RUN_GRAPH || mode == MF_RUN_FUSED_GRAPH) {
    auto fingerprint = [&]() {
      std::vector<uint64_t> fp;
      for (auto& c : b->cls) fp.push_back(has_bank(c) ? mf::plan_fingerprint(c.plan) : 0);
      if (fused) {
        fp.push_back((uint64_t)(uintptr_t)b->fscratch);
        fp.push_back((uint64_t)b->fscratch_series);
      }
      return fp;
    };
    std::vector<uint64_t> fp = fingerprint();
    bool ready = b->ran;
    for (auto& c : b->cls)
      if (has_bank(c)) ready = ready && mf::plan_capturable(c.plan);
    if (!ready) {  // one uncaptured pass does every first-call set-up (host syncs, allocations)
      s = mf_batch_run(b, strain, ld, fused ? MF_RUN_FUSED : MF_RUN_STREAMS);
      if (s != MF_OK) return s;
      cudaStreamSynchronize(b->main);
      fp = fingerprint();
    }
    if (!b->exec || b->g_mode != mode || b->g_strain != strain || b->g_ld != ld || b->g_fp != fp) {
      if (b->exec) cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return bcuda(b, e, "mf_batch_run capture");
      if (fused) {
        s = enqueue_fused(b, strain, ld);
      } else {
        cudaEvent_t fork = b->ev_in;
        e = cudaEventRecord(fork, b->main);
        for (auto& c : b->cls) {
          if (!has_bank(c) || e != cudaSuccess || s != MF_OK) continue;
          e = cudaStreamWaitEvent(c.st, fork, 0);
          if (e == cudaSuccess) s = enqueue_class(b, c, strain, ld);
          if (e == cudaSuccess && s == MF_OK) e = cudaEventRecord(c.join, c.st);
          if (e == cudaSuccess && s == MF_OK) e = cudaStreamWaitEvent(b->main, c.join, 0);
        }
      }
      cudaError_t e2 = cudaStreamEndCapture(b->main, &g);
      if (s != MF_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
      }
      if (e == cudaSuccess) e = e2;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) return bcuda(b, e, "mf_batch_run graph");
      b->g_mode = mode;
      b->g_strain = strain;
      b->g_ld = ld;
      b->g_fp = fp;
    }
    e = cudaGraphLaunch(b->exec, b->main);
    if (e != cudaSuccess) return bcuda(b, e, "mf_batch_run graph launch");
  } else if (mode == MF_RUN_FUSED) {
    if ((s = enqueue_fused(b, strain, ld)) != MF_OK) return s;
  } else {
    cudaEvent_t prev = b->ev_in;
    e = cudaEventRecord(prev, b->main);
    for (auto& c : b->cls) {
      if (!has_bank(c) || e != cudaSuccess) continue;
      e = cudaStreamWaitEvent(c.st, prev, 0);
      if (e != cudaSuccess) break;
      if (mode == MF_RUN_SERIAL) cudaEventRecord(c.t0, c.st);
      if ((s = enqueue_class(b, c, strain, ld)) != MF_OK) return s;
      if (mode == MF_RUN_SERIAL) {
        cudaEventRecord(c.t1, c.st);
        c.timed = true;
      }
      e = cudaEventRecord(c.join, c.st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->main, c.join, 0);
      if (mode == MF_RUN_SERIAL) prev = c.join;  // the next class starts when this one ends
    }
    if (e != cudaSuccess) return bcuda(b, e, "mf_batch_run order");
  }
  e = cudaEventRecord(b->ev_out, b->main);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->user, b->ev_out, 0);
  // a fused pass filtered on the main stream: later calls on a class's plan (its own stream) follow it
  for (auto& c : b->cls)
    if (fused && has_bank(c) && e == cudaSuccess) e = cudaStreamWaitEvent(c.st, b->ev_out, 0);
  if (e != cudaSuccess) return bcuda(b, e, "mf_batch_run join");
  b->ran = true;
  return MF_OK;
}

mf_status mf_batch_get_triggers(mf_batch_t b, mf_batch_trigger* out, int64_t cap, int64_t* n_found) {
  try {  // the host lists can be large: no allocation failure crosses the ABI
    if (!b || !n_found || (cap > 0 && !out)) return bfail(b, MF_EINVAL, "mf_batch_get_triggers: null argument");
    if (!b->ran) return bfail(b, MF_ESTATE, "mf_batch_get_triggers: no run");
    cudaError_t e = cudaStreamSynchronize(b->main);
    if (e != cudaSuccess) return bcuda(b, e, "mf_batch_get_triggers sync");
    std::vector<mf_batch_trigger> all;
    bool overflow = false;
    for (int ci = 0; ci < b->d.n_class; ++ci) {
      mf_batch_s::Cls& c = b->cls[ci];
      if (!has_bank(c)) continue;
      int64_t n = 0;
      mf_status s = mf_get_triggers(c.plan, nullptr, 0, &n);
      if (s != MF_OK && s != MF_EOVERFLOW) return bplan(b, c.plan, s, "mf_batch_get_triggers");
      std::vector<mf_trigger> t((size_t)std::min<int64_t>(n, b->d.max_triggers));
      s = mf_get_triggers(c.plan, t.data(), (int64_t)t.size(), &n);
      if (s == MF_EOVERFLOW) overflow = true;
      else if (s != MF_OK) return bplan(b, c.plan, s, "mf_batch_get_triggers");
      for (const mf_trigger& x : t) {
        const int64_t seg = x.det / b->d.n_det;
        mf_batch_trigger y{};
        y.det = (int32_t)(x.det - seg * b->d.n_det);
        y.cls = ci;
        y.tmpl = x.tmpl;
        y.sample = seg * c.stride + x.sample;
        y.snr = x.snr;
        y.phase = x.phase;
        all.push_back(y);
      }
    }
    std::sort(all.begin(), all.end(), [](const mf_batch_trigger& a, const mf_batch_trigger& c) {
      if (a.cls != c.cls) return a.cls < c.cls;
      if (a.det != c.det) return a.det < c.det;
      if (a.tmpl != c.tmpl) return a.tmpl < c.tmpl;
      return a.sample < c.sample;
    });
    *n_found = (int64_t)all.size();
    const int64_t m = std::min<int64_t>(cap, (int64_t)all.size());
    if (m > 0) std::copy(all.begin(), all.begin() + m, out);
    if (overflow || (int64_t)all.size() > cap)
      return bfail(b, MF_EOVERFLOW, "mf_batch_get_triggers: triggers exceed a buffer");
    return MF_OK;
  } catch (const std::bad_alloc&) {
    return bfail(b, MF_ENOMEM, "mf_batch_get_triggers: host memory");
  }
}

}  // extern "C"
