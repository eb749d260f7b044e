// Matched-filter kernels for sm_103a: weighted data, FP64 template norms,
// the fused product + inverse FFT + SNR/threshold/window-max filter, and the
// compaction of window maxima into triggers.
//
// The filter computes, for template h and detector data s (Eq. 1-2, Sec. V.C),
//   z[n] = sum_k w[k] s~[k] h~*[k] exp(+2 pi i n k / N),  w = 4 df / S_n on the band,
//   rho^2[n] = |z[n]|^2 / sigma^2,  sigma^2 = sum_k w |h~[k]|^2,
// keeps n with rho^2 >= rho_thr^2 (Sec. II, inclusive) and reduces them to one
// maximum per window of W samples.  The N-point transform is a four-step
// N = N1 * N2: pass 1 forms the product while loading and does N1-point column
// transforms (k = k1 N2 + k2, the upper half k1 >= N1/2 is the empty negative
// frequency half), multiplies by exp(+2 pi i j1 k2 / N) and writes an
// L2-resident scratch; pass 2 does N2-point row transforms and evaluates
// rho^2 of z[j1 + N1 j2] in registers, so the SNR series never reaches memory.
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "mf_common.cuh"
#include "mf_tma.cuh"

namespace mf {

namespace {

constexpr int kThreads = 256;

template <int N1>
struct P1Geo {
  using G = SubFft<N1>;
  static constexpr int C = kThreads / G::T;  // columns per CTA
  static constexpr int L = C >= 16 ? 1 : 16 / C;
  static constexpr int S = stride_for(G::PAD, L);
  static constexpr int SMEM = C * S * (int)sizeof(float2);
};

template <int N2>
struct P2Geo {
  using G = SubFft<N2>;
  static constexpr int RW = kThreads / G::T;  // rows per CTA
  static constexpr int L = G::T >= 16 ? 16 : G::T;
  static constexpr int S = stride_for(G::PAD, L);
  static constexpr int SMEM = RW * S * (int)sizeof(float2);
};

// u[r] *= b^r, r = 1..R-1 (running product)
template <int R>
__device__ __forceinline__ void twiddle_run(float2 (&u)[R], float2 b) {
  float2 w = b;
#pragma unroll
  for (int r = 1; r < R; ++r) {
    u[r] = cmul(u[r], w);
    if (r + 1 < R) w = cmul(w, b);
  }
}

// ---------------------------------------------------------------------------
// loaders (pass 1 input) and epilogues (pass 2 output)
// ---------------------------------------------------------------------------

// x[k] = q_d[k] conj(h_t[k]); series s = b * n_det + d, template t = sel[pos0 + b]
template <int BT>
struct FilterLoad {
  const void* bank;
  int64_t ld_bank;
  const float2* q;
  int64_t ld_q;
  const int32_t* sel;
  int64_t pos0;
  int n_det;
  int64_t nb;
  struct Ser {
    const float2* qd;
    int64_t hoff;
  };
  __device__ __forceinline__ Ser series(int s) const {
    const int d = s % n_det;
    const int64_t t = sel[pos0 + s / n_det];
    return Ser{q + (int64_t)d * ld_q, t * ld_bank};
  }
  __device__ __forceinline__ float2 value(const Ser& se, int64_t k) const {
    if (k >= nb) return make_float2(0.f, 0.f);
    float2 qv = __ldg(se.qd + k);
    float2 hv = BankElem<BT>::get(bank, se.hoff + k);
    return cmulc(qv, hv);
  }
};

// real strain -> complex input (forward transform via conjugation at the end)
struct RealLoad {
  const float* x;
  int64_t ld;
  struct Ser {
    const float* xd;
  };
  __device__ __forceinline__ Ser series(int s) const { return Ser{x + (int64_t)s * ld}; }
  __device__ __forceinline__ float2 value(const Ser& se, int64_t k) const {
    return make_float2(__ldg(se.xd + k), 0.f);
  }
};

// forward one-sided spectrum: dtilde[n] = dt * conj(z[n]) for n <= N/2
struct SpectrumEpi {
  float2* out;
  int64_t ld;
  int64_t nb;
  float dt;
  struct Ser {
    float2* o;
  };
  __device__ __forceinline__ Ser series(int s) const { return Ser{out + (int64_t)s * ld}; }
  __device__ __forceinline__ void operator()(const Ser& se, int64_t n, float2 z) const {
    if (n < nb) se.o[n] = make_float2(z.x * dt, -z.y * dt);
  }
};

// ---------------------------------------------------------------------------
// pass 1: column transforms (length N1) of series s, product fused into the load
// ---------------------------------------------------------------------------

template <int N1, int N2, bool HALF, class Load>
__global__ void __launch_bounds__(kThreads, 2) k_pass1(Load ld, float2* __restrict__ scratch, int n_series) {
  using G = SubFft<N1>;
  using P = P1Geo<N1>;
  constexpr int RA = G::RA, RB = G::RB, T = G::T, NB = G::NB, C = P::C;
  constexpr int NCB = N2 / C;
  constexpr uint32_t N = (uint32_t)N1 * (uint32_t)N2;
  extern __shared__ float2 sm[];
  const int c = threadIdx.x % C;
  const int t = threadIdx.x / C;
  float2* col = sm + c * P::S;
  const int n_items = n_series * NCB;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int s = item / NCB;
    const int k2 = (item % NCB) * C + c;
    const auto se = ld.series(s);
    float2 v[RA];
#pragma unroll
    for (int r = 0; r < RA; ++r) {
      if (HALF && r >= RA / 2) {
        v[r] = make_float2(0.f, 0.f);
      } else {
        const int k1 = t + r * RB;
        v[r] = ld.value(se, (int64_t)k1 * N2 + k2);
      }
    }
    dft<RA, HALF>(v);
    __syncthreads();
#pragma unroll
    for (int a = 0; a < RA; ++a) col[G::pidx(t * RA + a)] = v[a];
    __syncthreads();
    float2* out = scratch + (int64_t)s * N;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int j = t + T * i;
      float2 u[RB];
#pragma unroll
      for (int r = 0; r < RB; ++r) u[r] = col[G::pidx(j + r * RA)];
      twiddle_run<RB>(u, unit_root((uint32_t)j, (uint32_t)N1));
      dft<RB>(u);
      // four-step twiddle exp(+2 pi i j1 k2 / N), j1 = j + a RA
      float2 w = unit_root(((uint32_t)j * (uint32_t)k2) & (N - 1), N);
      const float2 st = unit_root(((uint32_t)RA * (uint32_t)k2) & (N - 1), N);
#pragma unroll
      for (int a = 0; a < RB; ++a) {
        out[(int64_t)(j + a * RA) * N2 + k2] = cmul(u[a], w);
        if (a + 1 < RB) w = cmul(w, st);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// pass 2: row transforms (length N2) + epilogue on z[j1 + N1 j2]
// ---------------------------------------------------------------------------

template <int N1, int N2, class Epi>
__global__ void __launch_bounds__(kThreads, 2) k_pass2(const float2* __restrict__ scratch, Epi epi, int n_series) {
  using G = SubFft<N2>;
  using P = P2Geo<N2>;
  constexpr int RA = G::RA, RB = G::RB, T = G::T, NB = G::NB, RW = P::RW;
  constexpr int NRB = N1 / RW;
  constexpr int64_t N = (int64_t)N1 * N2;
  extern __shared__ float2 sm[];
  const int t = threadIdx.x % T;
  const int row = threadIdx.x / T;
  float2* rs = sm + row * P::S;
  const int n_items = n_series * NRB;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int s = item / NRB;
    const int j1 = (item % NRB) * RW + row;
    const float2* in = scratch + (int64_t)s * N + (int64_t)j1 * N2;
    float2 v[RA];
#pragma unroll
    for (int r = 0; r < RA; ++r) v[r] = in[t + r * RB];
    dft<RA>(v);
    __syncthreads();
#pragma unroll
    for (int a = 0; a < RA; ++a) rs[G::pidx(t * RA + a)] = v[a];
    __syncthreads();
    const auto se = epi.series(s);
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int j = t + T * i;
      float2 u[RB];
#pragma unroll
      for (int r = 0; r < RB; ++r) u[r] = rs[G::pidx(j + r * RA)];
      twiddle_run<RB>(u, unit_root((uint32_t)j, (uint32_t)N2));
      dft<RB>(u);
#pragma unroll
      for (int a = 0; a < RB; ++a) epi(se, (int64_t)j1 + (int64_t)N1 * (j + a * RA), u[a]);
    }
  }
}

int g_num_sms = 0;
int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

template <class K>
cudaError_t set_smem(K kern, int bytes) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

int grid_for(int n_items, int per_sm) {
  int g = num_sms() * per_sm;
  return n_items < g ? n_items : g;
}

int64_t g_launches = 0;

template <int N1, int N2, int BT>
cudaError_t run_pass1(const FilterArgs& a, cudaStream_t st) {
  const int n_series = a.count * a.n_det;
  FilterLoad<BT> ld{a.bank, a.ld_bank, a.q, a.ld_q, a.sel, a.pos0, a.n_det, a.nb};
  auto k1 = k_pass1<N1, N2, true, FilterLoad<BT>>;
  cudaError_t e = set_smem(k1, P1Geo<N1>::SMEM);
  if (e != cudaSuccess) return e;
  const int items1 = n_series * (N2 / P1Geo<N1>::C);
  k1<<<grid_for(items1, 2), kThreads, P1Geo<N1>::SMEM, st>>>(ld, a.scratch, n_series);
  ++g_launches;
  return cudaGetLastError();
}

template <int N1, int N2>
cudaError_t run_pass2(const FilterArgs& a, cudaStream_t st) {
  const int n_series = a.count * a.n_det;
  FilterEpi ep{a.sel, a.inv_sigma, a.pos0, a.n_det, a.thr2, a.window, a.valid_begin, a.valid_end,
               a.n_win, a.n_sel_total, a.slots};
  auto k2 = k_pass2<N1, N2, FilterEpi>;
  cudaError_t e = set_smem(k2, P2Geo<N2>::SMEM);
  if (e != cudaSuccess) return e;
  const int items2 = n_series * (N1 / P2Geo<N2>::RW);
  k2<<<grid_for(items2, 2), kThreads, P2Geo<N2>::SMEM, st>>>(a.scratch, ep, n_series);
  ++g_launches;
  return cudaGetLastError();
}

template <int N1, int N2>
cudaError_t run_pass1_bt(const FilterArgs& a, cudaStream_t st) {
  switch (a.bank_type) {
    case kBankF32: return run_pass1<N1, N2, kBankF32>(a, st);
    case kBankF16: return run_pass1<N1, N2, kBankF16>(a, st);
    case kBankBF16: return run_pass1<N1, N2, kBankBF16>(a, st);
  }
  return cudaErrorInvalidValue;
}

// dispatch on N to the instantiation with N = N1 * N2 (N1 >= N2)
#define MF_DISPATCH_N(n, FN, ARGS)                   \
  switch (n) {                                       \
    case 1 << 12: return FN<64, 64> ARGS;            \
    case 1 << 13: return FN<128, 64> ARGS;           \
    case 1 << 14: return FN<128, 128> ARGS;          \
    case 1 << 15: return FN<256, 128> ARGS;          \
    case 1 << 16: return FN<256, 256> ARGS;          \
    case 1 << 17: return FN<512, 256> ARGS;          \
    case 1 << 18: return FN<512, 512> ARGS;          \
    case 1 << 19: return FN<1024, 512> ARGS;         \
    case 1 << 20: return FN<1024, 1024> ARGS;        \
  }                                                  \
  return cudaErrorInvalidValue;

template <int N1, int N2>
cudaError_t run_rfft(const float* x, int64_t ld_s, int n_det, double dt, float2* scratch, float2* out,
                     int64_t ld_d, cudaStream_t st) {
  RealLoad ld{x, ld_s};
  auto k1 = k_pass1<N1, N2, false, RealLoad>;
  cudaError_t e = set_smem(k1, P1Geo<N1>::SMEM);
  if (e != cudaSuccess) return e;
  k1<<<grid_for(n_det * (N2 / P1Geo<N1>::C), 2), kThreads, P1Geo<N1>::SMEM, st>>>(ld, scratch, n_det);
  SpectrumEpi ep{out, ld_d, (int64_t)N1 * N2 / 2 + 1, (float)dt};
  auto k2 = k_pass2<N1, N2, SpectrumEpi>;
  e = set_smem(k2, P2Geo<N2>::SMEM);
  if (e != cudaSuccess) return e;
  k2<<<grid_for(n_det * (N1 / P2Geo<N2>::RW), 2), kThreads, P2Geo<N2>::SMEM, st>>>(scratch, ep, n_det);
  g_launches += 2;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------

__global__ void k_prep(const float2* __restrict__ d, int64_t ld_d, const double* __restrict__ w, int64_t nb,
                       int n_det, float2* __restrict__ q, int64_t ld_q, double q_scale) {
  const int64_t total = nb * n_det;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int det = (int)(i / nb);
    const int64_t k = i - (int64_t)det * nb;
    const double wk = w[k] * q_scale;
    const float2 s = d[(int64_t)det * ld_d + k];
    q[(int64_t)det * ld_q + k] = make_float2((float)(wk * (double)s.x), (float)(wk * (double)s.y));
  }
}

__global__ void k_tmpl_scale(const float* __restrict__ inv_sigma, int64_t n, double sigma_ref, double thr2,
                             float* __restrict__ ratio, float* __restrict__ thr_raw) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double r = (double)inv_sigma[i] * sigma_ref;
    ratio[i] = (float)r;
    thr_raw[i] = r > 0.0 ? (float)(thr2 / (r * r)) : __int_as_float(0x7f800000);
  }
}

__global__ void k_zero_u64(unsigned long long* p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 0ull;
}

// n1 = 0: row t holds bins 0..nb-1; n1 > 0: column layout (stored index
// i = k2 n1/2 + k1 holds bin k = k1 n2 + k2, i < N/2)
template <int BT>
__global__ void k_sigmasq(const void* bank, int64_t ld_bank, const float* scales, int64_t row0,
                          const double* __restrict__ w, int64_t nb, double* sigmasq, float* inv_sigma, int n1,
                          int n2) {
  const int64_t t = row0 + blockIdx.x;
  double acc = 0.0;
  const int64_t count = n1 > 0 ? (int64_t)n1 * n2 / 2 : nb;
  const int R = n1 / 2;
  for (int64_t i = threadIdx.x; i < count; i += blockDim.x) {
    const int64_t k = n1 > 0 ? (int64_t)(i % R) * n2 + i / R : i;
    const double wk = w[k];
    if (wk != 0.0) {
      const float2 h = BankElem<BT>::get(bank, t * ld_bank + i);
      acc += wk * ((double)h.x * h.x + (double)h.y * h.y);
    }
  }
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) {
      const double sc = scales ? (double)scales[t] : 1.0;
      const double s2 = v * sc * sc;  // sigma^2 of the dequantised template
      sigmasq[t] = s2;
      inv_sigma[t] = s2 > 0.0 ? (float)(sc / sqrt(s2)) : 0.0f;  // scale folded in: z is of the stored values
    }
  }
}

// --- compaction of window maxima ------------------------------------------

struct TrigRec {
  int32_t det, tmpl;
  int64_t sample;
  float snr, phase;
};
static_assert(sizeof(TrigRec) == 24, "mf_trigger layout");

constexpr int kCompactBlock = 1024;        // threads
constexpr int kCompactPerThread = 4;       // slots per thread
constexpr int kCompactSpan = kCompactBlock * kCompactPerThread;

__global__ void k_compact_count(const unsigned long long* __restrict__ slots, int64_t n_slots, int64_t* bc) {
  const int64_t base = (int64_t)blockIdx.x * kCompactSpan;
  int cnt = 0;
#pragma unroll
  for (int i = 0; i < kCompactPerThread; ++i) {
    const int64_t idx = base + (int64_t)i * kCompactBlock + threadIdx.x;
    if (idx < n_slots && slots[idx] != 0ull) ++cnt;
  }
  __shared__ int red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x < 32) {
    int v = red[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) bc[blockIdx.x] = v;
  }
}

// single block: exclusive scan of bc[0..n) in place, total -> *count
__global__ void k_scan_blocks(int64_t* bc, int64_t n, int64_t* count) {
  __shared__ int64_t carry;
  __shared__ int64_t wsum[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < n; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const int64_t v = i < n ? bc[i] : 0;
    int64_t x = v;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int64_t s = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      wsum[lane] = s;  // inclusive over warps
    }
    __syncthreads();
    const int64_t incl = x + (wid > 0 ? wsum[wid - 1] : 0);
    if (i < n) bc[i] = carry + incl - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = carry;
}

__global__ void k_compact_write(const unsigned long long* __restrict__ slots, int64_t n_slots, int64_t n_sel,
                                int64_t n_win, int64_t window, const int32_t* __restrict__ sel,
                                const int64_t* __restrict__ bc, TrigRec* out, int64_t cap) {
  const int64_t base = (int64_t)blockIdx.x * kCompactSpan;
  __shared__ int wcount[32];
  __shared__ int tot;
  __shared__ int64_t run;
  if (threadIdx.x == 0) run = bc[blockIdx.x];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = 0; i < kCompactPerThread; ++i) {
    const int64_t idx = base + (int64_t)i * kCompactBlock + threadIdx.x;
    const unsigned long long key = idx < n_slots ? slots[idx] : 0ull;
    const bool has = key != 0ull;
    const unsigned m = __ballot_sync(0xffffffffu, has);
    if (lane == 0) wcount[wid] = __popc(m);
    __syncthreads();
    if (threadIdx.x < 32) {
      int v = wcount[threadIdx.x];
      int x = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      wcount[threadIdx.x] = x - v;  // exclusive
      if (threadIdx.x == 31) tot = x;
    }
    __syncthreads();
    if (has) {
      const int64_t pos = run + wcount[wid] + __popc(m & ((1u << lane) - 1u));
      if (pos < cap) {
        const int64_t w = idx % n_win;
        const int64_t ds = idx / n_win;
        const int64_t p = ds % n_sel;
        const int d = (int)(ds / n_sel);
        const uint32_t lo = (uint32_t)(key & 0xffffffffull);
        const int64_t n = (int64_t)(((1u << kSampleBits) - 1u) - (lo >> kPhaseBits));
        const float r2 = __uint_as_float((uint32_t)(key >> 32));
        const float ph = ((float)(lo & 2047u) / 2048.0f - 0.5f) * 6.283185307179586f;
        (void)w;
        (void)window;
        out[pos] = TrigRec{d, sel[p], n, sqrtf(r2), ph};
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) run += tot;
    __syncthreads();
  }
}


// --- FP32 FMA throughput probe (context for the ALU roofline) -----------------

// 8 independent FMA chains per thread, 16 x iters rounds; the result is
// written only if it is exactly zero so the work cannot be removed.
__global__ void __launch_bounds__(256) k_fma_probe(float* out, int iters, float a, float b) {
  float x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = (float)(threadIdx.x + i) * 1e-3f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], a, b);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == 0.0f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// --- failure detection without a fault ----------------------------------------

// One CTA waits on an mbarrier that no thread and no copy ever completes: every
// thread's bounded wait gives up after ~2^31 cycles, records kStatusTimeout in
// *status and returns; *returned counts the threads that came back.
__global__ void k_wait_selftest(int* status, int* returned) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (!mbar_wait_bounded(&bar, 0, status)) atomicAdd(returned, 1);
}

// --- column layout of spectra (the filter's bank and weighted-data layout) ----

// dst[r][k2 R + k1] = src[r][k1 n2 + k2], k1 < R = n1/2, k2 < n2: 32 x 32 tiles
// through shared memory, coalesced on both sides.  grid (n2/32, R/32, rows).
template <typename E>
__global__ void k_to_cols(const E* __restrict__ src, int64_t ld_src, E* __restrict__ dst, int64_t ld_dst, int n1,
                          int n2, int64_t row0) {
  __shared__ E tile[32][33];
  const int R = n1 / 2;
  const int64_t row = row0 + blockIdx.z;
  const int k1_0 = blockIdx.y * 32, k2_0 = blockIdx.x * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y)
    tile[y][threadIdx.x] = src[row * ld_src + (int64_t)(k1_0 + y) * n2 + k2_0 + threadIdx.x];
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y)
    dst[row * ld_dst + (int64_t)(k2_0 + y) * R + k1_0 + threadIdx.x] = tile[threadIdx.x][y];
}

// q[det][k2 R + k1] = q_scale w[k] s~[det][k], k = k1 n2 + k2 (FP64 product)
__global__ void k_prep_cols(const float2* __restrict__ d, int64_t ld_d, const double* __restrict__ w, int n1, int n2,
                            int n_det, float2* __restrict__ q, int64_t ld_q, double q_scale) {
  const int R = n1 / 2;
  const int64_t half = (int64_t)R * n2;
  const int64_t total = half * n_det;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int det = (int)(i / half);
    const int64_t ii = i - (int64_t)det * half;
    const int64_t k = (ii % R) * n2 + ii / R;
    const double wk = w[k] * q_scale;
    const float2 s = d[(int64_t)det * ld_d + k];
    q[(int64_t)det * ld_q + ii] = make_float2((float)(wk * (double)s.x), (float)(wk * (double)s.y));
  }
}

// --- 16-bit storage (bank and weighted data) ---------------------------------

// Power-of-two c with amax * c in [2^14, 2^15) (1 for amax = 0 or not finite):
// the largest 16-bit value then stays below FP16's 65504 with room for rounding,
// and scaling by c is exact in binary floating point.
__device__ __forceinline__ float pow2_scale(float amax) {
  if (!(amax > 0.f) || !(amax < INFINITY)) return 1.f;
  const int E = (int)((__float_as_uint(amax) >> 23) & 0xffu);  // amax < 2^(E - 126)
  int e = 141 - E;                                              // amax c < 2^15, >= 2^14 (normal amax)
  e = e > 126 ? 126 : (e < -126 ? -126 : e);
  return __uint_as_float((uint32_t)(e + 127) << 23);
}

template <int QT>
__device__ __forceinline__ void store_lp(void* base, int64_t i, float x, float y) {
  if constexpr (QT == kBankF16) {
    reinterpret_cast<__half2*>(base)[i] = __floats2half2_rn(x, y);
  } else {
    reinterpret_cast<__nv_bfloat162*>(base)[i] = __floats2bfloat162_rn(x, y);
  }
}

__device__ __forceinline__ float block_max(float m, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  float r = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmaxf(r, red[w]);
  return r;
}

// grid (blocks, n_det): per-detector max |component| of q into dmax (float bits, >= 0)
__global__ void k_qmax(const float2* __restrict__ q, int64_t ld_q, int64_t nb, unsigned* dmax) {
  __shared__ float red[32];
  const int d = blockIdx.y;
  float m = 0.f;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nb; k += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = q[(int64_t)d * ld_q + k];
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
  m = block_max(m, red);
  if (threadIdx.x == 0) atomicMax(dmax + d, __float_as_uint(m));
}

template <int QT>
__global__ void k_quant_q(const float2* __restrict__ q, int64_t ld_q, int64_t nb, const unsigned* __restrict__ dmax,
                          void* q_lp, float* dscale) {
  const int d = blockIdx.y;
  const float c = pow2_scale(__uint_as_float(dmax[d]));
  if (blockIdx.x == 0 && threadIdx.x == 0) dscale[d] = c;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nb; k += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = q[(int64_t)d * ld_q + k];
    store_lp<QT>(q_lp, (int64_t)d * ld_q + k, v.x * c, v.y * c);
  }
}

// one CTA per template row
template <int BT>
__global__ void k_quant_bank(const float2* __restrict__ src, int64_t ld_src, int64_t nb, void* dst, int64_t ld_dst,
                             float* scales) {
  __shared__ float red[32];
  const float2* row = src + blockIdx.x * ld_src;
  float m = 0.f;
  for (int64_t k = threadIdx.x; k < nb; k += blockDim.x) {
    const float2 v = row[k];
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
  const float c = pow2_scale(block_max(m, red));
  for (int64_t k = threadIdx.x; k < nb; k += blockDim.x) {
    const float2 v = row[k];
    store_lp<BT>(dst, blockIdx.x * ld_dst + k, v.x * c, v.y * c);
  }
  if (threadIdx.x == 0) scales[blockIdx.x] = 1.f / c;  // exact: c is a power of two
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

cudaError_t launch_fma_probe(float* out, int blocks, int iters, cudaStream_t st) {
  k_fma_probe<<<blocks, 256, 0, st>>>(out, iters, 0.999999f, 1e-7f);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t launch_wait_selftest(int* status, int* returned, cudaStream_t st) {
  k_wait_selftest<<<1, 128, 0, st>>>(status, returned);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t launch_tmpl_scale(const float* inv_sigma, int64_t n_tmpl, double sigma_ref, double thr2, float* ratio,
                              float* thr_raw, cudaStream_t st) {
  if (n_tmpl <= 0) return cudaSuccess;
  k_tmpl_scale<<<num_sms() * 2, 256, 0, st>>>(inv_sigma, n_tmpl, sigma_ref, thr2, ratio, thr_raw);
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t launch_prep(const float2* dtilde, int64_t ld_d, const double* w, int64_t nb, int n_det,
                        float2* q, int64_t ld_q, unsigned long long* slots, int64_t n_slots, cudaStream_t st,
                        double q_scale) {
  const int g = num_sms() * 4;
  k_prep<<<g, 256, 0, st>>>(dtilde, ld_d, w, nb, n_det, q, ld_q, q_scale);
  ++g_launches;
  if (slots && n_slots > 0) {
    k_zero_u64<<<g, 256, 0, st>>>(slots, n_slots);
    ++g_launches;
  }
  return cudaGetLastError();
}

int64_t launch_count() { return g_launches; }
void add_launches(int64_t n) { g_launches += n; }

cudaError_t launch_filter_pass1(const FilterArgs& a, cudaStream_t st) { MF_DISPATCH_N(a.n, run_pass1_bt, (a, st)) }

cudaError_t launch_filter_pass2(const FilterArgs& a, cudaStream_t st) { MF_DISPATCH_N(a.n, run_pass2, (a, st)) }

cudaError_t launch_filter_batch(const FilterArgs& a, cudaStream_t st) {
  cudaError_t e = launch_filter_pass1(a, st);
  if (e != cudaSuccess) return e;
  return launch_filter_pass2(a, st);
}

cudaError_t launch_rfft(const float* x, int64_t ld_s, int n_det, int64_t n, int n1, int n2, double dt,
                        float2* scratch, float2* out, int64_t ld_d, cudaStream_t st) {
  (void)n1;
  (void)n2;
  MF_DISPATCH_N(n, run_rfft, (x, ld_s, n_det, dt, scratch, out, ld_d, st))
}

cudaError_t launch_quant_q(const float2* q, int64_t ld_q, int64_t nb, int n_det, int q_type, void* q_lp,
                           unsigned* dmax, float* dscale, cudaStream_t st) {
  if (q_type != kBankF16 && q_type != kBankBF16) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(dmax, 0, n_det * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  const dim3 g((unsigned)std::max(1, std::min<int>(num_sms() * 2 / n_det + 1, (int)((nb + 255) / 256))), (unsigned)n_det);
  k_qmax<<<g, 256, 0, st>>>(q, ld_q, nb, dmax);
  if (q_type == kBankF16)
    k_quant_q<kBankF16><<<g, 256, 0, st>>>(q, ld_q, nb, dmax, q_lp, dscale);
  else
    k_quant_q<kBankBF16><<<g, 256, 0, st>>>(q, ld_q, nb, dmax, q_lp, dscale);
  g_launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_quant_bank(const float2* src, int64_t ld_src, int64_t n_rows, int64_t nb, int bank_type, void* dst,
                              int64_t ld_dst, float* scales, cudaStream_t st) {
  if (n_rows <= 0) return cudaSuccess;
  if (bank_type == kBankF16)
    k_quant_bank<kBankF16><<<(unsigned)n_rows, 256, 0, st>>>(src, ld_src, nb, dst, ld_dst, scales);
  else if (bank_type == kBankBF16)
    k_quant_bank<kBankBF16><<<(unsigned)n_rows, 256, 0, st>>>(src, ld_src, nb, dst, ld_dst, scales);
  else
    return cudaErrorInvalidValue;
  ++g_launches;
  return cudaGetLastError();
}

cudaError_t launch_to_cols(const void* src, int64_t ld_src, void* dst, int64_t ld_dst, int64_t n_rows, int n1, int n2,
                           int elem_bytes, cudaStream_t st) {
  if (n1 < 64 || n2 < 32 || (elem_bytes != 8 && elem_bytes != 4)) return cudaErrorInvalidValue;
  for (int64_t r0 = 0; r0 < n_rows; r0 += 65535) {
    const dim3 g((unsigned)(n2 / 32), (unsigned)(n1 / 2 / 32), (unsigned)std::min<int64_t>(65535, n_rows - r0));
    const dim3 b(32, 8);
    if (elem_bytes == 8)
      k_to_cols<float2><<<g, b, 0, st>>>(static_cast<const float2*>(src), ld_src, static_cast<float2*>(dst), ld_dst,
                                         n1, n2, r0);
    else
      k_to_cols<uint32_t><<<g, b, 0, st>>>(static_cast<const uint32_t*>(src), ld_src, static_cast<uint32_t*>(dst),
                                           ld_dst, n1, n2, r0);
    ++g_launches;
  }
  return cudaGetLastError();
}

cudaError_t launch_prep_cols(const float2* dtilde, int64_t ld_d, const double* w, int n1, int n2, int n_det,
                             float2* q, int64_t ld_q, unsigned long long* slots, int64_t n_slots, cudaStream_t st,
                             double q_scale) {
  const int g = num_sms() * 4;
  k_prep_cols<<<g, 256, 0, st>>>(dtilde, ld_d, w, n1, n2, n_det, q, ld_q, q_scale);
  ++g_launches;
  if (slots && n_slots > 0) {
    k_zero_u64<<<g, 256, 0, st>>>(slots, n_slots);
    ++g_launches;
  }
  return cudaGetLastError();
}

cudaError_t launch_sigmasq(const void* bank, int bank_type, int64_t ld_bank, const float* scales, int64_t row0,
                           int64_t n_rows, const double* w, int64_t nb, double* sigmasq, float* inv_sigma,
                           cudaStream_t st, int n1, int n2) {
  if (n_rows <= 0) return cudaSuccess;
  if (n_rows > 0x7fffffff) return cudaErrorInvalidValue;
  switch (bank_type) {
    case kBankF32:
      k_sigmasq<kBankF32><<<(unsigned)n_rows, 256, 0, st>>>(bank, ld_bank, scales, row0, w, nb, sigmasq, inv_sigma,
                                                             n1, n2);
      break;
    case kBankF16:
      k_sigmasq<kBankF16><<<(unsigned)n_rows, 256, 0, st>>>(bank, ld_bank, scales, row0, w, nb, sigmasq, inv_sigma,
                                                             n1, n2);
      break;
    case kBankBF16:
      k_sigmasq<kBankBF16><<<(unsigned)n_rows, 256, 0, st>>>(bank, ld_bank, scales, row0, w, nb, sigmasq, inv_sigma,
                                                             n1, n2);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  ++g_launches;
  return cudaGetLastError();
}

int64_t compact_blocks(int64_t n_slots) { return (n_slots + kCompactSpan - 1) / kCompactSpan; }

cudaError_t launch_compact(const unsigned long long* slots, int n_det, int64_t n_sel, int64_t n_win, int64_t window,
                           const int32_t* sel, void* trig_out, int64_t trig_cap, int64_t* count, int64_t* bc,
                           int64_t n_blocks_cap, cudaStream_t st) {
  const int64_t n_slots = (int64_t)n_det * n_sel * n_win;
  const int64_t nblk = compact_blocks(n_slots);
  if (nblk > n_blocks_cap || nblk > 0x7fffffff) return cudaErrorInvalidValue;
  if (nblk == 0) return cudaMemsetAsync(count, 0, sizeof(int64_t), st);
  k_compact_count<<<(unsigned)nblk, kCompactBlock, 0, st>>>(slots, n_slots, bc);
  k_scan_blocks<<<1, 1024, 0, st>>>(bc, nblk, count);
  k_compact_write<<<(unsigned)nblk, kCompactBlock, 0, st>>>(slots, n_slots, n_sel, n_win, window, sel, bc,
                                                            reinterpret_cast<TrigRec*>(trig_out), trig_cap);
  g_launches += 3;
  return cudaGetLastError();
}

cudaError_t launch_decimate(const float2* in, int64_t ld_in, float2* out, int64_t ld_out, int64_t nb_out, int n_det,
                            cudaStream_t st);

}  // namespace mf
