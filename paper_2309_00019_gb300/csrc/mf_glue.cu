// Hierarchy glue kernels (Sec. III): decimation of the frequency-domain data to
// the stage-1 rate, two-detector coincidence with time shifts on the stage-1
// window maxima, and the union of the neighbourhoods of followed-up coarse
// templates that becomes the stage-2 template selection.
#include "mf_internal.h"

namespace mf {

namespace {

int sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

__global__ void k_decimate(const float2* __restrict__ in, int64_t ld_in, float2* __restrict__ out, int64_t ld_out,
                           int64_t nb_out, int n_det) {
  const int64_t total = nb_out * n_det;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int d = (int)(i / nb_out);
    const int64_t k = i - (int64_t)d * nb_out;
    out[(int64_t)d * ld_out + k] = in[(int64_t)d * ld_in + k];
  }
}

// max rho^2 over the windows of detector 1, per selection position (a cheap
// bound that lets most detector-0 triggers skip the shift loop)
__global__ void k_max_rho2(const unsigned long long* __restrict__ slots, int64_t n_sel, int64_t n_win, float* out) {
  const int64_t p = blockIdx.x;
  const unsigned long long* row = slots + (n_sel + p) * n_win;  // detector 1
  unsigned int m = 0;
  for (int64_t w = threadIdx.x; w < n_win; w += blockDim.x) {
    const unsigned int hi = (unsigned int)(row[w] >> 32);
    m = hi > m ? hi : m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned int y = __shfl_xor_sync(0xffffffffu, m, o);
    m = y > m ? y : m;
  }
  __shared__ unsigned int red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = red[i] > m ? red[i] : m;
    m = red[0] > m ? red[0] : m;
    out[p] = __uint_as_float(m);
  }
}

struct CoincRec {
  int32_t tmpl, shift;
  int64_t sample0, sample1;
  float snr0, snr1, rho_c;
  int32_t pad;
};
static_assert(sizeof(CoincRec) == 40, "mf_coinc layout");

__device__ __forceinline__ int64_t key_sample(unsigned long long key) {
  const uint32_t lo = (uint32_t)(key & 0xffffffffull);
  return (int64_t)(((1u << kSampleBits) - 1u) - (lo >> kPhaseBits));
}
__device__ __forceinline__ float key_rho2(unsigned long long key) { return __uint_as_float((uint32_t)(key >> 32)); }

// One thread per detector-0 window maximum.  Sample positions are below 2^21, so the ring arithmetic is
// 32-bit, and the ring position of shift k follows from shift k - 1 by one subtraction.
__global__ void k_coinc(CoincArgs a) {
  const int64_t total = a.n_sel * a.n_win;
  const float need = fminf(a.rho_c_thr2, a.rho_c_store2);
  const int32_t R = (int32_t)(a.ring_end - a.ring_begin), rb = (int32_t)a.ring_begin;
  const int32_t win = (int32_t)a.window, cw = (int32_t)a.coinc_window;
  const int32_t step = (int32_t)(a.shift % (int64_t)R);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long kh = a.slots[i];  // detector 0, position p, window w
    if (kh == 0ull) continue;
    const int64_t p = i / a.n_win;
    const float r2h = key_rho2(kh);
    if (r2h + a.max_rho2_det1[p] < need) continue;
    const int64_t sh = key_sample(kh);
    const unsigned long long* row1 = a.slots + (a.n_sel + p) * a.n_win;
    const int32_t tmpl = a.sel[p];
    int32_t x = (int32_t)(sh - a.ring_begin);  // ring position of the detector-0 sample, in [0, R)
    for (int k = 0; k <= a.n_shifts; ++k) {
      // detector-1 triggers at ring position x +- window land on s_h after a shift of k * shift
      if (k > 0) {
        x -= step;
        if (x < 0) x += R;
      }
      int32_t lo[2], hi[2];
      int nint = 1;
      lo[0] = x - cw;
      hi[0] = x + cw;
      if (lo[0] < 0) {
        lo[1] = lo[0] + R; hi[1] = R - 1; lo[0] = 0; nint = 2;
      } else if (hi[0] >= R) {
        lo[1] = 0; hi[1] = hi[0] - R; hi[0] = R - 1; nint = 2;
      }
      for (int q = 0; q < nint; ++q) {
        const int32_t w0 = (lo[q] + rb) / win;
        const int32_t w1 = (hi[q] + rb) / win;
        for (int32_t w = w0; w <= w1; ++w) {
          const unsigned long long kl = row1[w];
          if (kl == 0ull) continue;
          const int32_t y = (int32_t)(key_sample(kl) - a.ring_begin);
          if (y < lo[q] || y > hi[q]) continue;
          const float r2l = key_rho2(kl);
          const float rc2 = r2h + r2l;
          if (rc2 >= a.rho_c_thr2) a.followed[tmpl] = 1;
          if (rc2 >= a.rho_c_store2) {
            const unsigned long long slot = atomicAdd(a.n_coinc, 1ull);
            if ((int64_t)slot < a.coinc_cap) {
              CoincRec* out = reinterpret_cast<CoincRec*>(a.coincs);
              out[slot] = CoincRec{tmpl, k, sh, (int64_t)y + a.ring_begin, sqrtf(r2h), sqrtf(r2l), sqrtf(rc2), 0};
            }
          }
        }
      }
    }
  }
}

__global__ void k_zero_i32(int32_t* p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 0;
}

__global__ void k_mark(const int64_t* __restrict__ ptr, const int32_t* __restrict__ idx, int64_t n_coarse,
                       const int32_t* __restrict__ followed, int32_t* flags, int64_t n_fine) {
  for (int64_t c = blockIdx.x; c < n_coarse; c += gridDim.x) {
    if (!followed[c]) continue;
    for (int64_t e = ptr[c] + threadIdx.x; e < ptr[c + 1]; e += blockDim.x) {
      const int32_t f = idx[e];
      if (f >= 0 && f < n_fine) flags[f] = 1;
    }
  }
}

constexpr int kFB = 1024;  // threads per flag-compaction block, one flag each

__global__ void k_flag_count(const int32_t* __restrict__ flags, int64_t n, int64_t* bc) {
  const int64_t i = (int64_t)blockIdx.x * kFB + threadIdx.x;
  const int has = (i < n && flags[i]) ? 1 : 0;
  const int c = __syncthreads_count(has);
  if (threadIdx.x == 0) bc[blockIdx.x] = c;
}

__global__ void k_flag_scan(int64_t* bc, int64_t nblk, int64_t* total) {
  // nblk is small (n_fine / 1024): one thread walks it
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int64_t run = 0;
    for (int64_t b = 0; b < nblk; ++b) {
      const int64_t v = bc[b];
      bc[b] = run;
      run += v;
    }
    *total = run;
  }
}

__global__ void k_flag_write(const int32_t* __restrict__ flags, int64_t n, const int64_t* __restrict__ bc,
                             int32_t* out) {
  __shared__ int wc[32];
  const int64_t i = (int64_t)blockIdx.x * kFB + threadIdx.x;
  const bool has = i < n && flags[i];
  const unsigned m = __ballot_sync(0xffffffffu, has);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) wc[wid] = __popc(m);
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int w = 0; w < 32; ++w) {
      const int v = wc[w];
      wc[w] = run;
      run += v;
    }
  }
  __syncthreads();
  if (has) out[bc[blockIdx.x] + wc[wid] + __popc(m & ((1u << lane) - 1u))] = (int32_t)i;
}

}  // namespace

cudaError_t launch_decimate(const float2* in, int64_t ld_in, float2* out, int64_t ld_out, int64_t nb_out, int n_det,
                            cudaStream_t st) {
  k_decimate<<<sms() * 4, 256, 0, st>>>(in, ld_in, out, ld_out, nb_out, n_det);
  add_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_coinc(const CoincArgs& a, float* max_rho2_det1, cudaStream_t st) {
  if (a.n_sel <= 0) return cudaSuccess;
  if (a.n_sel > 0x7fffffff) return cudaErrorInvalidValue;
  k_max_rho2<<<(unsigned)a.n_sel, 256, 0, st>>>(a.slots, a.n_sel, a.n_win, max_rho2_det1);
  CoincArgs b = a;
  b.max_rho2_det1 = max_rho2_det1;
  k_coinc<<<sms() * 8, 256, 0, st>>>(b);
  add_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_union(const int64_t* ptr, const int32_t* idx, int64_t n_coarse, const int32_t* followed,
                         int32_t* flags, int64_t n_fine, int32_t* subset, int64_t* n_subset, int64_t* bc,
                         cudaStream_t st) {
  const int g = sms() * 4;
  k_zero_i32<<<g, 256, 0, st>>>(flags, n_fine);
  if (n_coarse > 0) k_mark<<<g, 128, 0, st>>>(ptr, idx, n_coarse, followed, flags, n_fine);
  const int64_t nblk = (n_fine + kFB - 1) / kFB;
  if (nblk == 0) return cudaMemsetAsync(n_subset, 0, sizeof(int64_t), st);
  k_flag_count<<<(unsigned)nblk, kFB, 0, st>>>(flags, n_fine, bc);
  k_flag_scan<<<1, 32, 0, st>>>(bc, nblk, n_subset);
  k_flag_write<<<(unsigned)nblk, kFB, 0, st>>>(flags, n_fine, bc, subset);
  add_launches(n_coarse > 0 ? 5 : 4);
  return cudaGetLastError();
}

}  // namespace mf
