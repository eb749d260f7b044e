// Learned proposal network: training and inference kernels.
//
// A small MLP scores the neighbourhood slots of a stage-1 candidate so that
// stage 2 (Sec. III) can filter only the best-ranked fine templates, with the
// full neighbourhood as the fallback.  Layers: x -> depth x (affine + GELU)
// -> affine -> masked softmax over the candidate's n_valid slots.  Weights are
// kept in FP32 (master copy for AdamW) and cast to BF16 for the products;
// every matrix product runs on the tensor cores (mma.sync m16n8k16, BF16
// inputs, FP32 accumulation).  Parameter layout (flat, FP32): W_1 [n_in][width],
// b_1, ..., W_depth, b_depth, W_out [width][n_out], b_out.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/mf.h"
#include "mf_internal.h"

typedef __nv_bfloat16 bf16;

namespace {

// ---------------------------------------------------------------------------
// GEMM: C[M][N] (FP32) = op(A)[M][K] op(B)[K][N] (+ bias[n]); BF16 inputs.
//   A(m,k) = ta ? A[k lda + m] : A[m lda + k];  B(k,n) = tb ? B[n ldb + k] : B[k ldb + n]
// 64 x 64 tile per 128-thread CTA, 4 warps of 32 x 32, K step 32.
// ---------------------------------------------------------------------------

constexpr int kTM = 64, kTN = 64, kTK = 32, kPadK = kTK + 8;

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(128) k_gemm(int M, int N, int K, const bf16* __restrict__ A, int lda, int ta,
                                              const bf16* __restrict__ B, int ldb, int tb, float* __restrict__ C,
                                              int ldc, const float* __restrict__ bias) {
  __shared__ __align__(16) bf16 As[kTM][kPadK];  // [m][k]
  __shared__ __align__(16) bf16 Bs[kTN][kPadK];  // [n][k]
  const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int g = lane >> 2, tq = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
  const bf16 zero = __float2bfloat16(0.f);
  for (int k0 = 0; k0 < K; k0 += kTK) {
    for (int i = threadIdx.x; i < kTM * kTK; i += blockDim.x) {
      const int mm = ta ? (i % kTM) : (i / kTK), kk = ta ? (i / kTM) : (i % kTK);
      const int gm = m0 + mm, gk = k0 + kk;
      bf16 v = zero;
      if (gm < M && gk < K) v = ta ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk];
      As[mm][kk] = v;
    }
    for (int i = threadIdx.x; i < kTN * kTK; i += blockDim.x) {
      const int nn = tb ? (i / kTK) : (i % kTN), kk = tb ? (i % kTK) : (i / kTN);
      const int gn = n0 + nn, gk = k0 + kk;
      bf16 v = zero;
      if (gn < N && gk < K) v = tb ? B[(int64_t)gn * ldb + gk] : B[(int64_t)gk * ldb + gn];
      Bs[nn][kk] = v;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < kTK; ks += 16) {
      uint32_t af[2][4], bfg[4][2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int r = wm + mi * 16 + g, c = ks + tq * 2;
        af[mi][0] = *reinterpret_cast<const uint32_t*>(&As[r][c]);
        af[mi][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][c]);
        af[mi][2] = *reinterpret_cast<const uint32_t*>(&As[r][c + 8]);
        af[mi][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][c + 8]);
      }
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const int n = wn + ni * 8 + g, c = ks + tq * 2;
        bfg[ni][0] = *reinterpret_cast<const uint32_t*>(&Bs[n][c]);
        bfg[ni][1] = *reinterpret_cast<const uint32_t*>(&Bs[n][c + 8]);
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], af[mi], bfg[ni]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = m0 + wm + mi * 16 + g + 8 * h;
        const int c = n0 + wn + ni * 8 + tq * 2;
        if (r >= M) continue;
#pragma unroll
        for (int e = 0; e < 2; ++e)
          if (c + e < N) C[(int64_t)r * ldc + c + e] = acc[mi][ni][2 * h + e] + (bias ? bias[c + e] : 0.f);
      }
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

__global__ void k_to_bf16(const float* __restrict__ x, bf16* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

__global__ void k_gelu_fwd(const float* __restrict__ z, bf16* __restrict__ h, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    h[i] = __float2bfloat16(gelu(z[i]));
}

// dZ = dH * GELU'(Z), as FP32 (bias gradients) and BF16 (products)
__global__ void k_gelu_bwd(const float* __restrict__ dh, const float* __restrict__ z, float* __restrict__ dz,
                           bf16* __restrict__ dzb, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = dh[i] * gelu_grad(z[i]);
    dz[i] = v;
    dzb[i] = __float2bfloat16(v);
  }
}

// masked softmax cross-entropy, one CTA per row: loss += -log p[label] / B,
// grad = (p - onehot) / B on the valid slots, 0 elsewhere
__global__ void k_masked_ce(const float* __restrict__ logits, int n_out, const int32_t* __restrict__ n_valid,
                            const int32_t* __restrict__ label, int B, float* loss, float* __restrict__ g,
                            bf16* __restrict__ gb) {
  const int row = blockIdx.x;
  const float* l = logits + (int64_t)row * n_out;
  const int nv = min(max(n_valid[row], 1), n_out);
  __shared__ float red[32];
  float m = -INFINITY;
  for (int j = threadIdx.x; j < nv; j += blockDim.x) m = fmaxf(m, l[j]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : -INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  m = red[0];
  __syncthreads();
  float s = 0.f;
  for (int j = threadIdx.x; j < nv; j += blockDim.x) s += expf(l[j] - m);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  s = red[0];
  const int lab = label[row];
  const float invB = 1.f / (float)B;
  for (int j = threadIdx.x; j < n_out; j += blockDim.x) {
    float gv = 0.f;
    if (j < nv) gv = (expf(l[j] - m) / s - (j == lab ? 1.f : 0.f)) * invB;
    g[(int64_t)row * n_out + j] = gv;
    gb[(int64_t)row * n_out + j] = __float2bfloat16(gv);
  }
  if (threadIdx.x == 0 && lab >= 0 && lab < nv) atomicAdd(loss, -(l[lab] - m - logf(s)) * invB);
}

// db[n] = sum_b G[b][n]
__global__ void k_colsum(const float* __restrict__ G, int rows, int cols, float* __restrict__ db) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < cols; n += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int b = 0; b < rows; ++b) s += G[(int64_t)b * cols + n];
    db[n] = s;
  }
}

__global__ void k_adamw(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                        float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float wd, float c1,
                        float c2, bf16* __restrict__ thb) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float t = th[i] - lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * th[i]);
    th[i] = t;
    thb[i] = __float2bfloat16(t);
  }
}

// Best-scored valid slots per row (ties to the lower slot), in order, until
// their softmax probability (over the valid slots) reaches p_mass or k slots
// are taken; -1 padding; count[row] = slots taken.
__global__ void k_topk(const float* __restrict__ logits, int n_out, const int32_t* __restrict__ n_valid, int k,
                       float p_mass, int32_t* __restrict__ out, int32_t* __restrict__ count) {
  const int row = blockIdx.x;
  const float* l = logits + (int64_t)row * n_out;
  const int nv = min(max(n_valid[row], 0), n_out);
  __shared__ int chosen[64];
  __shared__ float bv[32];
  __shared__ int bi[32];
  __shared__ float s_max, s_sum, s_cum;
  __shared__ int s_done;
  // softmax normaliser over the valid slots
  float m = -INFINITY;
  for (int j = threadIdx.x; j < nv; j += blockDim.x) m = fmaxf(m, l[j]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) bv[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float mm = -INFINITY;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmaxf(mm, bv[w]);
    s_max = mm;
  }
  __syncthreads();
  float sum = 0.f;
  for (int j = threadIdx.x; j < nv; j += blockDim.x) sum += expf(l[j] - s_max);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) bv[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    float ss = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) ss += bv[w];
    s_sum = ss;
    s_cum = 0.f;
    s_done = 0;
  }
  __syncthreads();
  int taken = 0;
  for (int r = 0; r < k; ++r) {
    float best = -INFINITY;
    int besti = 0x7fffffff;
    if (!s_done) {
      for (int j = threadIdx.x; j < nv; j += blockDim.x) {
        bool used = false;
        for (int q = 0; q < r; ++q) used |= chosen[q] == j;
        if (used) continue;
        const float x = l[j];
        if (x > best || (x == best && j < besti)) {
          best = x;
          besti = j;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, besti, o);
      if (ob > best || (ob == best && oi < besti)) {
        best = ob;
        besti = oi;
      }
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
      bv[threadIdx.x >> 5] = best;
      bi[threadIdx.x >> 5] = besti;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float b = -INFINITY;
      int ii = 0x7fffffff;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
        if (bv[w] > b || (bv[w] == b && bi[w] < ii)) {
          b = bv[w];
          ii = bi[w];
        }
      const bool ok = !s_done && r < nv && ii != 0x7fffffff;
      chosen[r] = ok ? ii : -1;
      out[(int64_t)row * k + r] = chosen[r];
      if (ok) {
        s_cum += expf(b - s_max) / s_sum;
        if (s_cum >= p_mass) s_done = 1;
      }
    }
    __syncthreads();
    taken += chosen[r] >= 0 ? 1 : 0;
  }
  if (threadIdx.x == 0 && count) count[row] = taken;
}

int sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

}  // namespace

struct mf_mlp_s {
  int n_in = 0, width = 0, depth = 0, n_out = 0;
  int64_t max_batch = 0, n_params = 0, step = 0;
  cudaStream_t st = nullptr;
  std::string err;
  std::vector<int64_t> w_off, b_off;  // offsets of W_l, b_l in the flat parameter vector
  float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  bf16* thb = nullptr;                 // BF16 copy of the parameters (weights used by the products)
  bf16* xb = nullptr;                  // input [B][n_in]
  std::vector<float*> z;               // pre-activations [B][width], l = 1..depth
  std::vector<bf16*> h;                // activations [B][width]
  float* logits = nullptr;             // [B][n_out]
  float* dlog = nullptr;               // [B][n_out]
  bf16* dlogb = nullptr;
  float *dh = nullptr, *dz = nullptr;  // [B][width]
  bf16* dzb = nullptr;
  float* loss = nullptr;
};

namespace {

mf_status mfail(mf_mlp_t p, mf_status s, const std::string& m) {
  if (p) p->err = m;
  mf::set_global_error(m);
  return s;
}

template <class T>
bool dal(T** ptr, size_t n) {
  return cudaMalloc((void**)ptr, std::max<size_t>(n, 1) * sizeof(T)) == cudaSuccess;
}

cudaError_t gemm(cudaStream_t st, int M, int N, int K, const bf16* A, int lda, int ta, const bf16* B, int ldb, int tb,
                 float* C, int ldc, const float* bias) {
  dim3 grid((N + kTN - 1) / kTN, (M + kTM - 1) / kTM);
  k_gemm<<<grid, 128, 0, st>>>(M, N, K, A, lda, ta, B, ldb, tb, C, ldc, bias);
  mf::add_launches(1);
  return cudaGetLastError();
}

// forward of a batch of B rows whose input (FP32, device) is x; leaves logits in p->logits
cudaError_t forward(mf_mlp_t p, const float* x, int B) {
  const int g = sms() * 4;
  k_to_bf16<<<g, 256, 0, p->st>>>(x, p->xb, (int64_t)B * p->n_in);
  mf::add_launches(1);
  const bf16* hin = p->xb;
  int kin = p->n_in;
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < p->depth && e == cudaSuccess; ++l) {
    e = gemm(p->st, B, p->width, kin, hin, kin, 0, p->thb + p->w_off[l], p->width, 0, p->z[l], p->width,
             p->theta + p->b_off[l]);
    k_gelu_fwd<<<g, 256, 0, p->st>>>(p->z[l], p->h[l], (int64_t)B * p->width);
    mf::add_launches(1);
    hin = p->h[l];
    kin = p->width;
  }
  if (e == cudaSuccess)
    e = gemm(p->st, B, p->n_out, kin, hin, kin, 0, p->thb + p->w_off[p->depth], p->n_out, 0, p->logits, p->n_out,
             p->theta + p->b_off[p->depth]);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

}  // namespace

extern "C" {

mf_status mf_mlp_create(mf_mlp_t* out, int32_t n_in, int32_t width, int32_t depth, int32_t n_out, int64_t max_batch,
                        void* cuda_stream) {
  if (!out) return mfail(nullptr, MF_EINVAL, "mf_mlp_create: null out");
  if (n_in < 1 || n_in > 4096 || width < 1 || width > 8192 || depth < 1 || depth > 16 || n_out < 1 ||
      n_out > 65536 || max_batch < 1 || max_batch > (1 << 20))
    return mfail(nullptr, MF_EINVAL, "mf_mlp_create: sizes out of range");
  mf_mlp_t p = new (std::nothrow) mf_mlp_s();
  if (!p) return mfail(nullptr, MF_ENOMEM, "mf_mlp_create: host allocation");
  p->n_in = n_in;
  p->width = width;
  p->depth = depth;
  p->n_out = n_out;
  p->max_batch = max_batch;
  p->st = (cudaStream_t)cuda_stream;
  int64_t o = 0, din = n_in;
  for (int l = 0; l <= depth; ++l) {
    const int64_t dout = l < depth ? width : n_out;
    p->w_off.push_back(o);
    o += din * dout;
    p->b_off.push_back(o);
    o += dout;
    din = width;
  }
  p->n_params = o;
  const int64_t B = max_batch;
  bool ok = dal(&p->theta, o) && dal(&p->grad, o) && dal(&p->m, o) && dal(&p->v, o) && dal(&p->thb, o) &&
            dal(&p->xb, B * n_in) && dal(&p->logits, B * n_out) && dal(&p->dlog, B * n_out) &&
            dal(&p->dlogb, B * n_out) && dal(&p->dh, B * width) && dal(&p->dz, B * width) &&
            dal(&p->dzb, B * width) && dal(&p->loss, 1);
  for (int l = 0; ok && l < depth; ++l) {
    float* zz = nullptr;
    bf16* hh = nullptr;
    ok = dal(&zz, B * width) && dal(&hh, B * width);
    p->z.push_back(zz);
    p->h.push_back(hh);
  }
  if (!ok) {
    cudaGetLastError();
    mf_mlp_destroy(p);
    return mfail(nullptr, MF_ENOMEM, "mf_mlp_create: device allocation");
  }
  cudaMemsetAsync(p->theta, 0, o * sizeof(float), p->st);
  cudaMemsetAsync(p->thb, 0, o * sizeof(bf16), p->st);
  cudaMemsetAsync(p->m, 0, o * sizeof(float), p->st);
  cudaMemsetAsync(p->v, 0, o * sizeof(float), p->st);
  *out = p;
  return MF_OK;
}

void mf_mlp_destroy(mf_mlp_t p) {
  if (!p) return;
  if (p->st) cudaStreamSynchronize(p->st); else cudaDeviceSynchronize();
  for (void* q : {(void*)p->theta, (void*)p->grad, (void*)p->m, (void*)p->v, (void*)p->thb, (void*)p->xb,
                  (void*)p->logits, (void*)p->dlog, (void*)p->dlogb, (void*)p->dh, (void*)p->dz, (void*)p->dzb,
                  (void*)p->loss})
    if (q) cudaFree(q);
  for (auto* q : p->z) if (q) cudaFree(q);
  for (auto* q : p->h) if (q) cudaFree(q);
  delete p;
}

int64_t mf_mlp_num_params(mf_mlp_t p) { return p ? p->n_params : -1; }

mf_status mf_mlp_set_params(mf_mlp_t p, const float* theta, int64_t n, int on_device) {
  if (!p || !theta) return mfail(p, MF_EINVAL, "mf_mlp_set_params: null argument");
  if (n != p->n_params) return mfail(p, MF_EINVAL, "mf_mlp_set_params: n must equal mf_mlp_num_params");
  cudaError_t e = cudaMemcpyAsync(p->theta, theta, n * sizeof(float),
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, p->st);
  if (e == cudaSuccess) {
    k_to_bf16<<<sms() * 4, 256, 0, p->st>>>(p->theta, p->thb, n);
    mf::add_launches(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(p->m, 0, n * sizeof(float), p->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->v, 0, n * sizeof(float), p->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
  if (e != cudaSuccess) return mfail(p, MF_ECUDA, std::string("mf_mlp_set_params: ") + cudaGetErrorString(e));
  p->step = 0;
  return MF_OK;
}

mf_status mf_mlp_get_params(mf_mlp_t p, float* theta, int64_t n) {
  if (!p || !theta || n != p->n_params) return mfail(p, MF_EINVAL, "mf_mlp_get_params: bad argument");
  cudaError_t e = cudaMemcpyAsync(theta, p->theta, n * sizeof(float), cudaMemcpyDeviceToHost, p->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
  if (e != cudaSuccess) return mfail(p, MF_ECUDA, std::string("mf_mlp_get_params: ") + cudaGetErrorString(e));
  return MF_OK;
}

mf_status mf_mlp_forward(mf_mlp_t p, const float* x, int64_t B, float* logits) {
  if (!p || !x) return mfail(p, MF_EINVAL, "mf_mlp_forward: null argument");
  if (B < 1 || B > p->max_batch) return mfail(p, MF_EINVAL, "mf_mlp_forward: batch out of range");
  cudaError_t e = forward(p, x, (int)B);
  if (e == cudaSuccess && logits)
    e = cudaMemcpyAsync(logits, p->logits, B * p->n_out * sizeof(float), cudaMemcpyDeviceToDevice, p->st);
  if (e != cudaSuccess) return mfail(p, MF_ECUDA, std::string("mf_mlp_forward: ") + cudaGetErrorString(e));
  return MF_OK;
}

mf_status mf_mlp_loss_grad(mf_mlp_t p, const float* x, const int32_t* n_valid, const int32_t* label, int64_t B,
                           float* loss, float* grad) {
  if (!p || !x || !n_valid || !label) return mfail(p, MF_EINVAL, "mf_mlp_loss_grad: null argument");
  if (B < 1 || B > p->max_batch) return mfail(p, MF_EINVAL, "mf_mlp_loss_grad: batch out of range");
  const int Bi = (int)B, W = p->width, D = p->depth, g = sms() * 4;
  cudaError_t e = forward(p, x, Bi);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->loss, 0, sizeof(float), p->st);
  if (e != cudaSuccess) return mfail(p, MF_ECUDA, std::string("mf_mlp_loss_grad: ") + cudaGetErrorString(e));
  k_masked_ce<<<Bi, 256, 0, p->st>>>(p->logits, p->n_out, n_valid, label, Bi, p->loss, p->dlog, p->dlogb);
  mf::add_launches(1);
  // output layer
  const bf16* hlast = D > 0 ? p->h[D - 1] : p->xb;
  e = gemm(p->st, W, p->n_out, Bi, hlast, W, 1, p->dlogb, p->n_out, 0, p->grad + p->w_off[D], p->n_out, nullptr);
  k_colsum<<<(p->n_out + 255) / 256, 256, 0, p->st>>>(p->dlog, Bi, p->n_out, p->grad + p->b_off[D]);
  mf::add_launches(1);
  // dH_D = dlog W_out^T
  if (e == cudaSuccess) e = gemm(p->st, Bi, W, p->n_out, p->dlogb, p->n_out, 0, p->thb + p->w_off[D], p->n_out, 1,
                                 p->dh, W, nullptr);
  for (int l = D - 1; l >= 0 && e == cudaSuccess; --l) {
    k_gelu_bwd<<<g, 256, 0, p->st>>>(p->dh, p->z[l], p->dz, p->dzb, (int64_t)Bi * W);
    k_colsum<<<(W + 255) / 256, 256, 0, p->st>>>(p->dz, Bi, W, p->grad + p->b_off[l]);
    mf::add_launches(2);
    const bf16* hprev = l > 0 ? p->h[l - 1] : p->xb;
    const int kin = l > 0 ? W : p->n_in;
    e = gemm(p->st, kin, W, Bi, hprev, kin, 1, p->dzb, W, 0, p->grad + p->w_off[l], W, nullptr);
    if (e == cudaSuccess && l > 0)
      e = gemm(p->st, Bi, W, W, p->dzb, W, 0, p->thb + p->w_off[l], W, 1, p->dh, W, nullptr);
  }
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, p->loss, sizeof(float), cudaMemcpyDeviceToDevice, p->st);
  if (e == cudaSuccess && grad)
    e = cudaMemcpyAsync(grad, p->grad, p->n_params * sizeof(float), cudaMemcpyDeviceToDevice, p->st);
  if (e != cudaSuccess) return mfail(p, MF_ECUDA, std::string("mf_mlp_loss_grad: ") + cudaGetErrorString(e));
  return MF_OK;
}

mf_status mf_mlp_adamw_step(mf_mlp_t p, float lr, float beta1, float beta2, float eps, float weight_decay) {
  if (!p) return mfail(p, MF_EINVAL, "mf_mlp_adamw_step: null plan");
  p->step += 1;
  const float c1 = 1.f - std::pow(beta1, (float)p->step), c2 = 1.f - std::pow(beta2, (float)p->step);
  k_adamw<<<sms() * 4, 256, 0, p->st>>>(p->theta, p->grad, p->m, p->v, p->n_params, lr, beta1, beta2, eps,
                                         weight_decay, c1, c2, p->thb);
  mf::add_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return mfail(p, MF_ECUDA, std::string("mf_mlp_adamw_step: ") + cudaGetErrorString(e));
  return MF_OK;
}

mf_status mf_mlp_topk(mf_mlp_t p, const float* x, const int32_t* n_valid, int64_t B, int32_t k, float p_mass,
                      int32_t* out, int32_t* count) {
  if (!p || !x || !n_valid || !out) return mfail(p, MF_EINVAL, "mf_mlp_topk: null argument");
  if (B < 1 || B > p->max_batch || k < 1 || k > 64) return mfail(p, MF_EINVAL, "mf_mlp_topk: bad batch or k");
  cudaError_t e = forward(p, x, (int)B);
  if (e == cudaSuccess) {
    k_topk<<<(unsigned)B, 128, 0, p->st>>>(p->logits, p->n_out, n_valid, k, p_mass, out, count);
    mf::add_launches(1);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return mfail(p, MF_ECUDA, std::string("mf_mlp_topk: ") + cudaGetErrorString(e));
  return MF_OK;
}

const char* mf_mlp_last_error(mf_mlp_t p) { return p ? p->err.c_str() : ""; }

}  // extern "C"
