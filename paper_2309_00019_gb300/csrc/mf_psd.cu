// PSD estimation upstream of the filter: Welch's method on the GPU.
//
// The weights of Eq. (2) need the one-sided PSD S_n of the data; the paper
// takes it from the data without describing the estimate.  Reading: Welch
// segments of seg_len samples every stride samples with a periodic Hann
// window and no detrending, averaged by the mean or by the median divided by
// its bias for exponential periodogram values (FINDCHIRP, Appendix B).
//   k_welch_rows   gathers the windowed segments of every detector as rows;
//   the rows go through the library's real-input transform (k_pass1/k_pass2);
//   k_welch_reduce forms each bin's periodogram values in FP64 and reduces
//                  them over segments (fixed-order sum, or a bitonic sort in
//                  shared memory for the median), one CTA per (bin, detector).
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "../../include/mf.h"
#include "mf_common.cuh"

namespace mf {
namespace {

constexpr int kWT = 256;        // threads per reduction CTA
constexpr int kMaxSeg = 4096;   // segments held in shared memory by the median

// rows[s n_det + d][j] = w[j] x[d][s stride + j], w[j] = (1 - cos(2 pi j / n)) / 2
__global__ void k_welch_rows(const float* __restrict__ x, int64_t ld, int n_det, int64_t stride, int lg_n,
                             int64_t rows, float* __restrict__ out) {
  const int64_t n = int64_t(1) << lg_n;
  const int64_t total = rows << lg_n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i >> lg_n, j = i & (n - 1);
    const int64_t s = r / n_det;
    const int d = (int)(r - s * n_det);
    const float w = 0.5f - 0.5f * cospif(2.0f * (float)j / (float)n);
    out[i] = w * x[d * ld + s * stride + j];
  }
}

// psd[d][k] = average over segments s of c fs |X_s[k]|^2 / sum w^2, with X the
// dt-normalised spectrum of the windowed segment (so |FFT|^2 = fs^2 |X|^2),
// sum w^2 = 3n/8 and c = 2 off DC and Nyquist.
__global__ void __launch_bounds__(kWT) k_welch_reduce(const float2* __restrict__ fd, int64_t ld_fd, int n_det,
                                                      int64_t n_seg, int64_t n, double fs, int average,
                                                      double median_bias, double* __restrict__ psd) {
  __shared__ double v[kMaxSeg];
  __shared__ double red[kWT];
  const int64_t k = blockIdx.x;
  const int d = blockIdx.y;
  const double c = (k == 0 || k == n / 2) ? 1.0 : 2.0;
  const double norm = c * fs / (0.375 * (double)n);
  if (average == 0) {
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n_seg; i += kWT) {
      const float2 z = fd[(i * n_det + d) * ld_fd + k];
      s += norm * ((double)z.x * z.x + (double)z.y * z.y);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = kWT / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) psd[(int64_t)d * (n / 2 + 1) + k] = red[0] / (double)n_seg;
    return;
  }
  int m = 1;
  while (m < n_seg) m <<= 1;
  for (int i = threadIdx.x; i < m; i += kWT) {
    if (i < n_seg) {
      const float2 z = fd[((int64_t)i * n_det + d) * ld_fd + k];
      v[i] = norm * ((double)z.x * z.x + (double)z.y * z.y);
    } else {
      v[i] = INFINITY;
    }
  }
  __syncthreads();
  for (int size = 2; size <= m; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < m; i += kWT) {
        const int j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          const double a = v[i], b = v[j];
          if ((a > b) == up) {
            v[i] = b;
            v[j] = a;
          }
        }
      }
      __syncthreads();
    }
  if (threadIdx.x == 0) {
    const double med = (n_seg & 1) ? v[n_seg / 2] : 0.5 * (v[n_seg / 2 - 1] + v[n_seg / 2]);
    psd[(int64_t)d * (n / 2 + 1) + k] = med / median_bias;
  }
}

int sms_p() {
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
}  // namespace mf

extern "C" mf_status mf_psd_welch(double fs, int32_t n_det, int64_t n_samples, const float* strain, int64_t ld,
                                  int64_t seg_len, int64_t stride, int32_t average, double* psd, void* cuda_stream) {
  auto bad = [](const char* m) {
    mf::set_global_error(std::string("mf_psd_welch: ") + m);
    return MF_EINVAL;
  };
  if (!strain || !psd) return bad("null argument");
  if (!(fs > 0) || n_det < 1 || n_det > 8 || ld < n_samples) return bad("fs, n_det or ld");
  if (seg_len < 4096 || seg_len > mf::kMaxN || (seg_len & (seg_len - 1))) return bad("seg_len must be a power of two in [2^12, 2^20]");
  if (stride < 1 || n_samples < seg_len) return bad("stride < 1 or data shorter than one segment");
  if (average != 0 && average != 1) return bad("average must be 0 (mean) or 1 (median)");
  const int64_t n_seg = (n_samples - seg_len) / stride + 1;
  if (average == 1 && n_seg > mf::kMaxSeg) return bad("more than 4096 segments for the median");
  const int64_t rows = n_seg * n_det;
  int lg = 0;
  while ((int64_t(1) << lg) < seg_len) ++lg;
  const int n1 = 1 << ((lg + 1) / 2), n2 = 1 << (lg / 2);
  const int64_t nb = seg_len / 2 + 1, ld_fd = (nb + 63) / 64 * 64;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  float* seg = nullptr;
  float2 *scratch = nullptr, *fd = nullptr;
  cudaError_t e = cudaMalloc((void**)&seg, (size_t)rows * seg_len * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&scratch, (size_t)rows * seg_len * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc((void**)&fd, (size_t)rows * ld_fd * sizeof(float2));
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(seg);
    cudaFree(scratch);
    mf::set_global_error(std::string("mf_psd_welch: work space: ") + cudaGetErrorString(e));
    return MF_ENOMEM;
  }
  // median bias of n_seg exponential values: 1 - 1/2 + 1/3 - ... to 1/(2m+1), m = (n_seg - 1) / 2
  double bias = 1.0;
  for (int64_t i = 1; i <= (n_seg - 1) / 2; ++i) bias += 1.0 / (2.0 * i + 1.0) - 1.0 / (2.0 * i);
  const int64_t total = rows * seg_len;
  const int grid = (int)std::min<int64_t>((total + 255) / 256, (int64_t)mf::sms_p() * 8);
  mf::k_welch_rows<<<grid, 256, 0, st>>>(strain, ld, n_det, stride, lg, rows, seg);
  mf::add_launches(1);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = mf::launch_rfft(seg, seg_len, (int)rows, seg_len, n1, n2, 1.0 / fs, scratch, fd, ld_fd, st);
  if (e == cudaSuccess) {
    mf::k_welch_reduce<<<dim3((unsigned)nb, (unsigned)n_det), mf::kWT, 0, st>>>(fd, ld_fd, n_det, n_seg, seg_len, fs,
                                                                               average, bias, psd);
    mf::add_launches(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(seg);
  cudaFree(scratch);
  cudaFree(fd);
  if (e != cudaSuccess) {
    mf::set_global_error(std::string("mf_psd_welch: ") + cudaGetErrorString(e));
    return MF_ECUDA;
  }
  return MF_OK;
}
