/*
 * libmf - GB300 (sm_103a) hot path of a two-stage hierarchical matched-filter
 * search for compact-binary gravitational-wave signals.
 *
 * Plain C ABI: opaque handles, plain pointers and sizes, no exceptions.  Every
 * call returns an mf_status; on failure mf_last_error(plan) describes it.
 * "device" pointers are CUDA global-memory addresses of the current device
 * (e.g. torch.Tensor.data_ptr() of a CUDA tensor); "host" pointers are CPU
 * memory.  Unless stated otherwise the caller owns every buffer it passes and
 * the library copies what it keeps.  Work is enqueued asynchronously on the
 * plan's CUDA stream; calls that return data to the host synchronise it.
 * A plan is not thread-safe: use one plan per host thread.
 *
 * Conventions (shared with the documentation of every call):
 *   N = FFT length (samples per segment), fs = sampling rate, dt = 1/fs,
 *   df = fs/N, one-sided frequency bins k = 0..N/2 (nbins = N/2 + 1),
 *   x~[k] = dt * sum_j x[j] exp(-2 pi i j k / N).
 *   Complex arrays are interleaved (re, im) pairs: float32 pairs for MF_F32,
 *   IEEE half pairs for MF_F16, bfloat16 pairs for MF_BF16.
 */
#ifndef MF_H_
#define MF_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mf_plan_s* mf_plan_t;

typedef enum {
  MF_OK = 0,
  MF_EINVAL = 1,       /* bad argument (null pointer, size, unsupported N ...) */
  MF_ENOMEM = 2,       /* device or host allocation failed */
  MF_ECUDA = 3,        /* a CUDA runtime call or kernel launch failed */
  MF_ESTATE = 4,       /* call out of order (e.g. mf_filter before mf_set_psd) */
  MF_EOVERFLOW = 5,    /* more results than the buffer holds; the count is still exact */
  MF_ETIMEOUT = 6      /* a bounded device wait gave up (reported, never trapped) */
} mf_status;

typedef enum { MF_F32 = 0, MF_F16 = 1, MF_BF16 = 2, MF_F16X2 = 3 } mf_dtype;  /* MF_F16X2: intermediates only */

/* Plan description.  The matched filter of Eq. (1)-(2) (Sec. II) on segments
 * of N samples: the analysis band is f_low <= f_k < f_high, 0 < k < N/2, and
 * PSD bins that are positive and finite.  A trigger is kept when
 * rho >= snr_thr (Sec. II, inclusive); one trigger per (detector, template,
 * window of `window` samples aligned to sample 0), at the window's peak
 * (ties: lowest sample).  Only samples in [valid_begin, valid_end) count. */
typedef struct {
  double fs;             /* sampling rate, Hz (> 0) */
  int64_t n;             /* N, a power of two in [2^12, 2^20] */
  int32_t n_det;         /* data rows (detectors, or detector x segment), 1..65536 */
  double f_low, f_high;  /* band edges, Hz */
  mf_dtype dtype;        /* storage type of the template bank */
  double snr_thr;        /* rho threshold (> 0) */
  int64_t window;        /* clustering window, samples, 1 <= window <= N */
  int64_t valid_begin;   /* analysed range [valid_begin, valid_end), 0 <= b < e <= N */
  int64_t valid_end;
  int64_t max_triggers;  /* capacity of the device trigger buffer (>= 1) */
  void* cuda_stream;     /* cudaStream_t to enqueue on; NULL = legacy default stream */
} mf_plan_desc;

/* One trigger: detector, template id, sample index of the window peak,
 * rho at that sample and arg z (quantised to 2 pi / 2048). */
typedef struct {
  int32_t det;
  int32_t tmpl;
  int64_t sample;
  float snr;
  float phase;
} mf_trigger;

/* Create a plan (device buffers for the PSD weights and work space).
 * *out is set only on MF_OK.  Errors: MF_EINVAL for an invalid desc. */
mf_status mf_plan(mf_plan_t* out, const mf_plan_desc* desc);

/* Destroy a plan and free everything it owns (NULL is a no-op). */
void mf_destroy(mf_plan_t plan);

/* Message of the last failed call on this plan ("" if none).  Owned by the plan. */
const char* mf_last_error(mf_plan_t plan);

/* Set the one-sided PSD S_n(f_k) (Eq. 2), host float64 [nbins], nbins = N/2+1.
 * Copied.  Builds the weights w[k] = 4 df / S_n[k] on the band (0 elsewhere,
 * and 0 where S_n[k] <= 0 or is not finite).  Recomputes sigma^2 of a loaded
 * bank.  Errors: MF_EINVAL (null, nbins != N/2+1). */
mf_status mf_set_psd(mf_plan_t plan, const double* psd, int64_t nbins);

/* One-sided PSD S_n of long data by Welch's method (the weights of Eq. 2 need
 * the PSD of the data; the paper does not describe its estimate, this is the
 * reading): for each detector row of strain (device float32 [n_det][ld],
 * n_samples used), segments of seg_len samples (a power of two in
 * [2^12, 2^20]) every stride samples (those that fit), periodic Hann window
 * w[j] = (1 - cos(2 pi j / seg_len)) / 2, no detrending,
 *   P[k] = c |sum_j w[j] x[j] e^{-2 pi i j k / seg_len}|^2 / (fs sum_j w[j]^2),
 * c = 2 except at DC and Nyquist (c = 1), averaged over segments by the mean
 * (average = 0) or by the median divided by 1 - 1/2 + 1/3 - ... (m terms
 * after the first, m = (segments - 1) / 2; FINDCHIRP Appendix B; average = 1,
 * at most 4096 segments).  psd: device float64 [n_det][seg_len/2+1] (out).
 * Allocates segments x n_det x seg_len x 20 bytes of work space for the call.
 * Synchronises.  Errors (mf_last_error(NULL)): MF_EINVAL, MF_ENOMEM, MF_ECUDA. */
mf_status mf_psd_welch(double fs, int32_t n_det, int64_t n_samples, const float* strain, int64_t ld, int64_t seg_len,
                       int64_t stride, int32_t average, double* psd, void* cuda_stream);

/* Gating of loud short transients before the filter (Sec. VI: short-duration
 * artifacts are removed by gating before matched filtering; the paper cites
 * the method without its statistic or parameters, so these are readings).
 *
 * mf_load_gate_template replaces the plan's bank by one row,
 * h~[k] = sqrt(S_n[k]) on the band of Eq. (2) and 0 elsewhere, so that
 * mf_filter computes the gate statistic
 *   rho_g(t) = |z_g(t)| / sigma_g,
 *   z_g(t) = 4 df sum_{k in band} s~[k] / sqrt(S_n[k]) e^{+2 pi i t k / N},
 *   sigma_g^2 = 4 df n_band,
 * the envelope of the band-limited whitened strain in matched-filter SNR units
 * (rho_g^2 is chi^2 with 2 dof in Gaussian noise); the plan's triggers (per
 * window, the peak with rho_g >= the plan's threshold, tmpl 0) are the gates.
 * Needs the PSD (mf_set_psd).  Errors: MF_ESTATE, MF_ENOMEM, MF_ECUDA. */
mf_status mf_load_gate_template(mf_plan_t plan);

/* out[d][j] = strain[d][j] prod over the gates c of row d of W(|j - c| / fs),
 * W(t) = 0 for t <= t_zero, (1 - cos(pi (t - t_zero) / t_taper)) / 2 for
 * t_zero < t < t_zero + t_taper, 1 beyond (an inverse Tukey window; FP64).
 * gates: device mf_trigger list sorted by (det, sample), the first
 * min(*count, max_gates) used (mf_device_triggers of a plan loaded with
 * mf_load_gate_template); count: device int64.  strain, out: device float32
 * [n_det][ld], [n_det][ld_out] (out may be strain).  Asynchronous on
 * cuda_stream.  Errors: MF_EINVAL, MF_ECUDA. */
mf_status mf_gate_apply(const float* strain, int64_t ld, int32_t n_det, int64_t n, double fs, const mf_trigger* gates,
                        const int64_t* count, int64_t max_gates, double t_zero, double t_taper, float* out,
                        int64_t ld_out, void* cuda_stream);

/* Replace the template bank (Sec. II; Table I): n_tmpl one-sided templates
 * h~_t[k], row t at htilde + t*ld elements, k = 0..N/2 (ld >= N/2+1).  dtype
 * MF_F32 (scales must be NULL) or MF_F16 / MF_BF16 with host float32
 * scales[n_tmpl] (h~ = scale_t * stored value).  on_device != 0: htilde is a
 * device pointer, else host.  Device rows are read on the plan's stream after
 * the work already submitted to the legacy default stream (so rows written
 * there, or on a blocking stream, are complete); rows written on another
 * non-blocking stream must be complete before the call (the plans of an
 * mf_batch_t run on the batch's own streams).  Copied into plan-owned device
 * memory.  If the
 * PSD is set, sigma_t^2 = sum_k w[k] |h~_t[k]|^2 is computed in float64 on the
 * device (Eq. 2).  Errors: MF_EINVAL, MF_ENOMEM. */
mf_status mf_load_bank(mf_plan_t plan, const void* htilde, mf_dtype dtype, int64_t n_tmpl, int64_t ld,
                       const float* scales, int on_device);

/* Reserve an empty bank of n_tmpl templates (zeros) to be filled in row
 * blocks with mf_bank_set_rows; lets multi-GB banks be loaded piecewise. */
mf_status mf_bank_reserve(mf_plan_t plan, mf_dtype dtype, int64_t n_tmpl);

/* Copy rows [row0, row0+n_rows) of the bank (layout as mf_load_bank; scales
 * host float32 [n_rows] or NULL for MF_F32) and compute their sigma^2. */
mf_status mf_bank_set_rows(mf_plan_t plan, int64_t row0, int64_t n_rows, const void* htilde, int64_t ld,
                           const float* scales, int on_device);

/* TaylorF2 templates generated on the GPU (Sec. II: the bank's waveforms;
 * the paper does not name them, the bank here is non-spinning TaylorF2 with
 * the 3.5PN phase of Buonanno et al. 2009, Eq. 3.18, and Newtonian
 * amplitude): h~(f) = f^{-7/6} exp(-i Psi(f)) for f_low <= f <=
 * min(f_ISCO, fs/2), bin k < N/2, zero elsewhere, with t_c = phi_c = 0 and
 * f_ISCO = 1 / (6^{3/2} pi M).  Psi is evaluated in float64 at anchors at most
 * 0.25 Hz apart and interpolated (cubic) in float32 between them; the
 * template's match with the float64 formula is 1 to better than 1e-8.
 *   m1, m2: host float64 [n_tmpl], solar masses (copied)
 *   out:    device complex64 [n_tmpl][ld], ld >= N/2+1, bins 0..N/2 written
 * Synchronises cuda_stream.  Errors (mf_last_error(NULL)): MF_EINVAL (sizes,
 * masses <= 0, f_low <= 0), MF_ECUDA. */
mf_status mf_taylorf2(const double* m1, const double* m2, int64_t n_tmpl, double fs, int64_t n, double f_low,
                      void* out, int64_t ld, void* cuda_stream);

/* Generate bank rows [row0, row0+n_rows) of the plan on the GPU (as
 * mf_taylorf2 at the plan's fs and N, f_low given), store them in the bank's
 * layout and type (float32, or 16-bit as mf_bank_quantize_rows) and compute
 * their sigma^2: banks are filled without a host copy of the templates.
 * Synchronises.  Errors: MF_ESTATE (no bank), MF_EINVAL, MF_ENOMEM, MF_ECUDA. */
mf_status mf_bank_generate_taylorf2(mf_plan_t plan, int64_t row0, int64_t n_rows, const double* m1, const double* m2,
                                    double f_low);

/* Reduced-precision storage (no counterpart in the paper, which filters in
 * double precision on CPUs): quantise rows [row0, row0+n_rows) of a 16-bit
 * bank (reserved as MF_F16 or MF_BF16) from float32 complex templates
 * htilde [n_rows][ld] (device if on_device, else host).  Each template gets a
 * power-of-two scale s_t with max |h~_t / s_t| in [2^14, 2^15) (per real and
 * imaginary component), the stored value is h~_t / s_t rounded to nearest
 * even, and sigma_t^2 (Eq. 2) is computed in float64 from the stored values
 * times s_t, so the normalisation matches what is filtered.  Synchronises.
 * Errors: MF_ESTATE (no bank, or an MF_F32 bank), MF_EINVAL, MF_ENOMEM. */
mf_status mf_bank_quantize_rows(mf_plan_t plan, int64_t row0, int64_t n_rows, const void* htilde, int64_t ld,
                                int on_device);

/* Storage type of the weighted data w s~ that the filter reads (Eq. 2):
 * MF_F32 (default) or the bank's own 16-bit type.  With 16-bit data each
 * mf_filter quantises w s~ per detector with a power-of-two scale c_d
 * (max |c_d w s~| in [2^14, 2^15)) and the epilogue removes c_d exactly;
 * products and transforms stay float32.  A 16-bit type other than the bank's
 * makes mf_filter fail with MF_EINVAL.  Plans built with another filter
 * implementation switch to the TMA-staged one.  Errors: MF_EINVAL, MF_ENOMEM. */
mf_status mf_set_data_dtype(mf_plan_t plan, mf_dtype dtype);

/* Per-row analysed ranges for plans whose rows are overlapping segments of
 * longer data (Sec. V.C: the data are analysed in overlapping segments): row
 * d keeps only samples in [range[2d], range[2d+1]) (host int64 [2 n_det],
 * 0 <= begin <= end <= N; copied), replacing the plan's valid range for
 * every row; NULL restores it.  Plans built with another filter
 * implementation switch to the TMA-staged one.  Errors: MF_EINVAL, MF_ENOMEM. */
mf_status mf_set_row_valid(mf_plan_t plan, const int64_t* range);

/* Storage of the pass-1 -> pass-2 intermediate of mf_filter (Sec. V.C: the
 * FFT over coalescence time, here N = N1 N2 in two passes).  MF_F32
 * (default): complex64, and the row pass runs on the FP32 ALUs.  MF_F16
 * (N = 2^20 only): complex FP16, each series scaled by a power of two that
 * puts its values near RMS sqrt(2 / N2), in 8-row panels, and the row pass
 * runs on the tensor cores: each 1024-point row transform is two radix-32
 * stages, each a product with the 32 x 32 DFT matrix (FP16 operands, FP32
 * accumulation in tensor memory).  This halves the intermediate's HBM round
 * trip and moves the row transforms off the ALUs; SNR then agrees with the
 * FP64 filter to a few 1e-4 relative (within 1e-3) instead of 1e-6, so the
 * threshold and window peaks can differ at near-ties of that size.  MF_F16X2
 * (N = 2^20 only): each value as an FP16 pair hi + lo (hi = the value rounded
 * to FP16, lo = the remainder rounded to FP16), 8 bytes per point like
 * complex64, and the same tensor-core row pass with the stage operands and the
 * DFT matrices split the same way: three products per step (hi hi, lo hi,
 * hi lo), so each stage keeps about 22 significant bits and SNR stays at the
 * FP32 path's level (1e-4 and better).  Needs FP32 weighted data (MF_F32 data
 * dtype).  Synchronises.  Errors: MF_EINVAL (dtype, or MF_F16 / MF_F16X2 with
 * N != 2^20). */
mf_status mf_set_intermediate(mf_plan_t plan, mf_dtype dtype);

/* Templates per pass-1/pass-2 launch pair (the batch; default: as many as
 * fit a 1 GB intermediate).  Reallocates the intermediate (batch x n_det x
 * N x 8 bytes).  Errors: MF_EINVAL (batch < 1), MF_ENOMEM. */
mf_status mf_set_batch(mf_plan_t plan, int32_t batch);

/* sigma_t^2 of templates 0..n-1 (float64, Eq. 2) into host out[n]; synchronises. */
mf_status mf_get_sigmasq(mf_plan_t plan, double* out, int64_t n);

/* A1 (Eq. 2 input): one-sided dt-normalised spectrum of real strain.
 * strain: device float32 [n_det][ld_strain] (N samples used per detector);
 * dtilde: device complex64 [n_det][ld_dtilde], ld_dtilde >= N/2+1, receives
 * bins 0..N/2.  Asynchronous. */
mf_status mf_strain_to_fd(mf_plan_t plan, const float* strain, int64_t ld_strain, void* dtilde, int64_t ld_dtilde);

/* A2 (Sec. III, stage 1 at a reduced rate): the spectrum of the same data at
 * this plan's (lower) rate is bins 0..N/2 of the higher-rate spectrum.
 * dtilde_in: device complex64 [n_det][ld_in] with ld_in >= N/2+1 of this plan;
 * dtilde_out: device complex64 [n_det][ld_out].  Asynchronous. */
mf_status mf_decimate(mf_plan_t plan, const void* dtilde_in, int64_t ld_in, void* dtilde_out, int64_t ld_out);

/* A4-A7 (Eq. 1-2, Sec. II, Sec. V.C): filter every detector of dtilde
 * (device complex64 [n_det][ld_dtilde], one-sided spectra) against templates
 * subset[0..n_subset-1] (device int32 template ids, ascending for ordered
 * output); n_subset < 0 selects all templates (subset must then be NULL) and
 * n_subset == 0 selects none (the trigger list becomes empty).  Computes
 * z = IFFT(w s~ h~*), rho^2 = |z|^2 / sigma^2, threshold and window maxima
 * entirely on the device; the SNR series never leaves on-chip memory.
 * Asynchronous; results via mf_get_triggers.  Errors: MF_ESTATE (no PSD or
 * bank), MF_EINVAL (bad template id range is not checked on the device:
 * ids must be in [0, n_tmpl)). */
mf_status mf_filter(mf_plan_t plan, const void* dtilde, int64_t ld_dtilde, const int32_t* subset, int64_t n_subset);

/* Triggers of the last mf_filter, ordered by (det, position in the subset,
 * sample), into host out[cap]; *n_found = total number found.  Synchronises.
 * MF_EOVERFLOW if *n_found > cap or > max_triggers (the first
 * min(cap, max_triggers) are returned). */
mf_status mf_get_triggers(mf_plan_t plan, mf_trigger* out, int64_t cap, int64_t* n_found);

/* Device view of the last filter's results: *trig = device mf_trigger array,
 * *count = device int64 holding the number found (read after the stream
 * completes).  Valid until the next mf_filter or mf_destroy. */
mf_status mf_device_triggers(mf_plan_t plan, const mf_trigger** trig, const int64_t** count);

/* ---- instrumentation ---------------------------------------------------- */

/* Counters of one plan.  launches: kernels this plan enqueued.  When profiling
 * is on, CUDA events bracket the two filter kernels of each template batch on
 * the plan's stream (up to 4096 batches between reads; a batch runner's fused
 * launch pairs are reported by its first class's plan): pass1_* is the
 * product + column-transform kernel, pass2_* the row-transform + SNR /
 * threshold / window-max kernel; *_series = (template, detector) series they
 * processed, *_ms = summed device time. */
typedef struct {
  int64_t launches;
  int64_t pass1_launches, pass1_series;
  double pass1_ms;
  int64_t pass2_launches, pass2_series;
  double pass2_ms;
  int32_t impl;       /* filter kernels in use: 2 = k_cols / k_rows (FP32 intermediate), 3 = k_cols /
                         k_rows_tc (FP16 intermediate, tensor-core row pass), 4 = k_cols / k_rows_tc
                         with FP16 pairs (MF_F16X2) */
  int32_t batch;      /* templates per pass-1 / pass-2 launch pair */
} mf_plan_stats;

/* Event profiling of the filter kernels: enable = 0 off, 1 every template
 * batch, k > 1 every k-th batch (counted across calls).  The events between
 * the two kernels of a timed batch keep the second from launching early, so
 * a stride keeps that cost to the sampled batches.  Errors: MF_EINVAL
 * (enable < 0). */
mf_status mf_profile(mf_plan_t plan, int enable);

/* Read the counters into *out (synchronises the plan's stream); reset != 0
 * zeroes them afterwards. */
mf_status mf_get_stats(mf_plan_t plan, mf_plan_stats* out, int reset);

/* Signal-based veto at the triggers of the last mf_filter (Sec. II: triggers
 * are down-weighted by their chi^2; the re-weighted SNR is Eq. 4).  For each
 * trigger (det, tmpl, sample) of the device trigger list (mf_device_triggers
 * order, the first min(count, max_triggers)), with z the filter output at
 * the sample split over n_bands frequency bands of equal template power
 * (band l = bins k with floor(n_bands C(k) / sigma^2) = l, C(k) = the
 * template power sum_{k' < k} w |h~|^2 below k; the paper cites the test
 * without its bands, this is the reading):
 *   chi2[i]   = n_bands sum_l |z_l - z / n_bands|^2 / sigma^2  (2 n_bands - 2 dof),
 *   newsnr[i] = rho / [(1 + c^3) / 2]^{1/6} with c = chi2 / (2 n_bands - 2) if
 *               c >= 1, else rho  (Eq. 4).
 * chi2, newsnr: device float32 [max_triggers].  The band edges are computed
 * on the first call for a bank, PSD and n_bands (FP64).  Asynchronous on the
 * plan's stream.  Errors: MF_EINVAL (n_bands not in [2, 64]), MF_ESTATE (no
 * filter run), MF_ENOMEM. */
mf_status mf_chisq(mf_plan_t plan, int32_t n_bands, float* chi2, float* newsnr);

/* Sine-Gaussian veto of heavy templates at trigger times (Sec. III: triggers
 * of templates heavier than 30 M_sun are further re-weighted with chi^2_sg
 * against short glitches; the paper cites the test without its tiles or
 * normalisation, this is the reading).  For trigger i of the device trigger
 * list (template t, detector d, sample j) with mtotal[t] > m_min and
 * snr_in[i] >= snr_min, tiles l = 0..n_tiles-1 at f_l = f_final[t] +
 * offsets[l] (those at or above the band's upper edge skipped), spectra
 * g~_l[k] = exp(-(pi tau_l (f_k - f_l))^2), tau_l = q / (sqrt(2) pi f_l), give
 *   rho_l^2 = |sum_k w s~ g~_l e^{+2 pi i k j / N}|^2 / sum_k w g~_l^2
 * (w = 4 df / S_n on the band, Eq. 2), and
 *   chi2_r[i]  = sum_l rho_l^2 / (2 n_used)   (chi^2_sg, mean 1 in Gaussian noise),
 *   snr_hat[i] = snr_in[i] chi2_r^{-1/2} if chi2_r >= 6, else snr_in[i]  (Eq. 3);
 * other triggers get chi2_r 0 and snr_hat = snr_in.  f_final, mtotal: device
 * float [n_tmpl] (Hz, solar masses); offsets: host double [n_tiles] (Hz),
 * 1 <= n_tiles <= 16; snr_in (e.g. mf_chisq's newsnr), chi2_r, snr_hat:
 * device float [max_triggers] in trigger order.  Asynchronous on the plan's
 * stream.  Errors: MF_EINVAL, MF_ESTATE (no filter run), MF_ECUDA. */
mf_status mf_sgchisq(mf_plan_t plan, const float* f_final, const float* mtotal, float m_min, float snr_min,
                     int32_t n_tiles, const double* offsets, double q, const float* snr_in, float* chi2_r,
                     float* snr_hat);

/* Failure detection without a GPU fault (no counterpart in the paper): every
 * device wait in the filter kernels is bounded; on expiry it records a timeout
 * in the plan's status word, the kernel returns, and the next mf_get_triggers
 * returns MF_ETIMEOUT (clearing the word).  This call exercises that path: it
 * launches, on the plan's stream, one CTA of 128 threads that wait on a
 * barrier nothing completes, so each wait gives up after about 2^31 cycles
 * (about 1 s) and records the timeout.  *returned = threads that came back
 * (128 when the mechanism works).  The context stays usable.  Synchronises.
 * Errors: MF_EINVAL, MF_ENOMEM, MF_ECUDA. */
mf_status mf_selftest_wait(mf_plan_t plan, int32_t* returned);

/* Measured FP32 FMA throughput of the current device, TFLOP/s (2 flop per
 * FMA; 8 independent chains per thread, 8 CTAs of 256 threads per SM, timed
 * with CUDA events after a warm-up): context for the ALU roofline of the
 * filter kernels.  Synchronises.  Errors: MF_EINVAL, MF_ECUDA. */
mf_status mf_fma_probe(double* tflops, void* cuda_stream);

/* ---- two-detector coincidence and follow-up (Sec. III) ---------------- */

typedef struct {
  int64_t shift_samples;   /* time-shift step, samples (> 0) */
  int32_t n_shifts;        /* shifts k = 0..n_shifts (0 = zero lag only) */
  int64_t window_samples;  /* coincidence window, samples (2*window < ring length) */
  double rho_c_thr;        /* follow up a template when rho_c >= this */
  double rho_c_store;      /* record coincidences with rho_c >= this */
  int64_t max_coincs;      /* capacity of the coincidence record buffer */
} mf_coinc_desc;

typedef struct {
  int32_t tmpl;
  int32_t shift;      /* k */
  int64_t sample0;    /* detector-0 trigger sample */
  int64_t sample1;    /* detector-1 trigger sample (unshifted) */
  float snr0, snr1;
  float rho_c;        /* sqrt(snr0^2 + snr1^2) */
  int32_t reserved;
} mf_coinc;

/* A8: on the last mf_filter of a 2-detector plan, find coincidences of
 * detector-0 and detector-1 triggers of the same template: detector-1 times
 * shifted by k*shift_samples (k = 0..n_shifts) on the ring of analysed
 * samples [valid_begin, valid_end), circular distance <= window_samples.
 * followed: device int32 [n_tmpl], zeroed here, set to 1 for templates with
 * a coincidence of rho_c >= rho_c_thr.  Asynchronous. */
mf_status mf_coincide(mf_plan_t plan, const mf_coinc_desc* desc, int32_t* followed);

/* Coincidence records of the last mf_coincide, sorted by (tmpl, shift,
 * sample0, sample1), into host out[cap].  Synchronises.  MF_EOVERFLOW as for
 * triggers. */
mf_status mf_get_coincs(mf_plan_t plan, mf_coinc* out, int64_t cap, int64_t* n_found);

/* Background estimate from time-shifted coincidences (Sec. IV, Eq. 6).  For
 * each foreground statistic stat_fg[i] (host float32 [n_fg], e.g. rho_c of the
 * zero-lag coincidences) against the background stat_bg (host float32
 * [n_bg], the shifted coincidences), with n_b(x) = scale x #{bg >= x}
 * (scale: ratio of background volumes, Sec. IV):
 *   far_count[i] = (1 + n_b(stat_fg[i])) / t_bg                 (Eq. 6),
 *   far_fit[i]   = (1 + exp(alpha + beta stat_fg[i])) / t_bg,
 * where log n_b = alpha + beta x is the least-squares line through the
 * cumulative counts at every background value >= fit_min (natural log; the
 * Sec. IV tail fit).  t_bg: background time, s (> 0).  Outputs are host
 * float64 (far_fit, alpha, beta may be NULL; they are NaN when fewer than two
 * background values reach fit_min).  Host computation, no device work.
 * Errors: MF_EINVAL. */
mf_status mf_far(const float* stat_fg, int64_t n_fg, const float* stat_bg, int64_t n_bg, double t_bg, double scale,
                 double fit_min, double* far_count, double* far_fit, double* alpha, double* beta);

/* Neighbourhood map coarse -> fine (CSR: ptr int64 [n_coarse+1], idx int32
 * [ptr[n_coarse]] fine template ids of this plan's bank), copied to the
 * device; on_device selects the pointer kind. */
mf_status mf_set_nbhd(mf_plan_t plan, const int64_t* ptr, const int32_t* idx, int64_t n_coarse, int on_device);

/* A9: union of the neighbourhoods of coarse templates c with followed[c] != 0
 * (device int32 [n_coarse]) as ascending fine ids into device subset
 * [n_tmpl of this plan]; *n_subset (host) receives the count.  Synchronises. */
mf_status mf_nbhd_union(mf_plan_t plan, const int32_t* followed, int32_t* subset, int64_t* n_subset);

/* ---- learned proposal for the stage-2 follow-up ------------------------- */

/* Sec. III filters every fine template in the neighbourhood of a followed-up
 * coarse template.  This network (not in the paper; a ranking aid with the
 * full neighbourhood as the fallback) scores the n_valid[i] neighbourhood
 * slots of candidate i so that stage 2 can filter only the best-ranked
 * ones.  Architecture: x [n_in] -> depth x (affine + GELU, width) -> affine
 * [n_out] -> softmax over the first n_valid slots.  Parameters: FP32 master
 * copy, flat layout W_1 [n_in][width], b_1, ..., W_depth, b_depth,
 * W_out [width][n_out], b_out (row-major); products in BF16 on the tensor
 * cores with FP32 accumulation.  All arrays are device pointers unless
 * stated; calls are asynchronous on the network's stream except
 * set/get_params, which synchronise. */
typedef struct mf_mlp_s* mf_mlp_t;

/* Create a network with zero parameters for batches of up to max_batch rows.
 * Errors: MF_EINVAL (sizes), MF_ENOMEM. */
mf_status mf_mlp_create(mf_mlp_t* out, int32_t n_in, int32_t width, int32_t depth, int32_t n_out, int64_t max_batch,
                        void* cuda_stream);
void mf_mlp_destroy(mf_mlp_t net);
/* Number of FP32 parameters (layout above). */
int64_t mf_mlp_num_params(mf_mlp_t net);
/* Copy parameters in (host or device per on_device; resets the AdamW state) / out (to host). */
mf_status mf_mlp_set_params(mf_mlp_t net, const float* theta, int64_t n, int on_device);
mf_status mf_mlp_get_params(mf_mlp_t net, float* theta, int64_t n);
/* Forward pass of x [B][n_in] (FP32); logits [B][n_out] (FP32) if non-NULL. */
mf_status mf_mlp_forward(mf_mlp_t net, const float* x, int64_t B, float* logits);
/* Forward + backward of the mean masked softmax cross-entropy with labels
 * label[B] in [0, n_valid[i]); writes loss (1 float) and the gradient
 * (n_params floats) when those pointers are non-NULL; keeps the gradient for
 * mf_mlp_adamw_step. */
mf_status mf_mlp_loss_grad(mf_mlp_t net, const float* x, const int32_t* n_valid, const int32_t* label, int64_t B,
                           float* loss, float* grad);
/* One AdamW step (decoupled weight decay on every parameter) with the last gradient. */
mf_status mf_mlp_adamw_step(mf_mlp_t net, float lr, float beta1, float beta2, float eps, float weight_decay);
/* Proposal: the best-scored valid slots of each row in order (ties: lower
 * slot), until their softmax probability over the valid slots reaches p_mass
 * (p_mass >= 1: exactly min(k, n_valid) slots) or k (<= 64) are taken;
 * out [B][k] int32, -1 padded; count [B] int32 (may be NULL) = slots taken. */
mf_status mf_mlp_topk(mf_mlp_t net, const float* x, const int32_t* n_valid, int64_t B, int32_t k, float p_mass,
                      int32_t* out, int32_t* count);
/* Message of the last failed call on this network. */
const char* mf_mlp_last_error(mf_mlp_t net);

/* ---- long data in overlapping segments, by template-length class ------- */

/* The data of every detector are a long stream (n_samples samples) analysed
 * in overlapping segments (Sec. V.C).  Templates are grouped by duration into
 * length classes; class c holds templates of at most class_len[c] seconds and
 * filters them in segments of N_c samples (a power of two in [2^12, 2^20],
 * picked by mf_batch_autotune or set with mf_batch_set_segment).  With
 * L_c = class_len[c] fs rounded up to whole windows and stride
 * S_c = N_c - L_c rounded down to whole windows, segment s starts at sample
 * s S_c and analyses its local samples [L_c, min(L_c + S_c, n_samples - s S_c)):
 * the first L_c samples are where the circular filter wraps the template
 * around, and windows never straddle two segments.  Data past the end of the
 * stream are zero.  Every class is one plan (mf_batch_plan) whose data rows
 * are (segment, detector) pairs, row = s n_det + d; the batch owns it, sets
 * its PSD and row ranges, and the caller loads its bank at N_c (mf_bank_*).
 * Triggers are one per (detector, class, template, window of the stream). */
typedef struct mf_batch_s* mf_batch_t;

typedef struct {
  double fs;                /* sampling rate of the stream, Hz */
  int32_t n_det;            /* detectors, 1..8 */
  int64_t n_samples;        /* samples per detector */
  double f_low, f_high;     /* analysis band, Hz */
  double snr_thr;           /* rho threshold (Sec. II, inclusive) */
  int64_t window;           /* clustering window, samples */
  int32_t n_class;          /* length classes, 1..8 */
  const double* class_len;  /* host [n_class]: template duration bound of each class, s, increasing; copied */
  int64_t max_triggers;     /* trigger capacity of each class */
  void* cuda_stream;        /* stream that orders mf_batch_run with the caller's work */
} mf_batch_desc;

typedef struct {
  int32_t det, cls, tmpl;   /* detector, length class, template id within the class's bank */
  int32_t reserved;
  int64_t sample;           /* window peak, sample index in the stream */
  float snr, phase;         /* rho and arg z (quantised to 2 pi / 2048) */
} mf_batch_trigger;

enum { MF_RUN_SERIAL = 0, MF_RUN_STREAMS = 1, MF_RUN_GRAPH = 2, MF_RUN_FUSED = 3, MF_RUN_FUSED_GRAPH = 4 };

mf_status mf_batch_create(mf_batch_t* out, const mf_batch_desc* desc);
void mf_batch_destroy(mf_batch_t batch);
const char* mf_batch_last_error(mf_batch_t batch);

/* One-sided PSD on the grid of n_psd samples (host float64 [n_psd/2+1];
 * n_psd a power of two >= every N_c; copied): class c uses bins k n_psd/N_c. */
mf_status mf_batch_set_psd(mf_batch_t batch, const double* psd, int64_t n_psd);

/* Segment length of class c (power of two, > L_c + window, <= 2^20), with
 * templates per launch (0: the plan's default).  Creates the class's plan;
 * a plan of another length is destroyed with its bank. */
mf_status mf_batch_set_segment(mf_batch_t batch, int32_t cls, int64_t n, int32_t templates_per_launch);

/* Autotuner: for every class whose template count n_tmpl[c] > 0, time the
 * filter kernels on the actual row count of each admissible segment length
 * (probe banks of zeros, no triggers) and launch batch, and keep the pair
 * with the least estimated time per run, n_tmpl[c] x rows(N) x time per
 * series; then as mf_batch_set_segment.  Needs the PSD.  Synchronises. */
mf_status mf_batch_autotune(mf_batch_t batch, const int64_t* n_tmpl);

/* Autotuner for fused runs (MF_RUN_FUSED): the same probes, but one segment
 * length N for every class with n_tmpl[c] > 0, the admissible N with the
 * least summed estimate; each class keeps its own best launch batch at that N
 * (the fused launch holds the largest of those launches, batch x rows).  Then
 * as mf_batch_set_segment for each such class.  Synchronises. */
mf_status mf_batch_autotune_fused(mf_batch_t batch, const int64_t* n_tmpl);

/* Geometry of class c: N_c, L_c, S_c, segments, and the estimated and
 * measured milliseconds per run (measured: of the last MF_RUN_SERIAL run; 0 if none). */
mf_status mf_batch_segment(mf_batch_t batch, int32_t cls, int64_t* n, int64_t* tmpl_len, int64_t* stride,
                           int64_t* n_seg, double* est_ms, double* run_ms);

/* The class's plan (owned by the batch; valid until its segment length changes). */
mf_status mf_batch_plan(mf_batch_t batch, int32_t cls, mf_plan_t* plan);

/* Filter the stream with every class that has a bank: strain device float32
 * [n_det][ld], n_samples used per row.  MF_RUN_SERIAL: classes one after the
 * other; MF_RUN_STREAMS: each class on its own stream, joined at the end;
 * MF_RUN_GRAPH: as STREAMS, captured once into a CUDA graph per (strain, ld)
 * and replayed (the first run of a batch, or after a bank change, runs
 * uncaptured first).  MF_RUN_FUSED: every class's segment spectra on its own
 * stream, then one work queue over the (class, template, segment, detector)
 * series of all classes: each launch pair of the two filter passes takes the
 * next S series of the queue across class boundaries, S = the largest launch
 * a class makes alone (its batch x rows); the classes must share N, store an
 * FP32 bank and use the same intermediate (mf_set_intermediate on every class
 * plan; MF_ESTATE / MF_EINVAL otherwise).  Triggers are those of the
 * per-class modes, bit for bit.  A wait that timed out is reported by the
 * first class with a bank.  MF_RUN_FUSED_GRAPH: FUSED captured and replayed
 * as GRAPH.  Asynchronous on the batch's stream. */
mf_status mf_batch_run(mf_batch_t batch, const float* strain, int64_t ld, int32_t mode);

/* Triggers of the last run into host out[cap], ordered by (class, detector,
 * template, sample); *n_found = total.  Synchronises.  MF_EOVERFLOW as for
 * mf_get_triggers. */
mf_status mf_batch_get_triggers(mf_batch_t batch, mf_batch_trigger* out, int64_t cap, int64_t* n_found);

/* ---- filtering without device allocation ------------------------------- */

/* The matched filter of mf_filter for callers that cannot allocate GPU
 * memory, e.g. code that runs inside another framework's memory pool, a loop
 * that must never allocate, or a plug-in that is only handed buffers.  The
 * paper has no counterpart: it is an interface convenience of this library.
 * The threshold (inclusive), window rule and trigger order are mf_filter's;
 * the kernels are the per-thread-load filter (k_pass1 / k_pass2, 1/sigma
 * applied per sample) rather than mf_filter's (pre-scaled data and a
 * per-template raw threshold), so SNR agrees with mf_filter to 1e-4 relative
 * and a window peak or a sample at the threshold can differ at near-ties.
 *
 * No plan, no allocation: all working memory lives in one 32 MiB __device__
 * array compiled into the library (present on every GPU that loads it, until
 * the process exits).  Limits: N a power of two in [2^12, 2^16], n_det 1 or 2,
 * 1 <= n_tmpl <= 1024, at most 256 windows per segment; anything larger is
 * rejected with MF_EINVAL.  The whole segment is analysed (valid range [0, N)).
 *   psd:    device float64 [N/2+1], one-sided PSD (weights as in mf_set_psd)
 *   htilde: device complex64 templates [n_tmpl][ld_h] (float32 pairs)
 *   dtilde: device complex64 data [n_det][ld_d]
 *   trig:   device mf_trigger [trig_cap] (out), count: device int64 (out) =
 *           number found (may exceed trig_cap; only trig_cap are written)
 * Asynchronous on cuda_stream.  All calls share the one array: calls that
 * overlap on the GPU race, so serialise them; each call re-initialises what
 * must start at zero.  Each call looks up the array's address on the current
 * device (cudaGetSymbolAddress, a host-side query).  Errors are reported
 * through mf_last_error(NULL). */
mf_status mf_filter_noalloc(double fs, int64_t n, int32_t n_det, double f_low, double f_high, double snr_thr,
                            int64_t window, const double* psd, const void* htilde, int64_t n_tmpl, int64_t ld_h,
                            const void* dtilde, int64_t ld_d, mf_trigger* trig, int64_t trig_cap, int64_t* count,
                            void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* MF_H_ */
