// Internal launcher interface between the C-ABI layer (mf_api.cu) and the
// kernels (mf_kernels.cu, mf_glue.cu).  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

struct mf_plan_s;  // the plan (defined by the C-ABI layer)

namespace mf {

// Packed per-window maximum: [63:32] float bits of rho^2 (>= 0, so integer
// order = float order), [31:11] (2^21 - 1 - sample) so that ties go to the
// lowest sample, [10:0] phase of z quantised to 2 pi / 2048.
constexpr int kSampleBits = 21;
constexpr int kPhaseBits = 11;
constexpr int64_t kMaxN = int64_t(1) << 20;

enum BankType { kBankF32 = 0, kBankF16 = 1, kBankBF16 = 2 };

struct FilterArgs {
  // geometry
  int64_t n;          // FFT length N
  int n1, n2;         // N = n1 * n2 (pass-1 column length, pass-2 row length)
  int n_det;
  int64_t nb;         // N/2 + 1
  // inputs
  const void* bank;   // [n_tmpl][ld_bank] complex (f32 pairs or 16-bit pairs)
  int bank_type;
  int64_t ld_bank;
  const float* scales;      // per template (16-bit banks), may be null
  const float2* q;          // weighted data [n_det][ld_q]
  int64_t ld_q;
  const int32_t* sel;       // selection: position -> template id (device)
  const float* inv_sigma;   // per template id: 1 / sigma
  // this batch: selection positions [pos0, pos0 + count)
  int64_t pos0;
  int count;
  float2* scratch;          // [count * n_det][n1][n2]
  // epilogue
  float thr2;
  int64_t window;
  int64_t valid_begin, valid_end;
  int64_t n_win;
  int64_t n_sel_total;      // slots are [n_det][n_sel_total][n_win]
  unsigned long long* slots;
  int* status;              // device status word (bounded waits report here)
  const float2* tw1;        // sub-FFT twiddle tables (w_N1^{r j}, w_N2^{r j}), 8 KB max each
  const float2* tw2;
  const float* thr_raw;     // per template: rho_thr^2 / ratio^2 on the pre-scaled data (TMA kernels)
  const float2* tw4;        // four-step twiddles by column (launch_fill_tw4)
  int first_batch;          // 1: the weighted data were written by the kernel just before (PDL ordering)
  // 16-bit weighted data (TMA kernels): q_lp [n_det][ld_q] half2 / bfloat162 holding c_d q, with
  // c_d = dscale[d] a power of two; q_type = kBankF32 means the FP32 q above is used
  int q_type;
  const void* q_lp;
  const float* dscale;
  // per data row analysed range [x, y) (TMA kernels), or null: [valid_begin, valid_end) for all rows
  const int2* row_valid;
  // pass-1 -> pass-2 intermediate (N = 2^20 only for 1 and 2): 0 complex64, ALU row pass; 1 FP16 in
  // kPanel16-row panels, each series scaled by series_scale16(ratio[template]), tensor-core row pass;
  // 2 the same with every value an FP16 pair (hi image, then lo image, per panel) and split products
  int inter;
};

// rows per panel of the FP16 intermediate: a panel is one tensor-core row-pass item
constexpr int kPanel16 = 8;

// One plan's share of a fused launch (the length-class runner's work queue):
// `count` templates from selection position pos0 against its n_det data rows,
// the series [series0, series0 + count n_det) of the launch's scratch, in the
// plan's (template, row) order.  Every part of a launch shares N, the storage
// types (FP32 weighted data), the window, n_win, the intermediate and the
// twiddle tables of the FilterArgs it is launched with.
struct FilterPart {
  const void* bank;
  int64_t ld_bank;
  const float2* q;
  int64_t ld_q;
  const int32_t* sel;
  const float* inv_sigma;   // ratio per template id (as FilterArgs::inv_sigma)
  const float* thr_raw;
  int64_t pos0;
  int count, n_det;
  int64_t valid_begin, valid_end;
  int64_t n_sel_total;
  unsigned long long* slots;
  const int2* row_valid;
  int series0;
};
constexpr int kMaxParts = 8;
struct FilterParts {
  int n;         // parts of this launch, 1..kMaxParts (0: one plan, all of FilterArgs)
  int n_series;  // series of all parts
  FilterPart p[kMaxParts];
};

// part holding unit u of a launch whose parts own `per` consecutive units per series (uniform across a warp)
__host__ __device__ inline int part_of(const FilterParts& ps, int64_t u, int per) {
  int i = 0;
  while (i + 1 < ps.n && u >= (int64_t)ps.p[i + 1].series0 * per) ++i;
  return i;
}

// Quantise the FP32 weighted data q [n_det][ld_q] (nb bins per detector) to
// 16-bit (q_type) q_lp with a per-detector power-of-two scale c_d chosen so that
// max |c_d q| is in [2^14, 2^15); writes dscale[d] = c_d.  dmax: n_det words of
// scratch.
cudaError_t launch_quant_q(const float2* q, int64_t ld_q, int64_t nb, int n_det, int q_type, void* q_lp,
                           unsigned* dmax, float* dscale, cudaStream_t st);
// Quantise n_rows FP32 templates (src [n_rows][ld_src], nb bins) to the 16-bit
// bank rows dst [n_rows][ld_dst] with a per-template power-of-two scale:
// stored = h / scale, max |stored| in [2^14, 2^15); scales[i] = scale.
cudaError_t launch_quant_bank(const float2* src, int64_t ld_src, int64_t n_rows, int64_t nb, int bank_type, void* dst,
                              int64_t ld_dst, float* scales, cudaStream_t st);
// Plan introspection for the length-class runner (mf_batch.cu): templates in
// the bank; a fingerprint of everything a captured graph of mf_filter bakes in
// (buffers, batch, storage types); and whether mf_filter on the whole bank would
// run without host synchronisation or allocation (so that it can be captured).
int64_t plan_templates(const ::mf_plan_s* p);
uint64_t plan_fingerprint(const ::mf_plan_s* p);
bool plan_capturable(const ::mf_plan_s* p);
// templates per launch pair of a plan's own filter (mf_set_batch)
int plan_batch(const ::mf_plan_s* p);
// Fused filter of several plans (the length-class runner's work queue): each plan filters its whole
// bank against its own spectra dtilde[i] (rows ld[i] apart) exactly as mf_filter would, but the
// two passes take the series of all plans in (plan, template, row) order, one launch pair per
// scratch_series series across plan boundaries.  The plans share N, the window and the
// intermediate, with an FP32 bank and FP32 data; `scratch` holds scratch_series series of the
// intermediate (N x 8 bytes each; scratch_map encoded for it) and every step runs on st.  A wait
// that times out is reported by plans[0], and so are the launch counts and, when plans[0] is
// profiling (mf_profile), the launch pairs' CUDA-event times.  On failure *err holds the message.
int filter_fused(::mf_plan_s* const* plans, const void* const* dtilde, const int64_t* ld, int n_plans, void* scratch,
                 int64_t scratch_series, const CUtensorMap& scratch_map, cudaStream_t st, std::string* err);
// The TMA-staged filter passes (mf_filter.cu).  The bank rows and the
// weighted data are in column layout: element k = k1 N2 + k2 of the non-zero
// half (k1 < N1/2) at k2 N1/2 + k1 (see launch_to_cols).
cudaError_t launch_filter2_pass1(const FilterArgs& a, cudaStream_t st);
cudaError_t launch_filter2_pass2(const FilterArgs& a, const CUtensorMap& scratch_map, cudaStream_t st);
// the tensor-core row pass over the FP16 intermediate (mf_filter_tc.cu), N = 2^20
cudaError_t launch_filter2_pass2_tc(const FilterArgs& a, cudaStream_t st, const FilterParts* parts = nullptr);
// Both passes over the series of several plans' parts in one launch each (ps.n >= 1): the
// per-part fields come from ps, the rest (geometry, types, window, scratch, tables, status)
// from a; the scratch holds ps.n_series series (scratch_map encoded for at least as many).  `between`
// (optional) is recorded on st between the two launches.
cudaError_t launch_filter2_fused(const FilterArgs& a, const FilterParts& ps, const CUtensorMap& scratch_map,
                                 cudaStream_t st, cudaEvent_t between = nullptr);
// Tensor map of the pass-1 -> pass-2 scratch (`series` series of length n)
// through which pass 2 reads its items; all zero where pass 2 needs none.
cudaError_t encode_scratch_map(int64_t n, const float2* scratch, int64_t series, CUtensorMap* m);
cudaError_t launch_fill_twiddles(int64_t n, float2* tw1, float2* tw2, cudaStream_t st);
// four-step twiddles of k_cols by column: tw4[k2 (RA + 1) + j] = w_N^{j k2}, j <= RA(N1), k2 < N2;
// tw4_count(n) entries
cudaError_t launch_fill_tw4(int64_t n, float2* tw4, cudaStream_t st);
int64_t tw4_count(int64_t n);

// Column layout of spectra rows: dst[r][k2 N1/2 + k1] = src[r][k1 N2 + k2] for
// k1 < N1/2, k2 < N2 (the bins k < N/2), elem_bytes 8 (complex64) or 4 (16-bit
// pairs); src rows ld_src elements apart, dst rows ld_dst.
cudaError_t launch_to_cols(const void* src, int64_t ld_src, void* dst, int64_t ld_dst, int64_t n_rows, int n1, int n2,
                           int elem_bytes, cudaStream_t st);
// q = q_scale w s~ in column layout (q [n_det][ld_q], N/2 elements per row)
cudaError_t launch_prep_cols(const float2* dtilde, int64_t ld_d, const double* w, int n1, int n2, int n_det,
                             float2* q, int64_t ld_q, unsigned long long* slots, int64_t n_slots, cudaStream_t st,
                             double q_scale);

// chi^2 veto at trigger times (mf_chisq.cu): band edges of every template for
// p bands (bpow: n_tmpl x chisq_blocks scratch, edges: n_tmpl x (p + 1)), then
// chi^2 and the re-weighted SNR of the first min(*count, cap) triggers.
int64_t chisq_blocks(int n1, int n2);
cudaError_t launch_chisq_edges(const void* bank, int bank_type, int64_t ld_bank, int64_t n_tmpl, int n1, int n2,
                               const double* w, int64_t nb, double* bpow, int p, int32_t* edges, cudaStream_t st);
// Sine-Gaussian veto of heavy templates at trigger times (mf_chisq.cu): the tiles' offsets above each
// template's final frequency (Hz) and their quality factor.
constexpr int kMaxSgTiles = 16;
struct SgTiles {
  int n;
  double q;
  double offset[kMaxSgTiles];
};
cudaError_t launch_sgchisq(const void* trig, const int64_t* count, int64_t cap, const void* q, int q_type, int64_t ld_q,
                           int n1, int n2, const double* w, double df, double f_high, const float* f_final,
                           const float* mtotal, float m_min, float snr_min, const SgTiles& tiles, double q_to_true,
                           const float* dscale, const float* snr_in, float* chi2_r, float* snr_hat, cudaStream_t st);
cudaError_t launch_chisq(const void* trig, const int64_t* count, int64_t cap, const void* bank, int bank_type,
                         int64_t ld_bank, const void* q, int q_type, int64_t ld_q, int n1, int n2, const int32_t* edges,
                         int p, const float* ratio, const float* dscale, float* chi2, float* newsnr, cudaStream_t st);

// TaylorF2 templates (mf_taylorf2.cu): n_tmpl natural-order complex64 rows out [n_tmpl][ld] of an n-sample
// segment at fs, from host masses; synchronises the stream
cudaError_t launch_taylorf2(const double* m1, const double* m2, int64_t n_tmpl, double fs, int64_t n, double f_low,
                            float2* out, int64_t ld, cudaStream_t st);

// blocks x 256 threads, each 8 chains x 16 x iters FP32 FMAs (the ALU probe)
cudaError_t launch_fma_probe(float* out, int blocks, int iters, cudaStream_t st);

// One CTA of 128 threads waiting on a barrier nothing completes (bounded waits
// record a timeout in *status; *returned counts the threads that returned).
cudaError_t launch_wait_selftest(int* status, int* returned, cudaStream_t st);

// Message returned by mf_last_error(NULL) for calls without a plan.
void set_global_error(const char* msg);
inline void set_global_error(const std::string& msg) { set_global_error(msg.c_str()); }

// Number of kernels launched by this library (all plans, all threads).
int64_t launch_count();
void add_launches(int64_t n);

cudaError_t launch_prep(const float2* dtilde, int64_t ld_d, const double* w, int64_t nb, int n_det,
                        float2* q, int64_t ld_q, unsigned long long* slots, int64_t n_slots,
                        cudaStream_t st, double q_scale = 1.0);
// ratio[t] = inv_sigma[t] * sigma_ref, thr_raw[t] = thr2 / ratio[t]^2 (+inf when ratio is 0)
cudaError_t launch_tmpl_scale(const float* inv_sigma, int64_t n_tmpl, double sigma_ref, double thr2, float* ratio,
                              float* thr_raw, cudaStream_t st);
cudaError_t launch_filter_batch(const FilterArgs& a, cudaStream_t st);
// the two halves of launch_filter_batch, for per-kernel timing
cudaError_t launch_filter_pass1(const FilterArgs& a, cudaStream_t st);
cudaError_t launch_filter_pass2(const FilterArgs& a, cudaStream_t st);
// sigma^2 of bank rows [row0, row0 + n_rows) in natural layout (n1 = 0: bins
// 0..nb-1) or column layout (n1, n2 > 0: the N/2 bins of launch_to_cols)
cudaError_t launch_sigmasq(const void* bank, int bank_type, int64_t ld_bank, const float* scales,
                           int64_t row0, int64_t n_rows, const double* w, int64_t nb,
                           double* sigmasq, float* inv_sigma, cudaStream_t st, int n1 = 0, int n2 = 0);
// compaction of window maxima into mf_trigger records (layout of the public struct)
cudaError_t launch_compact(const unsigned long long* slots, int n_det, int64_t n_sel, int64_t n_win,
                           int64_t window, const int32_t* sel, void* trig_out, int64_t trig_cap,
                           int64_t* count, int64_t* block_counts, int64_t n_blocks_cap, cudaStream_t st);
int64_t compact_blocks(int64_t n_slots);
// time series -> one-sided dt-normalised spectrum (A1)
// Gate statistic's one-row bank (mf_gate.cu): row[k] = sqrt(4 df / w[k]) where
// w[k] > 0 (the PSD weights of Eq. 2), else 0; k < nb, complex64.
cudaError_t launch_gate_row(const double* w, int64_t nb, double df, float2* row, cudaStream_t st);
cudaError_t launch_rfft(const float* strain, int64_t ld_s, int n_det, int64_t n, int n1, int n2, double dt,
                        float2* scratch, float2* dtilde, int64_t ld_d, cudaStream_t st);
// keep bins 0..nb_out-1 (A2)
cudaError_t launch_decimate(const float2* in, int64_t ld_in, float2* out, int64_t ld_out, int64_t nb_out,
                            int n_det, cudaStream_t st);

struct CoincArgs {
  const unsigned long long* slots;  // stage-1 window maxima [2][n_sel][n_win]
  const int32_t* sel;
  int64_t n_sel, n_win, window;
  int64_t ring_begin, ring_end;
  int64_t shift;                    // samples per time shift
  int n_shifts;                     // k = 0..n_shifts
  int64_t coinc_window;             // samples
  float rho_c_thr2;                 // follow-up threshold on rho_c^2
  float rho_c_store2;               // store coincidences with rho_c^2 >= this
  int32_t* followed;                // [n_tmpl] flags (written 1)
  void* coincs;                     // mf_coinc records
  int64_t coinc_cap;
  unsigned long long* n_coinc;      // counter
  const float* max_rho2_det1;       // per selection position, max rho^2 of detector 1 (prefilter)
};
cudaError_t launch_coinc(const CoincArgs& a, float* max_rho2_det1, cudaStream_t st);
cudaError_t launch_union(const int64_t* ptr, const int32_t* idx, int64_t n_coarse, const int32_t* followed,
                         int32_t* flags, int64_t n_fine, int32_t* subset, int64_t* n_subset,
                         int64_t* block_counts, cudaStream_t st);

}  // namespace mf
