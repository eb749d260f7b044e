// Tensor-core row pass of the matched filter (Eq. 1-2, Sec. V.C: the inverse
// transform over coalescence time), N = N1 N2 with N2 = 1024, over the FP16
// pass-1 -> pass-2 intermediate that k_cols writes in 8-row panels.
//
// A row x[k2] (k2 = 32 p + q) has the 1024-point transform
//   z[u + 32 v] = sum_q w32^{q v} w1024^{q u} Y[u][q],   Y[u][q] = sum_p w32^{p u} x[32 p + q],
// (w_M = exp(+2 pi i / M)): two radix-32 stages, each a product with the
// complex 32 x 32 DFT matrix, which is a dense contraction and runs on the
// tensor cores as a real 64 x 64 matrix (real and imaginary parts interleaved
// along K and N) with FP16 operands and FP32 accumulation in tensor memory:
//   stage 1: D1[(q, r)][(u, c)] = sum_(p, c') A1[(q, r)][(p, c')] B[(u, c)][(p, c')]
//   stage 2: D2[(u, r)][(v, c)] = sum_(q, c') A2[(u, r)][(q, c')] B[(v, c)][(q, c')]
// with B the embedded DFT matrix, A1 a panel of 8 rows (r) exactly as k_cols
// stored it (the MN-major operand image, one 32 KB bulk copy) and A2 the
// stage-1 result times w1024^{q u}, rounded to FP16 (K-major).  M = 256 rows
// per stage, as two M = 128 tiles.
//
// One persistent CTA per SM, 832 threads.  Warp 24 copies items into six
// shared-memory slots (three with FP16 pairs); a slot holds its item's stage-1
// operand and then (written over it) its stage-2 operand, and is free again
// once stage 2 has read it.  Warp 25 owns all 512 tensor-memory columns (four
// buffers of 2 x 64) and one lane issues the MMAs in an event loop: stage 1 of
// item k into buffer k % 4 when its slot has landed and the buffer is free,
// stage 2 when its operand is written, in item order each.  Warps 0-23 are
// three consumer groups of eight warps; group g takes items k = g, g + 3, ...,
// so one buffer's stage 1 can complete while every group is busy.  In a group,
// warps 4 h .. 4 h + 3 own tile h, and thread t = TMEM lane t of that tile
// (q or u = t / 8 + 16 h, r = t % 8) applies the twiddles between the stages
// and runs the epilogue (raw |z|^2 against the per-template threshold, window
// maxima) on the stage-2 accumulators.  Barriers: per slot full / a2full /
// empty, per buffer d1 / d2 / tfree, and a drain barrier; every wait is bounded.
#include "mf_common.cuh"
#include "mf_tc.cuh"
#include "mf_tma.cuh"

namespace mf {

namespace {

constexpr int kGroupWarps = 8;                    // warps of one consumer group: 4 per operand tile
constexpr int kGroup = kGroupWarps * 32;          // threads of one consumer group
constexpr int kGroups = 3;
constexpr int kBufs = 4;                          // tensor-memory buffers: items from stage 1 to the epilogue
constexpr int kTcThreads = kGroups * kGroup + 64; // + producer warp + MMA warp
constexpr int kProdWarp = kGroups * kGroupWarps, kMmaWarp = kProdWarp + 1;
constexpr int kTcRows = kPanel16;                 // rows per item
constexpr int kTcK = 64;                          // 32 complex values, real and imaginary interleaved
constexpr int kLbo = 128, kSbo = 1024;            // unpadded core-matrix layouts
constexpr int kTileBytes = 128 * kTcK * 2;        // one M = 128 operand tile, 16 KB
constexpr int kBBytes = 64 * kTcK * 2;            // one image of the DFT matrix B (64 x 64), 8 KB
constexpr int kTwStride = 33;                     // padded rows of the w1024^{q u} table (float2)
constexpr uint32_t kBufCols = 128;                // 2 tiles x 64 FP32 columns
constexpr uint32_t kTmemCols = kBufs * kBufCols;  // all 512
constexpr uint32_t kIdesc2 = tc_idesc_f16(128, 64);          // A K-major (stage 2)
constexpr uint32_t kIdesc1 = kIdesc2 | (1u << 15);           // A MN-major (stage 1)

static_assert(cm_offset(255, 63, kLbo, kSbo) + 2 <= 2 * kTileBytes, "A2 layout");

// Shared memory: operand slots, B (hi, then lo when split), the twiddle table, the barriers.  SPLIT: every
// operand and B is a pair of FP16 images (hi, then lo), so an item is 64 KB and three slots fit.
template <bool SPLIT>
struct TcGeo {
  static constexpr int IMG = SPLIT ? 2 : 1;         // FP16 images per operand
  static constexpr int ITEM = IMG * 2 * kTileBytes;  // one item: 256 rows of every image
  static constexpr int SLOTS = SPLIT ? 3 : 6;
  static constexpr int B_OFF = SLOTS * ITEM;
  static constexpr int TW_OFF = B_OFF + IMG * kBBytes;
  static constexpr int BAR_OFF = TW_OFF + 32 * kTwStride * 8;
  static constexpr int NBAR = 3 * SLOTS + 3 * kBufs + 1;
  static constexpr int SMEM = BAR_OFF + NBAR * 8 + 16;
  static_assert(SMEM <= 232448, "k_rows_tc shared memory");
};

// generic-proxy writes of another grid -> async-proxy (bulk copy) reads of this one
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// One stage: two M = 128 tiles x four K = 16 steps into buffer columns [d, d + 128), 8 MMAs.  SPLIT: per
// step also A lo x B hi and A hi x B lo (the A lo image two tiles on, B lo one B image on), 24 MMAs.
template <bool SPLIT>
__device__ __forceinline__ void stage_mmas(uint32_t d, uint32_t a_addr, bool mn_major, uint32_t b_addr) {
  const uint32_t idesc = mn_major ? kIdesc1 : kIdesc2;
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int ks = 0; ks < kTcK / 16; ++ks) {
      // K steps: two core matrices along K, 128 B apart in both operand layouts
      const uint32_t ao = h * kTileBytes + ks * 2 * kLbo, bo = ks * 2 * kLbo;
      const uint64_t ad = tc_desc(a_addr + ao, kLbo, kSbo), bd = tc_desc(b_addr + bo, kLbo, kSbo);
      tc_mma_f16(d + 64 * h, ad, bd, idesc, ks > 0);
      if constexpr (SPLIT) {
        tc_mma_f16(d + 64 * h, tc_desc(a_addr + 2 * kTileBytes + ao, kLbo, kSbo), bd, idesc, true);
        tc_mma_f16(d + 64 * h, ad, tc_desc(b_addr + kBBytes + bo, kLbo, kSbo), idesc, true);
      }
    }
}

// parity of the n-th completion (n = 0, 1, ...) of a barrier
__device__ __forceinline__ uint32_t par(int n) { return (uint32_t)(n & 1); }

// MP: the series of several plans' parts (FilterParts), each with its own epilogue state.  SPLIT: the FP16-pair
// intermediate (FilterArgs::inter = 2) and split products.
template <int N1, bool MP, bool SPLIT>
__global__ void __launch_bounds__(kTcThreads, 1) k_rows_tc(FilterArgs a, const __grid_constant__ FilterParts ps) {
  using G = TcGeo<SPLIT>;
  constexpr int kSlots = G::SLOTS, kItemBytes = G::ITEM;
  constexpr int N2 = 1024;
  constexpr int64_t N = (int64_t)N1 * N2;
  constexpr int NP = N1 / kTcRows;  // panels (items) per series
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* sB = sm + G::B_OFF;
  float2* tw = reinterpret_cast<float2*>(sm + G::TW_OFF);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + G::BAR_OFF);  // [kSlots]
  uint64_t* a2full = full + kSlots;                              // [kSlots]
  uint64_t* empty = a2full + kSlots;                             // [kSlots]
  uint64_t* d1 = empty + kSlots;                                 // [kBufs]
  uint64_t* d2 = d1 + kBufs;
  uint64_t* tfree = d2 + kBufs;
  uint64_t* drain = tfree + kBufs;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + G::BAR_OFF + G::NBAR * 8);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid & 31;
  const int n_series = MP ? ps.n_series : a.count * a.n_det;
  const int n_items = n_series * NP;
  int n_mine = 0;  // items of this CTA: blockIdx.x + k gridDim.x
  for (int item = blockIdx.x; item < n_items; item += gridDim.x) ++n_mine;

  if (warp == kMmaWarp) tmem_alloc(tslot, kTmemCols);
  // B: the embedded DFT matrix, B[(u, c)][(p, c')] = Re / Im parts of w32^{p u} (SPLIT: hi, then lo)
  for (int i = tid; i < 64 * kTcK; i += kTcThreads) {
    const int n = i / kTcK, k = i % kTcK, u = n >> 1, c = n & 1, p = k >> 1, cp = k & 1;
    const float2 f = unit_root((uint32_t)((p * u) & 31), 32u);
    const float v = c == 0 ? (cp == 0 ? f.x : -f.y) : (cp == 0 ? f.y : f.x);
    const __half hi = __float2half_rn(v);
    *reinterpret_cast<__half*>(sB + cm_offset(n, k, kLbo, kSbo)) = hi;
    if constexpr (SPLIT)
      *reinterpret_cast<__half*>(sB + kBBytes + cm_offset(n, k, kLbo, kSbo)) = __float2half_rn(v - __half2float(hi));
  }
  for (int i = tid; i < 32 * 32; i += kTcThreads) {
    const int q = i >> 5, u = i & 31;
    tw[q * kTwStride + u] = unit_root((uint32_t)(q * u), 1024u);
  }
  if (tid == 0) {
    for (int i = 0; i < kSlots; ++i) {
      mbar_init(full + i, 1);
      mbar_init(a2full + i, kGroup);
      mbar_init(empty + i, 1);
    }
    for (int b = 0; b < kBufs; ++b) {
      mbar_init(d1 + b, 1);
      mbar_init(d2 + b, 1);
      mbar_init(tfree + b, kGroup);
    }
    mbar_init(drain, 1);
    fence_mbar_init();
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const __half* scratch = reinterpret_cast<const __half*>(a.scratch);

  if (warp == kProdWarp) {
    // ---- producer: item k into slot k % kSlots once stage 2 of item k - kSlots has read that slot ----
    if (lane == 0) {
      pdl_wait();  // the intermediate is written by the kernel just before
      fence_proxy_async_global();
      int k = 0;
      bool ok = true;
      for (; k < n_mine; ++k) {
        const int slot = k % kSlots;
        if (k >= kSlots && !(ok = mbar_wait_at(empty + slot, par(k / kSlots - 1), a.status, 11, k))) break;
        const int item = blockIdx.x + k * gridDim.x;
        const int s = n_series - 1 - item / NP;  // series in reverse: the last ones written are likeliest in L2
        const __half* src =
            scratch + (int64_t)s * 2 * G::IMG * N + (int64_t)(item % NP) * (2 * G::IMG * N2 * kTcRows);
        mbar_expect_tx(full + slot, (uint32_t)kItemBytes);
        bulk_g2s(sm + slot * kItemBytes, src, (uint32_t)kItemBytes, full + slot);
      }
      if (!ok)  // copies this lane issued that nobody may have waited for
        for (int m = k - kSlots; m < k; ++m)
          if (m >= 0) mbar_wait_bounded(full + (m % kSlots), par(m / kSlots), nullptr);
    }
  } else if (warp == kMmaWarp) {
    // ---- MMA issuer: whichever of stage 1 (next item) / stage 2 (oldest item) is ready ----
    if (lane == 0) {
      const uint32_t bb = smem_u32(sB);
      int n1 = 0, n2 = 0;  // items whose stage 1 / stage 2 have been issued
      bool ok = true;
      long long t0 = clock64();
      while (n2 < n_mine) {
        bool progress = false;
        if (n1 < n_mine) {
          const int slot = n1 % kSlots, b = n1 % kBufs;
          if (mbar_test_wait(full + slot, par(n1 / kSlots)) &&
              (n1 < kBufs || mbar_test_wait(tfree + b, par(n1 / kBufs - 1)))) {
            tc_fence_after();
            stage_mmas<SPLIT>(tmem + b * kBufCols, smem_u32(sm + slot * kItemBytes), true, bb);
            tc_commit(d1 + b);
            ++n1;
            progress = true;
          }
        }
        if (n2 < n1) {
          const int slot = n2 % kSlots, b = n2 % kBufs;
          if (mbar_test_wait(a2full + slot, par(n2 / kSlots))) {
            tc_fence_after();
            stage_mmas<SPLIT>(tmem + b * kBufCols, smem_u32(sm + slot * kItemBytes), false, bb);
            tc_commit(d2 + b);
            tc_commit(empty + slot);
            ++n2;
            progress = true;
          }
        }
        if (progress) {
          t0 = clock64();
        } else if (clock64() - t0 > (1LL << 31)) {
          atomicCAS(a.status, 0, kStatusTimeout | ((n1 < n_mine ? 12 : 13) << 8) | ((n1 < n_mine ? n1 : n2) << 16));
          ok = false;
          break;
        }
      }
      if (!ok) {  // the MMAs in flight: wait (bounded again) for everything this lane issued to retire
        tc_commit(drain);
        mbar_wait_bounded(drain, 0, nullptr);
      }
    }
  } else {
    // ---- consumer group g = warp / 8: items k = g, g + 3, ... in buffer k % 4; twiddle, then epilogue ----
    // warps 4 h .. 4 h + 3 of a group own tile h; thread = TMEM lane row of that tile in both stages
    const int g = warp / kGroupWarps, wg = warp % kGroupWarps, h = wg >> 2;
    const int row = 32 * (wg & 3) + lane;
    const int r = row & 7, qg = row >> 3;
    const int q = qg + 16 * h;  // stage-1 row (q, r) of tile h, then stage-2 row (u = q, r)
    const float2* twq = tw + q * kTwStride;
    for (int k = g; k < n_mine; k += kGroups) {
      // the epilogue's fields are kernel parameters, read where used (no registers held across the loop)
      const RawEpi ep{a.sel, a.inv_sigma, a.thr_raw, nullptr, a.pos0, a.n_det, a.window, a.valid_begin,
                      a.valid_end, a.n_win, a.n_sel_total, a.slots, a.row_valid};
      const int slot = k % kSlots, b = k % kBufs;
      unsigned char* sl = sm + slot * kItemBytes;
      const uint32_t tbuf = tmem + b * kBufCols + 64 * h + ((uint32_t)(32 * (wg & 3)) << 16);
      // the item's series state first: its dependent global loads overlap the waits below
      const int item = blockIdx.x + k * gridDim.x;
      const int s = n_series - 1 - item / NP;
      RawEpi::Ser se;
      float sc;
      if constexpr (MP) {
        const FilterPart& p = ps.p[part_of(ps, s, 1)];
        const RawEpi pe{p.sel,         p.inv_sigma, p.thr_raw, nullptr,       p.pos0,  p.n_det,    a.window,
                        p.valid_begin, p.valid_end, a.n_win,   p.n_sel_total, p.slots, p.row_valid};
        se = pe.series(s - p.series0);
        sc = series_scale16(__ldg(p.inv_sigma + p.sel[p.pos0 + (s - p.series0) / p.n_det]));
      } else {
        se = ep.series(s);
        sc = series_scale16(__ldg(a.inv_sigma + a.sel[a.pos0 + s / a.n_det]));
      }
      const int64_t j1 = (int64_t)(item % NP) * kTcRows + r;
      // twiddle w1024^{q u}, round to FP16, stage-2 operand row (u, r), K = (q, c), over the slot
      // (warp-uniform outcome: the tensor-memory loads below are warp-collective)
      if (!__all_sync(0xffffffffu, mbar_wait_at(d1 + b, par(k / kBufs), a.status, 14, k))) break;
      tc_fence_after();
      // four chunks of 16 columns (u = 8 t .. 8 t + 7); chunk t + 1 loads while t is used
      float ya[16], yb[16];
      tmem_ld16_issue(tbuf, ya);
      tmem_wait(ya);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        float(&cur)[16] = (t & 1) ? yb : ya;
        float(&nxt)[16] = (t & 1) ? ya : yb;
        if (t + 1 < 4) tmem_ld16_issue(tbuf + 16 * (t + 1), nxt);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int u = 8 * t + i;
          const float2 z = cmul(make_float2(cur[2 * i], cur[2 * i + 1]), twq[u]);
          const int off = cm_offset(u * 8 + r, 2 * q, kLbo, kSbo);
          const __half2 hi = __floats2half2_rn(z.x, z.y);
          *reinterpret_cast<__half2*>(sl + off) = hi;
          if constexpr (SPLIT) {  // the remainder, exact in FP32, into the lo image two tiles on
            const float2 hf = __half22float2(hi);
            *reinterpret_cast<__half2*>(sl + 2 * kTileBytes + off) = __floats2half2_rn(z.x - hf.x, z.y - hf.y);
          }
        }
        if (t + 1 < 4) tmem_wait(nxt);
      }
      fence_proxy_async();  // our operand writes before the MMAs that read them
      mbar_arrive(a2full + slot);
      // the series state is used from here on (its loads were issued before the stage-1 wait)
      se.ratio /= sc;  // exact: sc is a power of two
      se.thr *= sc * sc;
      // epilogue: row (u, r) of tile h holds z[u + 32 v], v = 0..31, of row j1 = 8 panel + r (u = q)
      if (!__all_sync(0xffffffffu, mbar_wait_at(d2 + b, par(k / kBufs), a.status, 15, k))) break;
      tc_fence_after();
      float za[16], zb[16];
      tmem_ld16_issue(tbuf, za);
      tmem_wait(za);
#pragma unroll
      for (int t = 0; t < 4; ++t) {  // v = 8 t .. 8 t + 7
        float(&cur)[16] = (t & 1) ? zb : za;
        float(&nxt)[16] = (t & 1) ? za : zb;
        if (t + 1 < 4) tmem_ld16_issue(tbuf + 16 * (t + 1), nxt);
        float mx = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) mx = fmaxf(mx, fmaf(cur[2 * i], cur[2 * i], cur[2 * i + 1] * cur[2 * i + 1]));
        if (mx >= se.thr) {  // rare: some sample of this row is over the threshold
#pragma unroll
          for (int i = 0; i < 8; ++i)
            ep(se, j1 + (int64_t)N1 * (q + 32 * (8 * t + i)), make_float2(cur[2 * i], cur[2 * i + 1]));
        }
        if (t + 1 < 4) tmem_wait(nxt);
      }
      tc_fence_before();  // our tensor-memory reads before the MMAs that reuse the buffer
      mbar_arrive(tfree + b);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kMmaWarp) tmem_free(tmem, kTmemCols);
  pdl_launch_dependents();
}

template <class K, class... Args>
cudaError_t launch_pdl_tc(K kern, int grid, int block, int smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

int sm_count_tc() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

template <bool MP, bool SPLIT>
cudaError_t run_rows_tc(const FilterArgs& a, const FilterParts& ps, cudaStream_t st) {
  using G = TcGeo<SPLIT>;
  auto k = k_rows_tc<1024, MP, SPLIT>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int items = (MP ? ps.n_series : a.count * a.n_det) * (1024 / kTcRows);
  const int g = sm_count_tc();  // one CTA (all 512 TMEM columns) per SM
  cudaError_t e = launch_pdl_tc(k, items < g ? items : g, kTcThreads, G::SMEM, st, a, ps);
  add_launches(1);
  return e;
}

}  // namespace

cudaError_t launch_filter2_pass2_tc(const FilterArgs& a, cudaStream_t st, const FilterParts* parts) {
  if (a.n != (int64_t(1) << 20) || a.n1 != 1024 || a.n2 != 1024 || a.q_type != kBankF32 ||
      (a.inter != 1 && a.inter != 2))
    return cudaErrorInvalidValue;
  const FilterParts one{};
  if (a.inter == 2) return parts ? run_rows_tc<true, true>(a, *parts, st) : run_rows_tc<false, true>(a, one, st);
  return parts ? run_rows_tc<true, false>(a, *parts, st) : run_rows_tc<false, false>(a, one, st);
}

}  // namespace mf
