// TMA-staged matched-filter kernels (the hot path of Eq. 1-2 / Sec. V.C).
//
// N = N1 N2 four-step transform on sm_103a: 128-thread CTAs, three per SM,
// each a persistent loop over work items whose inputs are brought into shared
// memory by the bulk-copy (TMA) engine while the previous item computes.
//   k_cols: item = C columns k2 of one (template, detector) series, the
//           detector fastest in the item order.  The
//           template bank and the weighted data are stored column-major over
//           the non-zero half (element k = k1 N2 + k2, k1 < N1/2, at
//           k2 N1/2 + k1), so an item's two tiles are two contiguous 1-D bulk
//           copies.  The product x = q conj(h) is formed on the shared-memory
//           read; N1-point column transforms, each column owned by one group
//           of T threads inside a warp (its exchange needs only a warp
//           barrier); the four-step twiddle exp(+2 pi i j1 k2 / N); stores to
//           the scratch in panels of P = max(T(N1) / 2, RW(N2)) rows:
//           element (j1, k2) of a series at (j1 / P) N2 P + k2 P + j1 % P,
//           so that a warp's store covers whole 128-byte lines.
//   k_rows: item = RW rows j1 of one panel, brought in by a 3-D tensor-map
//           copy (RW of the panel's P values at each k2; one 1-D bulk copy
//           when RW = P); N2-point row transforms; rho^2 = |z|^2 / sigma^2 of
//           z[j1 + N1 j2], threshold and window maxima in registers.
// Sub-FFT twiddles come from a per-CTA shared table.  All mbarrier waits are
// bounded (see mf_tma.cuh) and report through the plan's status word.
// Programmatic dependent launch: each kernel lets the next one launch only
// when a CTA has finished all its items, so the next kernel's CTAs (which wait
// for this one to complete before touching the scratch) take the slots of
// retiring CTAs instead of competing with this kernel's own CTAs for them.
#include "mf_common.cuh"
#include "mf_tma.cuh"

namespace mf {

namespace {

constexpr int kT2 = 128;  // threads per CTA

constexpr int round128(int x) { return (x + 127) / 128 * 128; }

// generic-proxy writes of another grid -> async-proxy (TMA) reads of this one
__device__ __forceinline__ void fence_proxy_async_global_fwd() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Padded exchange buffer of the row transforms: RW rows of M values, row
// stride S >= PAD with S = K (mod 16) so that 64-bit accesses of a half-warp
// (K lanes per row) hit 16 distinct bank pairs.
template <int M, int K>
struct Xch {
  using G = SubFft<M>;
  static constexpr int S = stride_for(G::PAD, K);
  __device__ __forceinline__ static int idx(int c, int i) { return c * S + G::pidx(i); }
};

// Column regions of k_cols: column c of an item owns S float2 of a slot,
// first its template tile then its weighted-data tile (N1/2 values each) and,
// once its threads hold those in registers, its exchange buffer.  Thread
// (c = tid / T, t = tid % T) writes logical t RA + q of column c in pass a
// and reads j + r RA (j = t + T i) in pass b.  S is the even candidate in
// [base, base + 32), base = max(tiles, PAD), with the fewest repeated 8-byte
// bank pairs over every half-warp of both patterns (half-warps span two
// columns when T = 8); even keeps every region 16-byte aligned for TMA.
template <int M, int C, int BASE>
struct ColStride {
  using G = SubFft<M>;
  static constexpr int RA = G::RA, RB = G::RB, T = G::T, NB = G::NB;
  static constexpr int conflicts(int S) {
    int total = 0;
    for (int hw = 0; hw < kT2 / 16; ++hw) {
      for (int q = 0; q < RA; ++q) {
        int cnt[16] = {};
        for (int l = 0; l < 16; ++l) {
          const int tid = hw * 16 + l, c = tid / T, t = tid % T;
          ++cnt[(c * S + t * RA + q + t) & 15];
        }
        for (int b = 0; b < 16; ++b) total += cnt[b] > 1 ? cnt[b] - 1 : 0;
      }
      for (int i = 0; i < NB; ++i)
        for (int r = 0; r < RB; ++r) {
          int cnt[16] = {};
          for (int l = 0; l < 16; ++l) {
            const int tid = hw * 16 + l, c = tid / T, j = tid % T + T * i;
            ++cnt[(c * S + j + r * RA + r) & 15];
          }
          for (int b = 0; b < 16; ++b) total += cnt[b] > 1 ? cnt[b] - 1 : 0;
        }
    }
    return total;
  }
  static constexpr int pick() {
    const int b0 = (BASE + 1) / 2 * 2;
    int best = b0, bc = conflicts(b0);
    for (int s = b0 + 2; s < b0 + 32; s += 2) {
      const int c = conflicts(s);
      if (c < bc) {
        bc = c;
        best = s;
      }
    }
    return best;
  }
  static constexpr int S = pick();
};

constexpr int kColConsumers = kT2;             // compute threads of k_cols (4 warps)
constexpr int kColThreads = kColConsumers + 32;  // plus one producer warp

// Shared-memory plan of k_cols: two slots of C column regions (ColStride),
// then the sub-FFT twiddles and the barriers full[2], empty[2], twiddles.
template <int N1, int BT, int QT>
struct ColGeo {
  using G = SubFft<N1>;
  static constexpr int T = G::T;                          // threads per column
  static constexpr int C = kColConsumers / T;             // columns per item
  static constexpr int R = N1 / 2;                        // non-zero half of k1
  static constexpr int HB = BT == kBankF32 ? 8 : 4;       // bytes per template element
  static constexpr int QB = QT == kBankF32 ? 8 : 4;       // bytes per weighted-data element
  static constexpr int H_COL = R * HB;                    // one column's template tile, bytes
  static constexpr int Q_COL = R * QB;
  static constexpr int TILES = (H_COL + Q_COL) / 8;
  static constexpr int S = ColStride<N1, C, (TILES > G::PAD ? TILES : G::PAD)>::S;
  static constexpr int SLOT = C * S * 8;
  static constexpr int TW_BYTES = G::RB * G::RA * 8;
  static constexpr int TW_OFF = 2 * SLOT;
  static constexpr int BAR_OFF = TW_OFF + round128(TW_BYTES);
  static constexpr int SMEM = BAR_OFF + 64;
};

template <int N2>
struct RowGeo {
  using G = SubFft<N2>;
  static constexpr int RW = kT2 / G::T;                   // rows per item (the scratch panel height)
  static constexpr int ITEM = RW * N2;                    // complex values per item
  static constexpr int K = 16 / RW;                       // threads of one row in a half-warp
  using X = Xch<N2, K>;
  static constexpr int XCH_BYTES = RW * X::S * 8;
  static constexpr int SLOT = round128(ITEM * 8 > XCH_BYTES ? ITEM * 8 : XCH_BYTES);
  static constexpr int TW_BYTES = G::RB * G::RA * 8;
  static constexpr int TW_OFF = 2 * SLOT;
  static constexpr int BAR_OFF = TW_OFF + round128(TW_BYTES);
  static constexpr int SMEM = BAR_OFF + 32;
};

// Panel height P of the pass-1 -> pass-2 scratch.  A pass-1 warp stores, per
// instruction, T(N1) consecutive j1 of 32 / T(N1) consecutive columns k2; with
// P >= T/2 those are whole 128-byte lines of at most two panels.  P is also a
// multiple of the rows of one pass-2 item (RW(N2)), which are contiguous when
// P = RW.
template <int N1, int N2>
struct ScratchGeo {
  static constexpr int RW = RowGeo<N2>::RW;
  static constexpr int HT = SubFft<N1>::T / 2;
  static constexpr int P = HT > RW ? HT : RW;
  static constexpr int BOXY = N2 < 256 ? N2 : 256;  // k2 per tensor-map box (256 at most)
  static_assert(P % RW == 0 && N1 % P == 0 && N2 % BOXY == 0, "scratch panel geometry");
};

template <int BT>
__device__ __forceinline__ float2 smem_h(const unsigned char* base, int idx) {
  if constexpr (BT == kBankF32) {
    return reinterpret_cast<const float2*>(base)[idx];
  } else if constexpr (BT == kBankF16) {
    return __half22float2(reinterpret_cast<const __half2*>(base)[idx]);
  } else {
    return __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(base)[idx]);
  }
}

// w_M^{r j}, j < RA fastest, r < RB, written to global memory once per plan
template <int M>
__global__ void k_fill_twiddles(float2* tw) {
  using G = SubFft<M>;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G::RB * G::RA; i += gridDim.x * blockDim.x) {
    const int r = i / G::RA, j = i % G::RA;
    tw[i] = unit_root((uint32_t)((r * j) % M), (uint32_t)M);
  }
}

// ---------------------------------------------------------------------------
// pass 1
// ---------------------------------------------------------------------------

// IM: the intermediate (FilterArgs::inter).  IM >= 1: FP16, each series scaled by series_scale16 of its
// template, in panels of kPanel16 rows that are the tensor-core row pass's stage-1 operand image: with
// k2 = 32 p + q, part c (0 real, 1 imaginary) of element (j1, k2) is the half at panel j1 / 8,
// ((q 32 + p) 2 + c) 8 + j1 % 8 (an image of 2 N2 8 halves), i.e. the MN-major layout of rows
// m = 8 q + j1 % 8 and columns k = 2 p + c.  IM = 2: each panel holds the image of hi = the value rounded
// to FP16, then the image of lo = the remainder rounded to FP16.
// MP: the series of several plans' parts (FilterParts), each with its own bank, data rows and selection
template <int N1, int N2, int BT, int QT, int IM, bool MP>
__global__ void __launch_bounds__(kColThreads, 3) k_cols(FilterArgs a, const __grid_constant__ FilterParts ps) {
  static_assert(!MP || QT == kBankF32, "fused launches take FP32 weighted data");
  constexpr bool H16 = IM >= 1;
  constexpr int IMG = IM == 2 ? 2 : 1;  // FP16 images per panel
  using G = SubFft<N1>;
  using P = ColGeo<N1, BT, QT>;
  constexpr int RA = G::RA, RB = G::RB, T = G::T, NB = G::NB, C = P::C, R = P::R, S = P::S;
  constexpr int NCB = N2 / C;
  constexpr uint32_t N = (uint32_t)N1 * (uint32_t)N2;
  constexpr int PH = H16 ? kPanel16 : ScratchGeo<N1, N2>::P;  // scratch panel height
  extern __shared__ __align__(128) unsigned char sm[];
  const float2* tw = reinterpret_cast<const float2*>(sm + P::TW_OFF);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + P::BAR_OFF);  // [0], [1]: tiles of the slot landed
  uint64_t* empty = full + 2;                                     // [0], [1]: every warp done with the slot
  uint64_t* twb = full + 4;                                       // the twiddle table landed
  const int tid = threadIdx.x;
  const int n_items = (MP ? ps.n_series : a.count * a.n_det) * NCB;
  if (tid == 0) {
    mbar_init(full + 0, 1);
    mbar_init(full + 1, 1);
    mbar_init(empty + 0, kColConsumers / 32);
    mbar_init(empty + 1, kColConsumers / 32);
    mbar_init(twb, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid >= kColConsumers) {
    // producer warp: one lane issues every item's tiles into the slot its consumers released
    if (tid == kColConsumers) {
      const unsigned char* qbase = static_cast<const unsigned char*>(QT == kBankF32 ? (const void*)a.q : a.q_lp);
      mbar_expect_tx(twb, (uint32_t)P::TW_BYTES);
      bulk_g2s(sm + P::TW_OFF, a.tw1, (uint32_t)P::TW_BYTES, twb);
      // the weighted data come from the kernel just before only for the first batch; otherwise
      // the first tiles (bank and data, both unchanged) load while the previous kernel drains
      if (a.first_batch) {
        pdl_wait();
        fence_proxy_async_global_fwd();
      }
      int k = 0;
      bool ok = true;
      for (int item = blockIdx.x; item < n_items; item += gridDim.x, ++k) {
        const int slot = k & 1;
        if (k >= 2 && !(ok = mbar_wait_bounded(empty + slot, (uint32_t)(((k >> 1) + 1) & 1), a.status))) break;
        fence_proxy_async();
        int li = item, nd = a.n_det;
        const int32_t* sel = a.sel;
        int64_t pos0 = a.pos0, ld_bank = a.ld_bank, ld_q = a.ld_q;
        const unsigned char *hb = static_cast<const unsigned char*>(a.bank), *qb = qbase;
        if constexpr (MP) {
          const FilterPart& p = ps.p[part_of(ps, item, NCB)];
          li = item - p.series0 * NCB;
          nd = p.n_det;
          sel = p.sel;
          pos0 = p.pos0;
          hb = static_cast<const unsigned char*>(p.bank);
          ld_bank = p.ld_bank;
          qb = reinterpret_cast<const unsigned char*>(p.q);
          ld_q = p.ld_q;
        }
        // detector fastest: the n_det items of one bank tile are issued back to back, so the
        // tile is read from HBM once and from L2 for the other detectors
        const int d = li % nd, cb = (li / nd) % NCB, b = li / (nd * NCB);
        const int64_t tmpl = sel[pos0 + b];
        unsigned char* dst = sm + slot * P::SLOT;
        mbar_expect_tx(full + slot, (uint32_t)(C * (P::H_COL + P::Q_COL)));
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const int64_t col = (int64_t)cb * C + c;
          // default L2 priority: the n_det - 1 later items of this tile read it from L2
          bulk_g2s(dst + c * S * 8, hb + (tmpl * ld_bank + col * R) * P::HB, (uint32_t)P::H_COL, full + slot);
          bulk_g2s(dst + c * S * 8 + P::H_COL, qb + ((int64_t)d * ld_q + col * R) * P::QB, (uint32_t)P::Q_COL,
                   full + slot);
        }
      }
      // the consumers' last items are done: then let the next kernel launch
      for (int m = k - 2; ok && m < k; ++m)
        if (m >= 0) ok = mbar_wait_bounded(empty + (m & 1), (uint32_t)((m >> 1) & 1), a.status);
      if (!ok) {
        // a wait gave up: before the CTA exits, wait (bounded again) for the copies this lane issued
        // that no consumer may have waited for (the twiddles and the last two items' tiles); no later
        // copy went into those slots, so their phases cannot have wrapped
        mbar_wait_bounded(twb, 0, nullptr);
        for (int m = k - 2; m < k; ++m)
          if (m >= 0) mbar_wait_bounded(full + (m & 1), (uint32_t)((m >> 1) & 1), nullptr);
      }
      pdl_launch_dependents();
    }
    return;
  }
  // consumer warps: column ca of every item, T threads per column
  const int ca = tid / T, ta = tid % T;
  pdl_wait();  // the previous kernel (reader of the scratch we are about to write) has completed
  if (!mbar_wait_bounded(twb, 0, a.status)) return;
  int k = 0;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x, ++k) {
    const int slot = k & 1;
    if (!mbar_wait_bounded(full + slot, (uint32_t)((k >> 1) & 1), a.status)) break;
    const unsigned char* col = sm + slot * P::SLOT + ca * S * 8;
    int li = item, nd = a.n_det, s0 = 0;
    const int32_t* sel = a.sel;
    const float* isg = a.inv_sigma;
    int64_t pos0 = a.pos0;
    if constexpr (MP) {
      const FilterPart& p = ps.p[part_of(ps, item, NCB)];
      li = item - p.series0 * NCB;
      nd = p.n_det;
      s0 = p.series0;
      sel = p.sel;
      isg = p.inv_sigma;
      pos0 = p.pos0;
    }
    const int s = s0 + (li / (nd * NCB)) * nd + li % nd;
    float2 v[RA];
#pragma unroll
    for (int r = 0; r < RA; ++r) {
      if (r >= RA / 2) {
        v[r] = make_float2(0.f, 0.f);
      } else {
        const int idx = ta + r * RB;  // k1 < N1/2
        v[r] = cmulc(smem_h<QT>(col + P::H_COL, idx), smem_h<BT>(col, idx));
      }
    }
    __syncwarp();  // the column's tiles are read: its region becomes the exchange buffer
    dft<RA, true>(v);
    float2* xb = reinterpret_cast<float2*>(sm + slot * P::SLOT) + ca * S;
#pragma unroll
    for (int q = 0; q < RA; ++q) xb[ta * RA + q + ta] = v[q];
    __syncwarp();
    float2* out = a.scratch + (int64_t)s * N;
    __half* out16 = reinterpret_cast<__half*>(a.scratch) + (int64_t)s * 2 * IMG * N;
    const int k2 = ((li / nd) % NCB) * C + ca;
    float sc = 1.f;
    if constexpr (H16) sc = series_scale16(__ldg(isg + sel[pos0 + li / (nd * NCB)]));
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int j = ta + T * i;
      float2 u[RB];
      u[0] = xb[j];
#pragma unroll
      for (int r = 1; r < RB; ++r) u[r] = cmul(xb[j + r * RA + r], tw[r * RA + j]);
      dft<RB>(u);
      // four-step twiddle w_N^{(j + q RA) k2} = w_N^{j k2} (w_N^{RA k2})^q; the table row of
      // column k2 holds w_N^{j k2} for j <= RA, so a warp's loads are contiguous
      const float2* twr = a.tw4 + (int64_t)k2 * (RA + 1);
      float2 w = __ldg(twr + j);
      const float2 st = __ldg(twr + RA);
      if constexpr (H16) {
        static_assert(RA % PH == 0 && N2 == 1024, "FP16 panels");
        w.x *= sc;
        w.y *= sc;
        // j1 = j + q RA: q RA / 8 whole panels past j's; within a panel, (k2 % 32, k2 / 32, part, j1 % 8).
        // Lanes j, j + 1 (j even) of the column swap halves so that each writes 4 bytes: j the real parts
        // of rows j, j + 1 and j + 1 their imaginary parts (one warp store: four whole 32-byte sectors)
        static_assert(T == 32, "lane pairs");
        const bool odd = (j & 1) != 0;
        constexpr int64_t IMAGE = 2 * N2 * PH;  // halves of one FP16 image of a panel
        __half* ob = out16 + (int64_t)(j / PH) * (IMG * IMAGE) + (((k2 & 31) * 32 + (k2 >> 5)) * 2) * PH +
                     (odd ? PH + (j % PH) - 1 : (j % PH));
        auto pair_store = [&](__half* dst, __half2 h) {
          const uint32_t mine = *reinterpret_cast<const uint32_t*>(&h);
          const uint32_t other = __shfl_xor_sync(0xffffffffu, mine, 1);
          *reinterpret_cast<uint32_t*>(dst) = odd ? __byte_perm(other, mine, 0x7632) : __byte_perm(mine, other, 0x5410);
        };
#pragma unroll
        for (int q = 0; q < RB; ++q) {
          const float2 z = cmul(u[q], w);
          const __half2 h = __float22half2_rn(z);
          __half* dq = ob + (int64_t)q * (RA / PH) * (IMG * IMAGE);
          pair_store(dq, h);
          if constexpr (IM == 2) {  // the remainder: z - hi is exact in FP32
            const float2 hf = __half22float2(h);
            pair_store(dq + IMAGE, __float22half2_rn(make_float2(z.x - hf.x, z.y - hf.y)));
          }
          if (q + 1 < RB) w = cmul(w, st);
        }
      } else if constexpr (RA % PH == 0) {  // j1 = j + q RA: q RA / PH whole panels past j's
        float2* ob = out + (int64_t)(j / PH) * (N2 * PH) + k2 * PH + (j % PH);
#pragma unroll
        for (int q = 0; q < RB; ++q) {
          ob[(int64_t)q * (RA / PH) * (N2 * PH)] = cmul(u[q], w);
          if (q + 1 < RB) w = cmul(w, st);
        }
      } else {
#pragma unroll
        for (int q = 0; q < RB; ++q) {
          const int j1 = j + q * RA;
          out[(int64_t)(j1 / PH) * (N2 * PH) + k2 * PH + (j1 % PH)] = cmul(u[q], w);
          if (q + 1 < RB) w = cmul(w, st);
        }
      }
    }
    // this warp is done with the slot: order its shared accesses before the next bulk copy into it
    fence_proxy_async();
    __syncwarp();
    if ((tid & 31) == 0) mbar_arrive(empty + slot);
  }
  pdl_launch_dependents();  // our items are done: the next kernel may launch
}

// ---------------------------------------------------------------------------
// pass 2
// ---------------------------------------------------------------------------

// tm: the scratch as [series * N1 / PH panels][N2][PH] of 8-byte values, box
// {RW, BOXY, 1} (unused when RW = PH: an item is then one contiguous panel)
// MP: the series of several plans' parts (FilterParts), each with its own epilogue state
template <int N1, int N2, bool MP>
__global__ void __launch_bounds__(kT2, 3) k_rows(const __grid_constant__ CUtensorMap tm, FilterArgs a,
                                                 const __grid_constant__ FilterParts ps) {
  using G = SubFft<N2>;
  using P = RowGeo<N2>;
  using X = typename P::X;
  using SG = ScratchGeo<N1, N2>;
  constexpr int RA = G::RA, RB = G::RB, T = G::T, NB = G::NB, RW = P::RW, PH = SG::P;
  constexpr int NRB = N1 / RW;
  constexpr int64_t N = (int64_t)N1 * N2;
  extern __shared__ __align__(128) unsigned char sm[];
  const float2* tw = reinterpret_cast<const float2*>(sm + P::TW_OFF);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + P::BAR_OFF);
  const int tid = threadIdx.x;
  const int row = tid % RW, t = tid / RW;  // rows fastest: the panel is [k2][row]
  // series in reverse order: the last ones pass 1 wrote are the likeliest to be still in L2
  const int n_series = MP ? ps.n_series : a.count * a.n_det;
  const int n_items = n_series * NRB;
  if (tid == 0) {
    mbar_init(bar + 0, 1);
    mbar_init(bar + 1, 1);
    mbar_init(bar + 2, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const uint64_t pol_last_use = policy_evict_first();
  auto issue = [&](int item, int slot) {
    const int s = n_series - 1 - item / NRB, j10 = (item % NRB) * RW;
    mbar_expect_tx(bar + slot, (uint32_t)(P::ITEM * 8));
    if constexpr (RW == PH) {
      bulk_g2s_hint(sm + slot * P::SLOT, a.scratch + (int64_t)s * N + (int64_t)j10 * N2, (uint32_t)(P::ITEM * 8),
                    bar + slot, pol_last_use);
    } else {
      // rows j10 .. j10 + RW - 1 of panel j10 / PH: RW * 8 bytes at each k2, landing as [k2][row]
      const int z = s * (N1 / PH) + j10 / PH;
#pragma unroll
      for (int y = 0; y < N2; y += SG::BOXY)
        tma_load_3d_hint(sm + slot * P::SLOT + (size_t)y * RW * 8, &tm, j10 % PH, y, z, bar + slot, pol_last_use);
    }
  };
  if (tid == 0) {
    mbar_expect_tx(bar + 2, (uint32_t)P::TW_BYTES);
    bulk_g2s(sm + P::TW_OFF, a.tw2, (uint32_t)P::TW_BYTES, bar + 2);
    pdl_wait();  // the scratch is written by the kernel just before
    fence_proxy_async_global_fwd();
    if ((int)blockIdx.x < n_items) issue(blockIdx.x, 0);
  }
  if (__syncthreads_or(!mbar_wait_bounded(bar + 2, 0, a.status))) {
    if (tid == 0) {  // drain (bounded) the copies issued above before the CTA exits
      mbar_wait_bounded(bar + 2, 0, nullptr);
      if ((int)blockIdx.x < n_items) mbar_wait_bounded(bar + 0, 0, nullptr);
    }
    return;
  }
  RawEpi ep{a.sel, a.inv_sigma, a.thr_raw, a.q_type == kBankF32 ? nullptr : a.dscale, a.pos0, a.n_det, a.window,
            a.valid_begin, a.valid_end, a.n_win, a.n_sel_total, a.slots, a.row_valid};
  int k = 0;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x, ++k) {
    const int slot = k & 1;
    const bool fail = !mbar_wait_bounded(bar + slot, (uint32_t)((k >> 1) & 1), a.status);
    const float2* stage = reinterpret_cast<const float2*>(sm + slot * P::SLOT);
    const int s = n_series - 1 - item / NRB;
    const int j1 = (item % NRB) * RW + row;
    float2 v[RA];
#pragma unroll
    for (int r = 0; r < RA; ++r) v[r] = stage[(t + r * RB) * RW + row];
    if (__syncthreads_or(fail)) {
      // the copy into this slot may still be in flight: wait for it (bounded) before the CTA exits;
      // nothing was issued into the other slot since its last wait completed
      if (tid == 0) mbar_wait_bounded(bar + slot, (uint32_t)((k >> 1) & 1), nullptr);
      return;
    }
    if (tid == 0 && item + (int)gridDim.x < n_items) {
      fence_proxy_async();
      issue(item + gridDim.x, slot ^ 1);
    }
    dft<RA>(v);
    float2* xb = reinterpret_cast<float2*>(sm + slot * P::SLOT);
#pragma unroll
    for (int q = 0; q < RA; ++q) xb[X::idx(row, t * RA + q)] = v[q];
    __syncthreads();
    RawEpi::Ser se;
    if constexpr (MP) {
      const FilterPart& p = ps.p[part_of(ps, s, 1)];
      const RawEpi pe{p.sel,           p.inv_sigma, p.thr_raw,     nullptr, p.pos0,   p.n_det,      a.window,
                      p.valid_begin,   p.valid_end, a.n_win,       p.n_sel_total,     p.slots,      p.row_valid};
      se = pe.series(s - p.series0);
    } else {
      se = ep.series(s);
    }
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int j = t + T * i;
      float2 u[RB];
      u[0] = xb[X::idx(row, j)];
#pragma unroll
      for (int r = 1; r < RB; ++r) u[r] = cmul(xb[X::idx(row, j + r * RA)], tw[r * RA + j]);
      dft<RB>(u);
#pragma unroll
      for (int q = 0; q < RB; ++q) ep(se, (int64_t)j1 + (int64_t)N1 * (j + q * RA), u[q]);
    }
  }
  pdl_launch_dependents();  // our items are done: the next kernel may launch
}

template <class K>
cudaError_t set_smem2(K kern, int bytes) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// launch with programmatic stream serialization (overlaps our prologue with the previous kernel's tail)
template <class K, class... Args>
cudaError_t launch_pdl(K kern, int grid, int block, int smem, cudaStream_t st, Args... args) {
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

int grid2(int items) {
  const int g = sm_count() * 3;
  return items < g ? items : g;
}

template <int N1, int N2, int BT, int QT, int IM = 0, bool MP = false>
cudaError_t run_cols(const FilterArgs& a, const FilterParts& ps, cudaStream_t st) {
  using P = ColGeo<N1, BT, QT>;
  static_assert(P::SMEM * 3 <= 230400, "k_cols: three CTAs per SM must fit in shared memory");
  auto k = k_cols<N1, N2, BT, QT, IM, MP>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = set_smem2(k, P::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int items = (MP ? ps.n_series : a.count * a.n_det) * (N2 / P::C);
  cudaError_t e = launch_pdl(k, grid2(items), kColThreads, P::SMEM, st, a, ps);
  add_launches(1);
  return e;
}

// (bank, data) storage pairs: FP32 data with any bank; 16-bit data with a bank of the same type.
// Fused launches (ps.n > 0): FP32 data, an FP32 bank.
template <int N1, int N2>
cudaError_t run_cols_bt(const FilterArgs& a, const FilterParts& ps, cudaStream_t st) {
  const bool mp = ps.n > 0;
  if (mp && (a.q_type != kBankF32 || a.bank_type != kBankF32)) return cudaErrorInvalidValue;
  if constexpr (N1 == 1024 && N2 == 1024) {
    // FP16 intermediates for the tensor-core row pass: FP32 data, any bank
    if (a.inter != 0 && a.q_type != kBankF32) return cudaErrorInvalidValue;
    if (a.inter == 1) {
      if (mp) return run_cols<N1, N2, kBankF32, kBankF32, 1, true>(a, ps, st);
      switch (a.bank_type) {
        case kBankF32: return run_cols<N1, N2, kBankF32, kBankF32, 1>(a, ps, st);
        case kBankF16: return run_cols<N1, N2, kBankF16, kBankF32, 1>(a, ps, st);
        case kBankBF16: return run_cols<N1, N2, kBankBF16, kBankF32, 1>(a, ps, st);
      }
      return cudaErrorInvalidValue;
    }
    if (a.inter == 2) {
      if (mp) return run_cols<N1, N2, kBankF32, kBankF32, 2, true>(a, ps, st);
      switch (a.bank_type) {
        case kBankF32: return run_cols<N1, N2, kBankF32, kBankF32, 2>(a, ps, st);
        case kBankF16: return run_cols<N1, N2, kBankF16, kBankF32, 2>(a, ps, st);
        case kBankBF16: return run_cols<N1, N2, kBankBF16, kBankF32, 2>(a, ps, st);
      }
      return cudaErrorInvalidValue;
    }
    if (a.inter != 0) return cudaErrorInvalidValue;
  } else {
    if (a.inter != 0) return cudaErrorInvalidValue;
  }
  if (mp) return run_cols<N1, N2, kBankF32, kBankF32, 0, true>(a, ps, st);
  if (a.q_type == kBankF32) {
    switch (a.bank_type) {
      case kBankF32: return run_cols<N1, N2, kBankF32, kBankF32>(a, ps, st);
      case kBankF16: return run_cols<N1, N2, kBankF16, kBankF32>(a, ps, st);
      case kBankBF16: return run_cols<N1, N2, kBankBF16, kBankF32>(a, ps, st);
    }
  } else if (a.q_type == a.bank_type) {
    switch (a.bank_type) {
      case kBankF16: return run_cols<N1, N2, kBankF16, kBankF16>(a, ps, st);
      case kBankBF16: return run_cols<N1, N2, kBankBF16, kBankBF16>(a, ps, st);
    }
  }
  return cudaErrorInvalidValue;
}

template <int N1, int N2, bool MP>
cudaError_t run_rows_mp(const FilterArgs& a, const FilterParts& ps, const CUtensorMap& tm, cudaStream_t st) {
  using P = RowGeo<N2>;
  static_assert(P::SMEM * 3 <= 230400, "k_rows: three CTAs per SM must fit in shared memory");
  auto k = k_rows<N1, N2, MP>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = set_smem2(k, P::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int items = (MP ? ps.n_series : a.count * a.n_det) * (N1 / P::RW);
  cudaError_t e = launch_pdl(k, grid2(items), kT2, P::SMEM, st, tm, a, ps);
  add_launches(1);
  return e;
}

template <int N1, int N2>
cudaError_t run_rows(const FilterArgs& a, const FilterParts& ps, const CUtensorMap& tm, cudaStream_t st) {
  if (ps.n > 0) {
    if (a.q_type != kBankF32) return cudaErrorInvalidValue;
    return run_rows_mp<N1, N2, true>(a, ps, tm, st);
  }
  return run_rows_mp<N1, N2, false>(a, ps, tm, st);
}

// signature of the driver's cuTensorMapEncodeTiled (CUDA 12.0 ABI), fetched at run time
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

template <int N1, int N2>
cudaError_t encode_scratch_of(const float2* scratch, int64_t series, CUtensorMap* m) {
  using SG = ScratchGeo<N1, N2>;
  *m = CUtensorMap{};
  if (SG::RW == SG::P) return cudaSuccess;  // contiguous items: no tensor map
  auto fn = encode_fn();
  if (!fn || !scratch || series < 1) return cudaErrorInvalidValue;
  cuuint64_t dims[3] = {(cuuint64_t)SG::P, (cuuint64_t)N2, (cuuint64_t)(series * (N1 / SG::P))};
  cuuint64_t strides[2] = {(cuuint64_t)SG::P * 8, (cuuint64_t)N2 * SG::P * 8};
  cuuint32_t box[3] = {(cuuint32_t)SG::RW, (cuuint32_t)SG::BOXY, 1u};
  cuuint32_t es[3] = {1u, 1u, 1u};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<float2*>(scratch), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

#define MF_DISPATCH2(n, FN, ARGS)            \
  switch (n) {                               \
    case 1 << 12: return FN<64, 64> ARGS;    \
    case 1 << 13: return FN<128, 64> ARGS;   \
    case 1 << 14: return FN<128, 128> ARGS;  \
    case 1 << 15: return FN<256, 128> ARGS;  \
    case 1 << 16: return FN<256, 256> ARGS;  \
    case 1 << 17: return FN<512, 256> ARGS;  \
    case 1 << 18: return FN<512, 512> ARGS;  \
    case 1 << 19: return FN<1024, 512> ARGS; \
    case 1 << 20: return FN<1024, 1024> ARGS;\
  }                                          \
  return cudaErrorInvalidValue;

template <int N1, int N2>
cudaError_t run_fill_tw(float2* tw1, float2* tw2, cudaStream_t st) {
  k_fill_twiddles<N1><<<4, 256, 0, st>>>(tw1);
  k_fill_twiddles<N2><<<4, 256, 0, st>>>(tw2);
  add_launches(2);
  return cudaGetLastError();
}

// four-step twiddles by column: tw4[k2 (ra + 1) + j] = w_N^{j k2}, j <= ra, k2 < n2
__global__ void k_fill_tw4(float2* tw4, int n2, int ra, uint32_t n) {
  const int64_t count = (int64_t)n2 * (ra + 1);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t k2 = (uint32_t)(i / (ra + 1)), j = (uint32_t)(i % (ra + 1));
    tw4[i] = unit_root((j * k2) % n, n);
  }
}

template <int N1, int N2>
cudaError_t run_fill_tw4(float2* tw4, cudaStream_t st) {
  k_fill_tw4<<<64, 256, 0, st>>>(tw4, N2, SubFft<N1>::RA, (uint32_t)N1 * (uint32_t)N2);
  add_launches(1);
  return cudaGetLastError();
}

template <int N1, int N2>
cudaError_t tw4_count_of(int64_t* c) {
  *c = (int64_t)N2 * (SubFft<N1>::RA + 1);
  return cudaSuccess;
}

}  // namespace

namespace {

const FilterParts kOnePlan{};  // n = 0: every per-series field from FilterArgs

cudaError_t pass1_parts(const FilterArgs& a, const FilterParts& ps, cudaStream_t st) {
  MF_DISPATCH2(a.n, run_cols_bt, (a, ps, st))
}

cudaError_t pass2_parts(const FilterArgs& a, const FilterParts& ps, const CUtensorMap& tm, cudaStream_t st) {
  if (a.inter != 0) return launch_filter2_pass2_tc(a, st, ps.n > 0 ? &ps : nullptr);
  MF_DISPATCH2(a.n, run_rows, (a, ps, tm, st))
}

}  // namespace

cudaError_t launch_filter2_pass1(const FilterArgs& a, cudaStream_t st) { return pass1_parts(a, kOnePlan, st); }

cudaError_t launch_filter2_pass2(const FilterArgs& a, const CUtensorMap& tm, cudaStream_t st) {
  return pass2_parts(a, kOnePlan, tm, st);
}

cudaError_t launch_filter2_fused(const FilterArgs& a, const FilterParts& ps, const CUtensorMap& tm, cudaStream_t st,
                                 cudaEvent_t between) {
  if (ps.n < 1 || ps.n > kMaxParts || ps.n_series < 1) return cudaErrorInvalidValue;
  cudaError_t e = pass1_parts(a, ps, st);
  if (e == cudaSuccess && between) e = cudaEventRecord(between, st);
  if (e == cudaSuccess) e = pass2_parts(a, ps, tm, st);
  return e;
}

cudaError_t encode_scratch_map(int64_t n, const float2* scratch, int64_t series, CUtensorMap* m) {
  MF_DISPATCH2(n, encode_scratch_of, (scratch, series, m))
}

cudaError_t launch_fill_tw4(int64_t n, float2* tw4, cudaStream_t st) { MF_DISPATCH2(n, run_fill_tw4, (tw4, st)) }

int64_t tw4_count(int64_t n) {
  int64_t c = 0;
  auto f = [&]() -> cudaError_t { MF_DISPATCH2(n, tw4_count_of, (&c)) };
  return f() == cudaSuccess ? c : 0;
}

cudaError_t launch_fill_twiddles(int64_t n, float2* tw1, float2* tw2, cudaStream_t st) {
  MF_DISPATCH2(n, run_fill_tw, (tw1, tw2, st))
}

}  // namespace mf
