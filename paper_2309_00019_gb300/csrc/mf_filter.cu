// TMA-staged matched-filter kernels (the hot path of Eq. 1-2 / Sec. V.C).
//
// Same four-step transform as the reference kernels in mf_kernels.cu, laid
// out for sm_103a: 128-thread CTAs, three per SM, each a persistent loop over
// work items whose inputs are brought into shared memory by the TMA engine
// while the previous item computes.
//   k_cols: item = C columns k2 of one (template, detector) series.  Two 3-D
//           tensor-map copies bring the template tile h[k1][k2] and the
//           weighted-data tile q_d[k1][k2] for the non-zero half k1 < N1/2;
//           the product x = q conj(h) is formed on the shared-memory read;
//           N1-point column transforms; the four-step twiddle
//           exp(+2 pi i j1 k2 / N); coalesced stores to the L2-resident scratch.
//   k_rows: item = RW consecutive rows j1 of one series, one 1-D bulk copy;
//           N2-point row transforms; rho^2 = |z|^2 / sigma^2 of
//           z[j1 + N1 j2], threshold and window maxima in registers.
// Sub-FFT twiddles come from a per-CTA shared table.  All mbarrier waits are
// bounded (see mf_tma.cuh) and report through the plan's status word.
#include "mf_common.cuh"
#include "mf_tma.cuh"

namespace mf {

namespace {

constexpr int kT2 = 128;  // threads per CTA

constexpr int round128(int x) { return (x + 127) / 128 * 128; }

// generic-proxy writes of another grid -> async-proxy (TMA) reads of this one
__device__ __forceinline__ void fence_proxy_async_global_fwd() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Exchange-buffer layout of G groups (columns or rows) of M complex values.
// For RA >= 16 the buffer is unpadded and XOR-swizzled: logical element i of
// group c lives at c M + (i & ~15) + ((i & 15) ^ ((i / RA + K c) & 15)), so
// that the pass-a writes (i = t RA + a) and the pass-b reads (i = j + r RA) of
// every half-warp touch 16 distinct 8-byte bank pairs; K = lanes a group
// contributes to a half-warp.  For RA = 8 (M = 64) rows are padded instead.
template <int M, int K, bool SWIZZLE = true>
struct Xch {
  using G = SubFft<M>;
  static constexpr bool SWZ = SWIZZLE && G::RA >= 16;
  static constexpr int S = SWZ ? M : stride_for(G::PAD, K);
  __device__ __forceinline__ static int idx(int c, int i) {
    if constexpr (SWZ) {
      return c * M + (i & ~15) + ((i & 15) ^ ((i / G::RA + K * c) & 15));
    } else {
      return c * S + G::pidx(i);
    }
  }
};

// Shared-memory plan of k_cols: two slots, each first the landing zone of an
// item's TMA tiles (template + weighted data) and then, once those are in
// registers, the padded exchange buffer of the same item; the next item's
// tiles land in the other slot.  Then the sub-FFT twiddle table and barriers.
template <int N1, int BT, int QT = kBankF32>
struct ColGeo {
  using G = SubFft<N1>;
  static constexpr int C = kT2 / G::T;                    // columns per item
  static constexpr int ROWS = N1 / 2;                     // non-zero half of k1
  static constexpr int BOXR = ROWS < 256 ? ROWS : 256;    // rows per TMA box
  static constexpr int NBOX = ROWS / BOXR;
  static constexpr int HB = BT == kBankF32 ? 8 : 4;       // bytes per template element
  static constexpr int QB = QT == kBankF32 ? 8 : 4;       // bytes per weighted-data element
  static constexpr int H_BYTES = ROWS * C * HB;
  static constexpr int Q_BYTES = ROWS * C * QB;
  static constexpr int K = C >= 16 ? 1 : 16 / C;
  using X = Xch<N1, K, false>;
  static constexpr int XCH_BYTES = C * X::S * 8;
  static constexpr int SLOT = round128(H_BYTES + Q_BYTES > XCH_BYTES ? H_BYTES + Q_BYTES : XCH_BYTES);
  static constexpr int TW_BYTES = G::RB * G::RA * 8;
  static constexpr int TW_OFF = 2 * SLOT;
  static constexpr int BAR_OFF = TW_OFF + round128(TW_BYTES);
  static constexpr int SMEM = BAR_OFF + 32;
};

template <int N2>
struct RowGeo {
  using G = SubFft<N2>;
  static constexpr int RW = kT2 / G::T;                   // rows per item
  static constexpr int ITEM = RW * N2;                    // complex values per item
  static constexpr int K = G::T >= 16 ? 0 : G::T;
  using X = Xch<N2, K == 0 ? 16 : K, false>;
  static constexpr int XCH_BYTES = RW * X::S * 8;
  static constexpr int SLOT = round128(ITEM * 8 > XCH_BYTES ? ITEM * 8 : XCH_BYTES);
  static constexpr int TW_BYTES = G::RB * G::RA * 8;
  static constexpr int TW_OFF = 2 * SLOT;
  static constexpr int BAR_OFF = TW_OFF + round128(TW_BYTES);
  static constexpr int SMEM = BAR_OFF + 32;
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

// Barrier wait of the whole CTA: thread 0 spins (bounded), the others then
// observe the completed phase.  Returns false (uniformly) on timeout.
__device__ __forceinline__ bool cta_wait(uint64_t* bar, uint32_t parity, int* status, int* ok) {
  if (threadIdx.x == 0) *ok = mbar_wait_bounded(bar, parity, status) ? 1 : 0;
  __syncthreads();
  if (!*ok) return false;
  if (threadIdx.x != 0) mbar_try_wait(bar, parity);
  return true;
}

// ---------------------------------------------------------------------------
// pass 1
// ---------------------------------------------------------------------------

template <int N1, int N2, int BT, int QT>
__global__ void __launch_bounds__(kT2, 3)
    k_cols(const __grid_constant__ CUtensorMap tm_h, const __grid_constant__ CUtensorMap tm_q, FilterArgs a) {
  using G = SubFft<N1>;
  using P = ColGeo<N1, BT, QT>;
  using X = typename P::X;
  constexpr int RA = G::RA, RB = G::RB, T = G::T, NB = G::NB, C = P::C;
  constexpr int NCB = N2 / C;
  constexpr uint32_t N = (uint32_t)N1 * (uint32_t)N2;
  extern __shared__ __align__(128) unsigned char sm[];
  const float2* tw = reinterpret_cast<const float2*>(sm + P::TW_OFF);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + P::BAR_OFF);  // [0], [1]: slots, [2]: twiddles
  const int tid = threadIdx.x;
  const int c = tid % C, t = tid / C;
  const int n_items = a.count * a.n_det * NCB;
  if (tid == 0) {
    mbar_init(bar + 0, 1);
    mbar_init(bar + 1, 1);
    mbar_init(bar + 2, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_keep = policy_evict_last();
  auto issue = [&](int item, int slot) {
    const int s = item / NCB, cb = item % NCB;
    const int b = s / a.n_det, d = s % a.n_det;
    const int tmpl = a.sel[a.pos0 + b];
    unsigned char* dst = sm + slot * P::SLOT;
    mbar_expect_tx(bar + slot, (uint32_t)(P::H_BYTES + P::Q_BYTES));
#pragma unroll
    for (int bx = 0; bx < P::NBOX; ++bx) {
      tma_load_3d_hint(dst + bx * P::BOXR * C * P::HB, &tm_h, cb * C, bx * P::BOXR, tmpl, bar + slot, pol_stream);
      tma_load_3d(dst + P::H_BYTES + bx * P::BOXR * C * P::QB, &tm_q, cb * C, bx * P::BOXR, d, bar + slot);
    }
  };
  pdl_launch_dependents();  // the next kernel may start its prologue as our CTAs retire
  if (tid == 0) {
    mbar_expect_tx(bar + 2, (uint32_t)P::TW_BYTES);
    bulk_g2s(sm + P::TW_OFF, a.tw1, (uint32_t)P::TW_BYTES, bar + 2);
    // the weighted data come from the kernel just before only for the first batch; otherwise
    // the first tiles (bank and data, both unchanged) load while the previous kernel drains
    if (a.first_batch) pdl_wait();
    if ((int)blockIdx.x < n_items) issue(blockIdx.x, 0);
  }
  pdl_wait();  // the previous kernel (reader of the scratch we are about to write) has completed
  if (__syncthreads_or(!mbar_wait_bounded(bar + 2, 0, a.status))) return;
  int k = 0;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x, ++k) {
    const int slot = k & 1;
    // every thread waits (bounded) for this item's tiles, reads its inputs, then one barrier
    const bool fail = !mbar_wait_bounded(bar + slot, (uint32_t)((k >> 1) & 1), a.status);
    const unsigned char* sh = sm + slot * P::SLOT;
    const int s = item / NCB;
    const int k2 = (item % NCB) * C + c;
    float2 v[RA];
#pragma unroll
    for (int r = 0; r < RA; ++r) {
      if (r >= RA / 2) {
        v[r] = make_float2(0.f, 0.f);
      } else {
        const int idx = (t + r * RB) * C + c;
        v[r] = cmulc(smem_h<QT>(sh + P::H_BYTES, idx), smem_h<BT>(sh, idx));
      }
    }
    // tiles consumed by every thread; the previous item (other slot) is finished too
    if (__syncthreads_or(fail)) return;
    if (tid == 0 && item + (int)gridDim.x < n_items) {
      fence_proxy_async();
      issue(item + gridDim.x, slot ^ 1);
    }
    dft<RA, true>(v);
    float2* xb = reinterpret_cast<float2*>(sm + slot * P::SLOT);
#pragma unroll
    for (int q = 0; q < RA; ++q) xb[X::idx(c, t * RA + q)] = v[q];
    __syncthreads();
    float2* out = a.scratch + (int64_t)s * N;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int j = t + T * i;
      float2 u[RB];
      u[0] = xb[X::idx(c, j)];
#pragma unroll
      for (int r = 1; r < RB; ++r) u[r] = cmul(xb[X::idx(c, j + r * RA)], tw[r * RA + j]);
      dft<RB>(u);
      // four-step twiddle w_N^{(j + q RA) k2} = w_N^{j k2} (w_N^{RA k2})^q, both from the table
      float2 w = __ldg(a.tw4 + (uint32_t)j * (uint32_t)k2);
      const float2 st = __ldg(a.tw4 + (uint32_t)RA * (uint32_t)k2);
#pragma unroll
      for (int q = 0; q < RB; ++q) {
        st_global_hint(out + (int64_t)(j + q * RA) * N2 + k2, cmul(u[q], w), pol_keep);
        if (q + 1 < RB) w = cmul(w, st);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// pass 2
// ---------------------------------------------------------------------------

template <int N1, int N2>
__global__ void __launch_bounds__(kT2, 3) k_rows(FilterArgs a) {
  using G = SubFft<N2>;
  using P = RowGeo<N2>;
  using X = typename P::X;
  constexpr int RA = G::RA, RB = G::RB, T = G::T, NB = G::NB, RW = P::RW;
  constexpr int NRB = N1 / RW;
  constexpr int64_t N = (int64_t)N1 * N2;
  extern __shared__ __align__(128) unsigned char sm[];
  const float2* tw = reinterpret_cast<const float2*>(sm + P::TW_OFF);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + P::BAR_OFF);
  const int tid = threadIdx.x;
  const int t = tid % T, row = tid / T;
  const int n_items = a.count * a.n_det * NRB;
  if (tid == 0) {
    mbar_init(bar + 0, 1);
    mbar_init(bar + 1, 1);
    mbar_init(bar + 2, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const uint64_t pol_last_use = policy_evict_first();
  auto issue = [&](int item, int slot) {
    const int s = item / NRB, j10 = (item % NRB) * RW;
    mbar_expect_tx(bar + slot, (uint32_t)(P::ITEM * 8));
    bulk_g2s_hint(sm + slot * P::SLOT, a.scratch + (int64_t)s * N + (int64_t)j10 * N2, (uint32_t)(P::ITEM * 8),
                  bar + slot, pol_last_use);
  };
  pdl_launch_dependents();
  if (tid == 0) {
    mbar_expect_tx(bar + 2, (uint32_t)P::TW_BYTES);
    bulk_g2s(sm + P::TW_OFF, a.tw2, (uint32_t)P::TW_BYTES, bar + 2);
    pdl_wait();  // the scratch is written by the kernel just before
    fence_proxy_async_global_fwd();
    if ((int)blockIdx.x < n_items) issue(blockIdx.x, 0);
  }
  if (__syncthreads_or(!mbar_wait_bounded(bar + 2, 0, a.status))) return;
  RawEpi ep{a.sel, a.inv_sigma, a.thr_raw, a.q_type == kBankF32 ? nullptr : a.dscale, a.pos0, a.n_det, a.window, a.valid_begin, a.valid_end,
            a.n_win, a.n_sel_total, a.slots, a.row_valid};
  int k = 0;
  for (int item = blockIdx.x; item < n_items; item += gridDim.x, ++k) {
    const int slot = k & 1;
    const bool fail = !mbar_wait_bounded(bar + slot, (uint32_t)((k >> 1) & 1), a.status);
    const float2* stage = reinterpret_cast<const float2*>(sm + slot * P::SLOT);
    const int s = item / NRB;
    const int j1 = (item % NRB) * RW + row;
    float2 v[RA];
#pragma unroll
    for (int r = 0; r < RA; ++r) v[r] = stage[row * N2 + t + r * RB];
    if (__syncthreads_or(fail)) return;
    if (tid == 0 && item + (int)gridDim.x < n_items) {
      fence_proxy_async();
      issue(item + gridDim.x, slot ^ 1);
    }
    dft<RA>(v);
    float2* xb = reinterpret_cast<float2*>(sm + slot * P::SLOT);
#pragma unroll
    for (int q = 0; q < RA; ++q) xb[X::idx(row, t * RA + q)] = v[q];
    __syncthreads();
    const auto se = ep.series(s);
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
}

// ---------------------------------------------------------------------------
// fused persistent filter: both passes of every batch from one work queue
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Work queue: phases P1(0), P1(1), P2(0), P1(2), P2(1), ..., P1(nb-1), P2(nb-2),
// P2(nb-1).  P2(b) needs every P1(b) item; P1(b) with b >= n_slots reuses the
// scratch slot of batch b - n_slots and needs every P2(b - n_slots) item.
// Every dependency points to earlier queue positions (n_slots >= 2), so the
// earliest unfinished item can always run.
__device__ __forceinline__ int fz_p1(const FusedSched& q, int b) { return b == q.nb - 1 ? q.L1 : q.F1; }
__device__ __forceinline__ int fz_p2(const FusedSched& q, int b) { return b == q.nb - 1 ? q.L2 : q.F2; }

__device__ __forceinline__ void fz_decode(const FusedSched& q, int g, int& kind, int& b, int& loc) {
  const int first = fz_p1(q, 0);
  if (g < first) {
    kind = 1; b = 0; loc = g;
    return;
  }
  g -= first;
  if (q.nb >= 2) {
    const int pair = q.F1 + q.F2;
    const int full = q.nb - 2;
    if (g < full * pair) {
      const int m = 1 + g / pair;
      const int r = g % pair;
      if (r < q.F1) { kind = 1; b = m; loc = r; }
      else { kind = 2; b = m - 1; loc = r - q.F1; }
      return;
    }
    g -= full * pair;
    if (g < q.L1) { kind = 1; b = q.nb - 1; loc = g; return; }
    g -= q.L1;
    if (g < q.F2) { kind = 2; b = q.nb - 2; loc = g; return; }
    g -= q.F2;
  }
  kind = 2; b = q.nb - 1; loc = g;
}

__device__ __forceinline__ bool fz_ready(const FusedSched& q, int kind, int b) {
  if (kind == 2) return ld_acquire_u32(q.done1 + b) >= (unsigned)fz_p1(q, b);
  if (b >= q.n_slots) return ld_acquire_u32(q.done2 + b - q.n_slots) >= (unsigned)fz_p2(q, b - q.n_slots);
  return true;
}

// bounded wait for a dependency (thread 0)
__device__ bool fz_wait_ready(const FusedSched& q, int kind, int b, int* status) {
  if (fz_ready(q, kind, b)) return true;
  const long long t0 = clock64();
  while (!fz_ready(q, kind, b)) {
    __nanosleep(200);
    if (clock64() - t0 > (1LL << 31)) {
      atomicExch(status, kStatusTimeout);
      return false;
    }
  }
  return true;
}

template <int M, int BT>
struct FusedGeo {
  using PC = ColGeo<M, BT>;
  using PR = RowGeo<M>;
  static constexpr int SLOT = PC::SLOT > PR::SLOT ? PC::SLOT : PR::SLOT;
  static constexpr int TW_BYTES = PC::TW_BYTES;
  static constexpr int TW_OFF = 2 * SLOT;
  static constexpr int BAR_OFF = TW_OFF + round128(TW_BYTES);
  static constexpr int SMEM = BAR_OFF + 32;
};

template <int M, int BT>
__global__ void __launch_bounds__(kT2, 3)
    k_fused(const __grid_constant__ CUtensorMap tm_h, const __grid_constant__ CUtensorMap tm_q, FilterArgs a,
            FusedSched q) {
  using G = SubFft<M>;
  using PC = ColGeo<M, BT>;
  using PR = RowGeo<M>;
  using F = FusedGeo<M, BT>;
  constexpr int RA = G::RA, RB = G::RB, T = G::T, NB = G::NB;
  constexpr int C = PC::C, RW = PR::RW;
  constexpr int NCB = M / C, NRB = M / RW;
  constexpr uint32_t N = (uint32_t)M * (uint32_t)M;
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ int ok;
  __shared__ int s_g[2], s_kind[2], s_b[2], s_loc[2], s_def[2];
  const float2* tw = reinterpret_cast<const float2*>(sm + F::TW_OFF);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + F::BAR_OFF);
  const int tid = threadIdx.x;
  const int total = q.total;
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_keep = policy_evict_last();
  const int64_t batch_series = (int64_t)q.B * q.n_det;

  auto scratch_of = [&](int b) { return a.scratch + (int64_t)(b % q.n_slots) * batch_series * N; };
  auto issue = [&](int kind, int b, int loc, int slot) {
    unsigned char* dst = sm + slot * F::SLOT;
    if (kind == 1) {
      const int s = loc / NCB, cb = loc % NCB;
      const int d = s % q.n_det;
      const int tmpl = a.sel[(int64_t)b * q.B + s / q.n_det];
      mbar_expect_tx(bar + slot, (uint32_t)(PC::H_BYTES + PC::Q_BYTES));
#pragma unroll
      for (int bx = 0; bx < PC::NBOX; ++bx) {
        tma_load_3d_hint(dst + bx * PC::BOXR * C * PC::HB, &tm_h, cb * C, bx * PC::BOXR, tmpl, bar + slot,
                         pol_stream);
        tma_load_3d(dst + PC::H_BYTES + bx * PC::BOXR * C * 8, &tm_q, cb * C, bx * PC::BOXR, d, bar + slot);
      }
    } else {
      const int s = loc / NRB, j10 = (loc % NRB) * RW;
      fence_proxy_async_global();
      mbar_expect_tx(bar + slot, (uint32_t)(PR::ITEM * 8));
      bulk_g2s_hint(dst, scratch_of(b) + (int64_t)s * N + (int64_t)j10 * M, (uint32_t)(PR::ITEM * 8), bar + slot,
                    pol_stream);
    }
  };
  // thread 0: dequeue the next item into descriptor slot `ds`, issuing its copy into
  // buffer `slot` when its dependency already holds (else mark it deferred)
  auto dequeue = [&](int ds, int slot) {
    const int g = (int)atomicAdd(q.head, 1u);
    s_g[ds] = g;
    if (g >= total) return;
    int kind, b, loc;
    fz_decode(q, g, kind, b, loc);
    s_kind[ds] = kind; s_b[ds] = b; s_loc[ds] = loc;
    if (fz_ready(q, kind, b)) {
      issue(kind, b, loc, slot);
      s_def[ds] = 0;
    } else {
      s_def[ds] = 1;
    }
  };

  if (tid == 0) {
    mbar_init(bar + 0, 1);
    mbar_init(bar + 1, 1);
    mbar_init(bar + 2, 1);
    fence_mbar_init();
    mbar_expect_tx(bar + 2, (uint32_t)F::TW_BYTES);
    bulk_g2s(sm + F::TW_OFF, a.tw1, (uint32_t)F::TW_BYTES, bar + 2);
    dequeue(0, 0);
  }
  if (!cta_wait(bar + 2, 0, a.status, &ok)) return;
  int prev_p1 = -1;  // batch of the P1 item this CTA just finished (thread 0 signals it)
  for (int k = 0;; ++k) {
    const int slot = k & 1;
    __syncthreads();  // the previous item is complete in every thread
    if (tid == 0) {
      if (prev_p1 >= 0) {
        fence_proxy_async_global();
        __threadfence();
        atomicAdd(q.done1 + prev_p1, 1u);
        prev_p1 = -1;
      }
      ok = 1;
      if (s_g[slot] < total) {
        if (s_def[slot]) {
          if (!fz_wait_ready(q, s_kind[slot], s_b[slot], a.status)) ok = 0;
          else issue(s_kind[slot], s_b[slot], s_loc[slot], slot);
        }
        if (ok) dequeue(slot ^ 1, slot ^ 1);
      }
    }
    __syncthreads();
    if (!ok) return;
    if (s_g[slot] >= total) break;
    const int kind = s_kind[slot], b = s_b[slot], loc = s_loc[slot];
    if (!cta_wait(bar + slot, (uint32_t)((k >> 1) & 1), a.status, &ok)) return;
    unsigned char* buf = sm + slot * F::SLOT;
    if (kind == 1) {
      const int s = loc / NCB;
      const int c = tid % C, t = tid / C;
      const int k2 = (loc % NCB) * C + c;
      const float2* sq = reinterpret_cast<const float2*>(buf + PC::H_BYTES);
      float2 v[RA];
#pragma unroll
      for (int r = 0; r < RA; ++r) {
        if (r >= RA / 2) {
          v[r] = make_float2(0.f, 0.f);
        } else {
          const int idx = (t + r * RB) * C + c;
          v[r] = cmulc(sq[idx], smem_h<BT>(buf, idx));
        }
      }
      __syncthreads();
      dft<RA, true>(v);
      float2* xb = reinterpret_cast<float2*>(buf);
      using XC = typename PC::X;
#pragma unroll
      for (int qq = 0; qq < RA; ++qq) xb[XC::idx(c, t * RA + qq)] = v[qq];
      __syncthreads();
      float2* out = scratch_of(b) + (int64_t)s * N;
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        const int j = t + T * i;
        float2 u[RB];
        u[0] = xb[XC::idx(c, j)];
#pragma unroll
        for (int r = 1; r < RB; ++r) u[r] = cmul(xb[XC::idx(c, j + r * RA)], tw[r * RA + j]);
        dft<RB>(u);
        float2 w = unit_root(((uint32_t)j * (uint32_t)k2) & (N - 1), N);
        const float2 st = unit_root(((uint32_t)RA * (uint32_t)k2) & (N - 1), N);
#pragma unroll
        for (int qq = 0; qq < RB; ++qq) {
          st_global_hint(out + (int64_t)(j + qq * RA) * M + k2, cmul(u[qq], w), pol_keep);
          if (qq + 1 < RB) w = cmul(w, st);
        }
      }
      prev_p1 = b;
    } else {
      if (tid == 0) atomicAdd(q.done2 + b, 1u);  // its scratch rows are in shared memory now
      const int s = loc / NRB;
      const int t = tid % T, row = tid / T;
      const int j1 = (loc % NRB) * RW + row;
      const float2* stage = reinterpret_cast<const float2*>(buf);
      float2 v[RA];
#pragma unroll
      for (int r = 0; r < RA; ++r) v[r] = stage[row * M + t + r * RB];
      __syncthreads();
      dft<RA>(v);
      float2* xb = reinterpret_cast<float2*>(buf);
      using XR = typename PR::X;
#pragma unroll
      for (int qq = 0; qq < RA; ++qq) xb[XR::idx(row, t * RA + qq)] = v[qq];
      __syncthreads();
      FilterEpi ep{a.sel, a.inv_sigma, (int64_t)b * q.B, q.n_det, a.thr2, a.window, a.valid_begin, a.valid_end,
                   a.n_win, a.n_sel_total, a.slots};
      const auto se = ep.series(s);
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        const int j = t + T * i;
        float2 u[RB];
        u[0] = xb[XR::idx(row, j)];
#pragma unroll
        for (int r = 1; r < RB; ++r) u[r] = cmul(xb[XR::idx(row, j + r * RA)], tw[r * RA + j]);
        dft<RB>(u);
#pragma unroll
        for (int qq = 0; qq < RB; ++qq) ep(se, (int64_t)j1 + (int64_t)M * (j + qq * RA), u[qq]);
      }
    }
  }
  // signal the last P1 item (all threads passed the loop-top barrier after it)
  if (tid == 0 && prev_p1 >= 0) {
    fence_proxy_async_global();
    __threadfence();
    atomicAdd(q.done1 + prev_p1, 1u);
  }
}

// ---------------------------------------------------------------------------
// register-pipelined variant: inputs go global -> registers directly; the
// next item's loads are issued as soon as the first sub-FFT's registers are
// free (after the exchange store), so they land while the second sub-FFT and
// the epilogue of the current item run.  Shared memory holds only the
// exchange buffer and the twiddle table.
// ---------------------------------------------------------------------------

__device__ __forceinline__ float2 ld_stream(const float2* p) { return __ldcs(p); }

template <int BT>
__device__ __forceinline__ float2 ld_bank(const void* base, int64_t i) {
  if constexpr (BT == kBankF32) {
    return __ldcs(reinterpret_cast<const float2*>(base) + i);
  } else if constexpr (BT == kBankF16) {
    const unsigned u = __ldcs(reinterpret_cast<const unsigned*>(base) + i);
    return __half22float2(*reinterpret_cast<const __half2*>(&u));
  } else {
    const unsigned u = __ldcs(reinterpret_cast<const unsigned*>(base) + i);
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u));
  }
}

template <int N1, int N2, int BT>
__global__ void __launch_bounds__(kT2, 3) k_cols4(FilterArgs a) {
  using G = SubFft<N1>;
  constexpr int RA = G::RA, RB = G::RB, T = G::T, NB = G::NB;
  constexpr int C = kT2 / T;
  constexpr int K = C >= 16 ? 1 : 16 / C;
  using X = Xch<N1, K>;
  constexpr int NCB = N2 / C;
  constexpr uint32_t N = (uint32_t)N1 * (uint32_t)N2;
  constexpr int H = RA / 2;  // non-zero inputs per thread (k1 < N1/2)
  extern __shared__ __align__(128) unsigned char sm[];
  float2* xb = reinterpret_cast<float2*>(sm);
  float2* tw = reinterpret_cast<float2*>(sm + C * X::S * 8);
  const int tid = threadIdx.x;
  const int c = tid % C, t = tid / C;
  for (int i = tid; i < RB * RA; i += kT2) tw[i] = a.tw1[i];
  const uint64_t pol_keep = policy_evict_last();
  const int n_items = a.count * a.n_det * NCB;
  float2 hv[H], qv[H];
  auto load = [&](int it) {
    const int s = it / NCB;
    const int k2 = (it % NCB) * C + c;
    const int64_t tmpl = a.sel[a.pos0 + s / a.n_det];
    const void* hrow = static_cast<const unsigned char*>(a.bank) + tmpl * a.ld_bank * (BT == kBankF32 ? 8 : 4);
    const float2* qrow = a.q + (int64_t)(s % a.n_det) * a.ld_q;
#pragma unroll
    for (int r = 0; r < H; ++r) {
      const int64_t k = (int64_t)(t + r * RB) * N2 + k2;
      hv[r] = ld_bank<BT>(hrow, k);
      qv[r] = __ldg(qrow + k);
    }
  };
  int item = blockIdx.x;
  if (item < n_items) load(item);
  for (; item < n_items; item += gridDim.x) {
    const int s = item / NCB;
    const int k2 = (item % NCB) * C + c;
    float2 v[RA];
#pragma unroll
    for (int r = 0; r < RA; ++r) v[r] = r < H ? cmulc(qv[r], hv[r]) : make_float2(0.f, 0.f);
    dft<RA, true>(v);
    __syncthreads();  // previous item's exchange reads (and the twiddle fill) are done
#pragma unroll
    for (int q = 0; q < RA; ++q) xb[X::idx(c, t * RA + q)] = v[q];
    __syncthreads();
    if (item + (int)gridDim.x < n_items) load(item + gridDim.x);
    float2* out = a.scratch + (int64_t)s * N;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int j = t + T * i;
      float2 u[RB];
      u[0] = xb[X::idx(c, j)];
#pragma unroll
      for (int r = 1; r < RB; ++r) u[r] = cmul(xb[X::idx(c, j + r * RA)], tw[r * RA + j]);
      dft<RB>(u);
      float2 w = unit_root(((uint32_t)j * (uint32_t)k2) & (N - 1), N);
      const float2 st = unit_root(((uint32_t)RA * (uint32_t)k2) & (N - 1), N);
#pragma unroll
      for (int q = 0; q < RB; ++q) {
        st_global_hint(out + (int64_t)(j + q * RA) * N2 + k2, cmul(u[q], w), pol_keep);
        if (q + 1 < RB) w = cmul(w, st);
      }
    }
  }
}

template <int N1, int N2>
__global__ void __launch_bounds__(kT2, 3) k_rows4(FilterArgs a) {
  using G = SubFft<N2>;
  constexpr int RA = G::RA, RB = G::RB, T = G::T, NB = G::NB;
  constexpr int RW = kT2 / T;
  using X = Xch<N2, (T >= 16 ? 16 : T)>;
  constexpr int NRB = N1 / RW;
  constexpr int64_t N = (int64_t)N1 * N2;
  extern __shared__ __align__(128) unsigned char sm[];
  float2* xb = reinterpret_cast<float2*>(sm);
  float2* tw = reinterpret_cast<float2*>(sm + RW * X::S * 8);
  const int tid = threadIdx.x;
  const int t = tid % T, row = tid / T;
  for (int i = tid; i < RB * RA; i += kT2) tw[i] = a.tw2[i];
  FilterEpi ep{a.sel, a.inv_sigma, a.pos0, a.n_det, a.thr2, a.window, a.valid_begin, a.valid_end,
               a.n_win, a.n_sel_total, a.slots};
  const int n_items = a.count * a.n_det * NRB;
  float2 v[RA];
  auto load = [&](int it) {
    const int s = it / NRB;
    const int j1 = (it % NRB) * RW + row;
    const float2* in = a.scratch + (int64_t)s * N + (int64_t)j1 * N2;
#pragma unroll
    for (int r = 0; r < RA; ++r) v[r] = ld_stream(in + t + r * RB);
  };
  int item = blockIdx.x;
  if (item < n_items) load(item);
  for (; item < n_items; item += gridDim.x) {
    const int s = item / NRB;
    const int j1 = (item % NRB) * RW + row;
    dft<RA>(v);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < RA; ++q) xb[X::idx(row, t * RA + q)] = v[q];
    __syncthreads();
    if (item + (int)gridDim.x < n_items) load(item + gridDim.x);
    const auto se = ep.series(s);
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
cudaError_t launch_pdl(K kern, int grid, int smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kT2);
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

template <int N1, int N2, int BT, int QT>
cudaError_t run_cols(const FilterArgs& a, const Filter2Maps& m, cudaStream_t st) {
  using P = ColGeo<N1, BT, QT>;
  auto k = k_cols<N1, N2, BT, QT>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = set_smem2(k, P::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int items = a.count * a.n_det * (N2 / P::C);
  cudaError_t e = launch_pdl(k, grid2(items), P::SMEM, st, m.h, m.q, a);
  add_launches(1);
  return e;
}

// (bank, data) storage pairs: FP32 data with any bank; 16-bit data with a bank of the same type
template <int N1, int N2>
cudaError_t run_cols_bt(const FilterArgs& a, const Filter2Maps& m, cudaStream_t st) {
  if (a.q_type == kBankF32) {
    switch (a.bank_type) {
      case kBankF32: return run_cols<N1, N2, kBankF32, kBankF32>(a, m, st);
      case kBankF16: return run_cols<N1, N2, kBankF16, kBankF32>(a, m, st);
      case kBankBF16: return run_cols<N1, N2, kBankBF16, kBankF32>(a, m, st);
    }
  } else if (a.q_type == a.bank_type) {
    switch (a.bank_type) {
      case kBankF16: return run_cols<N1, N2, kBankF16, kBankF16>(a, m, st);
      case kBankBF16: return run_cols<N1, N2, kBankBF16, kBankBF16>(a, m, st);
    }
  }
  return cudaErrorInvalidValue;
}

template <int N1, int N2>
cudaError_t run_rows(const FilterArgs& a, cudaStream_t st) {
  using P = RowGeo<N2>;
  auto k = k_rows<N1, N2>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = set_smem2(k, P::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int items = a.count * a.n_det * (N1 / P::RW);
  cudaError_t e = launch_pdl(k, grid2(items), P::SMEM, st, a);
  add_launches(1);
  return e;
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
int cols_of() {
  return ColGeo<N1, kBankF32>::C;
}
template <int N1, int N2>
int boxr_of() {
  return ColGeo<N1, kBankF32>::BOXR;
}
int dispatch_cols(int64_t n) {
  switch (n) {
    case 1 << 12: return cols_of<64, 64>();
    case 1 << 13: return cols_of<128, 64>();
    case 1 << 14: return cols_of<128, 128>();
    case 1 << 15: return cols_of<256, 128>();
    case 1 << 16: return cols_of<256, 256>();
    case 1 << 17: return cols_of<512, 256>();
    case 1 << 18: return cols_of<512, 512>();
    case 1 << 19: return cols_of<1024, 512>();
    case 1 << 20: return cols_of<1024, 1024>();
  }
  return 0;
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
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 3-D view [dim2][N1/2 rows][N2 cols] of rows of one-sided spectra k = k1 N2 + k2 < N/2
bool encode_view(CUtensorMap* m, const void* base, CUtensorMapDataType dt, int eb, int64_t n2, int64_t rows,
                 int64_t depth, int64_t ld_elems, int box_c, int box_r) {
  auto fn = encode_fn();
  if (!fn || !base || depth <= 0) return false;
  cuuint64_t dims[3] = {(cuuint64_t)n2, (cuuint64_t)rows, (cuuint64_t)depth};
  cuuint64_t strides[2] = {(cuuint64_t)(n2 * eb), (cuuint64_t)(ld_elems * eb)};
  cuuint32_t box[3] = {(cuuint32_t)box_c, (cuuint32_t)box_r, 1u};
  cuuint32_t es[3] = {1u, 1u, 1u};
  CUresult r = fn(m, dt, 3, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

namespace {
template <int N1, int N2, int BT>
cudaError_t run_cols4(const FilterArgs& a, cudaStream_t st) {
  using G = SubFft<N1>;
  constexpr int C = kT2 / G::T;
  constexpr int K = C >= 16 ? 1 : 16 / C;
  constexpr int SMEM = C * Xch<N1, K>::S * 8 + G::RB * G::RA * 8;
  auto k = k_cols4<N1, N2, BT>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = set_smem2(k, SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int items = a.count * a.n_det * (N2 / C);
  k<<<grid2(items), kT2, SMEM, st>>>(a);
  add_launches(1);
  return cudaGetLastError();
}
template <int N1, int N2>
cudaError_t run_cols4_bt(const FilterArgs& a, cudaStream_t st) {
  switch (a.bank_type) {
    case kBankF32: return run_cols4<N1, N2, kBankF32>(a, st);
    case kBankF16: return run_cols4<N1, N2, kBankF16>(a, st);
    case kBankBF16: return run_cols4<N1, N2, kBankBF16>(a, st);
  }
  return cudaErrorInvalidValue;
}
template <int N1, int N2>
cudaError_t run_rows4(const FilterArgs& a, cudaStream_t st) {
  using G = SubFft<N2>;
  constexpr int RW = kT2 / G::T;
  constexpr int SMEM = RW * Xch<N2, (G::T >= 16 ? 16 : G::T)>::S * 8 + G::RB * G::RA * 8;
  auto k = k_rows4<N1, N2>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = set_smem2(k, SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int items = a.count * a.n_det * (N1 / RW);
  k<<<grid2(items), kT2, SMEM, st>>>(a);
  add_launches(1);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_filter4_pass1(const FilterArgs& a, cudaStream_t st) { MF_DISPATCH2(a.n, run_cols4_bt, (a, st)) }
cudaError_t launch_filter4_pass2(const FilterArgs& a, cudaStream_t st) { MF_DISPATCH2(a.n, run_rows4, (a, st)) }

cudaError_t filter2_encode_maps(const FilterArgs& a, int64_t n_tmpl, Filter2Maps* m) {
  m->ok = false;
  const int n1 = a.n1, n2 = a.n2;
  const int C = dispatch_cols(a.n);
  if (C == 0) return cudaErrorInvalidValue;
  const int rows = n1 / 2;
  const int boxr = rows < 256 ? rows : 256;
  const bool f32 = a.bank_type == kBankF32;
  if (!encode_view(&m->h, a.bank, f32 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32, f32 ? 8 : 4,
                   n2, rows, n_tmpl, a.ld_bank, C, boxr))
    return cudaErrorInvalidValue;
  const bool q32 = a.q_type == kBankF32;
  if (!encode_view(&m->q, q32 ? (const void*)a.q : a.q_lp, q32 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32,
                   q32 ? 8 : 4, n2, rows, a.n_det, a.ld_q, C, boxr))
    return cudaErrorInvalidValue;
  m->ok = true;
  return cudaSuccess;
}

cudaError_t launch_filter2_pass1(const FilterArgs& a, const Filter2Maps& m, cudaStream_t st) {
  if (!m.ok) return cudaErrorInvalidValue;
  MF_DISPATCH2(a.n, run_cols_bt, (a, m, st))
}

cudaError_t launch_filter2_pass2(const FilterArgs& a, cudaStream_t st) { MF_DISPATCH2(a.n, run_rows, (a, st)) }

namespace {
template <int M, int BT>
cudaError_t run_fused(const FilterArgs& a, const Filter2Maps& m, const FusedSched& q, cudaStream_t st) {
  using F = FusedGeo<M, BT>;
  auto k = k_fused<M, BT>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = set_smem2(k, F::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int g = sm_count() * 3;
  if (q.total < g) g = q.total;
  if (g < 1) return cudaSuccess;
  k<<<g, kT2, F::SMEM, st>>>(m.h, m.q, a, q);
  add_launches(1);
  return cudaGetLastError();
}
template <int M>
cudaError_t run_fused_bt(const FilterArgs& a, const Filter2Maps& m, const FusedSched& q, cudaStream_t st) {
  switch (a.bank_type) {
    case kBankF32: return run_fused<M, kBankF32>(a, m, q, st);
    case kBankF16: return run_fused<M, kBankF16>(a, m, q, st);
    case kBankBF16: return run_fused<M, kBankBF16>(a, m, q, st);
  }
  return cudaErrorInvalidValue;
}
template <int M>
int items_per_series_p1() { return M / ColGeo<M, kBankF32>::C; }
template <int M>
int items_per_series_p2() { return M / RowGeo<M>::RW; }
}  // namespace

bool fused_supported(int64_t n) {
  return n == (1 << 12) || n == (1 << 14) || n == (1 << 16) || n == (1 << 18) || n == (1 << 20);
}

void fused_items(int64_t n, int* p1, int* p2) {
  switch (n) {
    case 1 << 12: *p1 = items_per_series_p1<64>(); *p2 = items_per_series_p2<64>(); return;
    case 1 << 14: *p1 = items_per_series_p1<128>(); *p2 = items_per_series_p2<128>(); return;
    case 1 << 16: *p1 = items_per_series_p1<256>(); *p2 = items_per_series_p2<256>(); return;
    case 1 << 18: *p1 = items_per_series_p1<512>(); *p2 = items_per_series_p2<512>(); return;
    case 1 << 20: *p1 = items_per_series_p1<1024>(); *p2 = items_per_series_p2<1024>(); return;
  }
  *p1 = *p2 = 0;
}

cudaError_t launch_filter_fused(const FilterArgs& a, const Filter2Maps& m, const FusedSched& q, cudaStream_t st) {
  if (!m.ok) return cudaErrorInvalidValue;
  switch (a.n) {
    case 1 << 12: return run_fused_bt<64>(a, m, q, st);
    case 1 << 14: return run_fused_bt<128>(a, m, q, st);
    case 1 << 16: return run_fused_bt<256>(a, m, q, st);
    case 1 << 18: return run_fused_bt<512>(a, m, q, st);
    case 1 << 20: return run_fused_bt<1024>(a, m, q, st);
  }
  return cudaErrorInvalidValue;
}

namespace {
template <int N1, int N2>
cudaError_t run_fill_tw(float2* tw1, float2* tw2, cudaStream_t st) {
  k_fill_twiddles<N1><<<4, 256, 0, st>>>(tw1);
  k_fill_twiddles<N2><<<4, 256, 0, st>>>(tw2);
  add_launches(2);
  return cudaGetLastError();
}
}  // namespace

namespace {
__global__ void k_fill_tw4(float2* tw4, int64_t count, uint32_t n) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < count; m += (int64_t)gridDim.x * blockDim.x)
    tw4[m] = unit_root((uint32_t)m, n);
}
}  // namespace

cudaError_t launch_fill_tw4(int64_t n, float2* tw4, int64_t count, cudaStream_t st) {
  k_fill_tw4<<<64, 256, 0, st>>>(tw4, count, (uint32_t)n);
  add_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_fill_twiddles(int64_t n, float2* tw1, float2* tw2, cudaStream_t st) {
  MF_DISPATCH2(n, run_fill_tw, (tw1, tw2, st))
}

}  // namespace mf
