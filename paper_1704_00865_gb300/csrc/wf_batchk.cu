// wf_batchk.cu -- the sweeps of a batch of maps of uneven sizes in one
// persistent cooperative launch (Huffenberger 2017, Sec. 2: every map runs
// the same messenger sweep; the maps are independent).
//
// Per sweep there are two phases, the row passes of every map and then the
// column passes of every map, separated by a grid barrier.  A phase is a
// device work queue: its items are (map, row group) or (map, column group)
// pairs listed on the host, largest maps first, and each CTA takes the next
// item with one atomic add until the list is exhausted, so CTAs that finish
// small items early go on to the next instead of idling while a large map
// finishes.  Items of a map whose solve is done (the per-map done flag its
// controller sets between launches) return at once.  The launch covers R
// sweeps; the residual checkpoints and lambda controllers of the maps run
// between launches.
//
// The items use 256 threads whatever the map size: a row item transforms
// 256 / (M / E) rows of M complex values with E values per thread, a column
// item 256 / (L / E) columns of length L.  Fields are read with loads that
// bypass L1 (another CTA may have written them earlier in the launch) and
// the transforms use shared memory only for their exchanges, so several
// CTAs share an SM.  Per size there are one or two compiled shapes (values
// per thread of the row and column transforms); the batch's tuner picks
// between them (wf_batch.cu).
#include <cuda_runtime.h>

#include <mutex>

#include "wf_cols_common.cuh"
#include "wf_device.cuh"
#include "wf_internal.h"
#include "wf_rows_common.cuh"

namespace wf {

constexpr int BT = 256;  // threads per CTA

// values per thread (row transform, column transform) of shape V of size N
template <int N, int V>
struct BShape {
  static constexpr int RE = (N % 3 == 0) ? 12 : (V == 0 ? 8 : (N <= 512 ? 4 : 16));
  static constexpr int CE = (N % 3 == 0) ? ((V == 1 && N == 1536) ? 24 : 12)
                                         : (V == 0 ? (N >= 1024 ? 16 : 8) : (N >= 1024 ? 8 : 16));
  static constexpr int M = N / 2, L = N;
  static constexpr int TPF = M / RE, ROWS = BT / TPF;
  static constexpr int TPC = L / CE, W = BT / TPC;
  static_assert(ROWS * TPF == BT && W * TPC == BT, "items use every thread");
  static constexpr int SP = SPad<L>::size;
  static constexpr int WANT = (W >= 32) ? 1 : (16 / W) % 16;
  static constexpr int STRIDE = SP + ((WANT - SP % 16) + 16) % 16;
  // Items whose inputs fit in shared memory beside their transform buffers
  // (two CTAs per SM) stage them first, all copies in flight at once: rows
  // of 8 values per thread (d_RF and the pixel table by bulk copies, t_RF
  // and d_2DF by 16-byte copies), columns up to 16 values per thread (the
  // messenger and (C, P1f) tiles).  The others load at the point of use.
  static constexpr bool ROW_STAGED = (RE == 8);
  static constexpr bool COL_STAGED = (CE <= 16) && (W >= 2);
  static constexpr bool COL_TILED = (W % WF_TW == 0);
  static constexpr size_t rows_in = (size_t)ROWS * M;  // complex values per row field
  static constexpr size_t row_fft = (size_t)ROWS * SPad<M>::size * 8;
  static constexpr size_t row_smem = row_fft + (ROW_STAGED ? rows_in * (8 + 16 + 8 + 8) : 0);
  static constexpr size_t col_tile = (size_t)W * L * 8;
  static constexpr size_t col_fft = (size_t)W * STRIDE * 8;
  static constexpr size_t col_smem = col_fft + (COL_STAGED ? 2 * col_tile : 0);
  static constexpr size_t smem = row_smem > col_smem ? row_smem : col_smem;
  // position of (ky, column c of the item) in a staged tile
  static __device__ __forceinline__ int sidx(int ky, int c) {
    if constexpr (COL_TILED) return (c / WF_TW) * L * WF_TW + ky * WF_TW + (c % WF_TW);
    else return ky * W + c;
  }
};

// Per-CTA staging state: the bulk-copy mbarrier and its next phase.
struct BatchStage {
  uint64_t* bar;
  uint32_t phase;
  bool ok;
};

// sizes in class order; class = 2 * (index of the size) + shape
constexpr int kBatchSizes[7] = {256, 384, 512, 768, 1024, 1536, 2048};
// sizes with a second shape
__host__ __device__ constexpr bool has_v1(int n) { return n == 256 || n == 512 || n == 1024 || n == 1536 || n == 2048; }

// The row pass of ROWS rows of one map (eq. 2mess_t1 analogue in pixels
// between the inverse and forward row DFTs, then the stripe-basis updates).
template <int N, int V>
__device__ __forceinline__ void batch_row_item(const BatchMapArgs& m, int grp, float2* sm) {
  using S = BShape<N, V>;
  constexpr int M = S::M, E = S::RE, TPF = S::TPF, ROWS = S::ROWS;
  const int g = threadIdx.x / TPF, t = threadIdx.x - g * TPF;
  const int y = grp * ROWS + g;
  const size_t row0 = (size_t)y * M;
  float2* sb = sm + g * SPad<M>::size;
  const float T2 = m.st->Tf[2], T1 = m.st->Tf[1], off1 = (float)m.st->off[1];
  float2 v[E];
#pragma unroll
  for (int k = 0; k < E; ++k) v[k] = __ldcg(&m.f_d1[row0 + t + k * TPF]);
  c2r_pre<M, E>(v, sb, t, m.twx);
  fft_block<M, E, true>(v, sb, t, m.twh, 1);
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const float4 q = __ldg(&m.dn[row0 + t + k * TPF]);
    v[k] = make_float2(tpx_update(q.x, q.y, v[k].x, T2), tpx_update(q.z, q.w, v[k].y, T2));
  }
  fft_block<M, E, false>(v, sb, t, m.twh, 1);
  r2c_post<M, E>(v, sb, t, m.twx);
  const float a2y = (m.a2 != nullptr) ? __ldg(&m.a2[y]) : 1.f;
  const float pkn = __ldg(&m.pst[M]);
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const int kk = t + k * TPF;
    const size_t ti = tidx(y, kk, N);
    float2 d1, t1;
    stripe_update(kk, v[k], __ldcg(&m.f_t1[ti]), __ldcg(&m.f_x[ti]), a2y, __ldg(&m.pst[kk]), pkn, off1, T2, T1, d1,
                  t1);
    m.f_d1[row0 + kk] = d1;
    m.f_t1[ti] = t1;
  }
}

// The row item with its inputs staged (ROW_STAGED shapes): the same
// arithmetic as batch_row_item, reading from shared memory.
template <int N, int V>
__device__ __forceinline__ void batch_row_item_staged(const BatchMapArgs& m, int grp, float2* sm, BatchStage& bs) {
  using S = BShape<N, V>;
  constexpr int M = S::M, E = S::RE, TPF = S::TPF, ROWS = S::ROWS;
  float2* s_fft = sm;
  float2* s_d1 = sm + S::row_fft / 8;
  float4* s_dn = reinterpret_cast<float4*>(s_d1 + S::rows_in);
  float2* s_t1 = reinterpret_cast<float2*>(s_dn + S::rows_in);
  float2* s_x = s_t1 + S::rows_in;
  const int g = threadIdx.x / TPF, t = threadIdx.x - g * TPF;
  const int y0 = grp * ROWS, y = y0 + g;
  const size_t row0 = (size_t)y * M;
  float2* sb = s_fft + g * SPad<M>::size;
  if (threadIdx.x == 0) {
    // d_RF was written by other CTAs' generic stores earlier in the launch
    asm volatile("fence.proxy.async.global;" ::: "memory");
    mbar_expect_tx(bs.bar, (uint32_t)(S::rows_in * (8 + 16)));
    bulk_g2s(s_d1, m.f_d1 + (size_t)y0 * M, (uint32_t)(S::rows_in * 8), bs.bar);
    bulk_g2s(s_dn, m.dn + (size_t)y0 * M, (uint32_t)(S::rows_in * 16), bs.bar);
  }
  for (int i = threadIdx.x; i < ROWS * (M / 2); i += BT) {
    const int r = i / (M / 2);
    const int k = (i - r * (M / 2)) * 2;
    cp_async16(s_t1 + r * M + k, m.f_t1 + tidx(y0 + r, k, N));
    cp_async16(s_x + r * M + k, m.f_x + tidx(y0 + r, k, N));
  }
  cp_async_commit();
  const float T2 = m.st->Tf[2], T1 = m.st->Tf[1], off1 = (float)m.st->off[1];
  const float a2y = (m.a2 != nullptr) ? __ldg(&m.a2[y]) : 1.f;
  const float pkn = __ldg(&m.pst[M]);
  if (!mbar_wait(bs.bar, bs.phase, WF_WAIT_TRIES)) bs.ok = false;
  bs.phase ^= 1u;
  float2 v[E];
#pragma unroll
  for (int k = 0; k < E; ++k) v[k] = s_d1[g * M + t + k * TPF];
  c2r_pre<M, E>(v, sb, t, m.twx);
  fft_block<M, E, true>(v, sb, t, m.twh, 1);
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const float4 q = s_dn[g * M + t + k * TPF];
    v[k] = make_float2(tpx_update(q.x, q.y, v[k].x, T2), tpx_update(q.z, q.w, v[k].y, T2));
  }
  fft_block<M, E, false>(v, sb, t, m.twh, 1);
  r2c_post<M, E>(v, sb, t, m.twx);
  cp_async_wait<0>();
  __syncthreads();
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const int kk = t + k * TPF;
    float2 d1, t1;
    stripe_update(kk, v[k], s_t1[g * M + kk], s_x[g * M + kk], a2y, __ldg(&m.pst[kk]), pkn, off1, T2, T1, d1, t1);
    m.f_d1[row0 + kk] = d1;
    m.f_t1[tidx(y, kk, N)] = t1;
  }
}

// The column pass of W columns of one map (the merged 2DF block between the
// forward and inverse column DFTs; with the defect-correction source when
// the map has one).
template <int N, int V>
__device__ __forceinline__ void batch_col_item(const BatchMapArgs& m, int grp, float2* sm, BatchStage& bs) {
  using S = BShape<N, V>;
  constexpr int L = S::L, E = S::CE, TPC = S::TPC, W = S::W;
  const int c = threadIdx.x % W, tc = threadIdx.x / W;
  const int col0 = grp * W, col = col0 + c;
  float2* sb = sm + c * S::STRIDE;
  float2* s_y = sm + S::col_fft / 8;
  float2* s_eig = s_y + S::col_tile / 8;
  const float Tl = m.st->Tf[1], off0 = (float)m.st->off[0];
  float2 u[E];
  if constexpr (S::COL_STAGED) {
    // the messenger tile (written by other CTAs earlier in the launch) and
    // the (C, P1f) tile
    if constexpr (S::COL_TILED) {
      if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.global;" ::: "memory");
        mbar_expect_tx(bs.bar, (uint32_t)(2 * S::col_tile));
        bulk_g2s(s_y, m.f_t1 + tidx(0, col0, N), (uint32_t)S::col_tile, bs.bar);
        bulk_g2s(s_eig, m.eig + tidx(0, col0, N), (uint32_t)S::col_tile, bs.bar);
      }
      if (!mbar_wait(bs.bar, bs.phase, WF_WAIT_TRIES)) bs.ok = false;
      bs.phase ^= 1u;
    } else {
      static_assert(S::COL_TILED || W == 2, "half-tile items are two columns wide");
      for (int ky = threadIdx.x; ky < L; ky += BT) {
        cp_async16(s_y + ky * 2, m.f_t1 + tidx(ky, col0, N));
        cp_async16(s_eig + ky * 2, m.eig + tidx(ky, col0, N));
      }
      cp_async_commit();
      cp_async_wait<0>();
      __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < E; ++k) u[k] = s_y[S::sidx(tc + k * TPC, c)];
  } else {
#pragma unroll
    for (int k = 0; k < E; ++k) u[k] = __ldcg(&m.f_t1[tidx(tc + k * TPC, col, N)]);
  }
  fft_block<L, E, false>(u, sb, tc, m.twy, 1);
  // partner values Z[-k] for the packed column 0, read from the exchange
  // buffer (first group only; uniform)
  const bool packed = (col == 0);
  if (col0 == 0) {
#pragma unroll
    for (int k = 0; k < E; ++k) sb[spad(tc + k * TPC)] = u[k];
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < E; ++k) {
    const int ky = tc + k * TPC;
    float2 eg;
    if constexpr (S::COL_STAGED) eg = s_eig[S::sidx(ky, c)];
    else eg = __ldg(&m.eig[tidx(ky, col, N)]);
    const float2 egb = packed ? __ldg(&m.eig_nyq[ky]) : eg;
    const float2 vp = packed ? sb[spad(neg_mod<L>(ky))] : u[k];
    if (m.src != nullptr) {
      const float2 jv = __ldg(&m.src[tidx(ky, col, N)]);
      const float2 jp = packed ? __ldg(&m.src[tidx(neg_mod<L>(ky), col, N)]) : jv;
      u[k] = merged_mode<true>(u[k], vp, eg, egb, off0, Tl, packed, jv, jp);
    } else {
      u[k] = merged_mode<false>(u[k], vp, eg, egb, off0, Tl, packed, eg, eg);
    }
  }
  if (col0 == 0) __syncthreads();  // the partner reads are done before the transform reuses sb
  fft_block<L, E, true>(u, sb, tc, m.twy, 1);
  const float sc = 1.0f / (float)L;
#pragma unroll
  for (int k = 0; k < E; ++k) m.f_x[tidx(tc + k * TPC, col, N)] = cscale(u[k], sc);
}

template <int N, int V>
__device__ __forceinline__ void batch_item(int phase, const BatchMapArgs& m, int grp, float2* sm, BatchStage& bs) {
  if (phase == 0) {
    if constexpr (BShape<N, V>::ROW_STAGED) batch_row_item_staged<N, V>(m, grp, sm, bs);
    else batch_row_item<N, V>(m, grp, sm);
  } else {
    batch_col_item<N, V>(m, grp, sm, bs);
  }
}

__device__ __forceinline__ void batch_dispatch(int phase, const BatchMapArgs& m, int grp, float2* sm, BatchStage& bs) {
  switch (m.cls) {
    case 0: batch_item<256, 0>(phase, m, grp, sm, bs); break;
    case 1: batch_item<256, 1>(phase, m, grp, sm, bs); break;
    case 2: batch_item<384, 0>(phase, m, grp, sm, bs); break;
    case 4: batch_item<512, 0>(phase, m, grp, sm, bs); break;
    case 5: batch_item<512, 1>(phase, m, grp, sm, bs); break;
    case 6: batch_item<768, 0>(phase, m, grp, sm, bs); break;
    case 8: batch_item<1024, 0>(phase, m, grp, sm, bs); break;
    case 9: batch_item<1024, 1>(phase, m, grp, sm, bs); break;
    case 10: batch_item<1536, 0>(phase, m, grp, sm, bs); break;
    case 11: batch_item<1536, 1>(phase, m, grp, sm, bs); break;
    case 12: batch_item<2048, 0>(phase, m, grp, sm, bs); break;
    case 13: batch_item<2048, 1>(phase, m, grp, sm, bs); break;
    default: break;
  }
}

// largest shared-memory need of any item
template <int N>
constexpr size_t bsm2() {
  return BShape<N, 0>::smem > BShape<N, 1>::smem ? BShape<N, 0>::smem : BShape<N, 1>::smem;
}
constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kBatchSmem =
    cmax(cmax(cmax(bsm2<256>(), BShape<384, 0>::smem), cmax(bsm2<512>(), BShape<768, 0>::smem)),
         cmax(cmax(bsm2<1024>(), bsm2<1536>()), bsm2<2048>()));
// two CTAs per SM: 228 KB of shared memory less 1 KB reserved per CTA and
// the static words
static_assert(kBatchSmem <= 112 * 1024, "two batch CTAs fit on an SM");

__global__ void __launch_bounds__(BT, 2) batch_sweep_kernel(BatchArgs a) {
  extern __shared__ __align__(16) float2 bsm[];
  __shared__ int s_item, s_ok;
  __shared__ __align__(8) uint64_t s_bar;
  unsigned nbar = 0;
  if (threadIdx.x == 0) {
    mbar_init(&s_bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  BatchStage bs{&s_bar, 0u, true};
  for (int it = 0; it < a.nsweeps; ++it) {
    for (int phase = 0; phase < 2; ++phase) {
      const int nitems = phase ? a.n_col : a.n_row;
      const int2* items = phase ? a.col_items : a.row_items;
      unsigned* q = a.queue + 2 * it + phase;
      for (;;) {
        // the last item's shared memory and s_item are free; a staging copy
        // that did not land within its bounded wait ends the launch (the
        // other CTAs leave at their next grid barrier)
        if (__syncthreads_or(bs.ok ? 0 : 1)) {
          if (threadIdx.x == 0) {
            atomicOr(a.err, WF_ERR_TIMEOUT);
            atomicExch(&a.bar[2], 1u);
            mbar_wait(bs.bar, bs.phase ^ 1u, WF_WAIT_TRIES);  // the copy still in flight
          }
          __syncthreads();
          return;
        }
        if (threadIdx.x == 0) s_item = (int)atomicAdd(q, 1u);
        __syncthreads();
        const int k = s_item;
        if (k >= nitems) break;
        const int2 w = items[k];
        const BatchMapArgs m = a.maps[w.x];
        if (m.st->done) continue;  // uniform: written between launches only
        batch_dispatch(phase, m, w.y, bsm, bs);
      }
      // the stores of this phase, seen by the next phase's bulk copies
      asm volatile("fence.proxy.async.global;" ::: "memory");
      if ((phase == 0 || it + 1 < a.nsweeps) && !grid_barrier(a.bar, ++nbar * gridDim.x, &s_ok, a.err)) return;
    }
  }
}

int batch_class(int n, int variant) {
  for (int i = 0; i < 7; ++i)
    if (kBatchSizes[i] == n) return (variant == 1 && has_v1(n)) ? 2 * i + 1 : 2 * i;
  return -1;
}

bool batch_has_second_shape(int n) { return has_v1(n); }

template <int N, int V>
static void shape_of(int* rows, int* cols, int* re, int* ce) {
  *rows = BShape<N, V>::ROWS;
  *cols = BShape<N, V>::W;
  *re = BShape<N, V>::RE;
  *ce = BShape<N, V>::CE;
}

int batch_item_shape(int cls, int* rows_per_item, int* cols_per_item, int* row_values, int* col_values) {
  switch (cls) {
    case 0: shape_of<256, 0>(rows_per_item, cols_per_item, row_values, col_values); return 0;
    case 1: shape_of<256, 1>(rows_per_item, cols_per_item, row_values, col_values); return 0;
    case 2: shape_of<384, 0>(rows_per_item, cols_per_item, row_values, col_values); return 0;
    case 4: shape_of<512, 0>(rows_per_item, cols_per_item, row_values, col_values); return 0;
    case 5: shape_of<512, 1>(rows_per_item, cols_per_item, row_values, col_values); return 0;
    case 6: shape_of<768, 0>(rows_per_item, cols_per_item, row_values, col_values); return 0;
    case 8: shape_of<1024, 0>(rows_per_item, cols_per_item, row_values, col_values); return 0;
    case 9: shape_of<1024, 1>(rows_per_item, cols_per_item, row_values, col_values); return 0;
    case 10: shape_of<1536, 0>(rows_per_item, cols_per_item, row_values, col_values); return 0;
    case 11: shape_of<1536, 1>(rows_per_item, cols_per_item, row_values, col_values); return 0;
    case 12: shape_of<2048, 0>(rows_per_item, cols_per_item, row_values, col_values); return 0;
    case 13: shape_of<2048, 1>(rows_per_item, cols_per_item, row_values, col_values); return 0;
    default: return -1;
  }
}

// CTAs of a persistent batch launch on the current device (all resident:
// the cooperative launch requires it), or 0 if it cannot be launched
int batch_grid() {
  static std::once_flag once;
  static cudaError_t cfg_err = cudaSuccess;
  std::call_once(once, [] {
    cfg_err = cudaFuncSetAttribute(batch_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem);
  });
  if (cfg_err != cudaSuccess) return 0;
  int dev = 0, sms = 0, coop = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_sweep_kernel, BT, kBatchSmem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return coop ? sms * per_sm : 0;
}

int launch_batch_sweeps(const BatchArgs& a, int grid, cudaStream_t s) {
  if (a.nsweeps < 1) return (int)cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(BT);
  cfg.dynamicSmemBytes = kBatchSmem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return (int)cudaLaunchKernelEx(&cfg, batch_sweep_kernel, a);
}

}  // namespace wf
