// wf_colpass.cuh -- the column pass of the messenger iteration (Huffenberger
// 2017, Sec. 2 and Appendix A): the forward column DFT that completes the 2D
// transform of the data-side messenger, the 2D-Fourier updates (the 1/f part
// and the signal prior are both diagonal there), and the inverse column DFT.
// One CTA owns W adjacent complex columns; the messenger tile, the (C, P1f)
// tile and the twiddle table are staged in shared memory by TMA bulk copies.
// PREC selects the radix-16 stages: FP32 (0) or the tensor-core DFT-as-GEMM
// stages of wf_device.cuh (1: split TF32, 2: TF32).
#pragma once

#include <mutex>

#include "wf_cols_common.cuh"

namespace wf {


// Column pass geometry: W columns per CTA, TPC = L/E threads per column.
// W is a whole number of column tiles (TMA bulk loads of contiguous tiles)
// unless the tiles would not fit in shared memory, then half a tile.
constexpr size_t kMaxSmem = 227 * 1024;  // dynamic shared memory per CTA

// Values per thread of the two shapes the autotuner chooses between (one
// where both coincide): 16 measured fastest for columns of 1024 and more,
// 8 for 512; 3 * 2^k columns take 12 or 24.
template <int L>
struct ColPassE {
  static constexpr int v0 = (L % 3 == 0) ? ((L >= 1536) ? 24 : 12) : ((L >= 512) ? 16 : 8);
  static constexpr int v1 = (L % 3 == 0 || L > 2048) ? v0 : ((L >= 512) ? 8 : (L >= 128 ? 16 : v0));
};

template <int L, int MODE, int EV>
struct ColPassCfg {
  static constexpr bool T0 = (MODE == COL_PASS_2DF);
  static constexpr bool SRC = (MODE == COL_PASS_MERGE_SRC);
  static constexpr bool EXTRA = T0 || SRC;  // a third staged tile
  static constexpr int E = EV;
  static constexpr int TPC = L / E;
  static constexpr int W_MIN = (TPC >= 32) ? 1 : 32 / TPC;  // at least one warp
  // widest staging that fits in 227 KB of shared memory
  static constexpr int W_FIT = EXTRA ? (L >= 4096 ? 1 : (L >= 2048 ? 2 : WF_TW)) : (L >= 4096 ? 2 : WF_TW);
  static constexpr int W_WANT = (W_MIN > W_FIT) ? ((W_MIN + WF_TW - 1) / WF_TW) * WF_TW : W_FIT;
  static constexpr int W_CAP = 1024 / TPC;  // at most 1024 threads per CTA
  static constexpr int W = (W_WANT <= W_CAP) ? W_WANT
                           : (W_CAP >= WF_TW ? (W_CAP / WF_TW) * WF_TW : (W_CAP >= 2 ? 2 : 1));
  static constexpr bool TILED = (W % WF_TW == 0);
  static constexpr int THREADS = W * TPC;
  static constexpr int SP = SPad<L>::size;
  static constexpr int WANT = (W >= 32) ? 1 : (16 / W) % 16;
  static constexpr int STRIDE = SP + ((WANT - SP % 16) + 16) % 16;
  static constexpr size_t tile = (size_t)L * W * 8;
  static constexpr size_t y_off = 16, eig_off = y_off + tile, t0_off = eig_off + tile;
  static constexpr size_t tw_off = t0_off + (EXTRA ? tile : 0);
  static constexpr size_t fft_bytes = (size_t)W * STRIDE * 8;
  // the twiddle table (L values) is staged too when it still fits and costs
  // no CTA per SM (228 KB per SM, 1 KB reserved per CTA)
  static constexpr size_t kSM = 228 * 1024, kRes = 1024;
  static constexpr bool TWS =
      tw_off + (size_t)L * 8 + fft_bytes <= kMaxSmem &&
      kSM / (tw_off + (size_t)L * 8 + fft_bytes + kRes) == kSM / (tw_off + fft_bytes + kRes);
  static constexpr size_t fft_off = tw_off + (TWS ? (size_t)L * 8 : 0);
  static constexpr size_t bytes = fft_off + fft_bytes;
  static_assert(bytes <= kMaxSmem, "column pass staging exceeds shared memory");
  // position of (ky, column c of the CTA) in the staged Y / eig tiles
  static __device__ __forceinline__ int sidx(int ky, int c) {
    if constexpr (TILED) return (c / WF_TW) * L * WF_TW + ky * WF_TW + (c % WF_TW);
    else return ky * W + c;
  }
};

// Stage W columns of a column-tiled field: one bulk copy of whole tiles, or
// 16-byte asynchronous copies of half-tile rows.
template <int L, int MODE, int EV>
__device__ __forceinline__ void stage_tiled(float2* dst, const float2* src, int col0, int ny, uint64_t* bar) {
  using Cfg = ColPassCfg<L, MODE, EV>;
  if constexpr (Cfg::TILED) {
    if (threadIdx.x == 0) bulk_g2s(dst, src + tidx(0, col0, ny), (uint32_t)(L * Cfg::W * 8), bar);
  } else {
    for (int ky = threadIdx.x; ky < L; ky += Cfg::THREADS) {
      if constexpr (Cfg::W == 2) cp_async16(dst + ky * 2, src + tidx(ky, col0, ny));
      else cp_async8(dst + ky, src + tidx(ky, col0, ny));
    }
  }
}

// Row-major source (t_2DF of the plain sweep): W columns by async copies.
template <int L, int W, int THREADS>
__device__ __forceinline__ void tile_load_rowmajor(float2* dst, const float2* src, int col0, int ncols) {
  constexpr int CB = (W * 8 >= 16) ? 16 : 8;
  constexpr int PER_ROW = W * 8 / CB;
  constexpr int VALS = CB / 8;
  for (int i = threadIdx.x; i < L * PER_ROW; i += THREADS) {
    const int ky = i / PER_ROW;
    const int j = (i - ky * PER_ROW) * VALS;
    const float2* g = src + (size_t)ky * ncols + col0 + j;
    if constexpr (CB == 16) cp_async16(dst + ky * W + j, g);
    else cp_async8(dst + ky * W + j, g);
  }
}

// Extra shared memory of the tcgen05 stages (PREC 3, 4) after the column
// pass's own: 1 KB of alignment slack, the A tiles (16 KB per 128 threads,
// twice for the split), the four 4 KB DFT matrices, the mbarrier.
template <int L, int MODE, int EV, int PREC>
struct Tc5Smem {
  static constexpr int tiles = ColPassCfg<L, MODE, EV>::THREADS / 128;
  static constexpr size_t bytes = PREC >= 3 ? 1024 + (size_t)tiles * 16384 * (PREC == 3 ? 2 : 1) + 16384 + 16 : 0;
};
template <int L, int MODE, int EV, int PREC>
__device__ __forceinline__ uint64_t* tc5_mbar(unsigned char* smem) {
  return reinterpret_cast<uint64_t*>(smem + ColPassCfg<L, MODE, EV>::bytes + Tc5Smem<L, MODE, EV, PREC>::bytes - 16);
}

// The column pass (Sec. 2 / Appendix A: the 2D-Fourier updates between the
// forward and inverse column DFTs).  The messenger tile and the (C, P1f)
// tile are staged in shared memory before the transform begins.
template <int L, int MODE, int EV, int PREC = 0>
__global__ void __launch_bounds__(ColPassCfg<L, MODE, EV>::THREADS)
col_pass_kernel(ColArgs a) {
  using Cfg = ColPassCfg<L, MODE, EV>;
  constexpr int E = Cfg::E, TPC = Cfg::TPC, W = Cfg::W;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  float2* s_y = reinterpret_cast<float2*>(smem + Cfg::y_off);
  float2* s_eig = reinterpret_cast<float2*>(smem + Cfg::eig_off);
  float2* s_t0 = reinterpret_cast<float2*>(smem + Cfg::t0_off);  // plain sweep: t_2DF; source: j^
  float2* s_tw = reinterpret_cast<float2*>(smem + Cfg::tw_off);
  float2* s_fft = reinterpret_cast<float2*>(smem + Cfg::fft_off);

  const int c = threadIdx.x % W;
  const int t = threadIdx.x / W;
  const int ncols = a.nx / 2;
  const int col0 = blockIdx.x * W;
  const int col = col0 + c;
  float2* sb = s_fft + c * Cfg::STRIDE;

  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  if constexpr (WF_PDL_EARLY) pdl_trigger();
  // before the previous kernel has finished: the (C, P1f) tile and the
  // twiddle table, fixed during a solve, on barrier 1
  if (threadIdx.x == 0)
    mbar_expect_tx(&bar[1], (Cfg::TILED ? (uint32_t)Cfg::tile : 0u) + (Cfg::TWS ? (uint32_t)(L * 8) : 0u));
  stage_tiled<L, MODE, EV>(s_eig, a.eig, col0, a.ny, &bar[1]);
  if constexpr (Cfg::TWS)
    if (threadIdx.x == 0) bulk_g2s(s_tw, a.twy, (uint32_t)(L * 8), &bar[1]);
  cp_async_commit();
  // Maps above L2: the CTA that will run on this SM one wave later (pf CTAs
  // on) finds its tiles in L2 -- (C, P1f) now, the messenger once the
  // previous kernel is done.  Half-tile CTAs hint the whole tile from the
  // first CTA of the tile.
  const int nb = blockIdx.x + a.pf;
  const bool pf = a.pf > 0 && nb < (int)gridDim.x && threadIdx.x == 0 && (Cfg::TILED || (nb * W) % WF_TW == 0);
  constexpr size_t pf_bytes = (size_t)L * (Cfg::TILED ? W : WF_TW) * 8;
  if (pf) prefetch_l2_range(a.eig + tidx(0, nb * W, a.ny), pf_bytes);
  // (C, P1f) at kx = nx/2 for the packed column (fixed during a solve)
  const bool packed = (blockIdx.x == 0 && c == 0);
  float2 egn[E];
  if (packed) {
#pragma unroll
    for (int m = 0; m < E; ++m) egn[m] = __ldg(&a.eig_nyq[t + m * TPC]);
  }
  pdl_wait();
  // the messenger tile (and the source tile) on barrier 0
  if (threadIdx.x == 0)
    mbar_expect_tx(&bar[0], Cfg::TILED ? (uint32_t)(Cfg::tile * (Cfg::SRC ? 2 : 1)) : 0u);
  stage_tiled<L, MODE, EV>(s_y, a.f_y, col0, a.ny, &bar[0]);
  cp_async_commit();
  if constexpr (Cfg::SRC) stage_tiled<L, MODE, EV>(s_t0, a.src, col0, a.ny, &bar[0]);
  if constexpr (Cfg::T0) tile_load_rowmajor<L, W, Cfg::THREADS>(s_t0, a.f_t0, col0, ncols);
  cp_async_commit();
  if (pf) {
    prefetch_l2_range(a.f_y + tidx(0, nb * W, a.ny), pf_bytes);
    if constexpr (Cfg::SRC) prefetch_l2_range(a.src + tidx(0, nb * W, a.ny), pf_bytes);
  }
  // link covariances of this lambda level (written by the controller)
  const float Tl = a.has_rf ? a.st->Tf[1] : a.st->Tf[2];  // link to the RF/PX messenger
  const float off0 = (float)a.st->off[0];
  const float T0 = Cfg::T0 ? a.st->Tf[0] : 0.f;
  const float T0s = Cfg::T0 ? a.st->T0s[a.parity] : 0.f;

  auto drain = [&]() {
    const bool ok0 = mbar_wait(&bar[0], 0, WF_WAIT_TRIES);
    const bool ok1 = mbar_wait(&bar[1], 0, WF_WAIT_TRIES);
    cp_async_wait<0>();
    if (!(ok0 && ok1)) atomicOr(&a.st->err, WF_ERR_TIMEOUT);
  };
  // uniform: the flag is set only between launches; the copies above are
  // already in flight, so they land before the block exits
  if (a.check_done && a.st->done) {
    drain();
    return;
  }
  cp_async_wait<1>();
  const bool ok0 = mbar_wait(&bar[0], 0, WF_WAIT_TRIES);
  const bool ok1 = ok0 && mbar_wait(&bar[1], 0, WF_WAIT_TRIES);
  if (__syncthreads_or(!ok1)) {
    drain();
    return;
  }
  // radix-16 stages on tcgen05: operand tiles, DFT matrices, TMEM (after the
  // early returns, so every path that allocates also releases)
  if constexpr (PREC >= 3)
    tc5_setup<L, PREC>(smem + Cfg::bytes, tc5_mbar<L, MODE, EV, PREC>(smem), Cfg::TWS ? s_tw : a.twy, 1);

  float2 v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = s_y[Cfg::sidx(t + m * TPC, c)];
  fft_block<L, E, false, false, Cfg::TWS, PREC>(v, sb, t, Cfg::TWS ? s_tw : a.twy, 1);

  // partner values Z[-k] for the packed column 0 (CTA 0 only; uniform)
  float2 vp[E];
  if (blockIdx.x == 0) {
#pragma unroll
    for (int m = 0; m < E; ++m) sb[spad(t + m * TPC)] = v[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; ++m) vp[m] = sb[spad(neg_mod<L>(t + m * TPC))];
    __syncthreads();
  }
  cp_async_wait<0>();
  __syncthreads();

#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int k = t + m * TPC;
    const float2 eg = s_eig[Cfg::sidx(k, c)];
    if constexpr (MODE == COL_PASS_MERGE || MODE == COL_PASS_MERGE_SRC) {
      constexpr bool SRC = (MODE == COL_PASS_MERGE_SRC);
      const float2 jv = SRC ? s_t0[Cfg::sidx(k, c)] : make_float2(0.f, 0.f);
      const float2 jp = (SRC && packed) ? s_t0[Cfg::sidx(neg_mod<L>(k), c)] : make_float2(0.f, 0.f);
      v[m] = merged_mode<SRC>(v[m], packed ? vp[m] : v[m], eg, packed ? egn[m] : eg, off0, Tl, packed, jv, jp);
    } else if constexpr (MODE == COL_PASS_2DF) {
      const float2 t0o = s_t0[k * W + c];
      float2 t0n, d0;
      if (packed) {
        const float2 egb = egn[m];
        const float2 t0p = s_t0[(neg_mod<L>(k)) * W + c];
        float2 yA, yB, tA, tB, tnA, tnB;
        unpack_pair(v[m], vp[m], yA, yB);
        unpack_pair(t0o, t0p, tA, tB);
        const float2 dA = mode_2df(yA, tA, eg.x, eg.y, off0, Tl, T0, T0s, tnA);
        const float2 dB = mode_2df(yB, tB, egb.x, egb.y, off0, Tl, T0, T0s, tnB);
        d0 = repack_pair(dA, dB);
        t0n = repack_pair(tnA, tnB);
      } else {
        d0 = mode_2df(v[m], t0o, eg.x, eg.y, off0, Tl, T0, T0s, t0n);
      }
      v[m] = d0;
      a.f_t0[(size_t)k * ncols + col] = t0n;
    } else {
      // no 1/f part: eq. (2mess_s), s = C/(C + T) y for the messenger next to s
      if (packed) {
        float2 yA, yB;
        unpack_pair(v[m], vp[m], yA, yB);
        const float2 egb = egn[m];
        v[m] = repack_pair(cscale(yA, __fdividef(eg.x, eg.x + Tl)), cscale(yB, __fdividef(egb.x, egb.x + Tl)));
      } else {
        v[m] = cscale(v[m], __fdividef(eg.x, eg.x + Tl));
      }
    }
  }
  if constexpr (Cfg::T0) {
    // publish the T_0 that the new t_2DF was made with (implicit s)
    if (blockIdx.x == 0 && threadIdx.x == 0) a.st->T0s[a.parity ^ 1] = T0;
  }
  fft_block<L, E, true, false, Cfg::TWS, PREC>(v, sb, t, Cfg::TWS ? s_tw : a.twy, 1);
  if constexpr (PREC >= 3) {
    tc5_teardown();
    if (threadIdx.x == 0 && !tc5_ctx().ok) atomicOr(&a.st->err, WF_ERR_TIMEOUT);
  }
  if constexpr (!WF_PDL_EARLY) pdl_trigger();
  const float sc = 1.0f / (float)L;
#pragma unroll
  for (int m = 0; m < E; ++m) a.f_x[tidx(t + m * TPC, col, a.ny)] = cscale(v[m], sc);
}

template <int L, int MODE, int EV, int PREC = 0>
static int launch_col_pass_e(const ColArgs& a, cudaStream_t s) {
  using Cfg = ColPassCfg<L, MODE, EV>;
  const int ncols = a.nx / 2;
  if (ncols % Cfg::W != 0) return (int)cudaErrorInvalidValue;
  constexpr size_t kBytes = Cfg::bytes + Tc5Smem<L, MODE, EV, PREC>::bytes;
  static_assert(kBytes <= kMaxSmem, "column pass staging exceeds shared memory");
  static_assert(PREC < 3 || Cfg::THREADS % 128 == 0, "tcgen05 tiles are 128 threads");
  // once per instantiation and process (plans may run on several host threads)
  static std::once_flag once;
  static cudaError_t cfg_err = cudaSuccess;
  static int dist = 0;  // CTAs one wave ahead
  std::call_once(once, [] {
    cfg_err = cudaFuncSetAttribute(col_pass_kernel<L, MODE, EV, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)kBytes);
    if (cfg_err == cudaSuccess) dist = resident_ctas(col_pass_kernel<L, MODE, EV, PREC>, Cfg::THREADS, kBytes);
  });
  if (cfg_err != cudaSuccess) return (int)cfg_err;
  const dim3 grid(ncols / Cfg::W), block(Cfg::THREADS);
  ColArgs b = a;
  b.pf = a.prefetch ? dist : 0;
  return launch_pdl(col_pass_kernel<L, MODE, EV, PREC>, grid, block, kBytes, s, b);
}

}  // namespace wf
