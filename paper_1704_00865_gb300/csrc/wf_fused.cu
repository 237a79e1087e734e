// wf_fused.cu -- the whole messenger sweep, R times, in one cooperative
// launch (Huffenberger 2017, Sec. 2: per iteration one transform pair and the
// diagonal updates between them), for 1024 x 1024 maps with a stripe part and
// the merged 2DF block.
//
// A sweep is the row pass (inverse row DFT, the pixel update, forward row
// DFT, the stripe-basis updates) and the column pass (forward column DFT, the
// 2D-Fourier block, inverse column DFT).  As two launches, every field is
// read from and written to global memory in every sweep (40 bytes per
// pixel).  Here 128 CTAs, one per SM, stay resident for R sweeps and
// separate the passes by grid barriers.  CTA b owns map rows 8b .. 8b+7 and
// the column tile 4b .. 4b+3 for the whole launch, so what only its own rows
// or its own tile use stays in its shared memory across sweeps: the pixel
// table (d, Nbar_PX) and the fields d_RF and t_RF of its rows, and the
// (C, P1f) eigenvalues of its tile.  Only what crosses between CTAs goes
// through global memory each sweep: t_RF (written by the row pass, read by
// the column pass of other CTAs) and d_2DF (the reverse), 16 bytes per
// pixel.  d_RF is written back once, at the end of the launch.
//
// The transforms and the updates are the row pass's and the column pass's
// own (wf_device.cuh, wf_rows_common.cuh, wf_cols_common.cuh), with 8 values
// per thread in both transforms.
//
// The grid barrier counts arrivals on a global word that is zeroed before
// each launch; its waits are bounded, and a CTA that gives up raises an
// abort word that ends every other wait, records WF_ERR_TIMEOUT and
// returns.  The cooperative launch guarantees that all 128 CTAs are
// resident at once (it fails instead of starting otherwise).
#include <cuda_runtime.h>

#include <mutex>

#include "wf_cols_common.cuh"
#include "wf_device.cuh"
#include "wf_internal.h"
#include "wf_rows_common.cuh"

namespace wf {

template <int N>
struct FusedCfg {
  static constexpr int M = N / 2;          // complex values per row (real length N)
  static constexpr int L = N;              // column length
  static constexpr int THREADS = 512;
  static constexpr int RE = 8;             // values per thread, row transforms
  static constexpr int TPF = M / RE;       // threads per row
  static constexpr int RPC = THREADS / TPF;  // rows per CTA
  static constexpr int W = WF_TW;          // columns per CTA: one column tile
  static constexpr int CE = 8;             // values per thread, column transforms
  static constexpr int TPC = L / CE;       // threads per column
  static constexpr int GRID = N / RPC;     // CTAs
  static_assert(W * TPC == THREADS, "the column pass must use every thread");
  static_assert(GRID * W == M, "one column tile per CTA");
  // padded per-column FFT buffers, as in the column pass for 4-column tiles
  static constexpr int SP = SPad<L>::size;
  static constexpr int STRIDE = SP + ((4 - SP % 16) + 16) % 16;
  // shared memory: header (mbarrier, flags), resident tables, then a region
  // the row phase and the column phase use in turn
  static constexpr size_t hdr = 64;
  static constexpr size_t dn_off = hdr;
  static constexpr size_t d1_off = dn_off + (size_t)RPC * M * 16;
  static constexpr size_t t1_off = d1_off + (size_t)RPC * M * 8;
  static constexpr size_t eig_off = t1_off + (size_t)RPC * M * 8;
  static constexpr size_t u_off = eig_off + (size_t)L * W * 8;
  static constexpr size_t fftr_bytes = (size_t)RPC * SPad<M>::size * 8;
  static constexpr size_t x_off = u_off + fftr_bytes;            // row phase: d_2DF rows
  static constexpr size_t fftc_bytes = (size_t)W * STRIDE * 8;
  static constexpr size_t src_off = u_off + fftc_bytes;          // column phase: source tile
  static constexpr size_t row_end = x_off + (size_t)RPC * M * 8;
  static constexpr size_t col_end = src_off + (size_t)L * W * 8;
  static constexpr size_t bytes = row_end > col_end ? row_end : col_end;
  static_assert(bytes <= 227 * 1024, "fused sweep staging exceeds shared memory");
  static_assert(src_off % 16 == 0 && x_off % 16 == 0, "16-byte aligned copies");
};

template <int N, bool SRC>
__global__ void __launch_bounds__(FusedCfg<N>::THREADS, 1)
fused_sweep_kernel(FusedArgs a) {
  using F = FusedCfg<N>;
  constexpr int M = F::M, L = F::L, RE = F::RE, TPF = F::TPF, RPC = F::RPC, W = F::W, CE = F::CE,
                TPC = F::TPC, NT = F::THREADS;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem);
  int* ok_s = reinterpret_cast<int*>(smem + 16);
  float4* s_dn = reinterpret_cast<float4*>(smem + F::dn_off);
  float2* s_d1 = reinterpret_cast<float2*>(smem + F::d1_off);
  float2* s_t1 = reinterpret_cast<float2*>(smem + F::t1_off);
  float2* s_eig = reinterpret_cast<float2*>(smem + F::eig_off);
  float2* s_fftr = reinterpret_cast<float2*>(smem + F::u_off);
  float2* s_x = reinterpret_cast<float2*>(smem + F::x_off);
  float2* s_fftc = reinterpret_cast<float2*>(smem + F::u_off);
  float2* s_src = reinterpret_cast<float2*>(smem + F::src_off);

  const int tid = threadIdx.x;
  const int b = blockIdx.x;
  const int y0 = b * RPC, col0 = b * W;
  const int ny = a.ny;
  // row phase: group g transforms row y0 + g with TPF threads
  const int g = tid / TPF, t = tid - g * TPF, y = y0 + g;
  float2* sbr = s_fftr + g * SPad<M>::size;
  // column phase: thread (c, tc) holds values tc + m TPC of column col0 + c
  const int c = tid % W, tc = tid / W;
  float2* sbc = s_fftc + c * F::STRIDE;
  const size_t tile0 = tidx(0, col0, ny);
  const bool packed = (b == 0 && c == 0);

  // uniform: the flag is written only between launches
  if (a.st->done) return;
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_fence_init();
  }
  __syncthreads();
  // resident tables: this CTA's rows of the pixel table and of d_RF, its
  // (C, P1f) tile (contiguous: bulk copies), its rows of t_RF (column-tiled:
  // 16-byte copies)
  if (tid == 0) {
    mbar_expect_tx(&mbar[0], (uint32_t)(RPC * M * 16 + RPC * M * 8 + L * W * 8));
    bulk_g2s(s_dn, a.dn + (size_t)y0 * M, RPC * M * 16, &mbar[0]);
    bulk_g2s(s_d1, a.f_d1 + (size_t)y0 * M, RPC * M * 8, &mbar[0]);
    bulk_g2s(s_eig, a.eig + tile0, L * W * 8, &mbar[0]);
  }
  for (int i = tid; i < RPC * (M / 2); i += NT) {
    const int r = i / (M / 2);
    const int k = (i - r * (M / 2)) * 2;
    cp_async16(s_t1 + r * M + k, a.f_t1 + tidx(y0 + r, k, ny));
  }
  cp_async_commit();
  // per-thread constants of the launch: real-FFT twiddles and stripe
  // eigenvalues of this thread's row modes, the kx = nx/2 eigenvalues of the
  // packed column, the link covariances of this lambda level
  float2 wk[RE];
  load_rtw<M, RE>(wk, t, a.twx);
  float pk[RE];
#pragma unroll
  for (int m = 0; m < RE; ++m) pk[m] = __ldg(&a.pst[t + m * TPF]);
  const float pkn = (t == 0) ? __ldg(&a.pst[M]) : 0.f;
  const float a2y = (a.a2 != nullptr) ? __ldg(&a.a2[y]) : 1.f;
  const float T2 = a.st->Tf[2], T1 = a.st->Tf[1];
  const float off1 = (float)a.st->off[1], off0 = (float)a.st->off[0];
  unsigned nbar = 0;  // barriers passed in this launch
  const bool ok0 = mbar_wait(&mbar[0], 0, WF_WAIT_TRIES);
  cp_async_wait<0>();
  if (__syncthreads_or(!ok0)) {
    if (tid == 0) atomicOr(&a.st->err, WF_ERR_TIMEOUT);
    return;
  }

  for (int it = 0; it < a.nsweeps; ++it) {
    // ---------------------------------------------------------------- rows
    // d_2DF of this CTA's rows (written by the column pass of every CTA)
    for (int i = tid; i < RPC * (M / 2); i += NT) {
      const int r = i / (M / 2);
      const int k = (i - r * (M / 2)) * 2;
      cp_async16(s_x + r * M + k, a.f_x + tidx(y0 + r, k, ny));
    }
    cp_async_commit();
    float2 v[RE];
#pragma unroll
    for (int m = 0; m < RE; ++m) v[m] = s_d1[g * M + t + m * TPF];
    c2r_pre_w<M, RE, false>(v, sbr, t, wk);
    fft_block<M, RE, true, false, false>(v, sbr, t, a.twh, 1);
    // eq. (2mess_t1) analogue in pixel space, two pixels per complex value
#pragma unroll
    for (int m = 0; m < RE; ++m) {
      const float4 q = s_dn[g * M + t + m * TPF];
      v[m] = make_float2(tpx_update(q.x, q.y, v[m].x, T2), tpx_update(q.z, q.w, v[m].y, T2));
    }
    fft_block<M, RE, false, false, false>(v, sbr, t, a.twh, 1);
    r2c_post_w<M, RE, false>(v, sbr, t, wk);
    cp_async_wait<0>();
    __syncthreads();
    // eqs. (2mess_d0), (2mess_t0) analogues in the stripe basis
#pragma unroll
    for (int m = 0; m < RE; ++m) {
      const int k = t + m * TPF;
      float2 d1, t1;
      stripe_update(k, v[m], s_t1[g * M + k], s_x[g * M + k], a2y, pk[m], pkn, off1, T2, T1, d1, t1);
      s_d1[g * M + k] = d1;
      s_t1[g * M + k] = t1;
      a.f_t1[tidx(y, k, ny)] = t1;
    }
    __syncthreads();  // s_x is free: the source tile may land there
    if constexpr (SRC) {
      for (int i = tid; i < L * W / 2; i += NT) cp_async16(s_src + 2 * i, a.src + tile0 + 2 * i);
      cp_async_commit();
    }
    if (!grid_barrier(a.bar, ++nbar * gridDim.x, ok_s, &a.st->err)) {
      cp_async_wait<0>();
      return;
    }
    // ------------------------------------------------------------- columns
    float2 u[CE];
#pragma unroll
    for (int m = 0; m < CE; ++m) u[m] = __ldcg(&a.f_t1[tile0 + (size_t)(tc + m * TPC) * W + c]);
    fft_block<L, CE, false, false, false>(u, sbc, tc, a.twy, 1);
    // partner values Z[-k] for the packed column 0 (CTA 0 only; uniform)
    float2 up[CE];
    if (b == 0) {
#pragma unroll
      for (int m = 0; m < CE; ++m) sbc[spad(tc + m * TPC)] = u[m];
      __syncthreads();
#pragma unroll
      for (int m = 0; m < CE; ++m) up[m] = sbc[spad(neg_mod<L>(tc + m * TPC))];
      __syncthreads();
    }
    if constexpr (SRC) {
      cp_async_wait<0>();
      __syncthreads();
    }
#pragma unroll
    for (int m = 0; m < CE; ++m) {
      const int k = tc + m * TPC;
      const float2 eg = s_eig[k * W + c];
      const float2 egb = packed ? __ldg(&a.eig_nyq[k]) : eg;
      const float2 jv = SRC ? s_src[k * W + c] : make_float2(0.f, 0.f);
      const float2 jp = (SRC && packed) ? s_src[neg_mod<L>(k) * W + c] : make_float2(0.f, 0.f);
      u[m] = merged_mode<SRC>(u[m], packed ? up[m] : u[m], eg, egb, off0, T1, packed, jv, jp);
    }
    fft_block<L, CE, true, false, false>(u, sbc, tc, a.twy, 1);
    const float sc = 1.0f / (float)L;
#pragma unroll
    for (int m = 0; m < CE; ++m) a.f_x[tile0 + (size_t)(tc + m * TPC) * W + c] = cscale(u[m], sc);
    // the next row pass reads d_2DF of every tile (none after the last sweep)
    if (it + 1 < a.nsweeps && !grid_barrier(a.bar, ++nbar * gridDim.x, ok_s, &a.st->err)) return;
  }
  // d_RF of this CTA's rows back to global memory
  __syncthreads();
  for (int i = tid; i < RPC * M; i += NT) a.f_d1[(size_t)y0 * M + i] = s_d1[i];
}

template <int N, bool SRC>
static int launch_fused_n(const FusedArgs& a, cudaStream_t s) {
  using F = FusedCfg<N>;
  static std::once_flag once;
  static cudaError_t cfg_err = cudaSuccess;
  std::call_once(once, [] {
    cfg_err = cudaFuncSetAttribute(fused_sweep_kernel<N, SRC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)F::bytes);
  });
  if (cfg_err != cudaSuccess) return (int)cfg_err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(F::GRID);
  cfg.blockDim = dim3(F::THREADS);
  cfg.dynamicSmemBytes = F::bytes;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return (int)cudaLaunchKernelEx(&cfg, fused_sweep_kernel<N, SRC>, a);
}

int launch_fused(const FusedArgs& a, cudaStream_t s) {
  if (a.nsweeps < 1) return (int)cudaSuccess;
  if (a.ny == 1024 && a.nx == 1024)
    return a.src != nullptr ? launch_fused_n<1024, true>(a, s) : launch_fused_n<1024, false>(a, s);
  return (int)cudaErrorInvalidValue;
}

bool fused_supported(int ny, int nx, int has_rf, int merged, int prec) {
  if (!(ny == 1024 && nx == 1024 && has_rf && merged && prec == 0)) return false;
  int dev = 0, sms = 0, coop = 0, smem = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) ||
      cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) {
    cudaGetLastError();
    return false;
  }
  return coop != 0 && sms >= FusedCfg<1024>::GRID && (size_t)smem >= FusedCfg<1024>::bytes;
}

}  // namespace wf
