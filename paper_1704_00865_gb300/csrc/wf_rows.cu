// wf_rows.cu -- the row pass of the messenger iteration and the row steps of
// the residual (Huffenberger 2017, Sec. 2).
//
// One CTA owns ROWS map rows; each row is a real length-nx signal handled by
// TPF = (nx/2)/E threads through a complex length-nx/2 Stockham FFT in
// shared memory.  The pixel-space messenger update (eq. 2mess_t1 analogue:
// white noise and mask, diagonal in pixels) sits between the inverse and the
// forward row transform, and the stripe-basis updates (eqs. 2mess_d0 and
// 2mess_t0 analogues: stripe noise, diagonal in the row-wise DFT) follow the
// forward transform, so a row is read and written once per iteration.
#include <mutex>

#include "wf_device.cuh"
#include "wf_internal.h"
#include "wf_rows_common.cuh"

namespace wf {

template <int M>
struct RowCfg {
  static constexpr int E = (M % 3 == 0) ? 12 : ((M >= 2048) ? 16 : 8);
  static constexpr int TPF = M / E;
  static constexpr int ROWS = (256 / TPF) >= 1 ? (256 / TPF) : 1;
  static constexpr int THREADS = ROWS * TPF;
};

// deterministic block sum of one double per thread (fixed tree)
template <int THREADS>
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  constexpr int NW = (THREADS + 31) / 32;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < NW; ++i) s += red[i];
  }
  return s;
}

template <int M, int MODE>
__global__ void __launch_bounds__(RowCfg<M>::THREADS)
row_kernel(RowArgs a) {
  using Cfg = RowCfg<M>;
  constexpr int E = Cfg::E, TPF = Cfg::TPF, ROWS = Cfg::ROWS;
  __shared__ float2 sbuf[ROWS][SPad<M>::size];
  __shared__ double red[(Cfg::THREADS + 31) / 32];
  pdl_trigger();
  pdl_wait();

  const int g = threadIdx.x / TPF;
  const int t = threadIdx.x - g * TPF;
  const int y = blockIdx.x * ROWS + g;
  const bool valid = y < a.ny;
  const size_t row0 = (size_t)(valid ? y : 0) * M;
  float2* sb = sbuf[g];

  // uniform: both flags are set only between launches
  if ((a.check_done && a.st->done) || (a.skip_ok && a.st->skip_resid)) return;

  float2 v[E];

  if constexpr (MODE == ROW_RESID_B) {
    // g = S^-1 s and s arrive in RF; go to pixels.
    float2 w[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
      v[m] = valid ? a.r_g[row0 + t + m * TPF] : make_float2(0.f, 0.f);
      w[m] = valid ? a.r_q[row0 + t + m * TPF] : make_float2(0.f, 0.f);
    }
    c2r_pre<M, E>(v, sb, t, a.twx);
    fft_block<M, E, true>(v, sb, t, a.twx, 2);
    c2r_pre<M, E>(w, sb, t, a.twx);
    fft_block<M, E, true>(w, sb, t, a.twx, 2);
    const float vshift = (float)a.st->var_shift;
    double gm2 = 0.0, g2 = 0.0;
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const float4 q = valid ? a.dn[row0 + t + m * TPF] : make_float4(0.f, -1.f, 0.f, -1.f);
      const float2 jm = (valid && a.src_px != nullptr) ? a.src_px[row0 + t + m * TPF] : make_float2(0.f, 0.f);
      float gp[2], qp[2], go[2];
      const float gv[2] = {v[m].x, v[m].y}, sv[2] = {w[m].x, w[m].y};
      const float dv[2] = {q.x, q.z}, nv[2] = {q.y, q.w}, jv[2] = {jm.x, jm.y};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const double gd = (double)gv[h];
        if (valid) g2 += gd * gd;
        if (nv[h] < 0.f) {  // masked: the residual there is S^-1 s (minus a source)
          const double rm = gd - (double)jv[h];
          if (valid) gm2 += rm * rm;
          gp[h] = 0.f;
          qp[h] = 0.f;
          go[h] = gv[h];
        } else {             // N_PX g' + s - d with the full pixel variance
          gp[h] = gv[h];
          qp[h] = fmaf(nv[h] + vshift, gv[h], sv[h] - dv[h]);
          go[h] = 0.f;
        }
      }
      if (valid && a.gm_out != nullptr) a.gm_out[row0 + t + m * TPF] = make_float2(go[0], go[1]);
      v[m] = make_float2(gp[0], gp[1]);
      w[m] = make_float2(qp[0], qp[1]);
    }
    fft_block<M, E, false>(v, sb, t, a.twx, 2);
    r2c_post<M, E>(v, sb, t, a.twx);
    fft_block<M, E, false>(w, sb, t, a.twx, 2);
    r2c_post<M, E>(w, sb, t, a.twx);
    if (valid) {
      const float a2y = (a.a2 != nullptr) ? a.a2[y] : 1.f;
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const int k = t + m * TPF;
        float2 q = w[m];
        if (a.has_rf) {  // + N_RF g' with the given stripe eigenvalues
          if (k == 0) {
            q.x = fmaf(a2y * a.pst[0], v[m].x, q.x);
            q.y = fmaf(a2y * a.pst[M], v[m].y, q.y);
          } else {
            const float n1 = a2y * a.pst[k];
            q = make_float2(fmaf(n1, v[m].x, q.x), fmaf(n1, v[m].y, q.y));
          }
        }
        a.r_g[row0 + k] = v[m];
        a.r_q[row0 + k] = q;
      }
    }
    double s0 = block_sum<Cfg::THREADS>(gm2, red);
    double s1 = block_sum<Cfg::THREADS>(g2, red);
    if (threadIdx.x == 0) {
      a.part0[blockIdx.x] = s0;
      a.part1[blockIdx.x] = s1;
    }
  } else if constexpr (MODE == ROW_RESID_D) {
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = valid ? a.r_q[row0 + t + m * TPF] : make_float2(0.f, 0.f);
    c2r_pre<M, E>(v, sb, t, a.twx);
    fft_block<M, E, true>(v, sb, t, a.twx, 2);
    double r2 = 0.0;
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const float4 q = valid ? a.dn[row0 + t + m * TPF] : make_float4(0.f, -1.f, 0.f, -1.f);
      if (valid) {
        if (q.y >= 0.f) r2 += (double)v[m].x * (double)v[m].x;
        if (q.w >= 0.f) r2 += (double)v[m].y * (double)v[m].y;
        // optional map of Delta d on unmasked pixels (defect correction)
        if (a.out_px != nullptr)
          a.out_px[row0 + t + m * TPF] = make_float2(q.y >= 0.f ? v[m].x : 0.f, q.w >= 0.f ? v[m].y : 0.f);
      }
    }
    double s0 = block_sum<Cfg::THREADS>(r2, red);
    if (threadIdx.x == 0) a.part0[blockIdx.x] = s0;
  } else if constexpr (MODE == ROW_C2R) {
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = valid ? a.in_rf[row0 + t + m * TPF] : make_float2(0.f, 0.f);
    c2r_pre<M, E>(v, sb, t, a.twx);
    fft_block<M, E, true>(v, sb, t, a.twx, 2);
    if (valid) {
#pragma unroll
      for (int m = 0; m < E; ++m) a.out_px[row0 + t + m * TPF] = v[m];
    }
  } else if constexpr (MODE == ROW_R2C) {
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = valid ? a.in_px[row0 + t + m * TPF] : make_float2(0.f, 0.f);
    fft_block<M, E, false>(v, sb, t, a.twx, 2);
    r2c_post<M, E>(v, sb, t, a.twx);
    if (valid) {
#pragma unroll
      for (int m = 0; m < E; ++m) a.out_rf[row0 + t + m * TPF] = v[m];
    }
  }
}


// Row pass geometry: each row is one real length-2M transform done by TPF
// threads with E values each -- a single warp per row up to M = 256 with 8
// values per thread (then the exchange steps need only warp barriers), two
// warps at M = 512.  Short rows are packed several to a warp.  One CTA = ROWS rows; the grid is ny / ROWS CTAs, small enough
// units that the SMs finish within one row of each other.
// Values per thread of the two shapes the autotuner chooses between (one
// where both coincide): 8 (two warps per 1024-point row) measured fastest at
// 1024^2 and above, 4 at 512^2 and below; 3 * 2^k rows take 12.
template <int M>
struct RowPassE {
  static constexpr int v0 = (M % 3 == 0) ? 12 : 8;
  static constexpr int v1 = (M % 3 == 0) ? 12 : 4;
};
template <int M, int EV>
struct RowPassCfg {
  static constexpr int E = EV;
  static constexpr int TPF = M / E;
  static constexpr int ROWS = (TPF >= 32) ? 1 : 32 / TPF;
  static constexpr int THREADS = ROWS * TPF;
  static constexpr bool WARP = (THREADS == 32);
};

template <int M, int MODE, int EV>
struct RowPassSmem {
  static constexpr int ROWS = RowPassCfg<M, EV>::ROWS;
  static constexpr bool RF = (MODE == ROW_PASS_RF);
  static constexpr size_t a_off = 16;
  static constexpr size_t dn_off = a_off + (size_t)ROWS * M * 8;
  static constexpr size_t t1_off = dn_off + (size_t)ROWS * M * 16;
  static constexpr size_t x_off = t1_off + (RF ? (size_t)ROWS * M * 8 : 0);
  static constexpr size_t tw_off = x_off + (RF ? (size_t)ROWS * M * 8 : 0);  // twh, M values
  static constexpr size_t fft_bytes = (size_t)ROWS * SPad<M>::size * 8;
  // the transform twiddles are staged too where that costs no CTA per SM
  // (228 KB per SM, 1 KB reserved per CTA); up to 512-point rows a whole
  // 1024^2 row pass is resident either way, and staging measured faster
  static constexpr size_t kSM = 228 * 1024, kRes = 1024;
  static constexpr size_t base_bytes = tw_off + fft_bytes;
  static constexpr bool TWS =
      M <= 512 || kSM / (base_bytes + (size_t)M * 8 + kRes) == kSM / (base_bytes + kRes);
  static constexpr size_t fft_off = tw_off + (TWS ? (size_t)M * 8 : 0);
  static constexpr size_t bytes = fft_off + fft_bytes;
};

// Gather rows y0 .. y0+nrows-1 of a column-tiled RF field into row-major
// shared memory, 16 bytes (two complex values) per asynchronous copy.
template <int M, int THREADS>
__device__ __forceinline__ void gather_tiled_rows(float2* dst, const float2* src, int y0, int nrows, int ny) {
  for (int i = threadIdx.x; i < nrows * (M / 2); i += THREADS) {
    const int r = i / (M / 2);
    const int k = (i - r * (M / 2)) * 2;
    cp_async16(dst + r * M + k, src + tidx(y0 + r, k, ny));
  }
}

// The row pass (Sec. 2: eq. 2mess_t1 analogue in pixels between the inverse
// and forward row DFTs, then the stripe-basis updates).  Row-major inputs
// (d_RF, the pixel table) arrive by TMA bulk copies on an mbarrier, the
// column-tiled ones (t_RF, the signal-side field) by 16-byte asynchronous
// copies; the first transform starts as soon as its own field is in.  Waits
// are bounded; on a timeout the CTA records WF_ERR_TIMEOUT, drains its
// copies (bounded) and returns.
template <int M, int MODE, int EV>
__global__ void __launch_bounds__(RowPassCfg<M, EV>::THREADS)
row_pass_kernel(RowArgs a) {
  using Cfg = RowPassCfg<M, EV>;
  using SM = RowPassSmem<M, MODE, EV>;
  constexpr int E = Cfg::E, TPF = Cfg::TPF, ROWS = Cfg::ROWS, NT = Cfg::THREADS;
  constexpr bool W = Cfg::WARP;
  constexpr bool RF = SM::RF;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  float2* s_a = reinterpret_cast<float2*>(smem + SM::a_off);
  float4* s_dn = reinterpret_cast<float4*>(smem + SM::dn_off);
  float2* s_t1 = reinterpret_cast<float2*>(smem + SM::t1_off);
  float2* s_x = reinterpret_cast<float2*>(smem + SM::x_off);
  float2* s_tw = reinterpret_cast<float2*>(smem + SM::tw_off);
  float2* s_fft = reinterpret_cast<float2*>(smem + SM::fft_off);

  const int g = threadIdx.x / TPF;
  const int t = threadIdx.x - g * TPF;
  const int y0 = blockIdx.x * ROWS;
  const int nval = min(ROWS, a.ny - y0);
  const int y = y0 + g;
  const bool valid = g < nval;
  float2* sb = s_fft + g * SPad<M>::size;

  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  fft_sync<W>();
  if constexpr (WF_PDL_EARLY) pdl_trigger();
  // before the previous kernel has finished: the pixel table (fixed during a
  // solve) and the transform twiddles
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bar[1], (uint32_t)(nval * M * 16 + (SM::TWS ? M * 8 : 0)));
    if constexpr (SM::TWS) bulk_g2s(s_tw, a.twh, (uint32_t)(M * 8), &bar[1]);
    for (int r = 0; r < nval; ++r) bulk_g2s(s_dn + r * M, a.dn + (size_t)(y0 + r) * M, M * 16, &bar[1]);
  }
  float2 wk[E];
  load_rtw<M, E>(wk, t, a.twx);
  // stripe spectrum a(y)^2 Pst(k) of this thread's modes (fixed during a solve)
  float pk[RF ? E : 1];
  float a2y = 1.f, pkn = 0.f;  // pkn: Pst at kx = M, packed with kx = 0
  if constexpr (RF) {
    if (a.a2 != nullptr && valid) a2y = __ldg(&a.a2[y]);
#pragma unroll
    for (int m = 0; m < E; ++m) pk[m] = __ldg(&a.pst[t + m * TPF]);
    if (t == 0) pkn = __ldg(&a.pst[M]);
  }
  pdl_wait();
  // the fields the previous kernels wrote
  if (threadIdx.x == 0) {
    if constexpr (RF) {
      mbar_expect_tx(&bar[0], (uint32_t)(nval * M * 8));
      for (int r = 0; r < nval; ++r) bulk_g2s(s_a + r * M, a.f_d1 + (size_t)(y0 + r) * M, M * 8, &bar[0]);
    } else {
      mbar_expect_tx(&bar[0], 0u);  // nothing on this barrier: completes at once
    }
  }
  if constexpr (RF) {
    gather_tiled_rows<M, NT>(s_t1, a.f_t1, y0, nval, a.ny);
    gather_tiled_rows<M, NT>(s_x, a.f_x, y0, nval, a.ny);
  } else {
    gather_tiled_rows<M, NT>(s_a, a.f_x, y0, nval, a.ny);
  }
  cp_async_commit();
  // link covariances of this lambda level (written by the controller)
  const float T2 = a.st->Tf[2];
  const float T1 = RF ? a.st->Tf[1] : 0.f;
  const float off1 = RF ? (float)a.st->off[1] : 0.f;

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
  bool ok = mbar_wait(&bar[0], 0, WF_WAIT_TRIES) && mbar_wait(&bar[1], 0, WF_WAIT_TRIES);
  if constexpr (!RF) cp_async_wait<0>();
  if (__syncthreads_or(!ok)) {
    drain();
    return;
  }

  float2 v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = s_a[g * M + t + m * TPF];
  c2r_pre_w<M, E, W>(v, sb, t, wk);
  fft_block<M, E, true, W, SM::TWS>(v, sb, t, SM::TWS ? s_tw : a.twh, 1);
  // eq. (2mess_t1) analogue in pixel space, two pixels per complex value
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const float4 q = s_dn[g * M + t + m * TPF];
    v[m] = make_float2(tpx_update(q.x, q.y, v[m].x, T2), tpx_update(q.z, q.w, v[m].y, T2));
  }
  fft_block<M, E, false, W, SM::TWS>(v, sb, t, SM::TWS ? s_tw : a.twh, 1);
  r2c_post_w<M, E, W>(v, sb, t, wk);
  if constexpr (!WF_PDL_EARLY) pdl_trigger();
  if constexpr (RF) {
    cp_async_wait<0>();
    fft_sync<W>();
  }
  if (!valid) return;
  const size_t row0 = (size_t)y * M;
  if constexpr (!RF) {
#pragma unroll
    for (int m = 0; m < E; ++m) a.f_y[tidx(y, t + m * TPF, a.ny)] = v[m];
  } else {
    // eqs. (2mess_d0), (2mess_t0) analogues in the stripe basis
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int k = t + m * TPF;
      const float2 t1o = s_t1[g * M + k];
      const float2 xo = s_x[g * M + k];
      const float2 t2 = v[m];
      float2 d1, t1;
      stripe_update(k, t2, t1o, xo, a2y, pk[m], pkn, off1, T2, T1, d1, t1);
      a.f_d1[row0 + k] = d1;
      a.f_t1[tidx(y, k, a.ny)] = t1;
    }
  }
}

template <int M, int MODE, int EV>
static int launch_row_pass_e(const RowArgs& a, cudaStream_t s) {
  using Cfg = RowPassCfg<M, EV>;
  constexpr size_t bytes = RowPassSmem<M, MODE, EV>::bytes;
  // once per instantiation and process (plans may run on several host threads)
  static std::once_flag once;
  static cudaError_t cfg_err = cudaSuccess;
  std::call_once(once, [] {
    cfg_err = cudaFuncSetAttribute(row_pass_kernel<M, MODE, EV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)bytes);
  });
  if (cfg_err != cudaSuccess) return (int)cfg_err;
  const dim3 grid((a.ny + Cfg::ROWS - 1) / Cfg::ROWS), block(Cfg::THREADS);
  return launch_pdl(row_pass_kernel<M, MODE, EV>, grid, block, bytes, s, a);
}

// a.variant selects the shape (0 or 1, RowPassE)
template <int M, int MODE>
static int launch_row_pass(const RowArgs& a, cudaStream_t s) {
  if constexpr (RowPassE<M>::v1 != RowPassE<M>::v0) {
    if (a.variant == 1) return launch_row_pass_e<M, MODE, RowPassE<M>::v1>(a, s);
  }
  return launch_row_pass_e<M, MODE, RowPassE<M>::v0>(a, s);
}

template <int M>
static int launch_row_M(int mode, const RowArgs& a, cudaStream_t s) {
  using Cfg = RowCfg<M>;
  const dim3 grid((a.ny + Cfg::ROWS - 1) / Cfg::ROWS), block(Cfg::THREADS);
  switch (mode) {
    case ROW_PASS_RF: return launch_row_pass<M, ROW_PASS_RF>(a, s);
    case ROW_PASS_NORF: return launch_row_pass<M, ROW_PASS_NORF>(a, s);
    case ROW_RESID_B: return launch_pdl(row_kernel<M, ROW_RESID_B>, grid, block, 0, s, a);
    case ROW_RESID_D: return launch_pdl(row_kernel<M, ROW_RESID_D>, grid, block, 0, s, a);
    case ROW_C2R: return launch_pdl(row_kernel<M, ROW_C2R>, grid, block, 0, s, a);
    case ROW_R2C: return launch_pdl(row_kernel<M, ROW_R2C>, grid, block, 0, s, a);
    default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

int launch_row(int mode, const RowArgs& a, cudaStream_t s) {
  switch (a.nx / 2) {
    case 16: return launch_row_M<16>(mode, a, s);
    case 32: return launch_row_M<32>(mode, a, s);
    case 64: return launch_row_M<64>(mode, a, s);
    case 128: return launch_row_M<128>(mode, a, s);
    case 256: return launch_row_M<256>(mode, a, s);
    case 192: return launch_row_M<192>(mode, a, s);
    case 384: return launch_row_M<384>(mode, a, s);
    case 512: return launch_row_M<512>(mode, a, s);
    case 768: return launch_row_M<768>(mode, a, s);
    case 1024: return launch_row_M<1024>(mode, a, s);
    case 2048: return launch_row_M<2048>(mode, a, s);
    default: return (int)cudaErrorInvalidValue;
  }
}

template <int M>
static int rows_per_cta() { return RowCfg<M>::ROWS; }

int row_grid(int nx, int ny) {
  int r = 1;
  switch (nx / 2) {
    case 16: r = rows_per_cta<16>(); break;
    case 32: r = rows_per_cta<32>(); break;
    case 64: r = rows_per_cta<64>(); break;
    case 128: r = rows_per_cta<128>(); break;
    case 256: r = rows_per_cta<256>(); break;
    case 192: r = rows_per_cta<192>(); break;
    case 384: r = rows_per_cta<384>(); break;
    case 512: r = rows_per_cta<512>(); break;
    case 768: r = rows_per_cta<768>(); break;
    case 1024: r = rows_per_cta<1024>(); break;
    case 2048: r = rows_per_cta<2048>(); break;
    default: r = 1;
  }
  return (ny + r - 1) / r;
}

template <int M>
static int row_e(int v) { return v == 1 ? RowPassE<M>::v1 : RowPassE<M>::v0; }

int row_pass_e(int M, int v) {
  switch (M) {
    case 16: return row_e<16>(v);
    case 32: return row_e<32>(v);
    case 64: return row_e<64>(v);
    case 128: return row_e<128>(v);
    case 192: return row_e<192>(v);
    case 256: return row_e<256>(v);
    case 384: return row_e<384>(v);
    case 512: return row_e<512>(v);
    case 768: return row_e<768>(v);
    case 1024: return row_e<1024>(v);
    case 2048: return row_e<2048>(v);
    default: return 0;
  }
}

bool size_supported(int n) {
  // powers of two from 32 to 4096, and 384, 768, 1536 (3 * 2^k, one radix-3 stage)
  return (n >= 32 && n <= 4096 && (n & (n - 1)) == 0) || n == 384 || n == 768 || n == 1536;
}

}  // namespace wf
