// wf_cols.cu -- the column pass of the messenger iteration and the column
// steps of the residual (Huffenberger 2017, Sec. 2).
//
// One CTA owns W adjacent complex columns (kx) of a row-transformed field;
// TPC = ny/E threads per column run a complex length-ny Stockham FFT in shared
// memory, which completes the 2D DFT.  The 2D-Fourier updates -- eqs.
// (2mess_d0), (2mess_t0) and (2mess_s) analogues: the 1/f part and the signal
// prior, both diagonal there -- run between the forward and the inverse
// column transform.  s is never stored: it is C t0 / (C + T_0) (eq. 2mess_s),
// recomputed with the T_0 in force when t0 was made.
//
// Column 0 packs the two real-signal columns kx = 0 and kx = nx/2 as
// Z = A + i B; after the column DFT, A[ky] = (Z[ky] + conj Z[-ky])/2 and
// B[ky] = (Z[ky] - conj Z[-ky])/(2i), which the updates treat as separate
// modes with their own eigenvalues.
#include "wf_device.cuh"
#include "wf_internal.h"

namespace wf {

template <int L>
struct ColCfg {
  static constexpr int E = (L >= 2048) ? 16 : 8;
  static constexpr int TPC = L / E;
  static constexpr int W0 = 256 / TPC;
  static constexpr int W = W0 < 1 ? 1 : (W0 > 32 ? 32 : W0);
  static constexpr int THREADS = W * TPC;
  // Stride between the per-column FFT buffers (complex values): a half-warp
  // covers W columns x 16/W consecutive indices, which are bank-conflict free
  // when the stride is congruent to 16/W modulo 16 (odd for W = 32).
  static constexpr int SP = SPad<L>::size;
  static constexpr int WANT = (W >= 32) ? 1 : (16 / W) % 16;
  static constexpr int STRIDE = SP + ((WANT - SP % 16) + 16) % 16;
};

__device__ __forceinline__ void unpack_pair(float2 Z, float2 Zp, float2& A, float2& B) {
  const float2 cz = cconj(Zp);
  A = cscale(cadd(Z, cz), 0.5f);
  const float2 D = cscale(csub(Z, cz), 0.5f);
  B = make_float2(D.y, -D.x);
}
__device__ __forceinline__ float2 repack_pair(float2 A, float2 B) {
  return make_float2(A.x - B.y, A.y + B.x);
}

// 2D-Fourier updates of one mode (real coefficients, complex values).
//   y    : data-side messenger (t_RF, or t_PX without stripes), this basis
//   t0o  : stored t_2DF;  C, P: signal and 1/f eigenvalues
// returns d_2DF and writes the new t_2DF
__device__ __forceinline__ float2 mode_2df(float2 yv, float2 t0o, float C, float P, float off0,
                                           float Tl, float T0, float T0s, float2& t0n) {
  const float nb0 = P + off0;                           // Nbar_2DF
  const float ws = __fdividef(C, C + T0s);              // s = C t0 / (C + T0)
  const float2 so = cscale(t0o, ws);
  const float wd = __fdividef(nb0, nb0 + Tl);          // d0 = (Nb y + Tl t0)/(Nb + Tl)
  const float2 d0 = make_float2(fmaf(wd, yv.x - t0o.x, t0o.x), fmaf(wd, yv.y - t0o.y, t0o.y));
  const float wt = __fdividef(nb0, nb0 + T0);          // t0 = (T0 d0 + Nb s)/(Nb + T0)
  t0n = make_float2(fmaf(wt, so.x - d0.x, d0.x), fmaf(wt, so.y - d0.y, d0.y));
  return d0;
}

template <int L, int MODE>
__global__ void __launch_bounds__(ColCfg<L>::THREADS)
col_kernel(ColArgs a) {
  using Cfg = ColCfg<L>;
  constexpr int E = Cfg::E, TPC = Cfg::TPC, W = Cfg::W;
  __shared__ float2 sbuf[W][Cfg::STRIDE];
  pdl_trigger();
  pdl_wait();

  const int c = threadIdx.x % W;
  const int t = threadIdx.x / W;
  const int ncols = a.nx / 2;
  const int col = blockIdx.x * W + c;
  const bool valid = col < ncols;
  const int colv = valid ? col : 0;
  float2* sb = sbuf[c];

  if (a.check_done && a.st->done) return;  // uniform: set only between launches

  auto at = [&](int k) -> size_t { return (size_t)k * ncols + colv; };       // row-major
  auto att = [&](int k) -> size_t { return tidx(k, colv, a.ny); };           // column-tiled
  float2 v[E];

  // Partner value Z[-k] of column 0 (only meaningful where col == 0).  Every
  // thread of CTA 0 takes part in the exchange; CTA 0 is uniform.
  auto exchange0 = [&](float2 (&u)[E], float2 (&up)[E]) {
#pragma unroll
    for (int m = 0; m < E; ++m) sb[spad(t + m * TPC)] = u[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int k = t + m * TPC;
      up[m] = sb[spad((L - k) & (L - 1))];
    }
    __syncthreads();
  };

  if constexpr (MODE == COL_RESID_A) {
    // g = S^-1 s and s = C g in RF, for the residual and the export of s:
    // from the data-side messenger (merged 2DF block, or no 1/f part), or
    // g = t0 / (C + T0) from the stored t_2DF (plain sweep)
    float2 vp[E];
    const float sc = 1.0f / (float)L;
    if (!a.has_f || a.merge) {
      // From the data-side messenger y that the last column pass used:
      // s = C/(C + N0 + T) y and g = S^-1 s = y/(C + N0 + T), with N0 = 0
      // without a 1/f part.  Forming g from y (not from the stored, high-k
      // suppressed d_2DF or s) keeps FP32 rounding out of the 1/C factor.
      const float Tl = a.has_rf ? a.st->Tf[1] : a.st->Tf[2];
      const float off0 = (float)a.st->off[0];
      float2 w[E];
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = valid ? a.f_y[att(t + m * TPC)] : make_float2(0.f, 0.f);
      fft_block<L, E, false>(v, sb, t, a.twy, 1);
      if (blockIdx.x == 0) exchange0(v, vp);
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const int k = t + m * TPC;
        const float2 eg = valid ? a.eig[att(k)] : make_float2(1.f, 1.f);
        // with a source j: g = (y + (N0 + T) j^) / (C + N0 + T)
        const float2 jv = (a.src != nullptr && valid) ? a.src[att(k)] : make_float2(0.f, 0.f);
        if (blockIdx.x == 0 && c == 0) {
          const float2 egb = a.eig_nyq[k];
          const float2 jp = (a.src != nullptr) ? a.src[att((L - k) & (L - 1))] : make_float2(0.f, 0.f);
          float2 A, B, JA, JB;
          unpack_pair(v[m], vp[m], A, B);
          unpack_pair(jv, jp, JA, JB);
          const float na = eg.y + off0 + Tl, nb = egb.y + off0 + Tl;
          const float2 gA = cscale(make_float2(fmaf(na, JA.x, A.x), fmaf(na, JA.y, A.y)), __fdividef(1.f, eg.x + na));
          const float2 gB = cscale(make_float2(fmaf(nb, JB.x, B.x), fmaf(nb, JB.y, B.y)), __fdividef(1.f, egb.x + nb));
          v[m] = repack_pair(gA, gB);
          w[m] = repack_pair(cscale(gA, eg.x), cscale(gB, egb.x));
        } else {
          const float na = eg.y + off0 + Tl;
          const float2 g = cscale(make_float2(fmaf(na, jv.x, v[m].x), fmaf(na, jv.y, v[m].y)),
                                  __fdividef(1.f, eg.x + na));
          v[m] = g;
          w[m] = cscale(g, eg.x);
        }
      }
      fft_block<L, E, true>(v, sb, t, a.twy, 1);
      fft_block<L, E, true>(w, sb, t, a.twy, 1);
      if (valid) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
          a.r_g[at(t + m * TPC)] = cscale(v[m], sc);
          a.r_q[at(t + m * TPC)] = cscale(w[m], sc);
        }
      }
    } else if (a.has_f) {
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = valid ? a.f_t0[at(t + m * TPC)] : make_float2(0.f, 0.f);
      const float T0s = a.st->T0s[a.parity];
      float2 w[E];
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const int k = t + m * TPC;
        const float2 eg = valid ? a.eig[att(k)] : make_float2(1.f, 1.f);
        if (blockIdx.x == 0 && c == 0) {
          const int kp = (L - k) & (L - 1);
          const float2 egb = a.eig_nyq[k];
          float2 A, B;
          unpack_pair(v[m], a.f_t0[at(kp)], A, B);
          const float ia = __fdividef(1.f, eg.x + T0s), ib = __fdividef(1.f, egb.x + T0s);
          const float2 gA = cscale(A, ia), gB = cscale(B, ib);
          v[m] = repack_pair(gA, gB);
          w[m] = repack_pair(cscale(gA, eg.x), cscale(gB, egb.x));
        } else {
          const float2 g = cscale(v[m], __fdividef(1.f, eg.x + T0s));
          v[m] = g;
          w[m] = cscale(g, eg.x);
        }
      }
      fft_block<L, E, true>(v, sb, t, a.twy, 1);
      fft_block<L, E, true>(w, sb, t, a.twy, 1);
      if (valid) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
          a.r_g[at(t + m * TPC)] = cscale(v[m], sc);
          a.r_q[at(t + m * TPC)] = cscale(w[m], sc);
        }
      }
    }
  } else if constexpr (MODE == COL_RESID_C) {
    // q += N_2DF g'  (the given 1/f eigenvalues)
    float2 vp[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = valid ? a.r_g[at(t + m * TPC)] : make_float2(0.f, 0.f);
    fft_block<L, E, false>(v, sb, t, a.twy, 1);
    if (blockIdx.x == 0) exchange0(v, vp);
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int k = t + m * TPC;
      const float2 eg = valid ? a.eig[att(k)] : make_float2(0.f, 0.f);
      if (blockIdx.x == 0 && c == 0) {
        float2 A, B;
        unpack_pair(v[m], vp[m], A, B);
        v[m] = repack_pair(cscale(A, eg.y), cscale(B, a.eig_nyq[k].y));
      } else {
        v[m] = cscale(v[m], eg.y);
      }
    }
    fft_block<L, E, true>(v, sb, t, a.twy, 1);
    const float sc = 1.0f / (float)L;
    if (valid) {
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const size_t i = at(t + m * TPC);
        const float2 q = a.r_q[i];
        a.r_q[i] = make_float2(fmaf(v[m].x, sc, q.x), fmaf(v[m].y, sc, q.y));
      }
    }
  } else if constexpr (MODE == COL_G_FROM_S) {
    // residual of a given s: r_q holds s in RF (kept); r_g <- S^-1 s in RF
    float2 vp[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = valid ? a.r_q[at(t + m * TPC)] : make_float2(0.f, 0.f);
    fft_block<L, E, false>(v, sb, t, a.twy, 1);
    if (blockIdx.x == 0) exchange0(v, vp);
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int k = t + m * TPC;
      const float2 eg = valid ? a.eig[att(k)] : make_float2(1.f, 1.f);
      if (blockIdx.x == 0 && c == 0) {
        float2 A, B;
        unpack_pair(v[m], vp[m], A, B);
        v[m] = repack_pair(cscale(A, __fdividef(1.f, eg.x)), cscale(B, __fdividef(1.f, a.eig_nyq[k].x)));
      } else {
        v[m] = cscale(v[m], __fdividef(1.f, eg.x));
      }
    }
    fft_block<L, E, true>(v, sb, t, a.twy, 1);
    const float sc = 1.0f / (float)L;
    if (valid) {
#pragma unroll
      for (int m = 0; m < E; ++m) a.r_g[at(t + m * TPC)] = cscale(v[m], sc);
    }
  } else if constexpr (MODE == COL_UNTILE) {
    if (valid) {
#pragma unroll
      for (int m = 0; m < E; ++m) a.out[at(t + m * TPC)] = a.in[att(t + m * TPC)];
    }
  } else if constexpr (MODE == COL_FWD || MODE == COL_INV || MODE == COL_FWD_TILED) {
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = valid ? a.in[at(t + m * TPC)] : make_float2(0.f, 0.f);
    fft_block<L, E, MODE == COL_INV>(v, sb, t, a.twy, 1);
    const float sc = (MODE == COL_INV) ? 1.0f / (float)L : 1.0f;
    if (valid) {
#pragma unroll
      for (int m = 0; m < E; ++m) {
        if constexpr (MODE == COL_FWD_TILED) a.out[att(t + m * TPC)] = cscale(v[m], sc);
        else a.out[at(t + m * TPC)] = cscale(v[m], sc);
      }
    }
  }
}


// Column pass geometry: W columns per CTA, TPC = L/E threads per column.
// W is a whole number of column tiles (TMA bulk loads of contiguous tiles)
// unless the tiles would not fit in shared memory, then half a tile.
#ifndef WF_COL_E
#define WF_COL_E 0  // 0: the default choice below; else values per thread (4, 8, 16)
#endif
constexpr size_t kMaxSmem = 227 * 1024;  // dynamic shared memory per CTA

template <int L, int MODE>
struct ColPassCfg {
  static constexpr bool T0 = (MODE == COL_PASS_2DF);
  static constexpr bool SRC = (MODE == COL_PASS_MERGE_SRC);
  static constexpr bool EXTRA = T0 || SRC;  // a third staged tile
  static constexpr int E = (WF_COL_E > 0 && WF_COL_E <= L / 2) ? WF_COL_E : ((L >= 512) ? 16 : 8);
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
  // the twiddle table (L values) is staged too when it still fits
  static constexpr bool TWS = tw_off + (size_t)L * 8 + fft_bytes <= kMaxSmem;
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
template <int L, int MODE>
__device__ __forceinline__ void stage_tiled(float2* dst, const float2* src, int col0, int ny, uint64_t* bar) {
  using Cfg = ColPassCfg<L, MODE>;
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

// The column pass (Sec. 2 / Appendix A: the 2D-Fourier updates between the
// forward and inverse column DFTs).  The messenger tile and the (C, P1f)
// tile are staged in shared memory before the transform begins.
template <int L, int MODE>
__global__ void __launch_bounds__(ColPassCfg<L, MODE>::THREADS)
col_pass_kernel(ColArgs a) {
  using Cfg = ColPassCfg<L, MODE>;
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
  stage_tiled<L, MODE>(s_eig, a.eig, col0, a.ny, &bar[1]);
  if constexpr (Cfg::TWS)
    if (threadIdx.x == 0) bulk_g2s(s_tw, a.twy, (uint32_t)(L * 8), &bar[1]);
  cp_async_commit();
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
  stage_tiled<L, MODE>(s_y, a.f_y, col0, a.ny, &bar[0]);
  cp_async_commit();
  if constexpr (Cfg::SRC) stage_tiled<L, MODE>(s_t0, a.src, col0, a.ny, &bar[0]);
  if constexpr (Cfg::T0) tile_load_rowmajor<L, W, Cfg::THREADS>(s_t0, a.f_t0, col0, ncols);
  cp_async_commit();
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

  float2 v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = s_y[Cfg::sidx(t + m * TPC, c)];
  fft_block<L, E, false, false, Cfg::TWS>(v, sb, t, Cfg::TWS ? s_tw : a.twy, 1);

  // partner values Z[-k] for the packed column 0 (CTA 0 only; uniform)
  float2 vp[E];
  if (blockIdx.x == 0) {
#pragma unroll
    for (int m = 0; m < E; ++m) sb[spad(t + m * TPC)] = v[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; ++m) vp[m] = sb[spad((L - (t + m * TPC)) & (L - 1))];
    __syncthreads();
  }
  cp_async_wait<0>();
  __syncthreads();

#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int k = t + m * TPC;
    const float2 eg = s_eig[Cfg::sidx(k, c)];
    if constexpr (MODE == COL_PASS_MERGE) {
      // joint update of the 2DF block given y (Appendix A shortcut):
      // d_2DF = (C + N0)/(C + N0 + T) y, s = C/(C + N0) d_2DF implicit
      const float pa = eg.x + eg.y + off0;
      if (packed) {
        const float2 egb = egn[m];
        const float pb = egb.x + egb.y + off0;
        float2 A, B;
        unpack_pair(v[m], vp[m], A, B);
        v[m] = repack_pair(cscale(A, __fdividef(pa, pa + Tl)), cscale(B, __fdividef(pb, pb + Tl)));
      } else {
        v[m] = cscale(v[m], __fdividef(pa, pa + Tl));
      }
    } else if constexpr (MODE == COL_PASS_MERGE_SRC) {
      // the same block with a source j in the objective (-2 s.j): the joint
      // minimiser is d_2DF = ((C + N0) y + T C j^) / (C + N0 + T)
      const float pa = eg.x + eg.y + off0;
      const float2 jv = s_t0[Cfg::sidx(k, c)];
      if (packed) {
        const float2 egb = egn[m];
        const float pb = egb.x + egb.y + off0;
        const float2 jp = s_t0[Cfg::sidx((L - k) & (L - 1), c)];
        float2 A, B, JA, JB;
        unpack_pair(v[m], vp[m], A, B);
        unpack_pair(jv, jp, JA, JB);
        const float ia = __fdividef(1.f, pa + Tl), ib = __fdividef(1.f, pb + Tl);
        const float2 dA = make_float2((pa * A.x + Tl * eg.x * JA.x) * ia, (pa * A.y + Tl * eg.x * JA.y) * ia);
        const float2 dB = make_float2((pb * B.x + Tl * egb.x * JB.x) * ib, (pb * B.y + Tl * egb.x * JB.y) * ib);
        v[m] = repack_pair(dA, dB);
      } else {
        const float ia = __fdividef(1.f, pa + Tl);
        v[m] = make_float2((pa * v[m].x + Tl * eg.x * jv.x) * ia, (pa * v[m].y + Tl * eg.x * jv.y) * ia);
      }
    } else if constexpr (MODE == COL_PASS_2DF) {
      const float2 t0o = s_t0[k * W + c];
      float2 t0n, d0;
      if (packed) {
        const float2 egb = egn[m];
        const float2 t0p = s_t0[((L - k) & (L - 1)) * W + c];
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
  fft_block<L, E, true, false, Cfg::TWS>(v, sb, t, Cfg::TWS ? s_tw : a.twy, 1);
  if constexpr (!WF_PDL_EARLY) pdl_trigger();
  const float sc = 1.0f / (float)L;
#pragma unroll
  for (int m = 0; m < E; ++m) a.f_x[tidx(t + m * TPC, col, a.ny)] = cscale(v[m], sc);
}

template <int L, int MODE>
static int launch_col_pass(const ColArgs& a, cudaStream_t s) {
  using Cfg = ColPassCfg<L, MODE>;
  const int ncols = a.nx / 2;
  if (ncols % Cfg::W != 0) return (int)cudaErrorInvalidValue;
  constexpr size_t kBytes = Cfg::bytes;
  static bool configured = false;  // per instantiation
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(col_pass_kernel<L, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBytes);
    if (e != cudaSuccess) return (int)e;
    configured = true;
  }
  const dim3 grid(ncols / Cfg::W), block(Cfg::THREADS);
  return launch_pdl(col_pass_kernel<L, MODE>, grid, block, kBytes, s, a);
}

template <int L>
static int launch_col_L(int mode, const ColArgs& a, cudaStream_t s) {
  using Cfg = ColCfg<L>;
  const int ncols = a.nx / 2;
  const dim3 grid((ncols + Cfg::W - 1) / Cfg::W), block(Cfg::THREADS);
  switch (mode) {
    case COL_PASS_2DF: return launch_col_pass<L, COL_PASS_2DF>(a, s);
    case COL_PASS_NO2DF: return launch_col_pass<L, COL_PASS_MERGE>(a, s);  // same update with N0 = 0
    case COL_RESID_A: return launch_pdl(col_kernel<L, COL_RESID_A>, grid, block, 0, s, a);
    case COL_RESID_C: return launch_pdl(col_kernel<L, COL_RESID_C>, grid, block, 0, s, a);
    case COL_FWD: return launch_pdl(col_kernel<L, COL_FWD>, grid, block, 0, s, a);
    case COL_INV: return launch_pdl(col_kernel<L, COL_INV>, grid, block, 0, s, a);
    case COL_PASS_MERGE: return launch_col_pass<L, COL_PASS_MERGE>(a, s);
    case COL_PASS_MERGE_SRC: return launch_col_pass<L, COL_PASS_MERGE_SRC>(a, s);
    case COL_G_FROM_S: return launch_pdl(col_kernel<L, COL_G_FROM_S>, grid, block, 0, s, a);
    case COL_UNTILE: return launch_pdl(col_kernel<L, COL_UNTILE>, grid, block, 0, s, a);
    case COL_FWD_TILED: return launch_pdl(col_kernel<L, COL_FWD_TILED>, grid, block, 0, s, a);
    default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

int launch_col(int mode, const ColArgs& a, cudaStream_t s) {
  switch (a.ny) {
    case 32: return launch_col_L<32>(mode, a, s);
    case 64: return launch_col_L<64>(mode, a, s);
    case 128: return launch_col_L<128>(mode, a, s);
    case 256: return launch_col_L<256>(mode, a, s);
    case 512: return launch_col_L<512>(mode, a, s);
    case 1024: return launch_col_L<1024>(mode, a, s);
    case 2048: return launch_col_L<2048>(mode, a, s);
    case 4096: return launch_col_L<4096>(mode, a, s);
    default: return (int)cudaErrorInvalidValue;
  }
}

}  // namespace wf
