// wf_cols.cu -- the column steps of the residual (Huffenberger 2017, Sec. 2)
// and the column transforms, plus the dispatch of every column kernel by
// column length (the column pass itself is in wf_colpass.cu).
//
// One CTA owns W adjacent complex columns (kx) of a row-transformed field;
// TPC = ny/E threads per column run a complex length-ny Stockham FFT in shared
// memory, which completes the 2D DFT.  s is never stored: it is
// C t0 / (C + T_0) (eq. 2mess_s), recomputed with the T_0 in force when t0
// was made, or C d0 / (C + N0) with the merged 2DF block.
//
// Column 0 packs the two real-signal columns kx = 0 and kx = nx/2 as
// Z = A + i B (see wf_cols_common.cuh), treated as separate modes with their
// own eigenvalues.
#include "wf_cols_common.cuh"

namespace wf {

template <int L>
struct ColCfg {
  static constexpr int E = (L % 3 == 0) ? 12 : ((L >= 2048) ? 16 : 8);
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

  // uniform: both flags are set only between launches
  if ((a.check_done && a.st->done) || (a.skip_ok && a.st->skip_resid)) return;

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
      up[m] = sb[spad(neg_mod<L>(k))];
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
          const float2 jp = (a.src != nullptr) ? a.src[att(neg_mod<L>(k))] : make_float2(0.f, 0.f);
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
          const int kp = neg_mod<L>(k);
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
  } else if constexpr (MODE == COL_WARM) {
    // warm start from s (in RF, row-major in a.in): the data-side messenger
    // gets s itself (tiled copy), the signal-side field d_2DF = (C + N_0)/C s
    // with the merged 2DF block (s = C/(C + N_0) d_2DF), or s itself
    float2 vp[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
      v[m] = valid ? a.in[at(t + m * TPC)] : make_float2(0.f, 0.f);
      if (valid) a.warm_copy[att(t + m * TPC)] = v[m];
    }
    if (a.has_f) {
      const float off0 = (float)a.st->off[0];
      fft_block<L, E, false>(v, sb, t, a.twy, 1);
      if (blockIdx.x == 0) exchange0(v, vp);
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const int k = t + m * TPC;
        const float2 eg = valid ? a.eig[att(k)] : make_float2(1.f, 0.f);
        const float fa = __fdividef(eg.x + eg.y + off0, eg.x);
        if (blockIdx.x == 0 && c == 0) {
          const float2 egb = a.eig_nyq[k];
          float2 A, B;
          unpack_pair(v[m], vp[m], A, B);
          v[m] = repack_pair(cscale(A, fa), cscale(B, __fdividef(egb.x + egb.y + off0, egb.x)));
        } else {
          v[m] = cscale(v[m], fa);
        }
      }
      fft_block<L, E, true>(v, sb, t, a.twy, 1);
      const float sc = 1.0f / (float)L;
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = cscale(v[m], sc);
    }
    if (valid) {
#pragma unroll
      for (int m = 0; m < E; ++m) a.out[att(t + m * TPC)] = v[m];
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

template <int L>
static int launch_col_L(int mode, const ColArgs& a, cudaStream_t s) {
  using Cfg = ColCfg<L>;
  const int ncols = a.nx / 2;
  const dim3 grid((ncols + Cfg::W - 1) / Cfg::W), block(Cfg::THREADS);
  switch (mode) {
    case COL_PASS_2DF:
    case COL_PASS_NO2DF:
    case COL_PASS_MERGE:
    case COL_PASS_MERGE_SRC: return launch_col_pass_any<L>(mode, a, s);
    case COL_RESID_A: return launch_pdl(col_kernel<L, COL_RESID_A>, grid, block, 0, s, a);
    case COL_RESID_C: return launch_pdl(col_kernel<L, COL_RESID_C>, grid, block, 0, s, a);
    case COL_FWD: return launch_pdl(col_kernel<L, COL_FWD>, grid, block, 0, s, a);
    case COL_INV: return launch_pdl(col_kernel<L, COL_INV>, grid, block, 0, s, a);
    case COL_G_FROM_S: return launch_pdl(col_kernel<L, COL_G_FROM_S>, grid, block, 0, s, a);
    case COL_UNTILE: return launch_pdl(col_kernel<L, COL_UNTILE>, grid, block, 0, s, a);
    case COL_FWD_TILED: return launch_pdl(col_kernel<L, COL_FWD_TILED>, grid, block, 0, s, a);
    case COL_WARM: return launch_pdl(col_kernel<L, COL_WARM>, grid, block, 0, s, a);
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
    case 384: return launch_col_L<384>(mode, a, s);
    case 512: return launch_col_L<512>(mode, a, s);
    case 768: return launch_col_L<768>(mode, a, s);
    case 1024: return launch_col_L<1024>(mode, a, s);
    case 1536: return launch_col_L<1536>(mode, a, s);
    case 2048: return launch_col_L<2048>(mode, a, s);
    case 4096: return launch_col_L<4096>(mode, a, s);
    default: return (int)cudaErrorInvalidValue;
  }
}

}  // namespace wf
