// wf_chi.cu -- the augmented objective of the messenger chain (Huffenberger
// 2017, Appendix A, eq. 2mess_prob) for the fields a plan keeps: the value
// the iteration lowers with every update (each update is the exact minimiser
// over one field), evaluated in FP64 from the FP32 fields.
//
// With the merged 2DF block the chain is s -N_0- d_0 -T- t -Nbar_RF- d_RF
// -T_PX- t_PX -Nbar_PX- d.  s and, with a stripe part, the pixel messenger
// t_PX are not stored; they are taken at their conditional means (s = C/(C +
// N_0) d_0, t_PX from d_RF and d), which turns their terms into
//   |d_0|^2 / (C + N_0)                       (2D Fourier basis)
//   |d - d_RF|^2 / (Nbar_PX + T_PX)            (pixels, unmasked)
// and leaves the stored links
//   |t - d_0|^2 / T,  |d_RF - t|^2 / Nbar_RF   (row basis)
// Without a stripe part t = t_PX is stored and its data link is
// |d - t_PX|^2 / Nbar_PX.  Sums over a basis use Parseval with the
// unnormalised transforms: sum_px x^2 = (1/n) sum_k |X_k|^2, the half
// spectra counting the modes 1 .. n/2 - 1 twice.
#include "wf_cols_common.cuh"

namespace wf {

struct ChiArgs {
  int ny, nx;
  int has_rf;
  const float2* d0;       // d_2DF (s without a 1/f part) in RF, column-tiled
  const float2* t;        // its data-side neighbour in RF, column-tiled: t_RF or t_PX
  const float2* d1;       // d_RF, row-major (stripe part) or nullptr
  const float4* dn;       // pixel pairs (d0, nb0, d1, nb1); nb < 0 = masked
  const float2* eig;      // (C, P1f), column-tiled
  const float2* eig_nyq;  // (C, P1f) at kx = nx/2
  const float* pst;       // [nx/2 + 1] stripe eigenvalues
  const float* a2;        // [ny] a(y)^2
  const float2* twx;      // exp(-2 pi i k/nx)
  const float2* twy;      // exp(-2 pi i k/ny)
  const WfState* st;
  double* part_col;       // per-CTA partials of the column kernel
  double* part_row;       // per-CTA partials of the row kernel
  double* out;            // the sum
};

namespace {

template <int NT>
__device__ __forceinline__ double cta_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (NT + 31) / 32; ++i) s += red[i];
  return s;
}

template <int L>
struct ChiColCfg {
  static constexpr int E = (L % 3 == 0) ? 12 : ((L >= 2048) ? 16 : 8);
  static constexpr int TPC = L / E;
  static constexpr int W0 = 256 / TPC;
  static constexpr int W = W0 < 1 ? 1 : (W0 > 32 ? 32 : W0);
  static constexpr int THREADS = W * TPC;
  static constexpr int STRIDE = SPad<L>::size + 1;
};

template <int M>
struct ChiRowCfg {
  static constexpr int E = (M % 3 == 0) ? 12 : ((M >= 2048) ? 16 : 8);
  static constexpr int TPF = M / E;
  static constexpr int ROWS = (256 / TPF) >= 1 ? (256 / TPF) : 1;
  static constexpr int THREADS = ROWS * TPF;
};

// The 2D-Fourier term and the row-basis terms, W complex columns per CTA.
template <int L>
__global__ void __launch_bounds__(ChiColCfg<L>::THREADS) chi_cols_kernel(ChiArgs a) {
  using Cfg = ChiColCfg<L>;
  constexpr int E = Cfg::E, TPC = Cfg::TPC, W = Cfg::W;
  __shared__ __align__(16) float2 sbuf[W][Cfg::STRIDE];
  __shared__ double red[(Cfg::THREADS + 31) / 32];
  pdl_trigger();
  pdl_wait();
  const int c = threadIdx.x % W;
  const int t = threadIdx.x / W;
  const int ncols = a.nx / 2;
  const int col = blockIdx.x * W + c;
  const bool valid = col < ncols;
  const int colv = valid ? col : 0;
  float2* sb = sbuf[c];
  const double off0 = a.st->off[0], off1 = a.st->off[1];
  const double T = a.has_rf ? (double)a.st->Tf[1] : (double)a.st->Tf[2];

  // |d_0|^2 / (C + N_0) over the 2D spectrum: column DFT of d_0 (RF)
  float2 v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = valid ? a.d0[tidx(t + m * TPC, colv, a.ny)] : make_float2(0.f, 0.f);
  fft_block<L, E, false>(v, sb, t, a.twy, 1);
  float2 vp[E];
  if (blockIdx.x == 0) {  // uniform: partners Z[-k] of the packed column
#pragma unroll
    for (int m = 0; m < E; ++m) sb[spad(t + m * TPC)] = v[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; ++m) vp[m] = sb[spad(neg_mod<L>(t + m * TPC))];
    __syncthreads();
  }
  double s2 = 0.0, srf = 0.0;
  if (valid) {
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int k = t + m * TPC;
      const float2 eg = a.eig[tidx(k, col, a.ny)];
      if (col == 0) {  // kx = 0 (A) and kx = nx/2 (B), each counted once
        float2 A, B;
        unpack_pair(v[m], vp[m], A, B);
        const float2 egb = a.eig_nyq[k];
        s2 += ((double)A.x * A.x + (double)A.y * A.y) / ((double)eg.x + eg.y + off0);
        s2 += ((double)B.x * B.x + (double)B.y * B.y) / ((double)egb.x + egb.y + off0);
      } else {
        s2 += 2.0 * ((double)v[m].x * v[m].x + (double)v[m].y * v[m].y) / ((double)eg.x + eg.y + off0);
      }
    }
    // row-basis links, row y = k of this column; slot 0 is the real pair
    // (X_0, X_{nx/2}), counted once each
    const double wk = (col == 0) ? 1.0 : 2.0;
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int y = t + m * TPC;
      const float2 dx = a.d0[tidx(y, col, a.ny)], ty = a.t[tidx(y, col, a.ny)];
      const double ex = (double)ty.x - dx.x, ey = (double)ty.y - dx.y;
      srf += wk * (ex * ex + ey * ey) / T;
      if (a.has_rf) {
        const float2 d1 = a.d1[(size_t)y * ncols + col];
        const double fx = (double)d1.x - ty.x, fy = (double)d1.y - ty.y;
        const double ay = a.a2[y];
        if (col == 0) {
          const double nr = ay * a.pst[0] + off1, ni = ay * a.pst[ncols] + off1;
          if (nr > 0.0) srf += fx * fx / nr;
          if (ni > 0.0) srf += fy * fy / ni;
        } else {
          const double nb = ay * a.pst[col] + off1;
          if (nb > 0.0) srf += 2.0 * (fx * fx + fy * fy) / nb;
        }
      }
    }
  }
  const double part = s2 / ((double)a.ny * (double)a.nx) + srf / (double)a.nx;
  const double tot = cta_sum<Cfg::THREADS>(part, red);
  if (threadIdx.x == 0) a.part_col[blockIdx.x] = tot;
}

// The pixel term: the field next to the pixel messenger, back in pixels.
template <int M>
__global__ void __launch_bounds__(ChiRowCfg<M>::THREADS) chi_rows_kernel(ChiArgs a) {
  using Cfg = ChiRowCfg<M>;
  constexpr int E = Cfg::E, TPF = Cfg::TPF, ROWS = Cfg::ROWS;
  __shared__ __align__(16) float2 sbuf[ROWS][SPad<M>::size];
  __shared__ double red[(Cfg::THREADS + 31) / 32];
  pdl_trigger();
  pdl_wait();
  const int g = threadIdx.x / TPF;
  const int t = threadIdx.x - g * TPF;
  const int y = blockIdx.x * ROWS + g;
  const bool valid = y < a.ny;
  const int yv = valid ? y : 0;
  float2* sb = sbuf[g];
  float2 v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int k = t + m * TPF;
    v[m] = !valid ? make_float2(0.f, 0.f) : (a.has_rf ? a.d1[(size_t)yv * M + k] : a.t[tidx(yv, k, a.ny)]);
  }
  c2r_pre<M, E>(v, sb, t, a.twx);
  fft_block<M, E, true>(v, sb, t, a.twx, 2);
  const double T2 = (double)a.st->Tf[2];
  double acc = 0.0;
  if (valid) {
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const float4 q = a.dn[(size_t)y * M + t + m * TPF];
      const float dv[2] = {q.x, q.z}, nv[2] = {q.y, q.w}, uv[2] = {v[m].x, v[m].y};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (nv[h] < 0.f) continue;  // masked: Nbar = inf
        const double e = (double)dv[h] - uv[h];
        if (a.has_rf) acc += e * e / ((double)nv[h] + T2);
        else if (nv[h] > 0.f) acc += e * e / (double)nv[h];  // Nbar = 0 pins t_PX = d
      }
    }
  }
  const double tot = cta_sum<Cfg::THREADS>(acc, red);
  if (threadIdx.x == 0) a.part_row[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(256) chi_fin_kernel(ChiArgs a, int ncol, int nrow) {
  __shared__ double red[8];
  pdl_trigger();
  pdl_wait();
  double s = 0.0;
  for (int i = threadIdx.x; i < ncol; i += blockDim.x) s += a.part_col[i];
  for (int i = threadIdx.x; i < nrow; i += blockDim.x) s += a.part_row[i];
  s = cta_sum<256>(s, red);
  if (threadIdx.x == 0) a.out[0] = s;
}

// launch = false only reports the grid size
template <int L>
int cols_L(const ChiArgs& a, cudaStream_t s, int* grid, bool launch) {
  using Cfg = ChiColCfg<L>;
  *grid = (a.nx / 2 + Cfg::W - 1) / Cfg::W;
  if (!launch) return 0;
  return launch_pdl(chi_cols_kernel<L>, dim3(*grid), dim3(Cfg::THREADS), 0, s, a);
}

template <int M>
int rows_M(const ChiArgs& a, cudaStream_t s, int* grid, bool launch) {
  using Cfg = ChiRowCfg<M>;
  *grid = (a.ny + Cfg::ROWS - 1) / Cfg::ROWS;
  if (!launch) return 0;
  return launch_pdl(chi_rows_kernel<M>, dim3(*grid), dim3(Cfg::THREADS), 0, s, a);
}

int cols_any(const ChiArgs& a, cudaStream_t s, int* grid, bool launch) {
  switch (a.ny) {
    case 32: return cols_L<32>(a, s, grid, launch);
    case 64: return cols_L<64>(a, s, grid, launch);
    case 128: return cols_L<128>(a, s, grid, launch);
    case 256: return cols_L<256>(a, s, grid, launch);
    case 384: return cols_L<384>(a, s, grid, launch);
    case 512: return cols_L<512>(a, s, grid, launch);
    case 768: return cols_L<768>(a, s, grid, launch);
    case 1024: return cols_L<1024>(a, s, grid, launch);
    case 1536: return cols_L<1536>(a, s, grid, launch);
    case 2048: return cols_L<2048>(a, s, grid, launch);
    case 4096: return cols_L<4096>(a, s, grid, launch);
    default: return (int)cudaErrorInvalidValue;
  }
}

int rows_any(const ChiArgs& a, cudaStream_t s, int* grid, bool launch) {
  switch (a.nx / 2) {
    case 16: return rows_M<16>(a, s, grid, launch);
    case 32: return rows_M<32>(a, s, grid, launch);
    case 64: return rows_M<64>(a, s, grid, launch);
    case 128: return rows_M<128>(a, s, grid, launch);
    case 192: return rows_M<192>(a, s, grid, launch);
    case 256: return rows_M<256>(a, s, grid, launch);
    case 384: return rows_M<384>(a, s, grid, launch);
    case 512: return rows_M<512>(a, s, grid, launch);
    case 768: return rows_M<768>(a, s, grid, launch);
    case 1024: return rows_M<1024>(a, s, grid, launch);
    case 2048: return rows_M<2048>(a, s, grid, launch);
    default: return (int)cudaErrorInvalidValue;
  }
}

}  // namespace

int chi2_scratch(int ny, int nx) {
  ChiArgs q{};
  q.ny = ny;
  q.nx = nx;
  int gc = 0, gr = 0;
  if (cols_any(q, nullptr, &gc, false) || rows_any(q, nullptr, &gr, false)) return 0;
  return gc + gr + 1;
}

int launch_chi2(const Chi2Fields& f, double* scratch, double* out, cudaStream_t s) {
  ChiArgs a{};
  a.ny = f.ny;
  a.nx = f.nx;
  a.has_rf = f.has_rf;
  a.d0 = f.d0;
  a.t = f.t;
  a.d1 = f.d1;
  a.dn = f.dn;
  a.eig = f.eig;
  a.eig_nyq = f.eig_nyq;
  a.pst = f.pst;
  a.a2 = f.a2;
  a.twx = f.twx;
  a.twy = f.twy;
  a.st = f.st;
  int gc = 0, gr = 0;
  int rc = cols_any(a, s, &gc, false);
  if (!rc) rc = rows_any(a, s, &gr, false);
  if (rc) return rc;
  a.part_col = scratch;
  a.part_row = scratch + gc;
  a.out = out;
  if ((rc = cols_any(a, s, &gc, true))) return rc;
  if ((rc = rows_any(a, s, &gr, true))) return rc;
  return launch_pdl(chi_fin_kernel, dim3(1), dim3(256), 0, s, a, gc, gr);
}

}  // namespace wf
