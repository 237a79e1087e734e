// wf_cols_common.cuh -- pieces shared by the column pass (wf_colpass.cu) and
// the other column kernels (wf_cols.cu): the packed column-0 pair and the
// per-mode 2D-Fourier update.
#pragma once

#include "wf_device.cuh"
#include "wf_internal.h"

namespace wf {

// Column 0 packs the two real-signal columns kx = 0 and kx = nx/2 as
// Z = A + i B; after the column DFT, A[ky] = (Z[ky] + conj Z[-ky])/2 and
// B[ky] = (Z[ky] - conj Z[-ky])/(2i).
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

// The column pass for one column length (wf_colpass.cu): modes COL_PASS_*.
template <int L>
int launch_col_pass_any(int mode, const ColArgs& a, cudaStream_t s);

}  // namespace wf
