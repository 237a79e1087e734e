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

// The merged 2DF block given the data-side messenger y, one mode (Appendix A
// shortcut): d_2DF = (C + N0)/(C + N0 + T) y, s = C/(C + N0) d_2DF implicit.
// With a source j in the objective (-2 s.j, defect correction) the joint
// minimiser is d_2DF = ((C + N0) y + T C j^) / (C + N0 + T).  For the packed
// column 0 (kx = 0 and kx = nx/2 as one complex column) the partner values
// at -ky (vp, jp) and the kx = nx/2 eigenvalues egb enter as well.
template <bool SRC>
__device__ __forceinline__ float2 merged_mode(float2 v, float2 vp, float2 eg, float2 egb, float off0, float Tl,
                                              bool packed, float2 jv, float2 jp) {
  const float pa = eg.x + eg.y + off0;
  if constexpr (!SRC) {
    if (packed) {
      const float pb = egb.x + egb.y + off0;
      float2 A, B;
      unpack_pair(v, vp, A, B);
      return repack_pair(cscale(A, __fdividef(pa, pa + Tl)), cscale(B, __fdividef(pb, pb + Tl)));
    }
    return cscale(v, __fdividef(pa, pa + Tl));
  } else {
    if (packed) {
      const float pb = egb.x + egb.y + off0;
      float2 A, B, JA, JB;
      unpack_pair(v, vp, A, B);
      unpack_pair(jv, jp, JA, JB);
      const float ia = __fdividef(1.f, pa + Tl), ib = __fdividef(1.f, pb + Tl);
      const float2 dA = make_float2((pa * A.x + Tl * eg.x * JA.x) * ia, (pa * A.y + Tl * eg.x * JA.y) * ia);
      const float2 dB = make_float2((pb * B.x + Tl * egb.x * JB.x) * ib, (pb * B.y + Tl * egb.x * JB.y) * ib);
      return repack_pair(dA, dB);
    }
    const float ia = __fdividef(1.f, pa + Tl);
    return make_float2((pa * v.x + Tl * eg.x * jv.x) * ia, (pa * v.y + Tl * eg.x * jv.y) * ia);
  }
}

// The column pass for one column length (wf_colpass.cu): modes COL_PASS_*.
template <int L>
int launch_col_pass_any(int mode, const ColArgs& a, cudaStream_t s);

}  // namespace wf
