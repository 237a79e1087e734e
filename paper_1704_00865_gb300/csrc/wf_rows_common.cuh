// wf_rows_common.cuh -- the per-element updates of the row pass (Huffenberger
// 2017, Sec. 2), shared by the row pass (wf_rows.cu) and the one-launch sweep
// (wf_fused.cu) so that both compute them with the same arithmetic.
#pragma once

#include "wf_device.cuh"

namespace wf {

// t_PX update for one pixel (eq. 2mess_t1 analogue): links Nbar_PX to d and
// T_PX to u (the field on the signal side); masked pixels (nb < 0, i.e.
// Nbar = inf) take u.
__device__ __forceinline__ float tpx_update(float d, float nb, float u, float T2) {
  return nb < 0.f ? u : __fdividef(fmaf(T2, d, nb * u), nb + T2);
}

// Stripe-basis updates of one row-DFT mode k (eqs. 2mess_d0 and 2mess_t0
// analogues): d_RF between t_PX (link T_PX) and the old t_RF (link Nbar_RF),
// then t_RF between the new d_RF (link T_RF) and the signal-side field x
// (link Nbar_RF).  Mode 0 holds the real pair (kx = 0, kx = nx/2); pk0 and
// pkn are their stripe eigenvalues, pk that of mode k (times a(y)^2 by a2y);
// off1 shifts Pst to Nbar_RF.
__device__ __forceinline__ void stripe_update(int k, float2 t2, float2 t1o, float2 xo, float a2y, float pk,
                                              float pkn, float off1, float T2, float T1, float2& d1,
                                              float2& t1) {
  if (k == 0) {  // packed (kx = 0, kx = M) real pair
    const float nr = fmaf(a2y, pk, off1), ni = fmaf(a2y, pkn, off1);
    d1.x = __fdividef(fmaf(nr, t2.x, T2 * t1o.x), nr + T2);
    d1.y = __fdividef(fmaf(ni, t2.y, T2 * t1o.y), ni + T2);
    t1.x = __fdividef(fmaf(T1, d1.x, nr * xo.x), nr + T1);
    t1.y = __fdividef(fmaf(T1, d1.y, ni * xo.y), ni + T1);
  } else {
    const float nb = fmaf(a2y, pk, off1);
    const float wa = __fdividef(nb, nb + T2);      // weight of t_PX
    d1 = make_float2(fmaf(wa, t2.x - t1o.x, t1o.x), fmaf(wa, t2.y - t1o.y, t1o.y));
    const float wb = __fdividef(nb, nb + T1);      // weight of x
    t1 = make_float2(fmaf(wb, xo.x - d1.x, d1.x), fmaf(wb, xo.y - d1.y, d1.y));
  }
}

}  // namespace wf
