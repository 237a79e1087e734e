// wf_ctrl.cu -- setup of one problem and the lambda controller.
//
// Setup (Huffenberger 2017, Sec. 2 and Appendix A): validate the inputs,
// find the minimum eigenvalue of each noise part, set tau_i = theta_i x that
// minimum (optionally after moving a white floor between parts, which leaves
// N unchanged), and lay out the per-pixel and per-mode tables the passes read.
//
// Controller (Sec. 2 cooling, Sec. 3.3 adaptive rule): after each residual
// evaluation, one CTA sums the per-CTA FP64 partials in a fixed order, forms
// ||Delta d_u|| / ||d_u|| and ||(S^-1 s)_m|| / ||S^-1 s||, applies the stop
// test and moves lambda.  Everything stays on the device; the host only polls
// the done flag.
#include <math.h>

#include "wf_device.cuh"
#include "wf_internal.h"

namespace wf {

constexpr int SETUP_CTAS = 256;
constexpr int SETUP_THREADS = 256;

__device__ __forceinline__ bool finite_pos(float x) { return isfinite(x) && x > 0.f; }

template <int NT>
__device__ double block_min(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double r = INFINITY;
  if (threadIdx.x == 0)
    for (int i = 0; i < NT / 32; ++i) r = fmin(r, red[i]);
  return r;
}

template <int NT>
__device__ double block_add(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < NT / 32; ++i) r += red[i];
  return r;
}

// pixel statistics: min unmasked variance, unmasked count, validity
__global__ void __launch_bounds__(SETUP_THREADS) setup_px(SetupArgs a) {
  __shared__ double red[SETUP_THREADS / 32];
  const size_t n = (size_t)a.ny * a.nx;
  double vmin = INFINITY, cnt = 0.0;
  unsigned err = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const bool masked = a.mask != nullptr && a.mask[i] != 0;
    if (masked) continue;
    const float v = a.var[i];
    const float dv = a.d[i];
    if (!finite_pos(v)) err |= WF_ERR_VAR;
    if (!isfinite(dv)) err |= WF_ERR_D_NONFINITE;
    vmin = fmin(vmin, (double)v);
    cnt += 1.0;
  }
  if (err) atomicOr(&a.st->err, err);
  double m = block_min<SETUP_THREADS>(vmin, red);
  double c = block_add<SETUP_THREADS>(cnt, red);
  if (threadIdx.x == 0) {
    a.part[blockIdx.x] = m;
    a.part[SETUP_CTAS + blockIdx.x] = c;
  }
}

// spectral tables, validity, min of the 1/f eigenvalues
__global__ void __launch_bounds__(SETUP_THREADS) setup_spec(SetupArgs a) {
  __shared__ double red[SETUP_THREADS / 32];
  const int h = a.nx / 2;
  const size_t n = (size_t)a.ny * (h + 1);
  double fmin_ = INFINITY;
  unsigned err = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int ky = (int)(i / (h + 1));
    const int kx = (int)(i - (size_t)ky * (h + 1));
    const float C = a.C[i];
    const float P = a.has_f ? a.P1f[i] : 0.f;
    if (!finite_pos(C)) err |= WF_ERR_C;
    if (a.has_f) {
      if (!finite_pos(P)) err |= WF_ERR_P1F;
      fmin_ = fmin(fmin_, (double)P);
    }
    if (kx == 0 || kx == h) {
      // a real covariance needs e(ky, kx) = e(-ky, kx) on these two columns
      const size_t j = (size_t)((a.ny - ky) % a.ny) * (h + 1) + kx;
      if (a.C[j] != C) err |= WF_ERR_ASYM;
      if (a.has_f && a.P1f[j] != P) err |= WF_ERR_ASYM;
    }
    if (kx < h) a.eig[tidx(ky, kx, a.ny)] = make_float2(C, P);  // column-tiled
    else a.eig_nyq[ky] = make_float2(C, P);
  }
  if (err) atomicOr(&a.st->err, err);
  double m = block_min<SETUP_THREADS>(fmin_, red);
  if (threadIdx.x == 0) a.part[2 * SETUP_CTAS + blockIdx.x] = m;
}

// one CTA: combine the minima, set tau_i and the offsets
__global__ void __launch_bounds__(SETUP_THREADS) setup_fin(SetupArgs a) {
  __shared__ double red[SETUP_THREADS / 32];
  WfState* st = a.st;
  double vmin = INFINITY, cnt = 0.0, fmin_ = INFINITY, smin = INFINITY, amin = INFINITY;
  unsigned err = 0;
  for (int i = threadIdx.x; i < SETUP_CTAS; i += blockDim.x) {
    vmin = fmin(vmin, a.part[i]);
    cnt += a.part[SETUP_CTAS + i];
    fmin_ = fmin(fmin_, a.part[2 * SETUP_CTAS + i]);
  }
  const int h = a.nx / 2;
  if (a.has_rf) {
    for (int k = threadIdx.x; k <= h; k += blockDim.x) {
      const float p = a.Pst[k];
      if (!finite_pos(p)) err |= WF_ERR_PST;
      smin = fmin(smin, (double)p);
      a.pst[k] = p;
    }
    for (int y = threadIdx.x; y < a.ny; y += blockDim.x) {
      const float q = a.a2 ? a.a2[y] : 1.f;
      if (!finite_pos(q)) err |= WF_ERR_A2;
      amin = fmin(amin, (double)q);
      a.a2_out[y] = q;
    }
  }
  if (err) atomicOr(&st->err, err);
  vmin = block_min<SETUP_THREADS>(vmin, red);
  cnt = block_add<SETUP_THREADS>(cnt, red);
  fmin_ = block_min<SETUP_THREADS>(fmin_, red);
  smin = block_min<SETUP_THREADS>(smin, red);
  amin = block_min<SETUP_THREADS>(amin, red);
  if (threadIdx.x == 0) {
    if (cnt < 0.5) st->err |= WF_ERR_ALLMASKED;
    st->n_unmasked = (int)cnt;
    st->min_v = vmin;
    st->min_f = a.has_f ? fmin_ : 0.0;
    st->min_s = a.has_rf ? smin : 0.0;
    st->min_a2 = a.has_rf ? amin : 0.0;
    // white floors moved between parts (N itself is unchanged): wf_ from the
    // 1/f part to the stripe part, wfp from the 1/f part to the white part,
    // ww from the white part to the stripe part
    const double wf_ = (a.has_f && a.has_rf) ? a.split_f * fmin_ : 0.0;
    const double wfp = a.has_f ? a.split_fp * fmin_ : 0.0;
    const double ww = a.has_rf ? a.split_w * vmin : 0.0;
    // merged 2DF block: the 1/f part needs no messenger covariance
    const double t0 = (a.has_f && !a.merge) ? a.theta[0] * (fmin_ - wf_ - wfp) : 0.0;
    const double t1 = a.has_rf ? a.theta[1] * (smin * amin + wf_ + ww) : 0.0;
    const double t2 = a.theta[2] * (vmin - ww + wfp);
    st->tau[0] = t0;
    st->tau[1] = t1;
    st->tau[2] = t2;
    st->off[0] = -wf_ - wfp - t0;
    st->off[1] = wf_ + ww - t1;
    st->off[2] = wfp - ww - t2;
    st->var_shift = -(wfp - ww - t2);
    st->lam = 1.0;
    st->Tf[0] = (float)t0;
    st->Tf[1] = (float)t1;
    st->Tf[2] = (float)t2;
    st->T0s[0] = st->T0s[1] = (float)t0;
    st->done = 0;
    st->status = 0;
    st->iter = 0;
    st->checkpoints = 0;
    st->prev_rho2 = -1.0;
  }
}

// per-pixel table (d, Nbar_PX) for pixel pairs; ||d_u||^2 partials
__global__ void __launch_bounds__(SETUP_THREADS) setup_pack_px(SetupArgs a) {
  __shared__ double red[SETUP_THREADS / 32];
  const float off2 = (float)a.st->off[2];
  const size_t npair = (size_t)a.ny * a.nx / 2;
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < npair; i += (size_t)gridDim.x * blockDim.x) {
    float o[4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const size_t p = 2 * i + h;
      const bool masked = a.mask != nullptr && a.mask[p] != 0;
      const float dv = masked ? 0.f : a.d[p];
      o[2 * h] = dv;
      o[2 * h + 1] = masked ? -1.f : fmaxf(a.var[p] + off2, 0.f);
      s += (double)dv * (double)dv;
    }
    a.dn[i] = make_float4(o[0], o[1], o[2], o[3]);
  }
  double t = block_add<SETUP_THREADS>(s, red);
  if (threadIdx.x == 0) a.part[3 * SETUP_CTAS + blockIdx.x] = t;
}

__global__ void __launch_bounds__(SETUP_THREADS) setup_fin2(SetupArgs a) {
  __shared__ double red[SETUP_THREADS / 32];
  double s = 0.0;
  for (int i = threadIdx.x; i < SETUP_CTAS; i += blockDim.x) s += a.part[3 * SETUP_CTAS + i];
  s = block_add<SETUP_THREADS>(s, red);
  if (threadIdx.x == 0) a.st->du2 = s;
}

int launch_setup(const SetupArgs& a, cudaStream_t s) {
  setup_px<<<SETUP_CTAS, SETUP_THREADS, 0, s>>>(a);
  setup_spec<<<SETUP_CTAS, SETUP_THREADS, 0, s>>>(a);
  setup_fin<<<1, SETUP_THREADS, 0, s>>>(a);
  setup_pack_px<<<SETUP_CTAS, SETUP_THREADS, 0, s>>>(a);
  setup_fin2<<<1, SETUP_THREADS, 0, s>>>(a);
  return (int)cudaGetLastError();
}

// ---------------------------------------------------------------- control
__device__ __forceinline__ void set_T(WfState* st) {
  st->Tf[0] = (float)(st->lam * st->tau[0]);
  st->Tf[1] = (float)(st->lam * st->tau[1]);
  st->Tf[2] = (float)(st->lam * st->tau[2]);
}

__global__ void set_lambda_kernel(WfState* st, double lam, int reset) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st->lam = lam;
  set_T(st);
  st->skip_resid = 0;
  if (reset) {
    st->done = 0;
    st->status = 0;
    st->iter = 0;
    st->checkpoints = 0;
    st->level = 0;
    st->in_level = 0;
    st->prev_rho2 = -1.0;
    st->stall_n = 0;
    st->stall_ref = -1.0;
  }
}

// data of a defect-correction solve: the pixel table with d replaced by rho
__global__ void __launch_bounds__(SETUP_THREADS)
pack_data_kernel(float4* dn_out, const float4* dn_in, const float2* rho, size_t npair, double* part) {
  __shared__ double red[SETUP_THREADS / 32];
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < npair; i += (size_t)gridDim.x * blockDim.x) {
    const float4 q = dn_in[i];
    const float2 r = rho[i];
    const float d0 = q.y < 0.f ? 0.f : r.x, d1 = q.w < 0.f ? 0.f : r.y;
    dn_out[i] = make_float4(d0, q.y, d1, q.w);
    s += (double)d0 * d0 + (double)d1 * d1;
  }
  double t = block_add<SETUP_THREADS>(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void __launch_bounds__(SETUP_THREADS) pack_data_fin(const double* part, WfState* st) {
  __shared__ double red[SETUP_THREADS / 32];
  double s = 0.0;
  for (int i = threadIdx.x; i < SETUP_CTAS; i += blockDim.x) s += part[i];
  s = block_add<SETUP_THREADS>(s, red);
  if (threadIdx.x == 0) st->du2 = s;
}

int launch_pack_data(float4* dn_out, const float4* dn_in, const float2* rho, size_t npair, double* part,
                     WfState* st, cudaStream_t s) {
  pack_data_kernel<<<SETUP_CTAS, SETUP_THREADS, 0, s>>>(dn_out, dn_in, rho, npair, part);
  pack_data_fin<<<1, SETUP_THREADS, 0, s>>>(part, st);
  return (int)cudaGetLastError();
}

__global__ void sub_kernel(float* y, const float* x, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] -= x[i];
}

int launch_sub(float* y, const float* x, size_t n, cudaStream_t s) {
  sub_kernel<<<SETUP_CTAS, SETUP_THREADS, 0, s>>>(y, x, n);
  return (int)cudaGetLastError();
}

__global__ void fill_kernel(float* y, float v, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) y[i] = v;
}

__global__ void scale_kernel(float* y, const float* x, float a, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}

int launch_fill(float* y, float v, size_t n, cudaStream_t s) {
  fill_kernel<<<SETUP_CTAS, SETUP_THREADS, 0, s>>>(y, v, n);
  return (int)cudaGetLastError();
}

int launch_scale(float* y, const float* x, float a, size_t n, cudaStream_t s) {
  scale_kernel<<<SETUP_CTAS, SETUP_THREADS, 0, s>>>(y, x, a, n);
  return (int)cudaGetLastError();
}

int launch_set_lambda(WfState* st, double lam, int reset, cudaStream_t s) {
  set_lambda_kernel<<<1, 32, 0, s>>>(st, lam, reset);
  return (int)cudaGetLastError();
}

constexpr int CTRL_THREADS = 256;

__global__ void __launch_bounds__(CTRL_THREADS) ctrl_kernel(CtrlArgs a) {
  __shared__ double red[CTRL_THREADS / 32];
  WfState* st = a.st;
  pdl_trigger();
  pdl_wait();
  if (a.count_iters && st->done) return;
  // the residual kernels of this checkpoint returned at once (uniform: the
  // flag changes below only after every thread has read it)
  const bool skipped = a.count_iters && st->skip_resid;
  __syncthreads();
  double gm2 = 0.0, g2 = 0.0, r2 = 0.0;
  if (!skipped) {
    for (int i = threadIdx.x; i < a.nrow; i += blockDim.x) {
      gm2 += a.part_g[i];
      g2 += a.part_g2[i];
      r2 += a.part_rho[i];
    }
    gm2 = block_add<CTRL_THREADS>(gm2, red);
    g2 = block_add<CTRL_THREADS>(g2, red);
    r2 = block_add<CTRL_THREADS>(r2, red);
  }
  if (threadIdx.x != 0) return;
  if (!skipped) {
    st->gm2 = gm2;
    st->g2 = g2;
    st->rho2 = r2;
    st->rel_u = st->du2 > 0 ? sqrt(r2 / st->du2) : 0.0;
    st->rel_m = g2 > 0 ? sqrt(gm2 / g2) : 0.0;
  }
  if (!a.count_iters) return;  // residual only
  st->iter += a.R;
  st->in_level += a.R;
  st->checkpoints += 1;
  if (a.trace != nullptr) {
    // one record per checkpoint: sweeps, the lambda they ran at, the
    // residual terms, chi^2_aug, the run
    const int i = *a.trace_n;
    if (i < a.trace_cap) {
      double* r = a.trace + (size_t)WF_TRACE_FIELDS * i;
      r[0] = (double)st->iter;
      r[1] = st->lam;
      r[2] = skipped ? nan("") : st->rel_u;
      r[3] = skipped ? nan("") : st->rel_m;
      r[4] = a.chi_val != nullptr ? *a.chi_val : nan("");
      r[5] = (double)a.run_index;
      *a.trace_n = i + 1;
    }
  }
  if (!skipped && a.tol > 0 && st->lam == 1.0 && st->rel_u <= a.tol_u && st->rel_m <= a.tol) {
    st->done = 1;
    st->status = 0;
    return;
  }
  if (st->iter >= a.max_iters) {
    st->done = 1;
    st->status = a.tol > 0 ? 3 : 0;  // WF_ENOCONV
    return;
  }
  // stagnation at lambda = 1: an FP32 iteration stops improving once the
  // slow links move their fields by less than one unit in the last place
  if (a.stall > 0 && a.tol > 0 && st->lam == 1.0) {
    if (st->stall_ref <= 0.0 || r2 < 0.99 * st->stall_ref) {
      st->stall_ref = r2;
      st->stall_n = 0;
    } else if (++st->stall_n >= a.stall) {
      st->done = 1;
      st->status = 4;  // WF_ESTALL
      return;
    }
  }
  if (a.mode == 0) {
    if (st->level < a.nlevels - 1 && st->in_level >= a.it_sched[st->level]) {
      st->level += 1;
      st->lam = a.lam_sched[st->level];
      st->in_level = 0;
      st->stall_ref = -1.0;
      st->stall_n = 0;
      set_T(st);
    }
    // a fixed schedule uses the residual only at lambda = 1 (stop and stall
    // tests) and at the checkpoint that ends the run (the reported values):
    // the next checkpoint skips it otherwise
    st->skip_resid = (a.skip_fixed && st->lam > 1.0 && st->iter + a.R < a.max_iters) ? 1 : 0;
  } else if (st->lam > 1.0) {
    // Sec. 3.3: lower lambda once Delta d^T Delta d changes by less than
    // `ratio` per iteration
    if (st->prev_rho2 > 0 && r2 > 0) {
      const double rate = fabs(1.0 - pow(r2 / st->prev_rho2, 1.0 / a.R));
      if (rate < a.ratio) {
        double lam = pow(st->lam, a.expo);
        if (lam < a.snap) lam = 1.0;
        st->lam = lam;
        st->in_level = 0;
        st->prev_rho2 = -1.0;
        st->stall_ref = -1.0;
        st->stall_n = 0;
        set_T(st);
        return;
      }
    }
    st->prev_rho2 = r2;
  }
}

int launch_ctrl(const CtrlArgs& a, cudaStream_t s) {
  return launch_pdl(ctrl_kernel, dim3(1), dim3(CTRL_THREADS), 0, s, a);
}

}  // namespace wf
