// wf_api.cu -- host side of the C ABI declared in include/wf.h: plans,
// workspace, input staging, the iteration driver and the exports.
//
// One iteration (Huffenberger 2017, Sec. 2, eqs. 2mess_t1 - 2mess_s for the
// chain s -T0- t_2DF -Nb0- d_2DF -T1- t_RF -Nb1- d_RF -T2- t_PX -Nb2- d) is
// two launches: the row pass (t_PX between the inverse and forward row
// transforms, then d_RF, t_RF) and the column pass (d_2DF, t_2DF between the
// forward and inverse column transforms; s implicit).  Every R iterations
// the residual (Sec. 2, Delta d) and the lambda controller run on the device.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/wf.h"
#include "wf_device.cuh"
#include "wf_internal.h"
#include "wf_ptr.h"

using namespace wf;

struct wf_plan_s {
  int ny = 0, nx = 0, M = 0;
  unsigned parts = 0;
  bool has_f = false, has_rf = false, merge = false, loaded = false;
  bool fused = false;       // sweeps run as one cooperative launch (wf_fused.cu)
  wf_params p{};
  cudaStream_t stream = nullptr;
  int nrow = 0;
  long long it_done = 0;
  long long launches = 0;   // kernels launched by this plan
  // device workspace
  float4* dn = nullptr;
  float2 *f_d1 = nullptr, *f_t1 = nullptr, *f_x = nullptr, *f_y = nullptr, *f_t0 = nullptr;
  float2 *eig = nullptr, *eig_nyq = nullptr;
  float *pst = nullptr, *a2 = nullptr;
  float2 *twx = nullptr, *twy = nullptr, *twh = nullptr;  // twh: exp(-2 pi i k/(nx/2))
  float2 *r_g = nullptr, *r_q = nullptr;
  double* part = nullptr;
  double* chi = nullptr;  // wf_chi2_aug: partial sums, then the value
  unsigned* fbar = nullptr;  // grid barrier words of the one-launch sweep
  double* trace = nullptr;   // per-checkpoint trace records (wf_params.trace)
  int* trace_n = nullptr;
  int run_index = 0;         // runs since the problem was loaded
  WfState* st = nullptr;
  double* lam_sched = nullptr;
  int* it_sched = nullptr;
  // staging for host-resident arguments
  float *stg_d = nullptr, *stg_var = nullptr, *stg_C = nullptr, *stg_P = nullptr;
  float *stg_pst = nullptr, *stg_a2 = nullptr, *stg_io = nullptr;
  uint8_t* stg_mask = nullptr;
  WfState* h_st = nullptr;  // pinned
  // defect correction (refine > 0)
  float4* dn_orig = nullptr;
  float *s_acc = nullptr, *s_corr = nullptr;
  float2* rho = nullptr;
  float2* jmap = nullptr;     // source j on masked pixels (pixel pairs)
  float2* src_2df = nullptr;  // its 2D DFT, column-tiled
  bool has_src = false;       // the loaded problem carries the source
  // Anderson-accelerated corrections (refine_accel = m > 0): the last f,
  // the last update, m differences of s and of f (ring), their Gram matrix
  float* aa_fprev = nullptr;
  float* aa_u = nullptr;
  float* aa_dx[WF_AA_MAX] = {};
  float* aa_df[WF_AA_MAX] = {};
  double* aa_part = nullptr;  // per-block partial dot products
  double* aa_G = nullptr;     // Gram matrix of the held Delta f (device)
  float* aa_gamma = nullptr;  // least-squares coefficients (device)
  int aa_n = 0, aa_head = 0;  // columns held, oldest column once the ring is full
  bool aa_have = false;       // aa_fprev holds the previous f
  // CUDA graph of one polling chunk of wf_run (K checkpoints of R sweeps),
  // captured and replayed on the plan's own stream (the caller's stream may
  // be the legacy default stream, which cannot be captured)
  cudaStream_t gstream = nullptr;
  // pass shapes (values per thread) picked by the autotuner, and a copy of
  // the state it restores after timing
  int row_variant = 0, col_variant = 0;
  bool tuned = false;
  // the column pass hints the next wave's tiles into L2 (maps whose sweep
  // moves more bytes than L2 holds)
  bool l2_prefetch = false;
  WfState* st_save = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // two cached chunk graphs: a solve and its correction solves alternate
  struct ChunkGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<unsigned char> key;
    long long launches = 0;
    long long last_use = 0;
  } chunk[2];
  long long chunk_clock = 0;
  // keys of the chunks that have run eagerly on this plan: a chunk is
  // captured only after its kernels have run once outside a capture, so
  // their one-time set-up (attributes, occupancy queries) is done
  std::vector<std::vector<unsigned char>> chunk_seen;
  std::vector<void*> allocs;
};

#define CK(x)                                      \
  do {                                             \
    cudaError_t e_ = (x);                          \
    if (e_ != cudaSuccess) {                       \
      fprintf(stderr, "libwf: %s:%d %s: %s\n", __FILE__, __LINE__, #x, cudaGetErrorString(e_)); \
      return e_ == cudaErrorMemoryAllocation ? WF_ENOMEM : WF_ECUDA; \
    }                                              \
  } while (0)
#define CKI(x)                                     \
  do {                                             \
    int e_ = (x);                                  \
    if (e_ != 0) {                                 \
      fprintf(stderr, "libwf: %s:%d launch: %s\n", __FILE__, __LINE__, cudaGetErrorString((cudaError_t)e_)); \
      return WF_ECUDA;                             \
    }                                              \
  } while (0)

template <class T>
static int dalloc(wf_plan_s* P, T** out, size_t n) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, n * sizeof(T) + 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return WF_ENOMEM;
  }
  P->allocs.push_back(q);
  *out = (T*)q;
  return WF_OK;
}

// where a caller's array lives (wf_ptr.h); another GPU's memory is rejected
static int ptr_where(const void* p) {
  if (!p) return PTR_HOST;
  cudaPointerAttributes at{};
  const cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) cudaGetLastError();
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) cudaGetLastError();
  return classify_ptr(e == cudaSuccess, (int)at.type, at.device, cur);
}

// device view of a caller array: the array itself, or a staged copy
template <class T>
static int to_device(wf_plan_s* P, const T* src, T* stage, size_t n, const T** out) {
  if (src == nullptr) {
    *out = nullptr;
    return WF_OK;
  }
  const int where = ptr_where(src);
  if (where == PTR_OTHER_DEVICE) return WF_EINVAL;
  if (where == PTR_DEVICE) {
    *out = src;
    return WF_OK;
  }
  CK(cudaMemcpyAsync(stage, src, n * sizeof(T), cudaMemcpyHostToDevice, P->stream));
  *out = stage;
  return WF_OK;
}

extern "C" {

int wf_version(void) { return WF_ABI_VERSION; }

const char* wf_strerror(int s) {
  switch (s) {
    case WF_OK: return "ok";
    case WF_EINVAL: return "invalid argument (size, NULL, non-finite or asymmetric input)";
    case WF_ENOTPD: return "a covariance eigenvalue is not positive";
    case WF_ENOCONV: return "no convergence within max_iters";
    case WF_ESTALL: return "the residual stopped falling above the tolerance";
    case WF_ETIMEOUT: return "a device wait timed out";
    case WF_ECUDA: return "CUDA runtime error";
    case WF_ENOMEM: return "device allocation failed";
    case WF_EUNSUPPORTED: return "unsupported size or option";
    default: return "unknown status";
  }
}

void wf_params_default(wf_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->theta[0] = 0.9;
  p->theta[1] = 0.9;
  p->theta[2] = 1.0;
  p->split_f = 0.5;
  p->split_fp = 0.5;
  p->split_w = 0.0;
  p->tol_u_scale = 1.0;
  p->merge_2df = 1;
  p->refine = 0;
  p->refine_tol_scale = 100.0;
  p->residual_every = 10;
  p->max_iters = 200000;
  p->check_every = 8;
  p->autotune = 1;
}

void wf_plan_destroy(wf_plan_t P) {
  if (!P) return;
  for (auto& g : P->chunk)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (P->ev_in) cudaEventDestroy(P->ev_in);
  if (P->ev_out) cudaEventDestroy(P->ev_out);
  if (P->gstream) cudaStreamDestroy(P->gstream);
  for (void* q : P->allocs) cudaFree(q);
  if (P->h_st) cudaFreeHost(P->h_st);
  delete P;
}

}  // extern "C"

// True when one sweep's fields (40 bytes per pixel: the row pass's 28 and
// the column pass's 12) exceed the current device's L2; then the column
// pass issues L2 prefetch hints one wave ahead (measured at 4096^2: 99.6 ->
// 96.0 us; the same hints in the row pass made 2048^2 slower).
static bool sweep_above_l2(int ny, int nx) {
  int dev = 0, l2 = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return 40.0 * ny * nx > (double)l2;
}

// Host-side validation shared by wf_plan_create and wf_batch_create (no CUDA call).
int wf::check_plan_args(int ny, int nx, unsigned parts, const wf_params* p) {
  if (!size_supported(nx) || !size_supported(ny)) return WF_EUNSUPPORTED;
  if (!(parts & WF_PART_WHITE) || (parts & ~7u)) return WF_EINVAL;
  wf_params prm;
  if (p) prm = *p;
  else wf_params_default(&prm);
  if (prm.residual_every < 1 || prm.max_iters < 1 || prm.check_every < 1) return WF_EINVAL;
  for (int i = 0; i < 3; ++i)
    if (!(prm.theta[i] > 0.0 && prm.theta[i] <= 1.0)) return WF_EINVAL;
  // the plain sweep needs tau_2DF > 0, i.e. split_f < 1; merged, N0 may reach 0
  const double fmax = prm.merge_2df ? 1.0 : 0.999999;
  if (!(prm.split_f >= 0.0 && prm.split_fp >= 0.0 && prm.split_f + prm.split_fp <= fmax) ||
      !(prm.split_w >= 0.0 && prm.split_w < 1.0))
    return WF_EINVAL;
  if (!(prm.tol_u_scale > 0.0) || (prm.merge_2df != 0 && prm.merge_2df != 1)) return WF_EINVAL;
  if (prm.refine < 0 || prm.refine > 32 || !(prm.refine_tol_scale >= 1.0) || prm.refine_max_iters < 0 ||
      prm.refine_lam1_iters < 0 || prm.stall_checks < 0 || prm.autotune < 0 || prm.autotune > 2 ||
      prm.refine_extra < 0 || prm.refine_extra > 32 ||
      prm.dft_precision < 0 || prm.dft_precision > 4 || prm.sweep_kernel < 0 || prm.sweep_kernel > 1 ||
      prm.trace < 0 || prm.trace > 2 || prm.refine_accel < 0 || prm.refine_accel > WF_AA_MAX)
    return WF_EINVAL;
  // tensor-core radix-16 stages: 16-value column shapes, merged 2DF block
  if (prm.dft_precision != 0 && (!col_tc_supported(ny) || prm.merge_2df != 1)) return WF_EUNSUPPORTED;
  if (prm.dft_precision >= 3 && !col_tc5_supported(ny)) return WF_EUNSUPPORTED;
  // chi^2_aug is summed for the merged 2DF block (or without a 1/f part)
  if (prm.trace == 2 && (parts & WF_PART_1F) && !prm.merge_2df) return WF_EUNSUPPORTED;
  return WF_OK;
}

extern "C" {

int wf_plan_create(wf_plan_t* out, int ny, int nx, unsigned parts, const wf_params* p, void* stream) {
  if (!out) return WF_EINVAL;
  const int chk = check_plan_args(ny, nx, parts, p);
  if (chk != WF_OK) return chk;
  wf_params prm;
  if (p) prm = *p;
  else wf_params_default(&prm);

  wf_plan_s* P = new wf_plan_s();
  P->ny = ny;
  P->nx = nx;
  P->M = nx / 2;
  P->parts = parts;
  P->has_f = parts & WF_PART_1F;
  P->has_rf = parts & WF_PART_STRIPE;
  P->merge = P->has_f && prm.merge_2df;
  P->p = prm;
  if (prm.autotune == 2) P->row_variant = P->col_variant = 1;  // the second shapes, untimed
  P->stream = (cudaStream_t)stream;
  P->nrow = row_grid(nx, ny);
  P->l2_prefetch = sweep_above_l2(ny, nx);
  const size_t npx = (size_t)ny * nx, nh = (size_t)ny * P->M;
  int rc = WF_OK;
#define AL(ptr, n)                                   \
  if (rc == WF_OK) rc = dalloc(P, &(ptr), (n));
  AL(P->dn, npx / 2);
  AL(P->f_x, nh);
  if (P->has_rf) {
    AL(P->f_d1, nh);
    AL(P->f_t1, nh);
  } else {
    AL(P->f_y, nh);
  }
  if (P->has_f && !P->merge) AL(P->f_t0, nh);
  AL(P->eig, nh);
  AL(P->eig_nyq, (size_t)ny);
  AL(P->pst, (size_t)P->M + 1);
  AL(P->a2, (size_t)ny);
  AL(P->twx, (size_t)nx);
  AL(P->twy, (size_t)ny);
  AL(P->twh, (size_t)(nx / 2));
  AL(P->r_g, nh);
  AL(P->r_q, nh);
  AL(P->part, (size_t)3 * P->nrow + 4 * 256 + 64);
  AL(P->chi, (size_t)chi2_scratch(ny, nx) + 1);
  AL(P->st, (size_t)1);
  AL(P->fbar, (size_t)4);
  if (prm.trace > 0) {
    AL(P->trace, (size_t)WF_TRACE_CAP * WF_TRACE_FIELDS);
    AL(P->trace_n, (size_t)1);
  }
  AL(P->st_save, (size_t)1);
  AL(P->lam_sched, (size_t)260);
  AL(P->it_sched, (size_t)260);
  AL(P->stg_d, npx);
  AL(P->stg_var, npx);
  AL(P->stg_mask, npx);
  AL(P->stg_C, (size_t)ny * (P->M + 1));
  if (P->has_f) AL(P->stg_P, (size_t)ny * (P->M + 1));
  AL(P->stg_pst, (size_t)P->M + 1);
  AL(P->stg_a2, (size_t)ny);
  AL(P->stg_io, npx + 64);
  if (prm.refine > 0) {
    AL(P->dn_orig, npx / 2);
    AL(P->s_acc, npx);
    AL(P->s_corr, npx);
    AL(P->rho, npx / 2);
    AL(P->jmap, npx / 2);
    AL(P->src_2df, nh);
    if (prm.refine_accel > 0) {
      AL(P->aa_fprev, npx);
      AL(P->aa_u, npx);
      for (int j = 0; j < prm.refine_accel; ++j) {
        AL(P->aa_dx[j], npx);
        AL(P->aa_df[j], npx);
      }
      AL(P->aa_part, (size_t)aa_dots_blocks() * 2 * WF_AA_MAX);
      AL(P->aa_G, (size_t)WF_AA_MAX * WF_AA_MAX);
      AL(P->aa_gamma, (size_t)WF_AA_MAX);
    }
  }
#undef AL
  if (rc != WF_OK) {
    wf_plan_destroy(P);
    return rc;
  }
  if (cudaMallocHost(&P->h_st, sizeof(WfState)) != cudaSuccess) {
    cudaGetLastError();
    P->h_st = nullptr;
    wf_plan_destroy(P);
    return WF_ENOMEM;
  }
  if (cudaStreamCreateWithFlags(&P->gstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    wf_plan_destroy(P);
    return WF_ECUDA;
  }
  if (cudaMemset(P->fbar, 0, 4 * sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    wf_plan_destroy(P);
    return WF_ECUDA;
  }
  // one cooperative launch per R sweeps, when asked for
  if (prm.sweep_kernel == 1) {
    P->fused = fused_supported(ny, nx, P->has_rf, P->merge || !P->has_f, prm.dft_precision);
    if (!P->fused) {
      wf_plan_destroy(P);
      return WF_EUNSUPPORTED;
    }
  }
  // twiddle tables exp(-2 pi i k / n), computed in double on the host
  std::vector<float2> tx(nx), ty(ny);
  for (int k = 0; k < nx; ++k) {
    const double a = 2.0 * M_PI * (double)k / (double)nx;
    tx[k] = make_float2((float)cos(a), (float)-sin(a));
  }
  for (int k = 0; k < ny; ++k) {
    const double a = 2.0 * M_PI * (double)k / (double)ny;
    ty[k] = make_float2((float)cos(a), (float)-sin(a));
  }
  // the half-length row transform's table is every other entry of twx
  std::vector<float2> th(nx / 2);
  for (int k = 0; k < nx / 2; ++k) th[k] = tx[2 * k];
  cudaError_t e1 = cudaMemcpy(P->twx, tx.data(), nx * sizeof(float2), cudaMemcpyHostToDevice);
  cudaError_t e2 = cudaMemcpy(P->twy, ty.data(), ny * sizeof(float2), cudaMemcpyHostToDevice);
  cudaError_t e3 = cudaMemcpy(P->twh, th.data(), nx / 2 * sizeof(float2), cudaMemcpyHostToDevice);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
    wf_plan_destroy(P);
    return WF_ECUDA;
  }
  *out = P;
  return WF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- helpers
static RowArgs row_args(wf_plan_s* P) {
  RowArgs a{};
  a.variant = P->row_variant;
  a.ny = P->ny;
  a.nx = P->nx;
  a.has_rf = P->has_rf;
  a.dn = P->dn;
  a.f_d1 = P->f_d1;
  a.f_t1 = P->f_t1;
  a.f_x = P->f_x;
  a.f_y = P->f_y;
  a.pst = P->pst;
  a.a2 = P->a2;
  a.twx = P->twx;
  a.twh = P->twh;
  a.st = P->st;
  a.r_g = P->r_g;
  a.r_q = P->r_q;
  a.src_px = P->has_src ? P->jmap : nullptr;
  return a;
}

static ColArgs col_args(wf_plan_s* P, int parity) {
  ColArgs a{};
  a.prec = P->p.dft_precision;
  a.variant = a.prec ? 0 : P->col_variant;  // the tensor-core stages use the 16-value shape
  a.prefetch = P->l2_prefetch;
  a.ny = P->ny;
  a.nx = P->nx;
  a.has_rf = P->has_rf;
  a.has_f = P->has_f;
  a.merge = P->merge;
  a.parity = parity & 1;
  a.f_y = P->has_rf ? P->f_t1 : P->f_y;
  a.f_x = P->f_x;
  a.f_t0 = P->f_t0;
  a.eig = P->eig;
  a.eig_nyq = P->eig_nyq;
  a.twy = P->twy;
  a.st = P->st;
  a.r_g = P->r_g;
  a.r_q = P->r_q;
  a.src = P->has_src ? P->src_2df : nullptr;
  return a;
}

// one sweep: row pass then column pass
static int enqueue_row_pass(wf_plan_s* P) {
  RowArgs ra = row_args(P);
  ra.check_done = 1;
  CKI(launch_row(P->has_rf ? ROW_PASS_RF : ROW_PASS_NORF, ra, P->stream));
  P->launches += 1;
  return WF_OK;
}

static int enqueue_col_pass(wf_plan_s* P, int parity) {
  ColArgs ca = col_args(P, parity);
  ca.check_done = 1;
  const int mode = (P->has_f && !P->merge) ? COL_PASS_2DF : (P->has_src ? COL_PASS_MERGE_SRC : COL_PASS_MERGE);
  CKI(launch_col(mode, ca, P->stream));
  P->launches += 1;
  return WF_OK;
}

static int enqueue_iteration(wf_plan_s* P, int parity) {
  int rc = enqueue_row_pass(P);
  if (rc) return rc;
  return enqueue_col_pass(P, parity);
}

// n sweeps from a sweep of the given parity: one cooperative launch for a
// fused plan, else n row-pass / column-pass pairs
static int enqueue_sweeps(wf_plan_s* P, int n, long long first) {
  if (!P->fused) {
    for (int i = 0; i < n; ++i) {
      int rc = enqueue_iteration(P, (int)((first + i) & 1));
      if (rc) return rc;
    }
    return WF_OK;
  }
  FusedArgs f{};
  f.ny = P->ny;
  f.nx = P->nx;
  f.nsweeps = n;
  f.dn = P->dn;
  f.f_d1 = P->f_d1;
  f.f_t1 = P->f_t1;
  f.f_x = P->f_x;
  f.eig = P->eig;
  f.eig_nyq = P->eig_nyq;
  f.pst = P->pst;
  f.a2 = P->a2;
  f.twx = P->twx;
  f.twh = P->twh;
  f.twy = P->twy;
  f.src = P->has_src ? P->src_2df : nullptr;
  f.st = P->st;
  f.bar = P->fbar;
  CK(cudaMemsetAsync(P->fbar, 0, sizeof(unsigned), P->stream));  // the arrival count
  CKI(launch_fused(f, P->stream));
  P->launches += 1;
  return WF_OK;
}

// residual passes; partials land in part[0 .. 3 nrow)
static int enqueue_residual(wf_plan_s* P, int parity, int check_done) {
  ColArgs ca = col_args(P, parity);
  ca.check_done = check_done;
  ca.skip_ok = check_done;  // iteration checkpoints only
  CKI(launch_col(COL_RESID_A, ca, P->stream));
  RowArgs ra = row_args(P);
  ra.check_done = check_done;
  ra.skip_ok = check_done;
  ra.part0 = P->part;
  ra.part1 = P->part + P->nrow;
  CKI(launch_row(ROW_RESID_B, ra, P->stream));
  if (P->has_f) CKI(launch_col(COL_RESID_C, ca, P->stream));
  ra.part0 = P->part + 2 * P->nrow;
  CKI(launch_row(ROW_RESID_D, ra, P->stream));
  P->launches += P->has_f ? 4 : 3;
  return WF_OK;
}

// Delta d of a pixel-space s against the original data (table dn_orig):
// rho map (unmasked pixels) and the partial sums of the residual.
static int enqueue_resid_map(wf_plan_s* P, const float* s_px, float2* rho_out, float2* gm_out) {
  RowArgs ra = row_args(P);
  ra.check_done = 0;
  ra.src_px = nullptr;  // the caller's problem has no source
  ra.gm_out = gm_out;
  ra.dn = P->dn_orig;
  ra.in_px = (const float2*)s_px;
  ra.out_rf = P->r_q;
  CKI(launch_row(ROW_R2C, ra, P->stream));
  ColArgs ca = col_args(P, 0);
  ca.check_done = 0;
  CKI(launch_col(COL_G_FROM_S, ca, P->stream));
  ra.part0 = P->part;
  ra.part1 = P->part + P->nrow;
  CKI(launch_row(ROW_RESID_B, ra, P->stream));
  ra.gm_out = nullptr;
  if (P->has_f) CKI(launch_col(COL_RESID_C, ca, P->stream));
  ra.part0 = P->part + 2 * P->nrow;
  ra.out_px = rho_out;
  CKI(launch_row(ROW_RESID_D, ra, P->stream));
  P->launches += P->has_f ? 5 : 4;
  return WF_OK;
}

static CtrlArgs ctrl_args(wf_plan_s* P) {
  CtrlArgs c{};
  c.st = P->st;
  c.part_g = P->part;
  c.part_g2 = P->part + P->nrow;
  c.part_rho = P->part + 2 * P->nrow;
  c.nrow = P->nrow;
  c.R = P->p.residual_every;
  c.max_iters = P->p.max_iters;
  c.stall = P->p.stall_checks;
  c.lam_sched = P->lam_sched;
  c.it_sched = P->it_sched;
  c.trace = P->trace;
  c.trace_n = P->trace_n;
  c.trace_cap = WF_TRACE_CAP;
  c.run_index = P->run_index;
  c.chi_val = nullptr;
  return c;
}

static int finish_status(unsigned err) {
  if (err & (WF_ERR_VAR | WF_ERR_C | WF_ERR_P1F | WF_ERR_PST | WF_ERR_A2)) return WF_ENOTPD;
  if (err) return WF_EINVAL;
  return WF_OK;
}

// ---------------------------------------------------------------- autotuner
// Each pass has two compiled shapes (values per thread, so threads per row or
// column); which is faster depends on the map size (measured: 4 values per
// thread for rows of 512 and fewer pixels, 8 above; 8 for 512-long columns,
// 16 above).  The first loaded problem of a plan times both shapes of each
// pass -- graph-replayed launches on the plan's buffers, as wf_time_passes
// does -- and keeps the faster one (the first unless the second wins by
// more than 3%), cached per device, map shape and sweep form for the rest of
// the process.  Results depend on the shape only through rounding order.

namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, unsigned, int, int>, std::pair<int, int>> g_tune;
}  // namespace

// mean time of n launches of one pass with shape `variant`, in microseconds
static int time_pass(wf_plan_s* P, int which, int variant, int n, cudaEvent_t e0, cudaEvent_t e1, double* us) {
  const int rv = P->row_variant, cv = P->col_variant;
  if (which == 0) P->row_variant = variant;
  else P->col_variant = variant;
  int rc = which == 0 ? enqueue_row_pass(P) : enqueue_col_pass(P, 0);  // un-captured: kernel attributes
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  if (!rc && cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = WF_ECUDA;
  if (!rc) {
    for (int i = 0; i < n && !rc; ++i) rc = which == 0 ? enqueue_row_pass(P) : enqueue_col_pass(P, 0);
    cudaError_t ce = cudaStreamEndCapture(P->stream, &g);
    if (!rc && (ce != cudaSuccess || cudaGraphInstantiate(&ge, g, 0) != cudaSuccess)) rc = WF_ECUDA;
  }
  float ms = 0.f;
  if (!rc && (cudaGraphLaunch(ge, P->stream) != cudaSuccess || cudaEventRecord(e0, P->stream) != cudaSuccess ||
              cudaGraphLaunch(ge, P->stream) != cudaSuccess || cudaEventRecord(e1, P->stream) != cudaSuccess ||
              cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
    rc = WF_ECUDA;
  if (ge) cudaGraphExecDestroy(ge);
  if (g) cudaGraphDestroy(g);
  P->row_variant = rv;
  P->col_variant = cv;
  if (rc) cudaGetLastError();
  *us = 1000.0 * ms / n;
  return rc;
}

static int autotune(wf_plan_s* P) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  const int prec = P->p.dft_precision;
  const auto key = std::make_tuple(dev, P->ny, P->nx, P->parts, (int)P->merge, prec);
  // held while timing: plans of one shape on other threads wait for the
  // answer instead of timing concurrently and possibly choosing differently
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(key);
  if (it != g_tune.end()) {
    P->row_variant = it->second.first;
    P->col_variant = it->second.second;
    P->tuned = true;
    return WF_OK;
  }
  const bool two_rows = row_pass_e(P->M, 0) != row_pass_e(P->M, 1);
  const bool two_cols = prec == 0 && col_pass_e(P->ny, 0) != col_pass_e(P->ny, 1);
  int rv = 0, cv = 0;
  if (two_rows || two_cols) {
    const int n = (int)std::min<size_t>(200, std::max<size_t>(8, (size_t)20000000 / ((size_t)P->ny * P->nx)));
    cudaStream_t user = P->stream;
    CK(cudaEventRecord(P->ev_in, user));
    CK(cudaStreamWaitEvent(P->gstream, P->ev_in, 0));
    P->stream = P->gstream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = WF_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = WF_ECUDA;
    // the passes run from the loaded problem's state at lambda = 1; state and
    // fields are put back afterwards
    if (!rc && cudaMemcpyAsync(P->st_save, P->st, sizeof(WfState), cudaMemcpyDeviceToDevice, P->stream) != cudaSuccess)
      rc = WF_ECUDA;
    if (!rc && launch_set_lambda(P->st, 1.0, 1, P->stream)) rc = WF_ECUDA;
    double t[2][2] = {{0, 0}, {0, 0}};
    for (int which = 0; which < 2 && !rc; ++which) {
      if (!(which == 0 ? two_rows : two_cols)) continue;
      for (int v = 0; v < 2 && !rc; ++v) rc = time_pass(P, which, v, n, e0, e1, &t[which][v]);
    }
    if (!rc) {
      rv = (two_rows && t[0][1] < 0.97 * t[0][0]) ? 1 : 0;
      cv = (two_cols && t[1][1] < 0.97 * t[1][0]) ? 1 : 0;
    }
    if (!rc && cudaMemcpyAsync(P->st, P->st_save, sizeof(WfState), cudaMemcpyDeviceToDevice, P->stream) != cudaSuccess)
      rc = WF_ECUDA;
    const size_t nhb = (size_t)P->ny * P->M * sizeof(float2);
    for (float2* f : {P->f_x, P->f_d1, P->f_t1, P->f_y, P->f_t0})
      if (!rc && f && cudaMemsetAsync(f, 0, nhb, P->stream) != cudaSuccess) rc = WF_ECUDA;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (cudaEventRecord(P->ev_out, P->gstream) != cudaSuccess || cudaStreamWaitEvent(user, P->ev_out, 0) != cudaSuccess)
      rc = rc ? rc : WF_ECUDA;
    P->stream = user;
    if (rc) return rc;
  }
  P->row_variant = rv;
  P->col_variant = cv;
  P->tuned = true;
  g_tune.emplace(key, std::make_pair(rv, cv));
  return WF_OK;
}

extern "C" {

int wf_set_problem(wf_plan_t P, const float* d, const float* pixel_var, const uint8_t* mask,
                   const float* C, const float* P1f, const float* Pst, const float* stripe_amp2) {
  if (!P || !d || !pixel_var || !C) return WF_EINVAL;
  if (P->has_f != (P1f != nullptr)) return WF_EINVAL;
  if (P->has_rf != (Pst != nullptr)) return WF_EINVAL;
  if (!P->has_rf && stripe_amp2) return WF_EINVAL;
  const size_t npx = (size_t)P->ny * P->nx, nspec = (size_t)P->ny * (P->M + 1);
  SetupArgs a{};
  a.ny = P->ny;
  a.nx = P->nx;
  int rc;
  if ((rc = to_device(P, d, P->stg_d, npx, &a.d))) return rc;
  if ((rc = to_device(P, pixel_var, P->stg_var, npx, &a.var))) return rc;
  if ((rc = to_device(P, mask, P->stg_mask, npx, &a.mask))) return rc;
  if ((rc = to_device(P, C, P->stg_C, nspec, &a.C))) return rc;
  if ((rc = to_device(P, P1f, P->stg_P, nspec, &a.P1f))) return rc;
  if ((rc = to_device(P, Pst, P->stg_pst, (size_t)P->M + 1, &a.Pst))) return rc;
  if ((rc = to_device(P, stripe_amp2, P->stg_a2, (size_t)P->ny, &a.a2))) return rc;
  a.dn = P->dn;
  a.eig = P->eig;
  a.eig_nyq = P->eig_nyq;
  a.pst = P->pst;
  a.a2_out = P->a2;
  a.part = P->part + 3 * P->nrow;
  a.st = P->st;
  for (int i = 0; i < 3; ++i) a.theta[i] = P->p.theta[i];
  a.split_f = P->p.split_f;
  a.split_fp = P->p.split_fp;
  a.split_w = P->p.split_w;
  a.has_rf = P->has_rf;
  a.has_f = P->has_f;
  a.merge = P->merge;
  CK(cudaMemsetAsync(P->st, 0, sizeof(WfState), P->stream));
  CK(cudaMemsetAsync(P->fbar, 0, 4 * sizeof(unsigned), P->stream));
  if (P->trace_n) CK(cudaMemsetAsync(P->trace_n, 0, sizeof(int), P->stream));
  P->run_index = 0;
  CKI(launch_setup(a, P->stream));
  P->launches += 5;
  // iteration starts from zero fields (Sec. 2)
  const size_t nhb = (size_t)P->ny * P->M * sizeof(float2);
  CK(cudaMemsetAsync(P->f_x, 0, nhb, P->stream));
  if (P->f_d1) CK(cudaMemsetAsync(P->f_d1, 0, nhb, P->stream));
  if (P->f_t1) CK(cudaMemsetAsync(P->f_t1, 0, nhb, P->stream));
  if (P->f_y) CK(cudaMemsetAsync(P->f_y, 0, nhb, P->stream));
  if (P->f_t0) CK(cudaMemsetAsync(P->f_t0, 0, nhb, P->stream));
  CK(cudaMemcpyAsync(P->h_st, P->st, sizeof(WfState), cudaMemcpyDeviceToHost, P->stream));
  CK(cudaStreamSynchronize(P->stream));
  P->it_done = 0;
  P->loaded = false;
  P->has_src = false;
  const int st = finish_status(P->h_st->err);
  if (st != WF_OK) return st;
  if (P->p.autotune == 1 && !P->tuned && (rc = autotune(P))) return rc;
  P->loaded = true;
  return WF_OK;
}

int wf_iterate(wf_plan_t P, double lam, int n) {
  if (!P || !P->loaded || n < 0 || !(lam >= 1.0) || !isfinite(lam)) return WF_EINVAL;
  CKI(launch_set_lambda(P->st, lam, 1, P->stream));
  P->launches += 1;
  int rc = enqueue_sweeps(P, n, P->it_done);
  if (rc) return rc;
  P->it_done += n;
  return WF_OK;
}

static void fill_stats(wf_plan_s* P, wf_stats* st, int status) {
  if (!st) return;
  const WfState& h = *P->h_st;
  st->iters = h.iter;
  st->checkpoints = h.checkpoints;
  st->lam_final = h.lam;
  st->rel_rho_u = h.rel_u;
  st->rel_rho_m = h.rel_m;
  for (int i = 0; i < 3; ++i) st->tau[i] = h.tau[i];
  st->status = status;
  st->parts = (int)P->parts;
}

}  // extern "C"

// the fields wf_chi2_aug sums (merged 2DF block or no 1/f part)
static Chi2Fields chi2_fields(wf_plan_s* P) {
  Chi2Fields f{};
  f.ny = P->ny;
  f.nx = P->nx;
  f.has_rf = P->has_rf;
  f.d0 = P->f_x;
  f.t = P->has_rf ? P->f_t1 : P->f_y;
  f.d1 = P->has_rf ? P->f_d1 : nullptr;
  f.dn = P->dn;
  f.eig = P->eig;
  f.eig_nyq = P->eig_nyq;
  f.pst = P->pst;
  f.a2 = P->a2;
  f.twx = P->twx;
  f.twy = P->twy;
  f.st = P->st;
  return f;
}

// ---------------------------------------------------------------- persistent batch
static int run_setup(wf_plan_t P, const wf_schedule* sch, double tol, CtrlArgs* out, double* lam0_out);

// The map's fields and tables as the persistent batch kernel takes them
// (merged 2DF block with a stripe part, square maps of the batch sizes).
int wf::plan_batch_map(wf_plan_t P, int variant, BatchMapArgs* out) {
  if (!P || P->ny != P->nx || !P->has_rf || (P->has_f && !P->merge) || P->p.dft_precision != 0) return WF_EUNSUPPORTED;
  const int cls = batch_class(P->ny, variant);
  if (cls < 0) return WF_EUNSUPPORTED;
  BatchMapArgs m{};
  m.cls = cls;
  m.dn = P->dn;
  m.f_d1 = P->f_d1;
  m.f_t1 = P->f_t1;
  m.f_x = P->f_x;
  m.eig = P->eig;
  m.eig_nyq = P->eig_nyq;
  m.pst = P->pst;
  m.a2 = P->a2;
  m.twx = P->twx;
  m.twh = P->twh;
  m.twy = P->twy;
  m.src = P->has_src ? P->src_2df : nullptr;
  m.st = P->st;
  *out = m;
  return WF_OK;
}

bool wf::plan_batch_ok(const wf_plan_t P) {
  return P && P->ny == P->nx && P->has_rf && !(P->has_f && !P->merge) && P->p.dft_precision == 0 &&
         batch_class(P->ny, 0) >= 0;
}

int wf::plan_size(const wf_plan_t P) { return P->ny; }
int wf::plan_autotune(const wf_plan_t P) { return P->p.autotune; }

// Runs the iteration of several loaded plans together (wf_run for each, with
// one schedule and stop tolerance): per checkpoint one persistent launch of
// R sweeps for all of them (wf_batchk.cu), then each plan's residual and
// controller; K checkpoints per CUDA graph, captured once and replayed on
// `s` until every plan is done or at its cap.  status[i] and st[i] receive
// what wf_run would return for plan i.
int wf::run_plans_persistent(const std::vector<wf_plan_t>& plans, const std::vector<int>& variant,
                             const wf_schedule* sch, double tol, BatchDevice& bd, cudaStream_t s,
                             std::vector<int>& status, std::vector<wf_stats>& st) {
  const size_t n = plans.size();
  status.assign(n, WF_OK);
  st.assign(n, wf_stats{});
  if (n == 0) return WF_OK;
  const int R = plans[0]->p.residual_every, K = plans[0]->p.check_every;
  std::vector<CtrlArgs> ctrl(n);
  std::vector<BatchMapArgs> maps(n);
  std::vector<cudaStream_t> own(n);
  long long cap = 0;
  for (size_t i = 0; i < n; ++i) {
    wf_plan_t P = plans[i];
    own[i] = P->stream;
    P->stream = s;
    double lam0 = 1.0;
    int rc = run_setup(P, sch, tol, &ctrl[i], &lam0);
    P->run_index += 1;
    if (!rc) rc = launch_set_lambda(P->st, lam0, 1, s) ? WF_ECUDA : WF_OK;
    if (!rc) rc = plan_batch_map(P, variant[i], &maps[i]);
    if (rc) {
      for (size_t j = 0; j <= i; ++j) plans[j]->stream = own[j];
      return rc;
    }
    P->launches += 1;
    cap = std::max<long long>(cap, ctrl[i].max_iters);
  }
  // work queues: the largest maps first, so the small ones fill in at the end
  std::vector<size_t> order(n);
  for (size_t i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return plans[a]->ny > plans[b]->ny; });
  bd.row_items.clear();
  bd.col_items.clear();
  for (size_t i : order) {
    int rows = 0, cols = 0, re = 0, ce = 0;
    batch_item_shape(maps[i].cls, &rows, &cols, &re, &ce);
    for (int g = 0; g < plans[i]->ny / rows; ++g) bd.row_items.push_back(make_int2((int)i, g));
    for (int g = 0; g < (plans[i]->nx / 2) / cols; ++g) bd.col_items.push_back(make_int2((int)i, g));
  }
  int rc = WF_OK;
  auto restore = [&]() {
    for (size_t i = 0; i < n; ++i) plans[i]->stream = own[i];
  };
  if (bd.row_items.size() > bd.cap_items || bd.col_items.size() > bd.cap_items || n > bd.cap_maps) {
    restore();
    return WF_EINVAL;
  }
  if (cudaMemcpyAsync(bd.maps, maps.data(), n * sizeof(BatchMapArgs), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(bd.rows, bd.row_items.data(), bd.row_items.size() * sizeof(int2), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(bd.cols, bd.col_items.data(), bd.col_items.size() * sizeof(int2), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemsetAsync(bd.err, 0, sizeof(unsigned), s) != cudaSuccess) {
    cudaGetLastError();
    restore();
    return WF_ECUDA;
  }
  BatchArgs a{};
  a.maps = bd.maps;
  a.row_items = bd.rows;
  a.col_items = bd.cols;
  a.n_row = (int)bd.row_items.size();
  a.n_col = (int)bd.col_items.size();
  a.nsweeps = R;
  a.bar = bd.bar;
  a.queue = bd.queue;
  a.err = bd.err;
  long long launches_per_chunk = 0;
  // one chunk: K checkpoints of one persistent launch and every plan's
  // residual and controller
  auto enqueue_chunk = [&]() -> int {
    for (int cp = 0; cp < K; ++cp) {
      if (cudaMemsetAsync(bd.bar, 0, 4 * sizeof(unsigned), s) != cudaSuccess ||
          cudaMemsetAsync(bd.queue, 0, 2 * (size_t)R * sizeof(unsigned), s) != cudaSuccess)
        return WF_ECUDA;
      if (launch_batch_sweeps(a, bd.grid, s)) return WF_ECUDA;
      launches_per_chunk += 1;
      for (size_t i = 0; i < n; ++i) {
        int r2 = enqueue_residual(plans[i], 0, 1);
        if (r2) return r2;
        if (launch_ctrl(ctrl[i], s)) return WF_ECUDA;
        plans[i]->launches += 1;
      }
    }
    return WF_OK;
  };
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = WF_ECUDA;
  if (!rc) {
    std::vector<long long> before(n);
    for (size_t i = 0; i < n; ++i) before[i] = plans[i]->launches;
    rc = enqueue_chunk();
    cudaError_t ce = cudaStreamEndCapture(s, &g);
    if (!rc && (ce != cudaSuccess || cudaGraphInstantiate(&ge, g, 0) != cudaSuccess)) rc = WF_ECUDA;
    // launches are counted per replay below
    for (size_t i = 0; i < n; ++i) bd.per_plan_launches = plans[i]->launches - before[i];
    for (size_t i = 0; i < n; ++i) plans[i]->launches = before[i];
  }
  long long enq = 0;
  std::vector<WfState> hst(n);
  while (!rc) {
    if (cudaGraphLaunch(ge, s) != cudaSuccess) {
      rc = WF_ECUDA;
      break;
    }
    bd.launches += launches_per_chunk;
    for (size_t i = 0; i < n; ++i) plans[i]->launches += bd.per_plan_launches;
    enq += (long long)K * R;
    for (size_t i = 0; i < n && !rc; ++i)
      if (cudaMemcpyAsync(plans[i]->h_st, plans[i]->st, sizeof(WfState), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        rc = WF_ECUDA;
    if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = WF_ECUDA;
    if (rc) break;
    bool all = true;
    for (size_t i = 0; i < n; ++i) all = all && plans[i]->h_st->done;
    if (all || enq >= cap) break;
  }
  if (ge) cudaGraphExecDestroy(ge);
  if (g) cudaGraphDestroy(g);
  unsigned err = 0;
  if (!rc && cudaMemcpy(&err, bd.err, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) rc = WF_ECUDA;
  restore();
  if (rc) {
    cudaGetLastError();
    return rc;
  }
  for (size_t i = 0; i < n; ++i) {
    wf_plan_t P = plans[i];
    P->it_done = P->h_st->iter;
    if ((P->h_st->err & WF_ERR_TIMEOUT) || (err & WF_ERR_TIMEOUT)) {
      status[i] = WF_ETIMEOUT;
      continue;
    }
    const int hs = P->h_st->status;
    status[i] = hs == 3 ? WF_ENOCONV : (hs == 4 ? WF_ESTALL : WF_OK);
    fill_stats(P, &st[i], status[i]);
  }
  return WF_OK;
}

// Mean time of one sweep of plan P alone in the persistent batch kernel with
// shape `variant` (the batch's tuner; overwrites P's fields and state).
int wf::time_batch_variant(wf_plan_t P, int variant, BatchDevice& bd, cudaStream_t s, double* us) {
  BatchMapArgs m{};
  int rc = plan_batch_map(P, variant, &m);
  if (rc) return rc;
  const int ns = std::max(1, std::min(4, P->p.residual_every));
  int rows = 0, cols = 0, re = 0, ce = 0;
  batch_item_shape(m.cls, &rows, &cols, &re, &ce);
  bd.row_items.clear();
  bd.col_items.clear();
  for (int g = 0; g < P->ny / rows; ++g) bd.row_items.push_back(make_int2(0, g));
  for (int g = 0; g < (P->nx / 2) / cols; ++g) bd.col_items.push_back(make_int2(0, g));
  BatchArgs a{};
  a.maps = bd.maps;
  a.row_items = bd.rows;
  a.col_items = bd.cols;
  a.n_row = (int)bd.row_items.size();
  a.n_col = (int)bd.col_items.size();
  a.nsweeps = ns;
  a.bar = bd.bar;
  a.queue = bd.queue;
  a.err = bd.err;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.f;
  rc = WF_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
      launch_set_lambda(P->st, 1.0, 1, s) ||
      cudaMemcpyAsync(bd.maps, &m, sizeof(m), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(bd.rows, bd.row_items.data(), bd.row_items.size() * sizeof(int2), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(bd.cols, bd.col_items.data(), bd.col_items.size() * sizeof(int2), cudaMemcpyHostToDevice, s) !=
          cudaSuccess)
    rc = WF_ECUDA;
  for (int rep = 0; rep < 2 && !rc; ++rep) {
    if (cudaMemsetAsync(bd.bar, 0, 4 * sizeof(unsigned), s) != cudaSuccess ||
        cudaMemsetAsync(bd.queue, 0, 2 * (size_t)ns * sizeof(unsigned), s) != cudaSuccess ||
        cudaEventRecord(e0, s) != cudaSuccess || launch_batch_sweeps(a, bd.grid, s) ||
        cudaEventRecord(e1, s) != cudaSuccess)
      rc = WF_ECUDA;
  }
  if (!rc && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)) rc = WF_ECUDA;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc) {
    cudaGetLastError();
    return rc;
  }
  P->launches += 3;
  P->loaded = false;
  *us = 1000.0 * ms / ns;
  return WF_OK;
}

// Controller arguments and device schedule of a run (wf_run and the
// persistent batch): validates the schedule, uploads a fixed schedule's
// levels to the plan, and gives the first lambda.
static int run_setup(wf_plan_t P, const wf_schedule* sch, double tol, CtrlArgs* out, double* lam0_out) {
  const int R = P->p.residual_every;
  CtrlArgs c = ctrl_args(P);
  c.tol = tol;
  c.tol_u = tol * P->p.tol_u_scale;
  c.count_iters = 1;
  c.max_iters = ((P->p.max_iters + R - 1) / R) * R;
  double lam0;
  if (sch->mode == WF_SCHED_FIXED) {
    if (sch->nlevels < 1 || sch->nlevels > 256 || !sch->lam || !sch->iters) return WF_EINVAL;
    std::vector<double> L(sch->lam, sch->lam + sch->nlevels);
    std::vector<int> I(sch->iters, sch->iters + sch->nlevels);
    for (size_t i = 0; i < L.size(); ++i)
      if (!(L[i] >= 1.0) || !isfinite(L[i]) || I[i] < 0) return WF_EINVAL;
    if (L.back() != 1.0) {
      L.push_back(1.0);
      I.push_back(0);
    }
    CK(cudaMemcpyAsync(P->lam_sched, L.data(), L.size() * sizeof(double), cudaMemcpyHostToDevice, P->stream));
    CK(cudaMemcpyAsync(P->it_sched, I.data(), I.size() * sizeof(int), cudaMemcpyHostToDevice, P->stream));
    c.mode = 0;
    c.skip_fixed = P->p.trace ? 0 : 1;  // a trace wants the residual at every checkpoint
    c.nlevels = (int)L.size();
    lam0 = L[0];
  } else if (sch->mode == WF_SCHED_ADAPTIVE) {
    if (!(sch->lam0 >= 1.0) || !(sch->expo > 0.0 && sch->expo < 1.0) || !(sch->ratio > 0.0) ||
        !(sch->snap >= 1.0))
      return WF_EINVAL;
    c.mode = 1;
    c.ratio = sch->ratio;
    c.expo = sch->expo;
    c.snap = sch->snap;
    lam0 = sch->lam0;
  } else {
    return WF_EINVAL;
  }
  *out = c;
  *lam0_out = lam0;
  return WF_OK;
}

extern "C" {

static int wf_run_on(wf_plan_t P, const wf_schedule* sch, double tol, wf_stats* st) {
  const int R = P->p.residual_every;
  CtrlArgs c;
  double lam0;
  int rc0 = run_setup(P, sch, tol, &c, &lam0);
  if (rc0) return rc0;
  P->run_index += 1;
  const int nchi = chi2_scratch(P->ny, P->nx);
  if (P->p.trace == 2) c.chi_val = P->chi + nchi;  // chi^2_aug at each checkpoint, before the controller
  CKI(launch_set_lambda(P->st, lam0, 1, P->stream));
  P->launches += 1;
  const long long it0 = P->it_done;
  long long enq = it0;
  // checkpoints per chunk: check_every, or fewer when the run's cap ends
  // sooner (a short correction solve is then one captured chunk)
  const int K = (int)std::max<long long>(1, std::min<long long>(P->p.check_every, ((long long)c.max_iters + R - 1) / R));
  const long long cap = it0 + (long long)c.max_iters;
  const long long per_chunk = (long long)K * R;
  // one chunk: K checkpoints, each R sweeps then the residual and the controller
  auto enqueue_chunk = [&](long long start) -> int {
    long long e = start;
    for (int cp = 0; cp < K && e < cap; ++cp) {
      int rc = enqueue_sweeps(P, R, e);
      if (rc) return rc;
      e += R;
      rc = enqueue_residual(P, (int)(e & 1), 1);
      if (rc) return rc;
      if (P->p.trace == 2) {
        CKI(launch_chi2(chi2_fields(P), P->chi, P->chi + nchi, P->stream));
        P->launches += 3;
      }
      CKI(launch_ctrl(c, P->stream));
      P->launches += 1;
    }
    return WF_OK;
  };
  // Full chunks start on the same sweep parity when K R is even, so one
  // captured graph replays them all; it is kept while the controller
  // arguments and the start parity stay the same.
  // (the kernel arguments also depend on whether a source is loaded)
  // (built field by field: struct padding must not make equal keys differ)
  std::vector<unsigned char> key;
  auto put = [&key](const void* p, size_t n) {
    const unsigned char* b = (const unsigned char*)p;
    key.insert(key.end(), b, b + n);
  };
  const long long par = it0 & 1, src = P->has_src ? 1 : 0;
  put(&c.tol, 8); put(&c.tol_u, 8); put(&c.ratio, 8); put(&c.expo, 8); put(&c.snap, 8);
  put(&c.mode, 4); put(&c.nlevels, 4); put(&c.R, 4); put(&c.max_iters, 4); put(&c.count_iters, 4);
  put(&c.skip_fixed, 4);
  put(&par, 8); put(&src, 8);
  if (P->p.trace) put(&c.run_index, 4);  // stamped into trace records
  const bool use_graph = (per_chunk % 2 == 0);
  bool seen = false;
  for (const auto& k : P->chunk_seen) seen = seen || (k == key);
  for (;;) {
    const bool full = enq + per_chunk <= cap;
    if (use_graph && full && seen) {
      wf_plan_s::ChunkGraph* G = nullptr;
      for (auto& g : P->chunk)
        if (g.exec && g.key == key) G = &g;
      if (!G) {
        // replace the least recently used slot
        G = (P->chunk[0].last_use <= P->chunk[1].last_use) ? &P->chunk[0] : &P->chunk[1];
        if (G->exec) {
          cudaGraphExecDestroy(G->exec);
          G->exec = nullptr;
        }
        cudaGraph_t g = nullptr;
        const long long l0 = P->launches;
        CK(cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_chunk(enq);
        cudaError_t ce = cudaStreamEndCapture(P->stream, &g);
        if (rc) {
          if (g) cudaGraphDestroy(g);
          return rc;
        }
        CK(ce);
        cudaError_t ie = cudaGraphInstantiate(&G->exec, g, 0);
        cudaGraphDestroy(g);
        CK(ie);
        G->launches = P->launches - l0;
        P->launches = l0;
        G->key = key;
      }
      G->last_use = ++P->chunk_clock;
      CK(cudaGraphLaunch(G->exec, P->stream));
      P->launches += G->launches;
      enq += per_chunk;
    } else {
      const long long e0 = enq;
      int rc = enqueue_chunk(enq);
      if (rc) return rc;
      enq = std::min(cap, e0 + per_chunk);
      if (!seen) {
        P->chunk_seen.push_back(key);
        seen = true;
      }
    }
    CK(cudaMemcpyAsync(P->h_st, P->st, sizeof(WfState), cudaMemcpyDeviceToHost, P->stream));
    CK(cudaStreamSynchronize(P->stream));
    if (P->h_st->done || enq >= cap) break;
  }
  P->it_done = it0 + P->h_st->iter;
  if (P->h_st->err & WF_ERR_TIMEOUT) return WF_ETIMEOUT;
  const int hs = P->h_st->status;
  int status = hs == 3 ? WF_ENOCONV : (hs == 4 ? WF_ESTALL : WF_OK);
  fill_stats(P, st, status);
  return status;
}

// The iteration runs on the plan's own stream, ordered after the caller's
// stream on entry and before it on exit.
int wf_run(wf_plan_t P, const wf_schedule* sch, double tol, wf_stats* st) {
  if (!P || !P->loaded || !sch) return WF_EINVAL;
  cudaStream_t user = P->stream;
  CK(cudaEventRecord(P->ev_in, user));
  CK(cudaStreamWaitEvent(P->gstream, P->ev_in, 0));
  P->stream = P->gstream;
  int rc = wf_run_on(P, sch, tol, st);
  P->stream = user;
  CK(cudaEventRecord(P->ev_out, P->gstream));
  CK(cudaStreamWaitEvent(user, P->ev_out, 0));
  return rc;
}

int wf_chi2_aug(wf_plan_t P, double* value) {
  if (!P || !P->loaded || !value) return WF_EINVAL;
  if (P->has_f && !P->merge) return WF_EUNSUPPORTED;  // the plain sweep's t_2DF links are not summed
  const Chi2Fields f = chi2_fields(P);
  const int n = chi2_scratch(P->ny, P->nx);
  CKI(launch_chi2(f, P->chi, P->chi + n, P->stream));
  P->launches += 3;
  double v = 0.0;
  CK(cudaMemcpyAsync(&v, P->chi + n, sizeof(double), cudaMemcpyDeviceToHost, P->stream));
  CK(cudaStreamSynchronize(P->stream));
  *value = v;
  return WF_OK;
}

int wf_residual(wf_plan_t P, double* rel_u, double* rel_m) {
  if (!P || !P->loaded) return WF_EINVAL;
  // a residual of the current state, without touching lambda or counters
  int rc = enqueue_residual(P, (int)(P->it_done & 1), 0);
  if (rc) return rc;
  CtrlArgs c = ctrl_args(P);
  c.count_iters = 0;
  CKI(launch_ctrl(c, P->stream));
  P->launches += 1;
  CK(cudaMemcpyAsync(P->h_st, P->st, sizeof(WfState), cudaMemcpyDeviceToHost, P->stream));
  CK(cudaStreamSynchronize(P->stream));
  if (P->h_st->err & WF_ERR_TIMEOUT) return WF_ETIMEOUT;
  if (rel_u) *rel_u = P->h_st->rel_u;
  if (rel_m) *rel_m = P->h_st->rel_m;
  return WF_OK;
}

int wf_get_field(wf_plan_t P, int field, float* out) {
  if (!P || !P->loaded || !out) return WF_EINVAL;
  const int where_ = ptr_where(out);
  if (where_ == PTR_OTHER_DEVICE) return WF_EINVAL;
  const bool dev = where_ == PTR_DEVICE;
  float2* dst = dev ? (float2*)out : (float2*)P->stg_io;
  RowArgs ra = row_args(P);
  ra.out_px = dst;
  switch (field) {
    case WF_FIELD_S: {
      ColArgs ca = col_args(P, (int)(P->it_done & 1));
      CKI(launch_col(COL_RESID_A, ca, P->stream));
      P->launches += 1;
      ra.in_rf = P->r_q;
      break;
    }
    case WF_FIELD_T_2DF: {
      if (!P->has_f || P->merge) return WF_EINVAL;
      ColArgs ca = col_args(P, 0);
      ca.in = P->f_t0;
      ca.out = P->r_g;
      CKI(launch_col(COL_INV, ca, P->stream));
      P->launches += 1;
      ra.in_rf = P->r_g;
      break;
    }
    case WF_FIELD_D_2DF:
    case WF_FIELD_T_RF: {
      // column-tiled fields: to row-major first
      if (field == WF_FIELD_D_2DF && !P->has_f) return WF_EINVAL;
      if (field == WF_FIELD_T_RF && !P->has_rf) return WF_EINVAL;
      ColArgs ca = col_args(P, 0);
      ca.in = field == WF_FIELD_D_2DF ? P->f_x : P->f_t1;
      ca.out = P->r_g;
      CKI(launch_col(COL_UNTILE, ca, P->stream));
      P->launches += 1;
      ra.in_rf = P->r_g;
      break;
    }
    case WF_FIELD_D_RF:
      if (!P->has_rf) return WF_EINVAL;
      ra.in_rf = P->f_d1;
      break;
    default:
      return WF_EINVAL;
  }
  CKI(launch_row(ROW_C2R, ra, P->stream));
  P->launches += 1;
  if (!dev)
    CK(cudaMemcpyAsync(out, dst, (size_t)P->ny * P->nx * sizeof(float), cudaMemcpyDeviceToHost, P->stream));
  CK(cudaStreamSynchronize(P->stream));
  return WF_OK;
}

}  // extern "C"

// Messenger fields from an estimate of s: the data-side messengers (t_RF and
// d_RF, or t_PX without stripes) take s itself in their basis, and the
// signal-side field the value whose implicit s is s_init.
static int warm_init(wf_plan_s* P, const float* s_init) {
  if (P->has_f && !P->merge) return WF_EUNSUPPORTED;  // t_2DF would need its own T_0 history
  const size_t npx = (size_t)P->ny * P->nx;
  const float* ds = nullptr;
  int rc = to_device(P, s_init, P->stg_io, npx, &ds);
  if (rc) return rc;
  RowArgs ra = row_args(P);
  ra.in_px = (const float2*)ds;
  ra.out_rf = P->r_q;
  CKI(launch_row(ROW_R2C, ra, P->stream));
  if (P->f_d1) CK(cudaMemcpyAsync(P->f_d1, P->r_q, npx / 2 * sizeof(float2), cudaMemcpyDeviceToDevice, P->stream));
  ColArgs ca = col_args(P, 0);
  ca.in = P->r_q;
  ca.out = P->f_x;
  ca.warm_copy = P->has_rf ? P->f_t1 : P->f_y;
  CKI(launch_col(COL_WARM, ca, P->stream));
  P->launches += 2;
  return WF_OK;
}

// One wf_solve as a sequence of steps: load the problem, the first run,
// then the defect-correction solves (each a preparation, a run and a
// subtraction), the residual of the refined s, and the output.  wf_solve
// takes the steps in order with wf_run between them; a persistent batch
// (wf_batch.cu) takes each step for all its maps and runs their iterations
// together.
static bool finished_rc(int r) { return r == WF_OK || r == WF_ENOCONV || r == WF_ESTALL; }

int wf::job_start(SolveJob& J, const float* d, const float* pixel_var, const uint8_t* mask, const float* C,
                  const float* P1f, const float* Pst, const float* stripe_amp2, const float* s_init) {
  wf_plan_t P = J.P;
  if (!P || !J.s_out || !J.sched) return WF_EINVAL;
  if (ptr_where(J.s_out) == PTR_OTHER_DEVICE) return WF_EINVAL;
  int rc = wf_set_problem(P, d, pixel_var, mask, C, P1f, Pst, stripe_amp2);
  if (rc) return rc;
  if (s_init && (rc = warm_init(P, s_init))) return rc;
  return WF_OK;
}

int wf::job_after_first(SolveJob& J, int run_status, const wf_stats& s0, bool* done) {
  wf_plan_t P = J.P;
  *done = true;
  J.status = run_status;
  if (!finished_rc(run_status)) return run_status;
  if (P->p.refine == 0) {
    int rc = wf_get_field(P, WF_FIELD_S, J.s_out);
    if (rc) return rc;
    if (J.st) *J.st = s0;
    return WF_OK;
  }
  // defect correction: s <- s - WF(Delta d_u(s)), Delta d against the original d
  const size_t npx = (size_t)P->ny * P->nx;
  J.du2 = P->h_st->du2;
  CK(cudaMemcpyAsync(P->dn_orig, P->dn, npx / 2 * sizeof(float4), cudaMemcpyDeviceToDevice, P->stream));
  int rc = wf_get_field(P, WF_FIELD_S, P->s_acc);
  if (rc) return rc;
  J.tot = s0;
  P->aa_n = P->aa_head = 0;
  P->aa_have = false;
  // a source on masked pixels needs the merged 2DF block (or no 1/f part)
  J.with_src = !(P->has_f && !P->merge);
  // A capped correction runs the fixed schedule's levels for at most
  // refine_max_iters - refine_lam1_iters sweeps, then lambda = 1 for the
  // rest: the cooling levels move the slow modes, the lambda = 1 sweeps
  // remove the bias the last level leaves in the fast ones.
  const wf_schedule* sched = J.sched;
  J.csched = *sched;
  J.clam.clear();
  J.citers.clear();
  const int cap = P->p.refine_max_iters;
  if (cap > 0 && sched->mode == WF_SCHED_FIXED && sched->lam && sched->iters && sched->nlevels > 0) {
    long long left = std::max(0, cap - P->p.refine_lam1_iters);
    for (int i = 0; i < sched->nlevels && left > 0; ++i) {
      const int n = (int)std::min<long long>(std::max(0, sched->iters[i]), left);
      if (n > 0 && sched->lam[i] > 1.0) {
        J.clam.push_back(sched->lam[i]);
        J.citers.push_back(n);
        left -= n;
      }
    }
    J.clam.push_back(1.0);
    J.citers.push_back(0);
    J.csched.lam = J.clam.data();
    J.csched.iters = J.citers.data();
    J.csched.nlevels = (int)J.clam.size();
  }
  *done = false;
  return WF_OK;
}

// Anderson step for the correction e = s_corr of x = s_acc (refine_accel):
// f = -e; the newest differences Delta f = f - f_prev and Delta x (the
// previous update) enter the ring; gamma minimises ||f - Delta F gamma||_2;
// x += f - (Delta X + Delta F) gamma.  The first correction is the plain one.
// Only launches: the ring's bookkeeping is on the host, the arithmetic
// (including the least squares) on the device.
static int anderson_step(wf_plan_s* P) {
  const size_t npx = (size_t)P->ny * P->nx;
  const int m = P->p.refine_accel;
  int slot = -1;
  if (P->aa_have) {
    slot = P->aa_n < m ? P->aa_n : P->aa_head;
    std::swap(P->aa_dx[slot], P->aa_u);  // Delta x of the new column: the previous update
  }
  CKI(launch_aa_diff(slot >= 0 ? P->aa_df[slot] : nullptr, P->aa_fprev, P->s_corr, npx, P->stream));
  P->launches += 1;
  if (slot >= 0) {
    if (P->aa_n < m) P->aa_n += 1;
    else P->aa_head = (P->aa_head + 1) % m;
  }
  P->aa_have = true;
  const int n = P->aa_n;
  if (n > 0) {
    // Delta f_new . Delta f_j and f . Delta f_j for every held column, the
    // Gram matrix's new row and the least-squares gamma, on the device
    AADots d{};
    d.a0 = P->aa_df[slot];
    d.a1 = P->aa_fprev;
    for (int j = 0; j < n; ++j) d.b[j] = P->aa_df[j];
    d.nb = n;
    CKI(launch_aa_lsq(d, npx, P->aa_part, slot, P->aa_G, P->aa_gamma, P->stream));
    P->launches += 2;
  }
  AAUpdate u{};
  u.x = P->s_acc;
  u.u = P->aa_u;
  u.f = P->aa_fprev;
  for (int j = 0; j < n; ++j) {
    u.dx[j] = P->aa_dx[j];
    u.df[j] = P->aa_df[j];
  }
  u.gamma = P->aa_gamma;
  u.nj = n;
  CKI(launch_aa_update(u, npx, P->stream));
  P->launches += 1;
  return WF_OK;
}

// s of the loaded problem's current state into the device map dst (the
// kernels of wf_get_field's WF_FIELD_S, without its host wait)
static int enqueue_s_field(wf_plan_s* P, float* dst) {
  ColArgs ca = col_args(P, (int)(P->it_done & 1));
  CKI(launch_col(COL_RESID_A, ca, P->stream));
  RowArgs ra = row_args(P);
  ra.out_px = (float2*)dst;
  ra.in_rf = P->r_q;
  CKI(launch_row(ROW_C2R, ra, P->stream));
  P->launches += 2;
  return WF_OK;
}

// one correction, s_acc <- s_acc - WF(residual of s_acc): the problem of the
// correction solve (its run follows with J.csched at J.tol * refine_tol_scale
// and the plan's max_iters set to the correction cap) ...
int wf::job_corr_begin(SolveJob& J) {
  wf_plan_t P = J.P;
  const size_t npx = (size_t)P->ny * P->nx;
  const size_t nhb = (size_t)P->ny * P->M * sizeof(float2);
  // residual of the accumulated s: Delta d_u (data) and (S^-1 s)_m (source)
  int rc = enqueue_resid_map(P, P->s_acc, P->rho, P->jmap);
  if (rc) return rc;
  CKI(launch_pack_data(P->dn, P->dn_orig, P->rho, npx / 2, P->part + 3 * P->nrow, P->st, P->stream));
  P->launches += 2;
  if (J.with_src) {
    // j^ = 2D DFT of the masked-pixel source, column-tiled
    RowArgs ra = row_args(P);
    ra.in_px = P->jmap;
    ra.out_rf = P->r_q;
    CKI(launch_row(ROW_R2C, ra, P->stream));
    ColArgs ca = col_args(P, 0);
    ca.in = P->r_q;
    ca.out = P->src_2df;
    CKI(launch_col(COL_FWD_TILED, ca, P->stream));
    P->launches += 2;
    P->has_src = true;
  }
  CK(cudaMemsetAsync(P->f_x, 0, nhb, P->stream));
  if (P->f_d1) CK(cudaMemsetAsync(P->f_d1, 0, nhb, P->stream));
  if (P->f_t1) CK(cudaMemsetAsync(P->f_t1, 0, nhb, P->stream));
  if (P->f_y) CK(cudaMemsetAsync(P->f_y, 0, nhb, P->stream));
  if (P->f_t0) CK(cudaMemsetAsync(P->f_t0, 0, nhb, P->stream));
  P->it_done = 0;
  J.main_cap = P->p.max_iters;
  if (P->p.refine_max_iters > 0) P->p.max_iters = P->p.refine_max_iters;
  return WF_OK;
}

// ... and, after that run, the subtraction
int wf::job_corr_end(SolveJob& J, int run_status, const wf_stats& sr) {
  wf_plan_t P = J.P;
  const size_t npx = (size_t)P->ny * P->nx;
  P->p.max_iters = J.main_cap;
  int rc = WF_OK;
  if (finished_rc(run_status)) rc = enqueue_s_field(P, P->s_corr);
  P->has_src = false;
  if (!finished_rc(run_status)) return run_status;
  if (rc) return rc;
  // a correction that runs to refine_max_iters has done what was asked
  if (run_status != WF_OK && P->p.refine_max_iters == 0 && J.status == WF_OK) J.status = run_status;
  J.tot.iters += sr.iters;
  J.tot.checkpoints += sr.checkpoints;
  if (P->p.refine_accel > 0) {
    if ((rc = anderson_step(P))) return rc;
  } else {
    CKI(launch_sub(P->s_acc, P->s_corr, npx, P->stream));
    P->launches += 1;
  }
  J.corrections += 1;
  return WF_OK;
}

// residual of the refined s against the original problem, into h_st
int wf::job_refined_residual(SolveJob& J) {
  wf_plan_t P = J.P;
  int rc = enqueue_resid_map(P, P->s_acc, P->rho, nullptr);
  if (rc) return rc;
  CK(cudaMemcpyAsync(&P->st->du2, &J.du2, sizeof(double), cudaMemcpyHostToDevice, P->stream));
  CtrlArgs c = ctrl_args(P);
  c.count_iters = 0;
  CKI(launch_ctrl(c, P->stream));
  P->launches += 1;
  CK(cudaMemcpyAsync(P->h_st, P->st, sizeof(WfState), cudaMemcpyDeviceToHost, P->stream));
  CK(cudaStreamSynchronize(P->stream));
  return WF_OK;
}

bool wf::job_passes(const SolveJob& J) {
  const wf_plan_t P = J.P;
  return P->h_st->rel_u <= J.tol * P->p.tol_u_scale && P->h_st->rel_m <= J.tol;
}

int wf::job_finish(SolveJob& J) {
  wf_plan_t P = J.P;
  const size_t npx = (size_t)P->ny * P->nx;
  const int where_ = ptr_where(J.s_out);
  if (where_ == PTR_OTHER_DEVICE) return WF_EINVAL;
  const bool dev = where_ == PTR_DEVICE;
  CK(cudaMemcpyAsync(J.s_out, P->s_acc, npx * sizeof(float), dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     P->stream));
  CK(cudaStreamSynchronize(P->stream));
  // the plan now holds the last correction problem, not the caller's
  P->loaded = false;
  J.tot.rel_rho_u = P->h_st->rel_u;
  J.tot.rel_rho_m = P->h_st->rel_m;
  if (J.tol > 0) {
    // the refined s is judged by the stop test itself
    J.status = job_passes(J) ? WF_OK : (J.status == WF_OK ? WF_ENOCONV : J.status);
  }
  J.tot.status = J.status;
  if (J.st) *J.st = J.tot;
  return WF_OK;
}

int wf::plan_refine(const wf_plan_t P) { return P->p.refine; }
int wf::plan_refine_extra(const wf_plan_t P) { return P->p.refine_extra; }
double wf::plan_refine_tol_scale(const wf_plan_t P) { return P->p.refine_tol_scale; }

static int solve_impl(wf_plan_t P, const float* d, const float* pixel_var, const uint8_t* mask, const float* C,
                      const float* P1f, const float* Pst, const float* stripe_amp2, const float* s_init,
                      const wf_schedule* sched, double tol, float* s_out, wf_stats* st) {
  SolveJob J;
  J.P = P;
  J.sched = sched;
  J.tol = tol;
  J.s_out = s_out;
  J.st = st;
  int rc = job_start(J, d, pixel_var, mask, C, P1f, Pst, stripe_amp2, s_init);
  if (rc) return rc;
  wf_stats s0{};
  bool done = false;
  rc = job_after_first(J, wf_run(P, sched, tol, &s0), s0, &done);
  if (rc || done) return rc ? rc : J.status;
  auto correction = [&]() -> int {
    int r = job_corr_begin(J);
    if (r) return r;
    wf_stats sr{};
    const int rs = wf_run(P, &J.csched, tol * P->p.refine_tol_scale, &sr);
    return job_corr_end(J, rs, sr);
  };
  for (int r = 0; r < P->p.refine; ++r)
    if ((rc = correction())) return rc;
  if ((rc = job_refined_residual(J))) return rc;
  // further corrections only while the refined s fails the stop test
  for (int r = 0; tol > 0 && r < P->p.refine_extra && !job_passes(J); ++r) {
    if ((rc = correction())) return rc;
    if ((rc = job_refined_residual(J))) return rc;
  }
  if ((rc = job_finish(J))) return rc;
  return J.status;
}

extern "C" {

int wf_solve(wf_plan_t P, const float* d, const float* pixel_var, const uint8_t* mask, const float* C,
             const float* P1f, const float* Pst, const float* stripe_amp2, const wf_schedule* sched,
             double tol, float* s_out, wf_stats* st) {
  return solve_impl(P, d, pixel_var, mask, C, P1f, Pst, stripe_amp2, nullptr, sched, tol, s_out, st);
}

int wf_inverse_noise(wf_plan_t P, const float* d, const float* pixel_var, const uint8_t* mask, const float* P1f,
                     const float* Pst, const float* stripe_amp2, double alpha, const wf_schedule* sched, double tol,
                     float* out, wf_stats* st) {
  if (!P || !out || !sched || !(alpha > 0.0) || !isfinite(alpha) || alpha > 1e30) return WF_EINVAL;
  const size_t npx = (size_t)P->ny * P->nx, nspec = (size_t)P->ny * (P->M + 1);
  // S = alpha I: every signal eigenvalue alpha (the staging table of C)
  CKI(launch_fill(P->stg_C, (float)alpha, nspec, P->stream));
  P->launches += 1;
  // s into the plan's device staging map, then scaled into out
  int rc = solve_impl(P, d, pixel_var, mask, P->stg_C, P1f, Pst, stripe_amp2, nullptr, sched, tol, P->stg_io, st);
  if (rc != WF_OK && rc != WF_ENOCONV && rc != WF_ESTALL) return rc;
  // N^-1 d ~ alpha^-1 [alpha (alpha I + N)^-1 d]
  const int where_ = ptr_where(out);
  if (where_ == PTR_OTHER_DEVICE) return WF_EINVAL;
  const bool dev = where_ == PTR_DEVICE;
  float* dst = dev ? out : P->stg_io;
  CKI(launch_scale(dst, P->stg_io, (float)(1.0 / alpha), npx, P->stream));
  P->launches += 1;
  if (!dev) CK(cudaMemcpyAsync(out, dst, npx * sizeof(float), cudaMemcpyDeviceToHost, P->stream));
  CK(cudaStreamSynchronize(P->stream));
  return rc;
}

int wf_solve_warm(wf_plan_t P, const float* d, const float* pixel_var, const uint8_t* mask, const float* C,
                  const float* P1f, const float* Pst, const float* stripe_amp2, const float* s_init,
                  const wf_schedule* sched, double tol, float* s_out, wf_stats* st) {
  if (!s_init) return WF_EINVAL;
  return solve_impl(P, d, pixel_var, mask, C, P1f, Pst, stripe_amp2, s_init, sched, tol, s_out, st);
}

int wf_fft2(wf_plan_t P, const float* in, float* out, int inverse, int rows_only) {
  if (!P || !in || !out) return WF_EINVAL;
  const size_t n = (size_t)P->ny * P->nx;
  const float* din;
  int rc = to_device(P, in, P->stg_d, n, &din);
  if (rc) return rc;
  const int where_ = ptr_where(out);
  if (where_ == PTR_OTHER_DEVICE) return WF_EINVAL;
  const bool dev = where_ == PTR_DEVICE;
  float* dout = dev ? out : P->stg_io;
  RowArgs ra = row_args(P);
  ColArgs ca = col_args(P, 0);
  if (!inverse) {
    ra.in_px = (const float2*)din;
    ra.out_rf = rows_only ? (float2*)dout : P->r_g;
    CKI(launch_row(ROW_R2C, ra, P->stream));
    P->launches += 1;
    if (!rows_only) {
      ca.in = P->r_g;
      ca.out = (float2*)dout;
      CKI(ca.prec ? launch_col_dft_tc(0, ca, P->stream) : launch_col(COL_FWD, ca, P->stream));
      P->launches += 1;
    }
  } else {
    const float2* rin = (const float2*)din;
    if (!rows_only) {
      ca.in = rin;
      ca.out = P->r_g;
      CKI(ca.prec ? launch_col_dft_tc(1, ca, P->stream) : launch_col(COL_INV, ca, P->stream));
      P->launches += 1;
      rin = P->r_g;
    }
    ra.in_rf = rin;
    ra.out_px = (float2*)dout;
    CKI(launch_row(ROW_C2R, ra, P->stream));
    P->launches += 1;
  }
  if (!dev) CK(cudaMemcpyAsync(out, dout, n * sizeof(float), cudaMemcpyDeviceToHost, P->stream));
  CK(cudaStreamSynchronize(P->stream));
  return WF_OK;
}

long long wf_launch_count(wf_plan_t P) { return P ? P->launches : -1; }

int wf_plan_shapes(wf_plan_t P, int* row_values, int* col_values) {
  if (!P) return WF_EINVAL;
  if (row_values) *row_values = row_pass_e(P->M, P->row_variant);
  if (col_values) *col_values = col_pass_e(P->ny, P->p.dft_precision ? 0 : P->col_variant);
  return WF_OK;
}

int wf_time_passes(wf_plan_t P, double lam, int n, double* us_row, double* us_col) {
  if (!P || !P->loaded || n < 1 || !(lam >= 1.0) || !isfinite(lam)) return WF_EINVAL;
  // n launches of one pass captured back to back in a graph on the plan's
  // stream, timed by events around the replay: the per-launch time without
  // host launch overhead.  The plan's stream starts after the work already
  // queued on the caller's stream (earlier iterations must not overlap the
  // timed replays).
  cudaStream_t user = P->stream;
  CK(cudaEventRecord(P->ev_in, user));
  CK(cudaStreamWaitEvent(P->gstream, P->ev_in, 0));
  P->stream = P->gstream;
  int rc = WF_OK;
  double res[2] = {0.0, 0.0};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = WF_ECUDA;
  if (!rc && launch_set_lambda(P->st, lam, 1, P->stream)) rc = WF_ECUDA;
  // one un-captured launch of each pass first (kernel attributes)
  if (!rc) rc = enqueue_row_pass(P);
  if (!rc) rc = enqueue_col_pass(P, (int)(P->it_done & 1));
  for (int which = 0; which < 2 && !rc; ++which) {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    if (cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      rc = WF_ECUDA;
      break;
    }
    for (int i = 0; i < n && !rc; ++i)
      rc = which == 0 ? enqueue_row_pass(P) : enqueue_col_pass(P, (int)(P->it_done & 1));
    cudaError_t ce = cudaStreamEndCapture(P->stream, &g);
    if (rc || ce != cudaSuccess || cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      rc = rc ? rc : WF_ECUDA;
      break;
    }
    cudaGraphDestroy(g);
    float ms = 0.f;
    if (cudaGraphLaunch(ge, P->stream) != cudaSuccess ||  // warm
        cudaEventRecord(e0, P->stream) != cudaSuccess || cudaGraphLaunch(ge, P->stream) != cudaSuccess ||
        cudaEventRecord(e1, P->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      rc = WF_ECUDA;
    res[which] = 1000.0 * ms / n;
    cudaGraphExecDestroy(ge);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(P->stream);
  P->stream = user;
  // the state has moved on by an unknown number of column passes
  P->loaded = false;
  if (rc) return rc;
  if (us_row) *us_row = res[0];
  if (us_col) *us_col = res[1];
  return WF_OK;
}

int wf_get_trace(wf_plan_t P, double* out, int max_records, int* n_out) {
  if (!P || !P->trace || max_records < 0 || (!out && max_records > 0)) return WF_EINVAL;
  int n = 0;
  CK(cudaMemcpyAsync(&n, P->trace_n, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
  CK(cudaStreamSynchronize(P->stream));
  n = std::min(n, WF_TRACE_CAP);
  const int k = std::min(n, max_records);
  if (k > 0) {
    const int where_ = ptr_where(out);
    if (where_ == PTR_OTHER_DEVICE) return WF_EINVAL;
    CK(cudaMemcpyAsync(out, P->trace, (size_t)k * WF_TRACE_FIELDS * sizeof(double),
                       where_ == PTR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, P->stream));
    CK(cudaStreamSynchronize(P->stream));
  }
  if (n_out) *n_out = n;
  return WF_OK;
}

int wf_time_sweeps(wf_plan_t P, double lam, int n, double* us_per_sweep, int* one_launch) {
  if (!P || !P->loaded || n < 1 || !(lam >= 1.0) || !isfinite(lam)) return WF_EINVAL;
  // n sweeps as the plan's iteration runs them (one cooperative launch, or
  // n row-pass / column-pass pairs), captured in a graph on the plan's
  // stream and timed by events around its replay, after the work already
  // queued on the caller's stream
  cudaStream_t user = P->stream;
  CK(cudaEventRecord(P->ev_in, user));
  CK(cudaStreamWaitEvent(P->gstream, P->ev_in, 0));
  P->stream = P->gstream;
  int rc = WF_OK;
  float ms = 0.f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = WF_ECUDA;
  if (!rc && launch_set_lambda(P->st, lam, 1, P->stream)) rc = WF_ECUDA;
  if (!rc) rc = enqueue_sweeps(P, 1, P->it_done);  // un-captured first: kernel attributes
  if (!rc && cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = WF_ECUDA;
  if (!rc) {
    rc = enqueue_sweeps(P, n, P->it_done);
    cudaError_t ce = cudaStreamEndCapture(P->stream, &g);
    if (!rc && (ce != cudaSuccess || cudaGraphInstantiate(&ge, g, 0) != cudaSuccess)) rc = WF_ECUDA;
  }
  if (!rc && (cudaGraphLaunch(ge, P->stream) != cudaSuccess ||  // warm
              cudaEventRecord(e0, P->stream) != cudaSuccess || cudaGraphLaunch(ge, P->stream) != cudaSuccess ||
              cudaEventRecord(e1, P->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
              cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
    rc = WF_ECUDA;
  if (ge) cudaGraphExecDestroy(ge);
  if (g) cudaGraphDestroy(g);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc) cudaGetLastError();
  cudaStreamSynchronize(P->stream);
  P->stream = user;
  // the state has moved on by 2n + 1 sweeps
  P->loaded = false;
  if (!rc && P->h_st && cudaMemcpy(P->h_st, P->st, sizeof(WfState), cudaMemcpyDeviceToHost) == cudaSuccess &&
      (P->h_st->err & WF_ERR_TIMEOUT))
    rc = WF_ETIMEOUT;
  if (rc) return rc;
  if (us_per_sweep) *us_per_sweep = 1000.0 * ms / n;
  if (one_launch) *one_launch = P->fused ? 1 : 0;
  return WF_OK;
}

}  // extern "C"
