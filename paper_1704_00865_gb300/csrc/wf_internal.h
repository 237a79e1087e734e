// wf_internal.h -- kernel argument blocks and launchers shared between the
// translation units of libwf (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/wf.h"

namespace wf {

struct WfState;

// Fields that both passes touch -- the data-side messenger in RF (t_RF, or
// t_PX without stripes), the field next to it on the signal side (d_2DF, or
// s without a 1/f part), and the (C, P1f) table -- are stored in column
// tiles of WF_TW complex columns: element (y, kx) lives at
//   (kx / WF_TW) * ny * WF_TW + y * WF_TW + kx % WF_TW,
// so a column pass reads whole tiles contiguously and a row pass reads
// 32-byte pieces.  Row-only fields (d_RF, the pixel table) stay row-major.
constexpr int WF_TW = 4;

// Kernels of the iteration are launched with programmatic stream
// serialisation: the next kernel's CTAs may start (and prefetch the tables
// that stay fixed during a solve) while the previous kernel drains; each
// kernel waits for its predecessor with griddepcontrol.wait before it reads
// anything the iteration writes.
#ifndef WF_PDL
#define WF_PDL 1
#endif
// 1: the passes release the next kernel at entry; 0: after their last
// transform, before the stores
#ifndef WF_PDL_EARLY
#define WF_PDL_EARLY 0
#endif
template <typename... KArgs, typename... Args>
inline int launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                      Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = WF_PDL;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  // the return value is this launch's own status (an error left pending by
  // an earlier, unrelated call is not collected here)
  return (int)cudaLaunchKernelEx(&cfg, kernel, args...);
}
__host__ __device__ __forceinline__ size_t tidx(int y, int kx, int ny) {
  return (size_t)(kx / WF_TW) * ny * WF_TW + (size_t)y * WF_TW + (kx % WF_TW);
}

// Row-pass modes (one CTA handles ROWS map rows; each row is one real DFT).
enum RowMode : int {
  ROW_PASS_RF = 0,    // t_PX update between the row transforms, then d_RF, t_RF
  ROW_PASS_NORF = 1,  // t_PX update only (no stripe part); writes t_PX in RF
  ROW_RESID_B = 2,    // residual: g, s to pixels; N_PX g' + s - d; N_RF g'
  ROW_RESID_D = 3,    // residual: Delta d to pixels; ||rho_u||^2
  ROW_C2R = 4,        // RF -> pixel (export)
  ROW_R2C = 5,        // pixel -> RF
  ROW_NMODES = 6
};

// Column-pass modes (one CTA handles W complex columns of length ny).
enum ColMode : int {
  COL_PASS_2DF = 0,   // d_2DF, t_2DF updates between the column transforms
  COL_PASS_NO2DF = 1, // s update only (no 1/f part); writes s in RF
  COL_RESID_A = 2,    // residual: g = S^-1 s and s, to RF
  COL_RESID_C = 3,    // residual: add N_2DF g' (in RF)
  COL_FWD = 4,        // RF -> 2D Fourier
  COL_INV = 5,        // 2D Fourier -> RF (with 1/ny)
  COL_PASS_MERGE = 6, // joint (s, t_2DF, d_2DF) update given the RF messenger
  COL_G_FROM_S = 7,   // residual of a given s: g = S^-1 s from s in RF
  COL_UNTILE = 8,     // column-tiled RF field -> row-major (exports)
  COL_FWD_TILED = 9,  // RF -> 2D Fourier, column-tiled output
  COL_PASS_MERGE_SRC = 10,  // COL_PASS_MERGE with a source term (defect correction)
  COL_WARM = 11,      // warm start: s in RF -> the signal-side field (tiled) and a tiled copy
  COL_NMODES = 11
};

struct RowArgs {
  int ny, nx;
  int has_rf;                 // stripe part present
  int check_done;             // return at once when the solver is done
  int skip_ok;                // residual kernels: return at once when st->skip_resid
  const float4* dn;           // [ny][nx/2] pixel pairs (d0, nb0, d1, nb1); nb < 0 = masked
  float2* f_d1;               // RF fields [ny][nx/2]
  float2* f_t1;
  const float2* f_x;          // signal-side neighbour in RF (d_2DF or s)
  float2* f_y;                // t_PX in RF (no stripe part)
  const float* pst;           // [nx/2+1] stripe eigenvalues
  const float* a2;            // [ny] a(y)^2 or nullptr
  const float2* twx;          // exp(-2 pi i k/nx), k < nx
  const float2* twh;          // exp(-2 pi i k/(nx/2)), k < nx/2 (row pass)
  WfState* st;
  float2* r_g;                // residual scratch (RF)
  float2* r_q;
  double* part0;              // per-CTA partial sums
  double* part1;
  const float2* in_rf;        // generic transforms
  float2* out_rf;
  const float2* in_px;        // pixel pairs
  float2* out_px;
  const float2* src_px;       // source j on masked pixels (pairs) or nullptr
  float2* gm_out;             // S^-1 s on masked pixels (pairs), 0 elsewhere, or nullptr
  int variant;                // row pass shape (0 or 1), chosen by the autotuner
};

struct ColArgs {
  int ny, nx;
  int has_rf, has_f;
  int merge;                  // 2DF block updated jointly (no stored t_2DF)
  int check_done;             // return at once when the solver is done
  int skip_ok;                // residual kernels: return at once when st->skip_resid
  int parity;                 // slot of T0s holding the stored t_2DF's T_0
  const float2* f_y;          // data-side messenger in RF (t_RF or t_PX)
  float2* f_x;                // output in RF (d_2DF or s)
  float2* f_t0;               // t_2DF [ny][nx/2] (2D Fourier)
  const float2* eig;          // [ny][nx/2] (C, P1f) for kx = col
  const float2* eig_nyq;      // [ny] (C, P1f) at kx = nx/2
  const float2* twy;          // exp(-2 pi i k/ny), k < ny
  WfState* st;
  float2* r_g;
  float2* r_q;
  const float2* in;           // generic transforms
  float2* out;
  const float2* src;          // 2D-Fourier source j^ (column-tiled) or nullptr
  float2* warm_copy;          // COL_WARM: tiled copy of the input (t_RF or t_PX)
  int variant;                // column pass shape (0 or 1), chosen by the autotuner
  int prec;                   // radix-16 stages of the column pass: 0 FP32, 1 split TF32, 2 TF32
  int prefetch;               // column pass: hint the tiles of the CTA one wave ahead into L2
  int pf;                     // (set by the launcher) that distance in CTAs, 0 = off
};

// CTAs of a kernel resident at once on the current device (SMs x CTAs per
// SM for the block and dynamic shared memory), or 0 if the query fails: the
// distance one wave ahead, for L2 prefetch hints
template <typename K>
int resident_ctas(K kernel, int threads, size_t smem) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return sms * per_sm;
}

// launchers (return a cudaError_t as int)
int launch_row(int mode, const RowArgs& a, cudaStream_t s);
int launch_col(int mode, const ColArgs& a, cudaStream_t s);
int row_grid(int nx, int ny);  // CTAs of a row pass (size of partial-sum arrays)
bool size_supported(int n);
// argument checks of wf_plan_create (host only; WF_OK or a WF_E* code)
int check_plan_args(int ny, int nx, unsigned parts, const wf_params* p);
// the column pass and the column transforms of wf_fft2 with tensor-core
// radix-16 stages (a.prec = 1 or 2; column lengths 512 to 4096, merged 2DF
// block); cudaErrorInvalidValue for other lengths or modes
int launch_col_pass_tc(int L, int mode, const ColArgs& a, cudaStream_t s);
int launch_col_dft_tc(int inverse, const ColArgs& a, cudaStream_t s);
bool col_tc_supported(int L);
bool col_tc5_supported(int L);  // tcgen05 stages (dft_precision 3, 4)
// values per thread of the row / column pass shape `variant` for a length
int row_pass_e(int M, int variant);
int col_pass_e(int L, int variant);

// The whole sweep, nsweeps times, in one cooperative launch (wf_fused.cu):
// 1024 x 1024 maps with a stripe part and the merged 2DF block.
struct FusedArgs {
  int ny, nx;
  int nsweeps;
  const float4* dn;           // pixel table
  float2* f_d1;               // d_RF, row-major RF
  float2* f_t1;               // t_RF, column-tiled RF
  float2* f_x;                // d_2DF, column-tiled RF
  const float2* eig;          // (C, P1f), column-tiled
  const float2* eig_nyq;      // (C, P1f) at kx = nx/2
  const float* pst;           // stripe eigenvalues
  const float* a2;            // a(y)^2 or nullptr
  const float2* twx;          // exp(-2 pi i k/nx)
  const float2* twh;          // exp(-2 pi i k/(nx/2))
  const float2* twy;          // exp(-2 pi i k/ny)
  const float2* src;          // 2D-Fourier source j^, column-tiled (src = 1)
  WfState* st;
  unsigned* bar;              // grid barrier words: arrivals (zeroed before each launch), -, abort
};
int launch_fused(const FusedArgs& a, cudaStream_t s);
// whether the one-launch sweep handles this plan on the current device
bool fused_supported(int ny, int nx, int has_rf, int merged, int prec);

// One map of a persistent batch (wf_batchk.cu): its size class and the
// fields and tables its row and column items use.
struct BatchMapArgs {
  int cls;                    // 2 * (index of the size) + shape, batch_class()
  const float4* dn;
  float2* f_d1;
  float2* f_t1;
  float2* f_x;
  const float2* eig;
  const float2* eig_nyq;
  const float* pst;
  const float* a2;            // or nullptr
  const float2* twx;
  const float2* twh;
  const float2* twy;
  const float2* src;          // 2D-Fourier source (defect correction) or nullptr
  WfState* st;
};
struct BatchArgs {
  const BatchMapArgs* maps;
  const int2* row_items;      // (map, row group) work queue of the row phase
  const int2* col_items;      // (map, column group) work queue of the column phase
  int n_row, n_col;
  int nsweeps;
  unsigned* bar;              // grid barrier words (zeroed before each launch)
  unsigned* queue;            // 2 nsweeps work counters (zeroed before each launch)
  unsigned* err;              // WF_ERR_TIMEOUT if a barrier wait gave up
};
int batch_class(int n, int variant);            // -1: size not handled
bool batch_has_second_shape(int n);
int batch_item_shape(int cls, int* rows_per_item, int* cols_per_item, int* row_values, int* col_values);
int batch_grid();                                 // CTAs of a launch (0: cannot launch)
int launch_batch_sweeps(const BatchArgs& a, int grid, cudaStream_t s);

// Device buffers of a persistent batch and the runner that iterates several
// loaded plans together (wf_api.cu).
struct BatchDevice {
  BatchMapArgs* maps = nullptr;
  int2* rows = nullptr;
  int2* cols = nullptr;
  unsigned* bar = nullptr;    // 4 words
  unsigned* queue = nullptr;  // 2 residual_every words
  unsigned* err = nullptr;
  size_t cap_maps = 0, cap_items = 0;
  int grid = 0;               // CTAs of a launch
  long long launches = 0;     // persistent launches so far
  long long per_plan_launches = 0;
  std::vector<int2> row_items, col_items;
};
int plan_batch_map(wf_plan_t P, int variant, BatchMapArgs* out);
bool plan_batch_ok(const wf_plan_t P);
int plan_size(const wf_plan_t P);
int plan_autotune(const wf_plan_t P);
int time_batch_variant(wf_plan_t P, int variant, BatchDevice& bd, cudaStream_t s, double* us);
int run_plans_persistent(const std::vector<wf_plan_t>& plans, const std::vector<int>& variant,
                         const wf_schedule* sch, double tol, BatchDevice& bd, cudaStream_t s,
                         std::vector<int>& status, std::vector<wf_stats>& st);

// The steps of one wf_solve (wf_api.cu): load, first run, corrections,
// refined residual, output.  A persistent batch takes each step for all its
// maps and runs their iterations together between the steps.
struct SolveJob {
  wf_plan_t P = nullptr;
  const wf_schedule* sched = nullptr;
  double tol = 0.0;
  float* s_out = nullptr;
  wf_stats* st = nullptr;
  int status = WF_OK;
  wf_stats tot{};
  double du2 = 0.0;
  bool with_src = false;
  wf_schedule csched{};        // schedule of the correction solves
  std::vector<double> clam;
  std::vector<int> citers;
  int main_cap = 0;            // max_iters while a correction's cap is in force
  int corrections = 0;
};
int job_start(SolveJob& J, const float* d, const float* pixel_var, const uint8_t* mask, const float* C,
              const float* P1f, const float* Pst, const float* stripe_amp2, const float* s_init);
int job_after_first(SolveJob& J, int run_status, const wf_stats& s0, bool* done);
int job_corr_begin(SolveJob& J);
int job_corr_end(SolveJob& J, int run_status, const wf_stats& sr);
int job_refined_residual(SolveJob& J);
bool job_passes(const SolveJob& J);
int job_finish(SolveJob& J);
int plan_refine(const wf_plan_t P);
int plan_refine_extra(const wf_plan_t P);
double plan_refine_tol_scale(const wf_plan_t P);

// setup / control kernels
struct SetupArgs {
  int ny, nx;
  const float* d;
  const float* var;
  const uint8_t* mask;
  const float* C;
  const float* P1f;
  const float* Pst;
  const float* a2;
  float4* dn;
  float2* eig;
  float2* eig_nyq;
  float* pst;
  float* a2_out;
  double* part;               // scratch for partial minima / sums
  WfState* st;
  double theta[3];
  double split_f, split_fp, split_w;
  int has_rf, has_f;
  int merge;
};
int launch_setup(const SetupArgs& a, cudaStream_t s);

struct CtrlArgs {
  WfState* st;
  const double* part_g;       // [nrow] (gm2, g2) partials from ROW_RESID_B
  const double* part_g2;
  const double* part_rho;     // [nrow] rho^2 partials from ROW_RESID_D
  int nrow;
  int R;
  int max_iters;
  double tol;
  double tol_u;
  int mode;                   // 0 fixed, 1 adaptive
  const double* lam_sched;    // fixed: device arrays
  const int* it_sched;
  int nlevels;
  double ratio, expo, snap;
  int count_iters;            // add R to iter (0 for a residual-only call)
  int skip_fixed;             // fixed schedule: skip residuals nothing uses (st->skip_resid)
  int stall;                  // stop after this many checkpoints at lambda = 1
                              // without a 1% drop of ||Delta d_u||^2 (0: never)
  double* trace;              // per-checkpoint records (6 doubles each) or nullptr
  int* trace_n;               // records written so far
  int trace_cap;
  int run_index;              // stamped into the records
  const double* chi_val;      // chi^2_aug of this checkpoint (trace = 2) or nullptr
};
constexpr int WF_TRACE_CAP = 8192;
constexpr int WF_TRACE_FIELDS = 6;
int launch_ctrl(const CtrlArgs& a, cudaStream_t s);
int launch_set_lambda(WfState* st, double lam, int reset, cudaStream_t s);
// refinement helpers: dn_out = (rho, Nbar of dn_in) per pixel and ||rho_u||^2
// into st->du2; and y -= x
int launch_pack_data(float4* dn_out, const float4* dn_in, const float2* rho, size_t npair,
                     double* part, WfState* st, cudaStream_t s);
int launch_sub(float* y, const float* x, size_t n, cudaStream_t s);

// Anderson-accelerated defect correction (wf_accel.cu): history of at most
// WF_AA_MAX corrections
constexpr int WF_AA_MAX = 16;
struct AADots {               // a0 . b_j and a1 . b_j, j < nb
  const float* a0;
  const float* a1;
  const float* b[WF_AA_MAX];
  int nb;
};
struct AAUpdate {             // u = f - sum_j gamma_j (dx_j + df_j); x += u
  float* x;
  float* u;
  const float* f;
  const float* dx[WF_AA_MAX];
  const float* df[WF_AA_MAX];
  const float* gamma;         // device, WF_AA_MAX values
  int nj;
};
int aa_dots_blocks();         // partial sums per dot product (upper bound)
int launch_aa_diff(float* df, float* fprev, const float* e, size_t n, cudaStream_t s);
// the dot products a0 . b_j, a1 . b_j, then row and column `slot` of the Gram
// matrix G (WF_AA_MAX x WF_AA_MAX doubles) and gamma (WF_AA_MAX floats) of
// (G + eps diag) gamma = (a1 . b_j), all in device memory
int launch_aa_lsq(const AADots& a, size_t n, double* part, int slot, double* G, float* gamma, cudaStream_t s);
int launch_aa_update(const AAUpdate& a, size_t n, cudaStream_t s);
// y[i] = v;  y[i] = a x[i]
int launch_fill(float* y, float v, size_t n, cudaStream_t s);

// augmented objective of the kept fields (wf_chi.cu)
struct Chi2Fields {
  int ny, nx, has_rf;
  const float2* d0;           // d_2DF (or s) in RF, column-tiled
  const float2* t;            // t_RF (stripe part) or t_PX, RF, column-tiled
  const float2* d1;           // d_RF row-major, or nullptr
  const float4* dn;
  const float2* eig;
  const float2* eig_nyq;
  const float* pst;
  const float* a2;
  const float2* twx;
  const float2* twy;
  const WfState* st;
};
int chi2_scratch(int ny, int nx);  // doubles of scratch launch_chi2 needs (0: unsupported size)
int launch_chi2(const Chi2Fields& f, double* scratch, double* out, cudaStream_t s);
int launch_scale(float* y, const float* x, float a, size_t n, cudaStream_t s);

}  // namespace wf
