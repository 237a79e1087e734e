// wf_colpass_tc.cu -- the column transforms with their radix-16 stages on the
// tensor cores (DFT as GEMM, wf_device.cuh): the column pass of the messenger
// iteration for the merged 2DF block (with and without a source) and the
// plain column DFTs of wf_fft2, for column lengths 512 to 4096, where every
// thread holds 16 values and all stages but the last are radix 16.
#include "wf_colpass.cuh"

namespace wf {
namespace {

template <int L, int PREC>
int col_pass_tc_L(int mode, const ColArgs& a, cudaStream_t s) {
  static_assert(ColPassE<L>::v0 == 16, "tensor-core stages need 16 values per thread");
  switch (mode) {
    case COL_PASS_NO2DF:  // the merged update with N0 = 0
    case COL_PASS_MERGE: return launch_col_pass_e<L, COL_PASS_MERGE, 16, PREC>(a, s);
    case COL_PASS_MERGE_SRC: return launch_col_pass_e<L, COL_PASS_MERGE_SRC, 16, PREC>(a, s);
    default: return (int)cudaErrorInvalidValue;
  }
}

template <int PREC>
int col_pass_tc_p(int L, int mode, const ColArgs& a, cudaStream_t s) {
  switch (L) {
    case 512: return col_pass_tc_L<512, PREC>(mode, a, s);
    case 1024: return col_pass_tc_L<1024, PREC>(mode, a, s);
    case 2048: return col_pass_tc_L<2048, PREC>(mode, a, s);
    case 4096: return col_pass_tc_L<4096, PREC>(mode, a, s);
    default: return (int)cudaErrorInvalidValue;
  }
}

// Column DFT of a row-major [L][ncols] complex field (wf_fft2): W columns per
// CTA, L/16 threads per column, 16 values per thread.
template <int L>
struct DftCfg {
  static constexpr int E = 16;
  static constexpr int TPC = L / E;
  static constexpr int W0 = 256 / TPC;
  static constexpr int W = W0 < 1 ? 1 : (W0 > 32 ? 32 : W0);
  static constexpr int THREADS = W * TPC;
  static constexpr int SP = SPad<L>::size;
  static constexpr int WANT = (W >= 32) ? 1 : (16 / W) % 16;
  static constexpr int STRIDE = SP + ((WANT - SP % 16) + 16) % 16;
};

template <int L, bool INV, int PREC>
__global__ void __launch_bounds__(DftCfg<L>::THREADS) col_dft_kernel(ColArgs a) {
  using Cfg = DftCfg<L>;
  constexpr int E = Cfg::E, TPC = Cfg::TPC, W = Cfg::W;
  __shared__ __align__(16) float2 sbuf[W][Cfg::STRIDE];
  pdl_trigger();
  pdl_wait();
  const int c = threadIdx.x % W;
  const int t = threadIdx.x / W;
  const int ncols = a.nx / 2;
  const int col = blockIdx.x * W + c;
  const bool valid = col < ncols;  // every thread takes part in the transform
  float2 v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = valid ? a.in[(size_t)(t + m * TPC) * ncols + col] : make_float2(0.f, 0.f);
  fft_block<L, E, INV, false, false, PREC>(v, sbuf[c], t, a.twy, 1);
  const float sc = INV ? 1.0f / (float)L : 1.0f;
  if (valid) {
#pragma unroll
    for (int m = 0; m < E; ++m) a.out[(size_t)(t + m * TPC) * ncols + col] = cscale(v[m], sc);
  }
}

template <int L, int PREC>
int col_dft_L(int inverse, const ColArgs& a, cudaStream_t s) {
  using Cfg = DftCfg<L>;
  const int ncols = a.nx / 2;
  const dim3 grid((ncols + Cfg::W - 1) / Cfg::W), block(Cfg::THREADS);
  if (inverse) return launch_pdl(col_dft_kernel<L, true, PREC>, grid, block, 0, s, a);
  return launch_pdl(col_dft_kernel<L, false, PREC>, grid, block, 0, s, a);
}

template <int PREC>
int col_dft_p(int inverse, const ColArgs& a, cudaStream_t s) {
  switch (a.ny) {
    case 512: return col_dft_L<512, PREC>(inverse, a, s);
    case 1024: return col_dft_L<1024, PREC>(inverse, a, s);
    case 2048: return col_dft_L<2048, PREC>(inverse, a, s);
    case 4096: return col_dft_L<4096, PREC>(inverse, a, s);
    default: return (int)cudaErrorInvalidValue;
  }
}

// tcgen05 stages (PREC 3, 4): the column pass for 512- and 1024-long
// columns, where the operand tiles fit beside the pass's own staging
template <int PREC>
int col_pass_tc5_p(int L, int mode, const ColArgs& a, cudaStream_t s) {
  switch (L) {
    case 512: return col_pass_tc_L<512, PREC>(mode, a, s);
    case 1024: return col_pass_tc_L<1024, PREC>(mode, a, s);
    default: return (int)cudaErrorInvalidValue;
  }
}

}  // namespace

bool col_tc_supported(int L) { return L == 512 || L == 1024 || L == 2048 || L == 4096; }
bool col_tc5_supported(int L) { return L == 512 || L == 1024; }

int launch_col_pass_tc(int L, int mode, const ColArgs& a, cudaStream_t s) {
  if (a.prec == 1) return col_pass_tc_p<1>(L, mode, a, s);
  if (a.prec == 2) return col_pass_tc_p<2>(L, mode, a, s);
  if (a.prec == 3) return col_pass_tc5_p<3>(L, mode, a, s);
  if (a.prec == 4) return col_pass_tc5_p<4>(L, mode, a, s);
  return (int)cudaErrorInvalidValue;
}

// wf_fft2's column DFTs: the tcgen05 precisions take the mma.sync stages of
// the same arithmetic (3 -> split TF32, 4 -> TF32)
int launch_col_dft_tc(int inverse, const ColArgs& a, cudaStream_t s) {
  if (a.prec == 1 || a.prec == 3) return col_dft_p<1>(inverse, a, s);
  if (a.prec == 2 || a.prec == 4) return col_dft_p<2>(inverse, a, s);
  return (int)cudaErrorInvalidValue;
}

}  // namespace wf
