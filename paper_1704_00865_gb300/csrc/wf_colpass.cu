// wf_colpass.cu -- dispatch of the column pass (wf_colpass.cuh) by column
// length, mode and shape, and its FP32 instantiations.
#include "wf_colpass.cuh"

namespace wf {

// a.variant selects the shape (0 or 1, ColPassE)
template <int L, int MODE>
static int launch_col_pass(const ColArgs& a, cudaStream_t s) {
  if constexpr (ColPassE<L>::v1 != ColPassE<L>::v0) {
    if (a.variant == 1) return launch_col_pass_e<L, MODE, ColPassE<L>::v1>(a, s);
  }
  return launch_col_pass_e<L, MODE, ColPassE<L>::v0>(a, s);
}

template <int L>
int launch_col_pass_any(int mode, const ColArgs& a, cudaStream_t s) {
  if (a.prec != 0) return launch_col_pass_tc(L, mode, a, s);
  switch (mode) {
    case COL_PASS_2DF: return launch_col_pass<L, COL_PASS_2DF>(a, s);
    case COL_PASS_NO2DF:  // the merged update with N0 = 0
    case COL_PASS_MERGE: return launch_col_pass<L, COL_PASS_MERGE>(a, s);
    case COL_PASS_MERGE_SRC: return launch_col_pass<L, COL_PASS_MERGE_SRC>(a, s);
    default: return (int)cudaErrorInvalidValue;
  }
}

template <int L>
static int col_e(int v) { return v == 1 ? ColPassE<L>::v1 : ColPassE<L>::v0; }

int col_pass_e(int L, int v) {
  switch (L) {
    case 32: return col_e<32>(v);
    case 64: return col_e<64>(v);
    case 128: return col_e<128>(v);
    case 256: return col_e<256>(v);
    case 384: return col_e<384>(v);
    case 512: return col_e<512>(v);
    case 768: return col_e<768>(v);
    case 1024: return col_e<1024>(v);
    case 1536: return col_e<1536>(v);
    case 2048: return col_e<2048>(v);
    case 4096: return col_e<4096>(v);
    default: return 0;
  }
}

template int launch_col_pass_any<32>(int, const ColArgs&, cudaStream_t);
template int launch_col_pass_any<64>(int, const ColArgs&, cudaStream_t);
template int launch_col_pass_any<128>(int, const ColArgs&, cudaStream_t);
template int launch_col_pass_any<256>(int, const ColArgs&, cudaStream_t);
template int launch_col_pass_any<384>(int, const ColArgs&, cudaStream_t);
template int launch_col_pass_any<512>(int, const ColArgs&, cudaStream_t);
template int launch_col_pass_any<768>(int, const ColArgs&, cudaStream_t);
template int launch_col_pass_any<1024>(int, const ColArgs&, cudaStream_t);
template int launch_col_pass_any<1536>(int, const ColArgs&, cudaStream_t);
template int launch_col_pass_any<2048>(int, const ColArgs&, cudaStream_t);
template int launch_col_pass_any<4096>(int, const ColArgs&, cudaStream_t);

}  // namespace wf
