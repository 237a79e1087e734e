// wf_accel.cu -- the device side of the Anderson-accelerated defect
// correction (wf_params.refine_accel): with x = s and f = -e the correction
// a solve returns for x, keep the differences of consecutive f and x, take
// the FP64 dot products, solve the small least-squares problem, and form
// the update -- all on the device, so a correction needs no host round trip.
// Every map is a flat array of n floats (n a multiple of 4, 16-byte aligned).
#include <cuda_runtime.h>

#include <algorithm>

#include "wf_internal.h"

namespace wf {
namespace {

constexpr int kThreads = 256;

// f = -e; with a previous f, df = f - f_prev; then f_prev = f
__global__ void aa_diff_kernel(float4* df, float4* fprev, const float4* e, size_t n4) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
    const float4 v = e[i];
    const float4 f = make_float4(-v.x, -v.y, -v.z, -v.w);
    if (df != nullptr) {
      const float4 p = fprev[i];
      df[i] = make_float4(f.x - p.x, f.y - p.y, f.z - p.z, f.w - p.w);
    }
    fprev[i] = f;
  }
}

__device__ __forceinline__ float dot4(const float4 a, const float4 b) {
  return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}

// Per-block partial sums of a0 . b_j and a1 . b_j (j < nb) in a fixed order:
// each thread its grid-stride share in FP32 (a few float4 per thread), the
// warp's 32 lanes in FP32 by a shuffle tree, then the block's warps in FP64.
// The FP64 units of this GPU are few, so FP64 is kept to the sums of
// partials (about 2.5e-7 relative error per warp sum of a few hundred
// products, below the FP32 maps' own precision).
__global__ void __launch_bounds__(kThreads) aa_dots_kernel(AADots a, size_t n4, double* part) {
  float acc[2 * WF_AA_MAX];
#pragma unroll
  for (int j = 0; j < 2 * WF_AA_MAX; ++j) acc[j] = 0.f;
  const float4* a0 = reinterpret_cast<const float4*>(a.a0);
  const float4* a1 = reinterpret_cast<const float4*>(a.a1);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
    const float4 x0 = a0[i], x1 = a1[i];
#pragma unroll
    for (int j = 0; j < WF_AA_MAX; ++j) {
      if (j < a.nb) {
        const float4 y = reinterpret_cast<const float4*>(a.b[j])[i];
        acc[j] += dot4(x0, y);
        acc[WF_AA_MAX + j] += dot4(x1, y);
      }
    }
  }
  __shared__ double sred[kThreads / 32][2 * WF_AA_MAX];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 2 * WF_AA_MAX; ++j) {
    float v = acc[j];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sred[w][j] = (double)v;
  }
  __syncthreads();
  if (threadIdx.x < 2 * WF_AA_MAX) {
    double v = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) v += sred[k][threadIdx.x];
    part[(size_t)blockIdx.x * 2 * WF_AA_MAX + threadIdx.x] = v;
  }
}

// The partials of all blocks summed in a fixed order -- warp j sums dot j,
// lane k the partials of blocks k, k + 32, ..., then a shuffle tree -- and,
// by one thread, the least-squares step: row and column `slot` of the Gram
// matrix G = Delta F^T Delta F (held in device memory across corrections)
// take the new products, and (G + eps diag) gamma = Delta F^T f is solved by
// Cholesky in FP64.  A column whose pivot falls below 1e-10 of the largest
// diagonal (dependent on the others to FP32 accuracy) gets gamma = 0.
constexpr int kSolveThreads = 2 * WF_AA_MAX * 32;
__global__ void __launch_bounds__(kSolveThreads) aa_solve_kernel(const double* part, int nblocks, int slot, int n,
                                                                 double* G, float* gamma) {
  __shared__ double dots[2 * WF_AA_MAX];
  __shared__ double L[WF_AA_MAX][WF_AA_MAX];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double v = 0.0;
  for (int b = lane; b < nblocks; b += 32) v += part[(size_t)b * 2 * WF_AA_MAX + w];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) dots[w] = v;
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int k = 0; k < n; ++k) G[slot * WF_AA_MAX + k] = G[k * WF_AA_MAX + slot] = dots[k];
  bool use[WF_AA_MAX];
  double g[WF_AA_MAX], y[WF_AA_MAX];
  double dmax = 0.0;
  for (int i = 0; i < n; ++i) dmax = fmax(dmax, G[i * WF_AA_MAX + i]);
  for (int i = 0; i < n; ++i) {
    use[i] = false;
    g[i] = y[i] = 0.0;
    if (!(dmax > 0.0)) continue;
    double d = G[i * WF_AA_MAX + i] * (1.0 + 1e-12);
    for (int k = 0; k < i; ++k)
      if (use[k]) d -= L[i][k] * L[i][k];
    if (!(d > 1e-10 * dmax)) continue;
    use[i] = true;
    L[i][i] = sqrt(d);
    for (int r = i + 1; r < n; ++r) {
      double x = G[r * WF_AA_MAX + i];
      for (int k = 0; k < i; ++k)
        if (use[k]) x -= L[r][k] * L[i][k];
      L[r][i] = x / L[i][i];
    }
  }
  for (int i = 0; i < n; ++i) {
    if (!use[i]) continue;
    double x = dots[WF_AA_MAX + i];
    for (int k = 0; k < i; ++k)
      if (use[k]) x -= L[i][k] * y[k];
    y[i] = x / L[i][i];
  }
  for (int i = n - 1; i >= 0; --i) {
    if (!use[i]) continue;
    double x = y[i];
    for (int k = i + 1; k < n; ++k)
      if (use[k]) x -= L[k][i] * g[k];
    g[i] = x / L[i][i];
  }
  for (int i = 0; i < WF_AA_MAX; ++i) gamma[i] = i < n ? (float)g[i] : 0.f;
}

// u = f - sum_j gamma_j (dx_j + df_j); x += u
__global__ void aa_update_kernel(AAUpdate a, size_t n4) {
  float4* x = reinterpret_cast<float4*>(a.x);
  float4* u = reinterpret_cast<float4*>(a.u);
  const float4* f = reinterpret_cast<const float4*>(a.f);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
    float4 v = f[i];
    for (int j = 0; j < a.nj; ++j) {
      const float4 p = reinterpret_cast<const float4*>(a.dx[j])[i];
      const float4 q = reinterpret_cast<const float4*>(a.df[j])[i];
      const float g = __ldg(&a.gamma[j]);
      v.x -= g * (p.x + q.x);
      v.y -= g * (p.y + q.y);
      v.z -= g * (p.z + q.z);
      v.w -= g * (p.w + q.w);
    }
    u[i] = v;
    const float4 o = x[i];
    x[i] = make_float4(o.x + v.x, o.y + v.y, o.z + v.z, o.w + v.w);
  }
}

int grid_for(size_t n4) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    sms = 1;
  }
  const size_t want = (n4 + kThreads - 1) / kThreads;
  return (int)std::min<size_t>(want, (size_t)sms * 4);
}

}  // namespace

int aa_dots_blocks() { return 1024; }  // upper bound of the partial-sum grid

int launch_aa_diff(float* df, float* fprev, const float* e, size_t n, cudaStream_t s) {
  const size_t n4 = n / 4;
  aa_diff_kernel<<<grid_for(n4), kThreads, 0, s>>>(reinterpret_cast<float4*>(df), reinterpret_cast<float4*>(fprev),
                                                   reinterpret_cast<const float4*>(e), n4);
  return (int)cudaGetLastError();
}

int launch_aa_lsq(const AADots& a, size_t n, double* part, int slot, double* G, float* gamma, cudaStream_t s) {
  const size_t n4 = n / 4;
  // two CTAs per SM: few partials for the one-block solve to sum
  const int g = std::min(std::max(1, grid_for(n4) / 2), aa_dots_blocks());
  aa_dots_kernel<<<g, kThreads, 0, s>>>(a, n4, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return (int)e;
  aa_solve_kernel<<<1, kSolveThreads, 0, s>>>(part, g, slot, a.nb, G, gamma);
  return (int)cudaGetLastError();
}

int launch_aa_update(const AAUpdate& a, size_t n, cudaStream_t s) {
  const size_t n4 = n / 4;
  aa_update_kernel<<<grid_for(n4), kThreads, 0, s>>>(a, n4);
  return (int)cudaGetLastError();
}

}  // namespace wf
