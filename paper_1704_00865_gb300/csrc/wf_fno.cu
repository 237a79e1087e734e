// wf_fno.cu -- a Fourier neural operator (FNO) that predicts the Wiener
// solution from the data and noise weights, trained on the GPU with hand-
// written forward and backward kernels and Adam, and used to start the
// messenger iteration (the paper has no network; this is an extension).
//
// Network, for input x [B, 2, N, N] (data and log noise weight):
//   h_0 = P x + p;   h_{l+1} = act(W_l h_l + w_l + K_l h_l), l < L
//   (act = GELU, identity after the last layer);   y = Q h_L + q.
// K_l is the spectral convolution on the retained modes k_x in [0, MX),
// k_y in [0, MY) U [N - MY, N): a truncated real 2D DFT of each channel, one
// complex width x width matrix per mode, and the truncated inverse
// (1/N^2, real part, k_x > 0 counted twice).  The truncated transforms are
// direct sums with twiddle tables: for 16 x 32 retained modes that is fewer
// operations than a full FFT and needs no transpose.
//
// Layout: activations [B][C][N][N] FP32.  Weights live as an FP32 master
// vector (the order of the test oracle's flatten: P, p, per layer W_l, w_l,
// R_l as interleaved (re, im), then Q, q) with Adam moments; the forward and
// backward passes read an FP16 copy of the matrices (P, W_l, R_l, Q) and the
// FP32 biases, and accumulate in FP32.  Gradients are with respect to the
// FP16-rounded weights and update the FP32 master.  Every reduction runs in
// a fixed order (per-block partial sums, then one block), so a training
// step repeats bit for bit.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <vector>

#include "../../include/wf.h"
#include "wf_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxWidth = 64;
constexpr int kMaxModes = 32;

struct Layout {
  int cin = 2, width = 0, mx = 0, my = 0, layers = 0;
  size_t oP = 0, op = 0, oQ = 0, oq = 0, total = 0;
  std::vector<size_t> oW, ow, oR;
  void build() {
    size_t o = 0;
    oP = o; o += (size_t)width * cin;
    op = o; o += width;
    oW.resize(layers); ow.resize(layers); oR.resize(layers);
    for (int l = 0; l < layers; ++l) {
      oW[l] = o; o += (size_t)width * width;
      ow[l] = o; o += width;
      oR[l] = o; o += (size_t)width * width * 2 * my * mx * 2;
    }
    oQ = o; o += width;
    oq = o; o += 1;
    total = o;
  }
};

// ------------------------------------------------------------------ kernels

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
// d/dz [z Phi(z)] = Phi(z) + z phi(z)
__device__ __forceinline__ float gelu_grad(float z) {
  const float Phi = 0.5f * (1.f + erff(z * 0.70710678118654752f));
  const float phi = 0.3989422804014327f * __expf(-0.5f * z * z);
  return Phi + z * phi;
}

__global__ void to_half_kernel(const float* __restrict__ src, __half* __restrict__ dst, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = __float2half_rn(src[i]);
}

// out[b][o][p] = act(sum_i W[o][i] in[b][i][p] + bias[o] + add[b][o][p]);
// pre (if not null) keeps the argument of act.
__global__ void pointwise_fwd(const float* __restrict__ in, const __half* __restrict__ W,
                              const float* __restrict__ bias, const float* __restrict__ add, float* __restrict__ pre,
                              float* __restrict__ out, int B, int CI, int CO, int P, int act) {
  __shared__ float sW[kMaxWidth * kMaxWidth];
  for (int k = threadIdx.x; k < CO * CI; k += blockDim.x) sW[k] = __half2float(W[k]);
  __syncthreads();
  const size_t total = (size_t)B * P;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(g / P), p = (int)(g % P);
    float xin[kMaxWidth];
    for (int i = 0; i < CI; ++i) xin[i] = in[((size_t)b * CI + i) * P + p];
    for (int o = 0; o < CO; ++o) {
      float z = bias[o];
      for (int i = 0; i < CI; ++i) z = fmaf(sW[o * CI + i], xin[i], z);
      const size_t idx = ((size_t)b * CO + o) * P + p;
      if (add) z += add[idx];
      if (pre) pre[idx] = z;
      out[idx] = act ? gelu_f(z) : z;
    }
  }
}

// g_pre = g_out * act'(pre) (in place into gz), g_in[b][i][p] (+)= sum_o W[o][i] g_pre[b][o][p]
__global__ void pointwise_bwd_in(const float* __restrict__ gout, const float* __restrict__ pre, float* __restrict__ gz,
                                 const __half* __restrict__ W, float* __restrict__ gin, int B, int CI, int CO, int P,
                                 int act, int accumulate) {
  __shared__ float sW[kMaxWidth * kMaxWidth];
  for (int k = threadIdx.x; k < CO * CI; k += blockDim.x) sW[k] = __half2float(W[k]);
  __syncthreads();
  const size_t total = (size_t)B * P;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(g / P), p = (int)(g % P);
    float gp[kMaxWidth];
    for (int o = 0; o < CO; ++o) {
      const size_t idx = ((size_t)b * CO + o) * P + p;
      float v = gout[idx];
      if (act) v *= gelu_grad(pre[idx]);
      gp[o] = v;
      if (gz) gz[idx] = v;
    }
    if (!gin) continue;
    for (int i = 0; i < CI; ++i) {
      float s = 0.f;
      for (int o = 0; o < CO; ++o) s = fmaf(sW[o * CI + i], gp[o], s);
      const size_t idx = ((size_t)b * CI + i) * P + p;
      gin[idx] = accumulate ? gin[idx] + s : s;
    }
  }
}

// partial[blk][o][i] = sum over this block's pixels of gz[b][o][p] in[b][i][p];
// partial[blk][o][CI] = sum of gz[b][o][p] (the bias gradient)
__global__ void pointwise_bwd_w(const float* __restrict__ gz, const float* __restrict__ in, float* __restrict__ partial,
                                int B, int CI, int CO, int P) {
  const int o = blockIdx.y;
  const int nblk = gridDim.x;
  float acc[kMaxWidth + 1];
  for (int i = 0; i <= CI; ++i) acc[i] = 0.f;
  const size_t total = (size_t)B * P;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)nblk * blockDim.x) {
    const int b = (int)(g / P), p = (int)(g % P);
    const float v = gz[((size_t)b * CO + o) * P + p];
    for (int i = 0; i < CI; ++i) acc[i] = fmaf(v, in[((size_t)b * CI + i) * P + p], acc[i]);
    acc[CI] += v;
  }
  __shared__ float red[kThreads / 32];
  for (int i = 0; i <= CI; ++i) {
    float v = acc[i];
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      partial[((size_t)blockIdx.x * CO + o) * (CI + 1) + i] = t;
    }
    __syncthreads();
  }
}

// grad[oW + o*CI + i] = sum_blk partial[blk][o][i]; grad[ob + o] = sum_blk partial[blk][o][CI]
__global__ void pointwise_bwd_w_fin(const float* __restrict__ partial, int nblk, int CI, int CO, float* __restrict__ gW,
                                    float* __restrict__ gb) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= CO * (CI + 1)) return;
  const int o = k / (CI + 1), i = k % (CI + 1);
  float s = 0.f;
  for (int b = 0; b < nblk; ++b) s += partial[((size_t)b * CO + o) * (CI + 1) + i];
  if (i < CI) gW[o * CI + i] = s;
  else gb[o] = s;
}

// Row transform of R real rows of length N onto MX modes:
// out[r][k] = scale_k * sum_x in[r][x] e^{-2 pi i k x / N}, scale_k = s0 (k=0) or s1.
__global__ void dft_rows(const float* __restrict__ in, float2* __restrict__ out, const float2* __restrict__ tw_x,
                         int R, int N, int MX, float s0, float s1) {
  extern __shared__ float srow[];
  for (int r = blockIdx.x; r < R; r += gridDim.x) {
    __syncthreads();
    for (int x = threadIdx.x; x < N; x += blockDim.x) srow[x] = in[(size_t)r * N + x];
    __syncthreads();
    // MX outputs, each a length-N sum split over the warp's lanes
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int k = warp; k < MX; k += nw) {
      float re = 0.f, im = 0.f;
      for (int x = lane; x < N; x += 32) {
        const float2 w = tw_x[(size_t)k * N + x];  // e^{-2 pi i k x / N}
        re = fmaf(srow[x], w.x, re);
        im = fmaf(srow[x], w.y, im);
      }
      for (int s = 16; s > 0; s >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, s);
        im += __shfl_xor_sync(0xffffffffu, im, s);
      }
      if (lane == 0) {
        const float sc = k == 0 ? s0 : s1;
        out[(size_t)r * MX + k] = make_float2(re * sc, im * sc);
      }
    }
  }
}

// Column transform between N rows and the 2 MY retained k_y (per slice of
// [N][MX] or [2MY][MX] complex values):
//   forward (dir = -1): out[j][k] = sum_y in[y][k] e^{-2 pi i ky_j y / N}
//   inverse (dir = +1): out[y][k] = sum_j in[j][k] e^{+2 pi i ky_j y / N}
// tw_y[j][y] = e^{-2 pi i ky_j y / N}.
__global__ void dft_cols(const float2* __restrict__ in, float2* __restrict__ out, const float2* __restrict__ tw_y,
                         int S, int N, int MX, int MY2, int dir) {
  const int nout = (dir < 0) ? MY2 : N;
  const size_t total = (size_t)S * nout * MX;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(g % MX);
    const int j = (int)((g / MX) % nout);
    const size_t sl = g / ((size_t)MX * nout);
    float re = 0.f, im = 0.f;
    if (dir < 0) {
      const float2* src = in + sl * (size_t)N * MX + k;
      const float2* w = tw_y + (size_t)j * N;
      for (int y = 0; y < N; ++y) {
        const float2 a = src[(size_t)y * MX], t = w[y];
        re = fmaf(a.x, t.x, fmaf(-a.y, t.y, re));
        im = fmaf(a.x, t.y, fmaf(a.y, t.x, im));
      }
    } else {
      const float2* src = in + sl * (size_t)MY2 * MX + k;
      for (int jj = 0; jj < MY2; ++jj) {
        const float2 a = src[(size_t)jj * MX], t0 = tw_y[(size_t)jj * N + j];
        const float2 t = make_float2(t0.x, -t0.y);  // conjugate: e^{+...}
        re = fmaf(a.x, t.x, fmaf(-a.y, t.y, re));
        im = fmaf(a.x, t.y, fmaf(a.y, t.x, im));
      }
    }
    out[g] = make_float2(re, im);
  }
}

// out[r][x] (+)= scale * ( c0 Re(in[r][0]) + c1 sum_{k>=1} Re(in[r][k] e^{+2 pi i k x / N}) )
__global__ void idft_rows(const float2* __restrict__ in, float* __restrict__ out, const float2* __restrict__ tw_x,
                          int R, int N, int MX, float c0, float c1, float scale, int accumulate) {
  extern __shared__ float2 srowc[];
  for (int r = blockIdx.x; r < R; r += gridDim.x) {
    __syncthreads();
    for (int k = threadIdx.x; k < MX; k += blockDim.x) srowc[k] = in[(size_t)r * MX + k];
    __syncthreads();
    for (int x = threadIdx.x; x < N; x += blockDim.x) {
      float s = c0 * srowc[0].x;
      for (int k = 1; k < MX; ++k) {
        const float2 a = srowc[k], t = tw_x[(size_t)k * N + x];  // e^{-i}; Re(a e^{+i}) = a.x t.x + a.y t.y
        s = fmaf(c1, fmaf(a.x, t.x, a.y * t.y), s);
      }
      const size_t idx = (size_t)r * N + x;
      out[idx] = accumulate ? out[idx] + scale * s : scale * s;
    }
  }
}

// Y[b][o][m] = sum_i R[i][o][m] X[b][i][m]  (complex; R in FP16 pairs)
__global__ void mix_fwd(const float2* __restrict__ X, const __half2* __restrict__ R, float2* __restrict__ Y, int B,
                        int C, int NM) {
  const size_t total = (size_t)B * C * NM;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(g % NM), o = (int)((g / NM) % C);
    const int b = (int)(g / ((size_t)NM * C));
    float re = 0.f, im = 0.f;
    for (int i = 0; i < C; ++i) {
      const float2 r = __half22float2(R[((size_t)i * C + o) * NM + m]);
      const float2 x = X[((size_t)b * C + i) * NM + m];
      re = fmaf(r.x, x.x, fmaf(-r.y, x.y, re));
      im = fmaf(r.x, x.y, fmaf(r.y, x.x, im));
    }
    Y[g] = make_float2(re, im);
  }
}

// g_X[b][i][m] = sum_o conj(R[i][o][m]) g_Y[b][o][m]
__global__ void mix_bwd_x(const float2* __restrict__ gY, const __half2* __restrict__ R, float2* __restrict__ gX, int B,
                          int C, int NM) {
  const size_t total = (size_t)B * C * NM;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(g % NM), i = (int)((g / NM) % C);
    const int b = (int)(g / ((size_t)NM * C));
    float re = 0.f, im = 0.f;
    for (int o = 0; o < C; ++o) {
      const float2 r = __half22float2(R[((size_t)i * C + o) * NM + m]);
      const float2 y = gY[((size_t)b * C + o) * NM + m];
      re = fmaf(r.x, y.x, fmaf(r.y, y.y, re));
      im = fmaf(r.x, y.y, fmaf(-r.y, y.x, im));
    }
    gX[g] = make_float2(re, im);
  }
}

// g_R[i][o][m] = sum_b g_Y[b][o][m] conj(X[b][i][m]), written as (re, im) pairs
__global__ void mix_bwd_r(const float2* __restrict__ gY, const float2* __restrict__ X, float* __restrict__ gR, int B,
                          int C, int NM) {
  const size_t total = (size_t)C * C * NM;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(g % NM), o = (int)((g / NM) % C);
    const int i = (int)(g / ((size_t)NM * C));
    float re = 0.f, im = 0.f;
    for (int b = 0; b < B; ++b) {
      const float2 y = gY[((size_t)b * C + o) * NM + m];
      const float2 x = X[((size_t)b * C + i) * NM + m];
      re = fmaf(y.x, x.x, fmaf(y.y, x.y, re));
      im = fmaf(y.y, x.x, fmaf(-y.x, x.y, im));
    }
    gR[2 * g] = re;
    gR[2 * g + 1] = im;
  }
}

// per-sample sums of (y - t)^2 and t^2
__global__ void loss_partial(const float* __restrict__ y, const float* __restrict__ t, double* __restrict__ part,
                             int P) {
  const int b = blockIdx.y;
  double num = 0.0, den = 0.0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    const double d = (double)y[(size_t)b * P + p] - (double)t[(size_t)b * P + p];
    const double tv = t[(size_t)b * P + p];
    num += d * d;
    den += tv * tv;
  }
  __shared__ double rn[kThreads / 32], rd[kThreads / 32];
  for (int s = 16; s > 0; s >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, s);
    den += __shfl_xor_sync(0xffffffffu, den, s);
  }
  if ((threadIdx.x & 31) == 0) {
    rn[threadIdx.x >> 5] = num;
    rd[threadIdx.x >> 5] = den;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += rn[w];
      c += rd[w];
    }
    part[((size_t)b * gridDim.x + blockIdx.x) * 2] = a;
    part[((size_t)b * gridDim.x + blockIdx.x) * 2 + 1] = c;
  }
}

// loss = mean_b num_b / den_b; inv[b] = 1 / (B den_b)
__global__ void loss_fin(const double* __restrict__ part, int nblk, int B, double* __restrict__ loss,
                         float* __restrict__ inv) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double L = 0.0;
  for (int b = 0; b < B; ++b) {
    double n = 0.0, d = 0.0;
    for (int k = 0; k < nblk; ++k) {
      n += part[((size_t)b * nblk + k) * 2];
      d += part[((size_t)b * nblk + k) * 2 + 1];
    }
    d = d > 0.0 ? d : 1.0;
    L += n / d;
    inv[b] = (float)(1.0 / (B * d));
  }
  *loss = L / B;
}

// g_y = 2 (y - t) inv[b]
__global__ void loss_grad(const float* __restrict__ y, const float* __restrict__ t, const float* __restrict__ inv,
                          float* __restrict__ gy, int B, int P) {
  const size_t total = (size_t)B * P;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x)
    gy[g] = 2.f * (y[g] - t[g]) * inv[g / P];
}

__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// Inputs of the network for one map: x0 = d / sigma (0 on masked pixels),
// x1 = log(sigma^2 / pixel_var) (masked: log of a 1e-6 weight), with sigma^2
// the mean pixel variance over unmasked pixels (reduced in part/fin).
__global__ void feat_partial(const float* __restrict__ var, const uint8_t* __restrict__ mask, double* __restrict__ part,
                             size_t n) {
  double s = 0.0, c = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if (mask && mask[i]) continue;
    s += var[i];
    c += 1.0;
  }
  __shared__ double rs[kThreads / 32], rc[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if ((threadIdx.x & 31) == 0) {
    rs[threadIdx.x >> 5] = s;
    rc[threadIdx.x >> 5] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += rs[w];
      b += rc[w];
    }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

__global__ void feat_fin(const double* __restrict__ part, int nblk, float* __restrict__ sigma) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int k = 0; k < nblk; ++k) {
    a += part[2 * k];
    b += part[2 * k + 1];
  }
  *sigma = (float)sqrt(b > 0.0 ? a / b : 1.0);
}

__global__ void feat_map(const float* __restrict__ d, const float* __restrict__ var, const uint8_t* __restrict__ mask,
                         const float* __restrict__ sigma, float* __restrict__ x, size_t n) {
  const float sg = *sigma;
  const float s2 = sg * sg;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const bool m = mask && mask[i];
    x[i] = m ? 0.f : d[i] / sg;
    x[n + i] = m ? logf(1e-6f) : logf(s2 / var[i]);
  }
}

int grid_for(size_t n) {
  const size_t g = (n + kThreads - 1) / kThreads;
  return (int)(g < 4096 ? (g > 0 ? g : 1) : 4096);
}

}  // namespace

struct wf_fno_s {
  Layout lay;
  int n = 0, batch = 0;
  cudaStream_t stream = nullptr;
  float *master = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
  __half* half = nullptr;     // FP16 copy of the whole vector (matrices read from it)
  long long step = 0;
  // activations
  float* h = nullptr;         // [L+1][B][C][P]
  float* z = nullptr;         // [L][B][C][P] pre-activations
  float* kbuf = nullptr;      // [B][C][P] spectral branch output
  float* y = nullptr;         // [B][P]
  float* gh = nullptr;        // [B][C][P] gradient wrt h_l
  float* gz = nullptr;        // [B][C][P]
  float* gy = nullptr;        // [B][P]
  float2 *A = nullptr, *X = nullptr, *Y = nullptr;  // [L][B][C][N][MX], [L][B][C][2MY][MX], scratch
  float2 *tw_x = nullptr, *tw_y = nullptr;
  float* wpart = nullptr;
  double* lpart = nullptr;
  double* dloss = nullptr;
  float* inv = nullptr;
  int wblk = 0, lblk = 0;
  std::vector<void*> allocs;
};

namespace {

template <typename T>
bool alloc(wf_fno_s* F, T** p, size_t n) {
  if (cudaMalloc((void**)p, n * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  F->allocs.push_back(*p);
  return true;
}

size_t P_(const wf_fno_s* F) { return (size_t)F->n * F->n; }
size_t act_(const wf_fno_s* F) { return (size_t)F->batch * F->lay.width * P_(F); }
size_t spec_(const wf_fno_s* F) { return (size_t)F->batch * F->lay.width * F->n * F->lay.mx; }
size_t modes_(const wf_fno_s* F) { return (size_t)2 * F->lay.my * F->lay.mx; }

// spectral convolution of h_l (B*C slices) into kbuf, keeping A and X of layer l
int spectral_fwd(wf_fno_s* F, int l, const float* hin, int B) {
  const int C = F->lay.width, N = F->n, MX = F->lay.mx, MY2 = 2 * F->lay.my;
  const int S = B * C;
  float2* A = F->A + (size_t)l * spec_(F);
  float2* X = F->X + (size_t)l * F->batch * C * modes_(F);
  dft_rows<<<grid_for((size_t)S * N * 32) / 8 + 1, kThreads, N * sizeof(float), F->stream>>>(hin, A, F->tw_x, S * N, N,
                                                                                             MX, 1.f, 1.f);
  dft_cols<<<grid_for((size_t)S * MY2 * MX), kThreads, 0, F->stream>>>(A, X, F->tw_y, S, N, MX, MY2, -1);
  const __half2* R = reinterpret_cast<const __half2*>(F->half + F->lay.oR[l]);
  mix_fwd<<<grid_for((size_t)S * MY2 * MX), kThreads, 0, F->stream>>>(X, R, F->Y, B, C, MY2 * MX);
  // the inverse: columns back to N rows (reuse A's space of this call as scratch in Y order)
  float2* Bm = F->A + (size_t)F->lay.layers * spec_(F);  // one extra slot
  dft_cols<<<grid_for((size_t)S * N * MX), kThreads, 0, F->stream>>>(F->Y, Bm, F->tw_y, S, N, MX, MY2, +1);
  const float sc = 1.f / ((float)N * (float)N);
  idft_rows<<<grid_for((size_t)S * N) / 4 + 1, kThreads, MX * sizeof(float2), F->stream>>>(Bm, F->kbuf, F->tw_x, S * N,
                                                                                            N, MX, 1.f, 2.f, sc, 0);
  return (int)cudaGetLastError();
}

int forward(wf_fno_s* F, const float* x, int B) {
  const Layout& L = F->lay;
  const int C = L.width;
  const int P = (int)P_(F);
  const size_t gsz = grid_for((size_t)B * P);
  pointwise_fwd<<<gsz, kThreads, 0, F->stream>>>(x, F->half + L.oP, F->master + L.op, nullptr, nullptr, F->h, B,
                                                 L.cin, C, P, 0);
  for (int l = 0; l < L.layers; ++l) {
    float* hin = F->h + (size_t)l * act_(F);
    float* hout = F->h + (size_t)(l + 1) * act_(F);
    int rc = spectral_fwd(F, l, hin, B);
    if (rc) return rc;
    pointwise_fwd<<<gsz, kThreads, 0, F->stream>>>(hin, F->half + L.oW[l], F->master + L.ow[l], F->kbuf,
                                                   F->z + (size_t)l * act_(F), hout, B, C, C, P,
                                                   l < L.layers - 1 ? 1 : 0);
  }
  pointwise_fwd<<<gsz, kThreads, 0, F->stream>>>(F->h + (size_t)L.layers * act_(F), F->half + L.oQ, F->master + L.oq,
                                                 nullptr, nullptr, F->y, B, C, 1, P, 0);
  return (int)cudaGetLastError();
}

int pointwise_weight_grad(wf_fno_s* F, const float* gz, const float* in, int B, int CI, int CO, float* gW,
                          float* gb) {
  const int P = (int)P_(F);
  dim3 grid(F->wblk, CO);
  pointwise_bwd_w<<<grid, kThreads, 0, F->stream>>>(gz, in, F->wpart, B, CI, CO, P);
  pointwise_bwd_w_fin<<<(CO * (CI + 1) + 255) / 256, 256, 0, F->stream>>>(F->wpart, F->wblk, CI, CO, gW, gb);
  return (int)cudaGetLastError();
}

// loss and gradient of the loss into F->grad (x, t device arrays)
int backward(wf_fno_s* F, const float* x, const float* t, int B) {
  const Layout& L = F->lay;
  const int C = L.width, N = F->n, MX = L.mx, MY2 = 2 * L.my;
  const int P = (int)P_(F);
  const size_t gsz = grid_for((size_t)B * P);
  // loss and dL/dy
  dim3 lg(F->lblk, B);
  loss_partial<<<lg, kThreads, 0, F->stream>>>(F->y, t, F->lpart, P);
  loss_fin<<<1, 32, 0, F->stream>>>(F->lpart, F->lblk, B, F->dloss, F->inv);
  loss_grad<<<gsz, kThreads, 0, F->stream>>>(F->y, t, F->inv, F->gy, B, P);
  // projection Q
  const float* hL = F->h + (size_t)L.layers * act_(F);
  pointwise_weight_grad(F, F->gy, hL, B, C, 1, F->grad + L.oQ, F->grad + L.oq);
  pointwise_bwd_in<<<gsz, kThreads, 0, F->stream>>>(F->gy, nullptr, nullptr, F->half + L.oQ, F->gh, B, C, 1, P, 0, 0);
  const int S = B * C;
  const float sc = 1.f / ((float)N * (float)N);
  for (int l = L.layers - 1; l >= 0; --l) {
    const float* hin = F->h + (size_t)l * act_(F);
    // through the activation: gz = gh * act'(z)
    pointwise_bwd_in<<<gsz, kThreads, 0, F->stream>>>(F->gh, F->z + (size_t)l * act_(F), F->gz, F->half + L.oW[l],
                                                      nullptr, B, C, C, P, l < L.layers - 1 ? 1 : 0, 0);
    pointwise_weight_grad(F, F->gz, hin, B, C, C, F->grad + L.oW[l], F->grad + L.ow[l]);
    // spectral branch: g_Bm = (c_k / N^2) rowDFT(gz), g_Y = colDFT(g_Bm), then R and X
    float2* gB = F->A + (size_t)L.layers * spec_(F);
    dft_rows<<<grid_for((size_t)S * N * 32) / 8 + 1, kThreads, N * sizeof(float), F->stream>>>(F->gz, gB, F->tw_x,
                                                                                               S * N, N, MX, sc,
                                                                                               2.f * sc);
    dft_cols<<<grid_for((size_t)S * MY2 * MX), kThreads, 0, F->stream>>>(gB, F->Y, F->tw_y, S, N, MX, MY2, -1);
    const float2* X = F->X + (size_t)l * F->batch * C * modes_(F);
    mix_bwd_r<<<grid_for((size_t)C * C * MY2 * MX), kThreads, 0, F->stream>>>(F->Y, X, F->grad + L.oR[l], B, C,
                                                                               MY2 * MX);
    const __half2* R = reinterpret_cast<const __half2*>(F->half + L.oR[l]);
    float2* gX = F->A + (size_t)l * spec_(F);  // A of layer l is no longer needed: scratch for g_X
    mix_bwd_x<<<grid_for((size_t)S * MY2 * MX), kThreads, 0, F->stream>>>(F->Y, R, gX, B, C, MY2 * MX);
    // g_A = colIDFT(g_X) into gB, then g_h = Re rowIDFT(g_A) (weights 1, no scale)
    dft_cols<<<grid_for((size_t)S * N * MX), kThreads, 0, F->stream>>>(gX, gB, F->tw_y, S, N, MX, MY2, +1);
    // pointwise branch of g_h, then add the spectral branch
    pointwise_bwd_in<<<gsz, kThreads, 0, F->stream>>>(F->gz, nullptr, nullptr, F->half + L.oW[l], F->gh, B, C, C, P, 0,
                                                      0);
    idft_rows<<<grid_for((size_t)S * N) / 4 + 1, kThreads, MX * sizeof(float2), F->stream>>>(gB, F->gh, F->tw_x,
                                                                                              S * N, N, MX, 1.f, 1.f,
                                                                                              1.f, 1);
  }
  // lift P
  pointwise_weight_grad(F, F->gh, x, B, L.cin, C, F->grad + L.oP, F->grad + L.op);
  return (int)cudaGetLastError();
}

int refresh_half(wf_fno_s* F) {
  to_half_kernel<<<grid_for(F->lay.total), kThreads, 0, F->stream>>>(F->master, F->half, F->lay.total);
  return (int)cudaGetLastError();
}

bool dev_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

int wf_fno_create(wf_fno_t* out, int n, int batch, int width, int mx, int my, int layers, const float* params,
                  void* stream) {
  if (!out || !params || n < 16 || n > 1024 || (n & (n - 1)) != 0 || batch < 1 || batch > 64 || width < 1 ||
      width > kMaxWidth || (width & 1) || mx < 1 || mx > kMaxModes || my < 1 || my > kMaxModes || 2 * my > n || mx > n / 2 ||
      layers < 1 || layers > 8)
    return WF_EINVAL;
  wf_fno_s* F = new wf_fno_s();
  F->lay.width = width;
  F->lay.mx = mx;
  F->lay.my = my;
  F->lay.layers = layers;
  F->lay.build();
  F->n = n;
  F->batch = batch;
  F->stream = (cudaStream_t)stream;
  const size_t T = F->lay.total, P = (size_t)n * n;
  F->wblk = 64;
  F->lblk = 32;
  bool ok = alloc(F, &F->master, T) && alloc(F, &F->grad, T) && alloc(F, &F->m1, T) && alloc(F, &F->m2, T) &&
            alloc(F, &F->half, T) && alloc(F, &F->h, (size_t)(layers + 1) * act_(F)) &&
            alloc(F, &F->z, (size_t)layers * act_(F)) && alloc(F, &F->kbuf, act_(F)) &&
            alloc(F, &F->y, (size_t)batch * P) && alloc(F, &F->gh, act_(F)) && alloc(F, &F->gz, act_(F)) &&
            alloc(F, &F->gy, (size_t)batch * P) && alloc(F, &F->A, (size_t)(layers + 1) * spec_(F)) &&
            alloc(F, &F->X, (size_t)layers * batch * width * modes_(F)) &&
            alloc(F, &F->Y, (size_t)batch * width * modes_(F)) && alloc(F, &F->tw_x, (size_t)mx * n) &&
            alloc(F, &F->tw_y, (size_t)2 * my * n) &&
            alloc(F, &F->wpart, (size_t)F->wblk * width * (kMaxWidth + 1)) &&
            alloc(F, &F->lpart, (size_t)batch * F->lblk * 2) && alloc(F, &F->dloss, 1) && alloc(F, &F->inv, batch);
  if (!ok) {
    wf_fno_destroy(F);
    return WF_ENOMEM;
  }
  // twiddles in double, rounded once
  std::vector<float2> tx((size_t)mx * n), ty((size_t)2 * my * n);
  for (int k = 0; k < mx; ++k)
    for (int x = 0; x < n; ++x) {
      const double a = 2.0 * M_PI * (double)((long long)k * x % n) / n;
      tx[(size_t)k * n + x] = make_float2((float)cos(a), (float)-sin(a));
    }
  for (int j = 0; j < 2 * my; ++j) {
    const int ky = j < my ? j : n - 2 * my + j;
    for (int y = 0; y < n; ++y) {
      const double a = 2.0 * M_PI * (double)((long long)ky * y % n) / n;
      ty[(size_t)j * n + y] = make_float2((float)cos(a), (float)-sin(a));
    }
  }
  const cudaMemcpyKind k = dev_ptr(params) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  ok = cudaMemcpy(F->tw_x, tx.data(), tx.size() * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(F->tw_y, ty.data(), ty.size() * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(F->master, params, T * sizeof(float), k) == cudaSuccess &&
       cudaMemset(F->m1, 0, T * sizeof(float)) == cudaSuccess && cudaMemset(F->m2, 0, T * sizeof(float)) == cudaSuccess &&
       cudaMemset(F->grad, 0, T * sizeof(float)) == cudaSuccess;
  if (!ok || refresh_half(F) != cudaSuccess || cudaStreamSynchronize(F->stream) != cudaSuccess) {
    cudaGetLastError();
    wf_fno_destroy(F);
    return WF_ECUDA;
  }
  *out = F;
  return WF_OK;
}

void wf_fno_destroy(wf_fno_t F) {
  if (!F) return;
  for (void* p : F->allocs) cudaFree(p);
  delete F;
}

long long wf_fno_num_params(wf_fno_t F) { return F ? (long long)F->lay.total : -1; }

int wf_fno_forward(wf_fno_t F, const float* x, float* y, int nb) {
  if (!F || !x || !y || nb < 1 || nb > F->batch || !dev_ptr(x) || !dev_ptr(y)) return WF_EINVAL;
  int rc = forward(F, x, nb);
  if (rc) return WF_ECUDA;
  if (cudaMemcpyAsync(y, F->y, (size_t)nb * P_(F) * sizeof(float), cudaMemcpyDeviceToDevice, F->stream) != cudaSuccess)
    return WF_ECUDA;
  return cudaStreamSynchronize(F->stream) == cudaSuccess ? WF_OK : WF_ECUDA;
}

int wf_fno_gradient(wf_fno_t F, const float* x, const float* t, int nb, float* grad, double* loss) {
  if (!F || !x || !t || nb < 1 || nb > F->batch || !dev_ptr(x) || !dev_ptr(t)) return WF_EINVAL;
  if (forward(F, x, nb) || backward(F, x, t, nb)) return WF_ECUDA;
  if (grad && cudaMemcpyAsync(grad, F->grad, F->lay.total * sizeof(float), cudaMemcpyDefault, F->stream) != cudaSuccess)
    return WF_ECUDA;
  double l = 0.0;
  if (cudaMemcpyAsync(&l, F->dloss, sizeof(double), cudaMemcpyDeviceToHost, F->stream) != cudaSuccess ||
      cudaStreamSynchronize(F->stream) != cudaSuccess)
    return WF_ECUDA;
  if (loss) *loss = l;
  return WF_OK;
}

int wf_fno_train_step(wf_fno_t F, const float* x, const float* t, int nb, double lr, double* loss) {
  if (!F || !x || !t || nb < 1 || nb > F->batch || !(lr > 0.0) || !dev_ptr(x) || !dev_ptr(t)) return WF_EINVAL;
  if (forward(F, x, nb) || backward(F, x, t, nb)) return WF_ECUDA;
  F->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)F->step), c2 = 1.f - powf(b2, (float)F->step);
  adam_kernel<<<grid_for(F->lay.total), kThreads, 0, F->stream>>>(F->master, F->grad, F->m1, F->m2, F->lay.total,
                                                                  (float)lr, b1, b2, 1e-8f, c1, c2);
  if (refresh_half(F) != cudaSuccess) return WF_ECUDA;
  double l = 0.0;
  if (cudaMemcpyAsync(&l, F->dloss, sizeof(double), cudaMemcpyDeviceToHost, F->stream) != cudaSuccess ||
      cudaStreamSynchronize(F->stream) != cudaSuccess)
    return WF_ECUDA;
  if (loss) *loss = l;
  return WF_OK;
}

int wf_fno_get_params(wf_fno_t F, float* out, int rounded) {
  if (!F || !out) return WF_EINVAL;
  if (!rounded) {
    if (cudaMemcpy(out, F->master, F->lay.total * sizeof(float), cudaMemcpyDefault) != cudaSuccess) return WF_ECUDA;
    return WF_OK;
  }
  // the values the forward pass uses: FP16 matrices, FP32 biases
  std::vector<__half> hh(F->lay.total);
  std::vector<float> mm(F->lay.total);
  if (cudaMemcpy(hh.data(), F->half, F->lay.total * sizeof(__half), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(mm.data(), F->master, F->lay.total * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return WF_ECUDA;
  std::vector<char> is_bias(F->lay.total, 0);
  for (int o = 0; o < F->lay.width; ++o) is_bias[F->lay.op + o] = 1;
  for (int l = 0; l < F->lay.layers; ++l)
    for (int o = 0; o < F->lay.width; ++o) is_bias[F->lay.ow[l] + o] = 1;
  is_bias[F->lay.oq] = 1;
  for (size_t i = 0; i < F->lay.total; ++i) mm[i] = is_bias[i] ? mm[i] : __half2float(hh[i]);
  return cudaMemcpy(out, mm.data(), F->lay.total * sizeof(float), cudaMemcpyDefault) == cudaSuccess ? WF_OK : WF_ECUDA;
}

int wf_fno_features(int ny, int nx, const float* d, const float* pixel_var, const uint8_t* mask, float* x_out,
                    float* sigma_out, void* stream) {
  if (!d || !pixel_var || !x_out || !sigma_out || ny < 1 || nx < 1) return WF_EINVAL;
  if (!dev_ptr(d) || !dev_ptr(pixel_var) || !dev_ptr(x_out) || !dev_ptr(sigma_out) || (mask && !dev_ptr(mask)))
    return WF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)ny * nx;
  constexpr int nblk = 64;
  double* part = nullptr;
  if (cudaMallocAsync((void**)&part, 2 * nblk * sizeof(double), s) != cudaSuccess) {
    cudaGetLastError();
    return WF_ENOMEM;
  }
  feat_partial<<<nblk, kThreads, 0, s>>>(pixel_var, mask, part, n);
  feat_fin<<<1, 32, 0, s>>>(part, nblk, sigma_out);
  feat_map<<<grid_for(n), kThreads, 0, s>>>(d, pixel_var, mask, sigma_out, x_out, n);
  cudaFreeAsync(part, s);
  return cudaGetLastError() == cudaSuccess ? WF_OK : WF_ECUDA;
}

}  // extern "C"
