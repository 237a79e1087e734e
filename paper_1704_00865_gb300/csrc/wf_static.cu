// wf_static.cu -- wf_fft2_noalloc: the 2D transform of wf_fft2 for callers
// that may not allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code embedded in a host
// application whose own allocator owns every byte of device memory, and
// pipelines that forbid allocation once they have started running (an
// allocation can block, fail, or synchronise the device at an unpredictable
// moment).  wf_fft2 needs a plan, and a plan allocates.  This entry point
// takes the two working buffers it needs -- the intermediate row-transformed
// spectrum and the twiddle tables -- from one file-scope device array whose
// size is fixed when the library is loaded.
//
// The array lives on every GPU that loads this library, until the process
// exits.  Host code may not use its name as an address (on the host it names
// a stand-in object), so each device's address is fetched once with
// cudaGetSymbolAddress, with that device current, and handed to the kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <mutex>

#include "../../include/wf.h"
#include "wf_internal.h"
#include "wf_ptr.h"

namespace {

constexpr int kMaxSide = 4096;                 // twiddle table length per axis
constexpr size_t kMaxSpectrum = (size_t)1 << 19;  // complex values: ny * nx / 2 <= 2^19
constexpr size_t kStaticComplex = 2 * (size_t)kMaxSide + kMaxSpectrum;  // 4 MiB + 64 KiB

// [0, 4096): exp(-2 pi i k / nx); [4096, 8192): exp(-2 pi i k / ny);
// [8192, ...): the row-transformed spectrum between the two passes.
static __device__ __align__(256) float2 wf_static_scratch[kStaticComplex];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float2* g_addr[kMaxDevices] = {};

// twiddles in double precision (sincospi), rounded once to float
__global__ void static_twiddles(float2* tw, int nx, int ny) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nx) {
    double s, c;
    sincospi(2.0 * (double)i / (double)nx, &s, &c);
    tw[i] = make_float2((float)c, (float)-s);
  }
  if (i < ny) {
    double s, c;
    sincospi(2.0 * (double)i / (double)ny, &s, &c);
    tw[kMaxSide + i] = make_float2((float)c, (float)-s);
  }
}

// Device address of the array on the current device (set up on first use).
int static_base(float2** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return WF_ECUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_addr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, wf_static_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return WF_ECUDA;
    }
    g_addr[dev] = static_cast<float2*>(p);
  }
  *out = g_addr[dev];
  return WF_OK;
}

// device memory of the current GPU (or managed memory); host memory and
// another GPU's memory are rejected
bool on_device(const void* p) {
  cudaPointerAttributes at{};
  const cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) cudaGetLastError();
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) cudaGetLastError();
  return wf::classify_ptr(e == cudaSuccess, (int)at.type, at.device, cur) == wf::PTR_DEVICE;
}

}  // namespace

extern "C" int wf_fft2_noalloc(int ny, int nx, const float* in, float* out, int inverse, void* stream) {
  if (!in || !out) return WF_EINVAL;
  if (!wf::size_supported(nx) || !wf::size_supported(ny)) return WF_EUNSUPPORTED;
  if ((size_t)ny * (size_t)(nx / 2) > kMaxSpectrum) return WF_EUNSUPPORTED;
  if (!on_device(in) || !on_device(out)) return WF_EINVAL;
  float2* base = nullptr;
  int rc = static_base(&base);
  if (rc != WF_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  float2* twx = base;
  float2* twy = base + kMaxSide;
  float2* spec = base + 2 * kMaxSide;
  const int nmax = nx > ny ? nx : ny;
  // launched with cudaLaunchKernelEx, whose return value is this launch's
  // own status (an error some earlier call left pending is not collected)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((nmax + 255) / 256);
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  if (cudaLaunchKernelEx(&cfg, static_twiddles, base, nx, ny) != cudaSuccess) return WF_ECUDA;

  wf::RowArgs ra{};
  ra.ny = ny;
  ra.nx = nx;
  ra.twx = twx;
  wf::ColArgs ca{};
  ca.ny = ny;
  ca.nx = nx;
  ca.twy = twy;
  if (!inverse) {
    ra.in_px = (const float2*)in;
    ra.out_rf = spec;
    if (wf::launch_row(wf::ROW_R2C, ra, s)) return WF_ECUDA;
    ca.in = spec;
    ca.out = (float2*)out;
    if (wf::launch_col(wf::COL_FWD, ca, s)) return WF_ECUDA;
  } else {
    ca.in = (const float2*)in;
    ca.out = spec;
    if (wf::launch_col(wf::COL_INV, ca, s)) return WF_ECUDA;
    ra.in_rf = spec;
    ra.out_px = (float2*)out;
    if (wf::launch_row(wf::ROW_C2R, ra, s)) return WF_ECUDA;
  }
  return WF_OK;
}
